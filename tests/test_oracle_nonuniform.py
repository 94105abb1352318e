"""Pins of the oracle on a non-uniform wall-normal grid (Section 2: variable
cell size in the wall-normal direction; Eqs. NS_prov, elliptic, projection,
update_pressure with the y spacings of each row).

Every check builds its reference from the face positions with numpy, not
from the oracle's formulas:
 - uniform face positions given explicitly reproduce the uniform oracle;
 - the Poisson solve satisfies L_c phi = rhs with L_c assembled here
   (zero flux through the walls) and a zero volume-weighted mean;
 - the projected field's divergence (computed here) vanishes;
 - the y sweep solves (1 - beta L_y) x = r with L_y assembled here;
 - the wall-normal viscous operator converges at second order on a
   smoothly stretched grid.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import OracleSim
from paper_2606_09799_gb300 import inputs


def spacings(yf):
    """Cell heights hc (ny), centre distances across faces hf (ny + 1; the wall
    faces measure to the mirrored first/last centre), centres yc."""
    hc = np.diff(yf)
    yc = 0.5 * (yf[:-1] + yf[1:])
    hf = np.empty(len(yf))
    hf[1:-1] = np.diff(yc)
    hf[0], hf[-1] = hc[0], hc[-1]
    return hc, hf, yc


def lap_c_dense_y(yf):
    """Wall-normal part of L_c (centres, zero flux through the walls)."""
    hc, hf, _ = spacings(yf)
    ny = len(hc)
    A = np.zeros((ny, ny))
    for j in range(ny):
        if j + 1 < ny:
            A[j, j + 1] += 1.0 / (hc[j] * hf[j + 1])
            A[j, j] -= 1.0 / (hc[j] * hf[j + 1])
        if j > 0:
            A[j, j - 1] += 1.0 / (hc[j] * hf[j])
            A[j, j] -= 1.0 / (hc[j] * hf[j])
    return A


def apply_lap_c(g, yf, phi):
    nz, ny, nx = phi.shape
    out = (np.roll(phi, -1, 2) - 2 * phi + np.roll(phi, 1, 2)) / g.dx ** 2
    out += (np.roll(phi, -1, 0) - 2 * phi + np.roll(phi, 1, 0)) / g.dz ** 2
    out += np.einsum("ab,kbi->kai", lap_c_dense_y(yf), phi)
    return out


def divergence_np(g, yf, u, v, w):
    hc = np.diff(yf)
    return ((np.roll(u, -1, 2) - u) / g.dx + (v[:, 1:, :] - v[:, :-1, :]) / hc[None, :, None]
            + (np.roll(w, -1, 0) - w) / g.dz)


def test_uniform_faces_reproduce_the_uniform_oracle():
    nx, ny, nz = 12, 10, 8
    u, v, w, p = inputs.random_fields(nx, ny, nz, seed=3, amp=0.2)
    a = OracleSim(nx, ny, nz, re=80.0, dt=2e-3)
    b = OracleSim(nx, ny, nz, re=80.0, dt=2e-3, yfaces=np.linspace(0.0, 1.0, ny + 1))
    for s in (a, b):
        s.set_fields(u, v, w, p)
        s.set_body_force(1.5, 0.0, 0.2)
        s.step(3)
    for x, y in zip(a.fields(), b.fields()):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12)


def test_poisson_solve_satisfies_the_assembled_operator():
    nx, ny, nz = 8, 12, 6
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    rng = np.random.default_rng(7)
    hc = np.diff(yf)
    rhs = rng.standard_normal((nz, ny, nx))
    rhs -= (rhs * hc[None, :, None]).sum() / (hc.sum() * nx * nz)   # compatible: zero volume integral
    phi = orc.poisson(g, rhs)
    np.testing.assert_allclose(apply_lap_c(g, yf, phi), rhs, rtol=0, atol=1e-9 * np.abs(rhs).max())
    assert abs((phi * hc[None, :, None]).sum()) <= 1e-10 * np.abs(phi).sum()
    np.testing.assert_allclose(orc.lap_c(g, phi), apply_lap_c(g, yf, phi), rtol=0, atol=1e-9)


def test_projection_leaves_no_divergence():
    nx, ny, nz = 8, 12, 6
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    u, v, w, p = inputs.random_fields(nx, ny, nz, seed=5)
    adt = 0.01
    div = divergence_np(g, yf, u, v, w)
    np.testing.assert_allclose(orc.divergence(g, u, v, w), div, rtol=0, atol=1e-12 * np.abs(div).max())
    phi = orc.poisson(g, div / adt)
    orc.project(g, u, v, w, p, phi, adt, 100.0)
    assert np.abs(divergence_np(g, yf, u, v, w)).max() <= 1e-10 * np.abs(div).max()


@pytest.mark.parametrize("c", [0, 1])
def test_y_sweep_solves_the_assembled_factor(c):
    nx, ny, nz = 4, 14, 3
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    hc, hf, _ = spacings(yf)
    beta = 3e-3
    rng = np.random.default_rng(11 + c)
    shape = orc.field_shape(g, c)
    r = rng.standard_normal(shape)
    if c == 1:
        r[:, 0, :] = r[:, ny, :] = 0.0
    x = r.copy()
    orc.sweep(g, c, 1, x, np.full(shape, -1, dtype=np.int32), beta)
    # L_y applied here: centres with no-slip ghosts (u_{-1} = -u_0), faces with v = 0 on the walls
    if c == 0:
        Ly = np.zeros((ny, ny))
        for j in range(ny):
            up = 1.0 / (hc[j] * hf[j + 1])
            dn = 1.0 / (hc[j] * hf[j])
            Ly[j, j] -= up + dn
            if j + 1 < ny:
                Ly[j, j + 1] += up
            else:
                Ly[j, j] -= up          # ghost -u_{ny-1}
            if j > 0:
                Ly[j, j - 1] += dn
            else:
                Ly[j, j] -= dn          # ghost -u_0
        lhs = x - beta * np.einsum("ab,kbi->kai", Ly, x)
        np.testing.assert_allclose(lhs, r, rtol=0, atol=1e-12)
    else:
        Ly = np.zeros((ny + 1, ny + 1))
        for j in range(1, ny):
            up = 1.0 / (hf[j] * hc[j])
            dn = 1.0 / (hf[j] * hc[j - 1])
            Ly[j, j] -= up + dn
            Ly[j, j + 1] += up
            Ly[j, j - 1] += dn
        lhs = x - beta * np.einsum("ab,kbi->kai", Ly, x)
        np.testing.assert_allclose(lhs[:, 1:ny, :], r[:, 1:ny, :], rtol=0, atol=1e-12)


def test_wall_normal_viscous_term_is_second_order():
    """R = dt (alpha/Re) L u for u = sin(pi y), no advection (gamma = 0):
    the error against -pi^2 sin(pi y) falls as h^2 on the stretched grid."""
    errs = []
    for ny in (16, 32, 64):
        nx = nz = 4
        yf = inputs.stretched_faces(ny)
        g = orc.make_grid(nx, ny, nz, yfaces=yf)
        _, _, yc = spacings(yf)
        u = np.broadcast_to(np.sin(np.pi * yc)[None, :, None], (nz, ny, nx)).copy()
        v = np.zeros(orc.field_shape(g, 1))
        w = np.zeros(orc.field_shape(g, 2))
        p = np.zeros((nz, ny, nx))
        R, _ = orc.rhs(g, u, v, w, p, orc.no_tags(g), gam=0.0, rho=0.0, alp=1.0, dt=1.0, re=1.0)
        exact = -np.pi ** 2 * np.sin(np.pi * yc)
        errs.append(np.abs(R[0][0, :, 0] - exact).max())
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > 1.8), (errs, slopes)


def row_coords(yf, c):
    """Wall-normal row coordinates of component c's lattice with one mirrored
    row beyond each wall (index 0 of the result is row -1), and the local cell
    size of every stored row (cell height for u, w; centre distance for v)."""
    hc, hf, yc = spacings(yf)
    if c == 1:
        rows = np.concatenate([[-yf[1]], yf, [2 * yf[-1] - yf[-2]]])
        return rows, hf
    rows = np.concatenate([[-yc[0]], yc, [2 * yf[-1] - yc[-1]]])
    return rows, hc


def brute_tags(g, yf, xyz, tri):
    """Algorithm 1 restated with the local cell of each node (box margin and
    diagonal from that node's row), every node and periodic image against
    every triangle; owner = smallest |N|^2, ties to the smallest index."""
    nx, ny, nz = g.nx, g.ny, g.nz
    out = []
    for c in range(3):
        rows, hy = row_coords(yf, c)
        nyc = ny + 1 if c == 1 else ny
        own = np.full((nz, nyc, nx), -1, dtype=np.int32)
        best = np.full((nz, nyc, nx), np.inf)
        jlo, jhi = (1, ny - 1) if c == 1 else (0, ny - 1)
        ox = 0.0 if c == 0 else 0.5
        oz = 0.0 if c == 2 else 0.5

        def pos(i, j, k):
            return np.array([(i + ox) * g.dx, rows[j + 1], (k + oz) * g.dz])

        for t, (a, b, cc) in enumerate(xyz[tri]):
            mn = np.minimum(np.minimum(a, b), cc)
            mx = np.maximum(np.maximum(a, b), cc)
            for k in range(nz):
                for j in range(jlo, jhi + 1):
                    for i in range(nx):
                        for mk in (-1, 0, 1):
                            for mi in (-1, 0, 1):
                                ii, kk = i + mi * nx, k + mk * nz
                                x = pos(ii, j, kk)
                                dl = (g.dx, hy[j], g.dz)
                                if not all(mn[d] - dl[d] < x[d] < mx[d] + dl[d] for d in range(3)):
                                    continue
                                X, _ = orc.closest_point(x, a, b, cc)
                                N = x - X
                                n2 = N[0] * N[0] + N[1] * N[1] + N[2] * N[2]
                                if not n2 <= (g.dx * g.dx + hy[j] * hy[j]) + g.dz * g.dz:
                                    continue
                                hit = n2 == 0.0
                                for di, dj, dk in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1),
                                                   (0, 0, 1)):
                                    vn = pos(ii + di, j + dj, kk + dk) - X
                                    if N[0] * vn[0] + N[1] * vn[1] + N[2] * vn[2] < 0.0:
                                        hit = True
                                if hit and (own[k, j, i] < 0 or n2 < best[k, j, i]):
                                    own[k, j, i] = t
                                    best[k, j, i] = n2
        out.append(own)
    return out


def test_uniform_faces_reproduce_uniform_surface_path():
    """Face positions j/ny given explicitly (exact binary fractions) tag, force
    and measure slip exactly as the uniform grid does."""
    nx, ny, nz = 16, 16, 16
    yf = np.arange(ny + 1) / ny
    gu = orc.make_grid(nx, ny, nz)
    gs = orc.make_grid(nx, ny, nz, yfaces=yf)
    xyz, tri = inputs.icosphere(1, 0.18, (0.48, 0.47, 0.53))
    ou, du = orc.tag(gu, xyz, tri)
    os_, ds = orc.tag(gs, xyz, tri)
    for c in range(3):
        np.testing.assert_array_equal(ou[c], os_[c])
        np.testing.assert_array_equal(du[c], ds[c])
    rng = np.random.default_rng(3)
    vel = rng.standard_normal(xyz.shape)
    h = 2.0 * np.sqrt((gu.dx * gu.dx + gu.dy * gu.dy) + gu.dz * gu.dz)
    for c in range(3):
        src = rng.standard_normal(orc.field_shape(gu, c))
        a, b = src.copy(), src.copy()
        assert orc.force(gu, c, src, a, ou[c], xyz, vel, tri, h) == 0
        assert orc.force(gs, c, src, b, ou[c], xyz, vel, tri, -1.0) == 0
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_stretched_tagging_matches_independent_brute_force(seed):
    nx, ny, nz = 6, 10, 6
    yf = inputs.stretched_faces(ny, beta=2.2)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    xyz, tri = inputs.random_triangles(6, seed, lo=0.15, hi=0.85, size=0.3)
    own, _ = orc.tag(g, xyz, tri)
    own_b, _ = orc.tag(g, xyz, tri, brute=True)
    ref = brute_tags(g, yf, xyz, tri)
    for c in range(3):
        np.testing.assert_array_equal(own[c], ref[c])
        np.testing.assert_array_equal(own_b[c], ref[c])
    assert sum(int((o >= 0).sum()) for o in own) > 20


@pytest.mark.parametrize("yw", [0.0371, 0.2013, 0.5 + 1e-3])
def test_stretched_flat_plane_closed_form(yw):
    """A plane y = yw across the periodic box: a node is tagged iff it lies
    within its own cell size of the plane (the box of Algorithm 1) and one of
    its wall-normal neighbours lies across the plane."""
    nx, ny, nz = 64, 24, 64
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    # a plate wider than the box; near its edges (and its diagonal) Algorithm 1
    # also tags nodes whose height above the plane is below about dx / 2, so
    # dx is kept well below the distance of any non-bracketing row
    big = 0.3
    xyz = np.array([[-big, yw, -big], [1 + big, yw, -big], [-big, yw, 1 + big], [1 + big, yw, 1 + big]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    own, _ = orc.tag(g, xyz, tri)
    for c in range(3):
        rows, hy = row_coords(yf, c)
        y = rows[1:-1]
        s = y - yw
        across = (s * (rows[:-2] - yw) < 0) | (s * (rows[2:] - yw) < 0)
        expect = (np.abs(s) > 0) & (np.abs(s) < hy) & across
        if c == 1:
            expect[0] = expect[-1] = False
        got = own[c] >= 0
        np.testing.assert_array_equal(got, np.broadcast_to(expect[None, :, None], got.shape))
        assert expect.sum() >= 1


def test_stretched_forcing_is_exact_for_affine_fields():
    """Eq. new_IB with u^e trilinear on the stretched rows reproduces an
    affine field at every forcing node (the interpolant, the wall value and
    the blend are all exact for affine data)."""
    nx, ny, nz = 24, 24, 24
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    xyz, tri = inputs.icosphere(2, 0.2, (0.5, 0.47, 0.5))
    own, _ = orc.tag(g, xyz, tri)
    grad = np.array([[0.3, -1.1, 0.7], [1.3, 0.4, -0.2], [-0.6, 0.9, 0.25]])
    base = np.array([0.2, -0.5, 1.0])
    for c in range(3):
        rows, _ = row_coords(yf, c)
        nyc = ny + 1 if c == 1 else ny
        x = (np.arange(nx) + (0.0 if c == 0 else 0.5)) * g.dx
        z = (np.arange(nz) + (0.0 if c == 2 else 0.5)) * g.dz
        y = rows[1:nyc + 1]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        f = base[c] + grad[c, 0] * X + grad[c, 1] * Y + grad[c, 2] * Z
        vel = np.zeros_like(xyz)
        vel[:, c] = base[c] + xyz @ grad[c]
        dst = np.zeros_like(f)
        assert orc.force(g, c, f, dst, own[c], xyz, vel, tri, -1.0) == 0
        m = own[c] >= 0
        assert m.sum() > 50
        np.testing.assert_allclose(dst[m], f[m], rtol=0, atol=1e-12)


def test_stretched_probe_length_is_twice_the_local_diagonal():
    """Plane y = yw, field (y - yw)^2 and U = 0: a forcing node at distance d
    takes alpha * I(yw +- h) with h = 2 sqrt(dx^2 + hy^2 + dz^2) from its own
    row and I the piecewise-linear interpolant along the rows (Eq. probe)."""
    nx, ny, nz = 64, 24, 64
    yf = inputs.stretched_faces(ny)
    g = orc.make_grid(nx, ny, nz, yfaces=yf)
    yw = 0.2013
    # a plate wider than the box; near its edges (and its diagonal) Algorithm 1
    # also tags nodes whose height above the plane is below about dx / 2, so
    # dx is kept well below the distance of any non-bracketing row
    big = 0.3
    xyz = np.array([[-big, yw, -big], [1 + big, yw, -big], [-big, yw, 1 + big], [1 + big, yw, 1 + big]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    own, _ = orc.tag(g, xyz, tri)
    for c in range(3):
        rows, hy = row_coords(yf, c)
        nyc = ny + 1 if c == 1 else ny
        y = rows[1:nyc + 1]
        f = np.broadcast_to(((y - yw) ** 2)[None, :, None], (nz, nyc, nx)).copy()
        dst = np.zeros_like(f)
        assert orc.force(g, c, f, dst, own[c], xyz, np.zeros_like(xyz), tri, -1.0) == 0
        ko, io = 40, 10   # a column far from the plate's edges and diagonal
        tagged = np.nonzero((own[c] >= 0)[ko, :, io])[0]
        assert len(tagged) >= 1
        for j in tagged:
            d = abs(y[j] - yw)
            h = 2.0 * np.sqrt((g.dx * g.dx + hy[j] * hy[j]) + g.dz * g.dz)
            ye = yw + np.sign(y[j] - yw) * h
            expect = (d / h) * np.interp(ye, y, (y - yw) ** 2)
            np.testing.assert_allclose(dst[ko, j, io], expect, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------
# immersed-plane flows on the stretched grid (Section 4.2's configuration:
# an immersed wall on a non-uniform wall-normal grid)
# ---------------------------------------------------------------------------
def _wall(yw, lx, lz, vel=(0.0, 0.0, 0.0)):
    """A plane y = yw wider than the periodic box (two triangles)."""
    b = 0.3 * max(lx, lz)
    xyz = np.array([[-b, yw, -b], [lx + b, yw, -b], [-b, yw, lz + b], [lx + b, yw, lz + b]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    return xyz, np.tile(np.asarray(vel, dtype=float), (4, 1)), tri


def test_stretched_immersed_plane_couette_is_exact():
    """A plane at y_w moving at U_p between resting walls: on the stretched
    grid too the steady discrete solution is the exact piecewise-linear
    profile (the flux-form second difference and the row-weighted linear
    reconstruction of Eq. new_IB are both exact for it)."""
    yw, up, ny = 0.4137, 0.8, 24
    yf = inputs.stretched_faces(ny)
    L = 4.0 / ny
    sim = OracleSim(4, ny, 4, lx=L, lz=L, re=1.0, dt=0.01, yfaces=yf)
    xyz, vel, tri = _wall(yw, L, L, (up, 0.0, 0.0))
    sim.set_surface(xyz, vel, tri)
    sim.step(400)
    _, _, yc = spacings(yf)
    Y = np.broadcast_to(yc[None, :, None], sim.u.shape)
    ex = np.where(Y < yw, up * Y / yw, up * (1 - Y) / (1 - yw))
    fluid = sim.owners[0] < 0
    err = np.abs(sim.u - ex)[fluid].max()
    assert err < 1e-10, err
    assert sim.last["slip"] < 1e-10


def _poiseuille_stretched(ny, frac=0.37, s_w=0.43):
    """Steady immersed-plane Poiseuille flow on the tanh-stretched grid.  The
    wall sits at a fixed fraction of its cell (the cell at the fraction s_w
    of the rows), as Section 4.2 builds its grids so the surface keeps its
    place relative to the nodes at every N; the error constant of the IB
    reconstruction depends on that place."""
    G, re = 1.0, 1.0
    yf = inputs.stretched_faces(ny)
    jw = int(np.floor(s_w * ny))
    yw = yf[jw] + frac * (yf[jw + 1] - yf[jw])
    L = 4.0 / ny
    sim = OracleSim(4, ny, 4, lx=L, lz=L, re=re, dt=0.01, yfaces=yf)
    xyz, vel, tri = _wall(yw, L, L)
    sim.set_surface(xyz, vel, tri)
    sim.set_body_force(G, 0.0, 0.0)
    sim.step(300)
    _, _, yc = spacings(yf)
    Y = np.broadcast_to(yc[None, :, None], sim.u.shape)
    ex = np.where(Y < yw, 0.5 * G * re * Y * (yw - Y), 0.5 * G * re * (Y - yw) * (1 - Y))
    up = (sim.owners[0] < 0) & (Y > yw)
    sel = yc > yw
    coef = np.polynomial.chebyshev.chebfit(yc[sel], sim.u[0, sel, 0], 4)
    wall = abs(np.polynomial.chebyshev.chebval(yw, coef))
    return np.abs(sim.u - ex)[up].mean(), wall


def test_stretched_immersed_plane_poiseuille_second_order():
    """Section 4.2's claim on a smoothly stretched wall-normal grid: the bulk
    L1 error on the driven side and the no-slip error at the immersed wall
    (4th-order Chebyshev fit extrapolated to it) both fall at second order."""
    e = [_poiseuille_stretched(n) for n in (32, 64, 128)]
    l1 = [x[0] for x in e]
    wall = [x[1] for x in e]
    slopes_l1 = [np.log2(l1[i] / l1[i + 1]) for i in range(2)]
    slopes_w = [np.log2(wall[i] / wall[i + 1]) for i in range(2)]
    assert min(slopes_l1) > 1.7, (l1, slopes_l1)
    assert min(slopes_w) > 1.8, (wall, slopes_w)
