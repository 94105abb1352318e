"""Pins of the oracle's discrete operators against the mathematics they
approximate: the discrete divergence theorem (Appendix A), L_c = D G with
Neumann walls (Eq. elliptic), the Poisson solve (discrete eigenfunctions,
dense brute force, manufactured solution), the explicit terms of Eq. NS_prov
(second-order convergence of each term to its analytic value) and the
tridiagonal sweeps of the approximate factorisation (dense solve)."""
import numpy as np
import pytest

from oracle import oracle as orc
from helpers import node_coords, sample, ddx, order

PI = np.pi


def test_discrete_divergence_theorem():
    """Appendix A: sum_c D u dV equals the net flux through the box faces
    for any field (periodic faces cancel, the y walls remain)."""
    g = orc.make_grid(10, 7, 9, 1.3, 0.8, 1.1)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(orc.field_shape(g, 0))
    v = rng.standard_normal(orc.field_shape(g, 1))
    w = rng.standard_normal(orc.field_shape(g, 2))
    d = orc.divergence(g, u, v, w)
    dV = g.dx * g.dy * g.dz
    flux = (v[:, -1, :].sum() - v[:, 0, :].sum()) * g.dx * g.dz
    np.testing.assert_allclose((d * dV).sum(), flux, rtol=0, atol=1e-12 * np.abs(d).sum() * dV)


def test_divergence_cellwise_definition_linear_field():
    """Eq. discrete_div is exact for fields linear along their own direction."""
    g = orc.make_grid(6, 5, 4, 1.0, 2.0, 1.0)
    u = sample(g, 0, lambda X, Y, Z: 0 * X + 0.7 * Y)          # no x-variation, periodic-safe
    v = sample(g, 1, lambda X, Y, Z: 0.3 * Y + 0 * X)
    w = sample(g, 2, lambda X, Y, Z: 0 * Z + X * 0)
    d = orc.divergence(g, u, v, w)
    np.testing.assert_allclose(d, 0.3, atol=1e-14)


def test_lap_c_equals_div_of_grad():
    """L_c = D G with homogeneous Neumann walls: compare with D applied to a
    face gradient built here (zero normal gradient on the wall faces)."""
    g = orc.make_grid(8, 6, 5, 1.0, 1.5, 0.7)
    phi = np.random.default_rng(4).standard_normal((g.nz, g.ny, g.nx))
    gu = (phi - np.roll(phi, 1, axis=2)) / g.dx
    gw = (phi - np.roll(phi, 1, axis=0)) / g.dz
    gv = np.zeros(orc.field_shape(g, 1))
    gv[:, 1:g.ny, :] = (phi[:, 1:, :] - phi[:, :-1, :]) / g.dy
    ref = orc.divergence(g, gu, gv, gw)
    np.testing.assert_allclose(orc.lap_c(g, phi), ref, atol=1e-11)


@pytest.mark.parametrize("modes", [(1, 0, 1), (0, 3, 0), (2, 1, 0), (3, 2, 2), (0, 0, 4)])
def test_poisson_discrete_eigenfunction(modes):
    """cos(2 pi m x/Lx) cos(2 pi n z/Lz) cos(pi l (j+1/2)/Ny) is an
    eigenvector of L_c; the solver must return it from rhs = -lambda phi."""
    m, l, n = modes
    g = orc.make_grid(16, 12, 8, 1.0, 1.0, 2.0)
    Z, Y, X = node_coords(g, 3)
    phi = np.cos(2 * PI * m * X / g.lx) * np.cos(2 * PI * n * Z / g.lz) * np.cos(PI * l * Y / g.ly)
    phi = np.ascontiguousarray(np.broadcast_to(phi, (g.nz, g.ny, g.nx)))
    lam = ((2 - 2 * np.cos(2 * PI * m / g.nx)) / g.dx ** 2 + (2 - 2 * np.cos(2 * PI * n / g.nz)) / g.dz ** 2
           + (2 - 2 * np.cos(PI * l / g.ny)) / g.dy ** 2)
    np.testing.assert_allclose(orc.lap_c(g, phi), -lam * phi, atol=1e-10 * lam)
    sol = orc.poisson(g, np.ascontiguousarray(-lam * phi))
    np.testing.assert_allclose(sol, phi, atol=1e-12)


def test_poisson_dense_brute_force():
    """Tiny grid: assemble L_c column by column, solve the singular system
    with the zero-mean constraint by least squares, compare."""
    g = orc.make_grid(4, 5, 6, 1.0, 0.9, 1.4)
    n = g.nx * g.ny * g.nz
    Am = np.zeros((n, n))
    for col in range(n):
        e = np.zeros(n)
        e[col] = 1.0
        Am[:, col] = orc.lap_c(g, e.reshape(g.nz, g.ny, g.nx)).ravel()
    rng = np.random.default_rng(9)
    r = rng.standard_normal(n)
    r -= r.mean()                                            # compatibility
    K = np.vstack([Am, np.ones((1, n))])
    ref = np.linalg.lstsq(K, np.concatenate([r, [0.0]]), rcond=None)[0]
    sol = orc.poisson(g, r.reshape(g.nz, g.ny, g.nx)).ravel()
    np.testing.assert_allclose(sol, ref, atol=1e-11)
    np.testing.assert_allclose(Am @ sol, r, atol=1e-10)


def test_poisson_manufactured_second_order():
    """phi = cos(2 pi x) cos(pi y) cos(2 pi z) (Neumann at y = 0, 1):
    solving with the continuous Laplacian as rhs converges as O(dx^2)."""
    errs = []
    for n in (16, 32):
        g = orc.make_grid(n, n, n)
        Z, Y, X = node_coords(g, 3)
        phi = np.broadcast_to(np.cos(2 * PI * X) * np.cos(PI * Y) * np.cos(2 * PI * Z), (n, n, n))
        rhs = np.ascontiguousarray(-9 * PI ** 2 * phi)
        sol = orc.poisson(g, rhs)
        errs.append(np.abs(sol - (phi - phi.mean())).max())
    assert abs(order(*errs) - 2.0) < 0.1


# --- explicit terms of Eq. NS_prov -------------------------------------------------
def _fields():
    # smooth, x/z periodic, every component vanishing on the walls (so the
    # tangential ghost u_{-1} = -u_0 is consistent)
    uf = lambda X, Y, Z: np.sin(2 * PI * X + 1.0) * np.sin(PI * Y) * np.cos(2 * PI * Z)
    vf = lambda X, Y, Z: np.sin(PI * Y) * np.cos(2 * PI * X) * np.sin(2 * PI * Z + 0.5)
    wf = lambda X, Y, Z: np.cos(2 * PI * X) * np.sin(PI * Y) * (1.0 + 0.3 * np.sin(2 * PI * Z))
    pf = lambda X, Y, Z: np.cos(2 * PI * X + 0.2) * np.cos(1.3 * Y) * np.sin(2 * PI * Z)
    return uf, vf, wf, pf


def _analytic_H():
    uf, vf, wf, _ = _fields()
    fl = [uf, vf, wf]
    out = []
    for c in range(3):
        terms = [(lambda X, Y, Z, a=a, c=c: fl[a](X, Y, Z) * fl[c](X, Y, Z)) for a in range(3)]
        d = [ddx(terms[a], a) for a in range(3)]
        out.append(lambda X, Y, Z, d=d: -(d[0](X, Y, Z) + d[1](X, Y, Z) + d[2](X, Y, Z)))
    return out


def _analytic_L():
    uf, vf, wf, _ = _fields()
    out = []
    for f in (uf, vf, wf):
        d2 = [ddx(ddx(f, a, 1e-4), a, 1e-4) for a in range(3)]
        out.append(lambda X, Y, Z, d2=d2: d2[0](X, Y, Z) + d2[1](X, Y, Z) + d2[2](X, Y, Z))
    return out


def _interior(g, c, a):
    return a[:, 1:-1, :] if c == 1 else a


@pytest.mark.parametrize("term", ["H", "L", "G", "f"])
def test_explicit_terms_converge(term):
    """Each term of R (conservative advection H, viscous L, pressure gradient
    G, body force) against its analytic value: second order (a transposed
    operand, a wrong index or a sign error breaks the limit)."""
    uf, vf, wf, pf = _fields()
    Hx, Lx = _analytic_H(), _analytic_L()
    errs = [[], [], []]
    for n in (16, 32):
        g = orc.make_grid(n, n, n, 1.0, 1.0, 1.0)
        u, v, w, p = sample(g, 0, uf), sample(g, 1, vf), sample(g, 2, wf), sample(g, 3, pf)
        own = orc.no_tags(g)
        zero = [np.zeros(orc.field_shape(g, c)) for c in range(3)]
        if term == "H":
            R, H = orc.rhs(g, u, v, w, np.zeros_like(p), own, 1.0, 0.0, 0.0, 1.0, 1.0)
            ref = [sample(g, c, Hx[c]) for c in range(3)]
            np.testing.assert_allclose(R[0], H[0], atol=1e-15)
        elif term == "L":
            R, _ = orc.rhs(g, u, v, w, np.zeros_like(p), own, 0.0, 0.0, 1.0, 1.0, 1.0)
            ref = [sample(g, c, Lx[c]) for c in range(3)]
        elif term == "G":
            R, _ = orc.rhs(g, *zero, p, own, 0.0, 0.0, 1.0, 1.0, 1.0)
            ref = [-sample(g, c, ddx(pf, c)) for c in range(3)]
        else:
            R, _ = orc.rhs(g, *zero, np.zeros_like(p), own, 0.0, 0.0, 0.5, 2.0, 1.0, fb=(0.3, -0.2, 0.7))
            for c, fc in enumerate((0.3, -0.2, 0.7)):
                r = _interior(g, c, R[c])
                np.testing.assert_allclose(r, 0.5 * 2.0 * fc, atol=1e-15)
            return
        for c in range(3):
            errs[c].append(np.abs(_interior(g, c, R[c] - ref[c])).max())
    for c in range(3):
        assert errs[c][1] < 0.05 * max(1.0, np.abs(ref[c]).max()), (term, c, errs[c])
        assert order(*errs[c]) > 1.8, (term, c, errs[c])


def test_rhs_zero_on_forcing_nodes_and_h_prev_weight():
    g = orc.make_grid(8, 8, 8)
    rng = np.random.default_rng(1)
    u, v, w, p = (rng.standard_normal(orc.field_shape(g, c)) for c in (0, 1, 2, 0))
    v[:, 0] = v[:, -1] = 0
    own = orc.no_tags(g)
    own[1][2, 3, 4] = 7
    own[0][1, 1, 1] = 0
    Hp = [rng.standard_normal(orc.field_shape(g, c)) for c in range(3)]
    R0, H0 = orc.rhs(g, u, v, w, p, own, 1.5, 0.0, 1.0, 0.1, 50.0)
    R1, H1 = orc.rhs(g, u, v, w, p, own, 1.5, -0.5, 1.0, 0.1, 50.0, Hprev=Hp)
    assert R1[1][2, 3, 4] == 0.0 and R1[0][1, 1, 1] == 0.0
    m = own[0] < 0
    np.testing.assert_allclose((R1[0] - R0[0])[m], 0.1 * -0.5 * Hp[0][m], atol=1e-14)
    np.testing.assert_allclose(H0[0], H1[0])


def test_shear_flow_has_no_advection():
    """u = u(y), v = w = 0: the conservative term vanishes identically."""
    g = orc.make_grid(8, 12, 6)
    u = sample(g, 0, lambda X, Y, Z: np.sin(PI * Y) + 0 * X)
    z = [np.zeros(orc.field_shape(g, c)) for c in range(3)]
    R, H = orc.rhs(g, u, z[1], z[2], np.zeros((6, 12, 8)), orc.no_tags(g), 1.0, 0.0, 0.0, 1.0, 1.0)
    for c in range(3):
        assert np.abs(H[c]).max() == 0.0


# --- tridiagonal sweeps ------------------------------------------------------------
def _second_diff_periodic(n, d):
    M = -2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    M[0, -1] = M[-1, 0] = 1
    return M / d ** 2


@pytest.mark.parametrize("c,direction", [(0, 0), (1, 0), (2, 2), (0, 2), (0, 1), (1, 1), (2, 1)])
@pytest.mark.parametrize("ybc", [0, 1])
def test_sweep_matches_dense_solve(c, direction, ybc):
    """(1 - beta L_dir) x = r with identity rows at forcing nodes, solved by a
    dense LU of the operator assembled here."""
    g = orc.make_grid(9, 7, 6, 1.0, 0.8, 1.1, ybc=ybc)
    beta = 0.37 * g.dx ** 2
    rng = np.random.default_rng(c * 10 + direction)
    shape = orc.field_shape(g, c)
    r = rng.standard_normal(shape)
    own = np.full(shape, -1, dtype=np.int32)
    own[rng.random(shape) < 0.15] = 3
    if c == 1:
        r[:, 0] = r[:, -1] = 0
    f = r.copy()
    orc.sweep(g, c, direction, f, own, beta)
    nx, nz = g.nx, g.nz
    if direction in (0, 2):
        n = nx if direction == 0 else nz
        d = g.dx if direction == 0 else g.dz
        Lm = _second_diff_periodic(n, d)
        jr = range(1, g.ny) if c == 1 else range(g.ny)
        for j in jr:
            for o in range(nz if direction == 0 else nx):
                sl = (o, j, slice(None)) if direction == 0 else (slice(None), j, o)
                M = np.eye(n) - beta * Lm
                fr = own[sl] >= 0
                M[fr] = 0
                M[fr, fr] = 1
                np.testing.assert_allclose(f[sl], np.linalg.solve(M, r[sl]), atol=1e-12)
    else:
        if c == 1:
            n = g.ny - 1
            Lm = (-2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)) / g.dy ** 2
            js = slice(1, g.ny)
        else:
            n = g.ny
            gs = -1.0 if ybc == 0 else 1.0
            Lm = (-2 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))
            Lm[0, 0] += gs
            Lm[-1, -1] += gs
            Lm /= g.dy ** 2
            js = slice(0, g.ny)
        for k in range(nz):
            for i in range(nx):
                M = np.eye(n) - beta * Lm
                fr = own[k, js, i] >= 0
                M[fr] = 0
                M[fr, fr] = 1
                np.testing.assert_allclose(f[k, js, i], np.linalg.solve(M, r[k, js, i]), atol=1e-12)
