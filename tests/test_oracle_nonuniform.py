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


def test_surfaces_are_refused_on_a_stretched_grid():
    sim = OracleSim(8, 8, 8, yfaces=inputs.stretched_faces(8))
    xyz, tri = inputs.icosphere(1, 0.2, (0.5, 0.5, 0.5))
    with pytest.raises(ValueError):
        sim.set_surface(xyz, np.zeros_like(xyz), tri)
