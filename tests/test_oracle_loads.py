"""Pins of the oracle's hydrodynamic loads (Section 3.3: MLS probes at the
triangle centroids, Taylor series back to the wall, traction, force and
torque) and of the boundary-cell pressure (Section 3.2, post-processing).

 - a linear pressure on a closed polyhedron: F = -V grad p exactly (the
   divergence theorem holds for linear integrands on flat faces), V the
   polyhedron's volume computed here from its faces;
 - a quadratic pressure: the second-order fit and Taylor series return the
   exact wall value at every centroid;
 - a linear shear over a plate: traction (dU/dy)/Re along the flow on the
   normal's side, zero net load with both sides;
 - the pressure of a boundary cell next to a flat plate is the value at
   the probe point: p + (h - |y - y_w|) dp/dn for a linear field.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2606_09799_gb300 import inputs


def centres(g):
    i = (np.arange(g.nx) + 0.5) * g.dx
    j = (np.arange(g.ny) + 0.5) * g.dy
    k = (np.arange(g.nz) + 0.5) * g.dz
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return X, Y, Z


def faces(g, c):
    off = [0.5, 0.5, 0.5]
    off[c] = 0.0
    n = [g.nx, g.ny + 1 if c == 1 else g.ny, g.nz]
    ax = [(np.arange(n[d]) + off[d]) * [g.dx, g.dy, g.dz][d] for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def polyhedron_volume(xyz, tri):
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    return np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0


def test_linear_pressure_on_closed_body_gives_minus_volume_times_gradient():
    g = orc.make_grid(40, 40, 40)
    xyz, tri = inputs.icosphere(2, 0.22, (0.5, 0.5, 0.5))
    X, Y, Z = centres(g)
    a = np.array([0.3, -1.2, 0.7])
    p = a[0] * X + a[1] * Y + a[2] * Z
    zero = [np.zeros(orc.field_shape(g, c)) for c in range(3)]
    isb = np.zeros(p.shape, dtype=np.uint8)
    tr, pw, F, M = orc.loads(g, xyz, tri, *zero, p, isb, re=100.0, sides=1)
    V = polyhedron_volume(xyz, tri)
    assert V > 0
    np.testing.assert_allclose(F, -V * a, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(F, tr[:, :3].sum(0), rtol=1e-13)
    # torque about a pole: -V (x_c - pole) x a, x_c the polyhedron's centroid
    # (divergence theorem on x_j p n_k with a linear p)
    A, B, C = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    vt = np.einsum("ij,ij->i", A, np.cross(B, C)) / 6.0
    xc = (vt[:, None] * (A + B + C) / 4.0).sum(0) / vt.sum()
    pole = np.array([0.1, 0.8, -0.3])
    _, _, F2, M2 = orc.loads(g, xyz, tri, *zero, p, isb, re=100.0, sides=1, pole=pole)
    np.testing.assert_allclose(F2, F, rtol=1e-13)
    np.testing.assert_allclose(M2, -V * np.cross(xc - pole, a), rtol=1e-8, atol=1e-12)


def test_quadratic_pressure_is_exact_at_the_wall():
    g = orc.make_grid(32, 32, 32)
    xyz, tri = inputs.icosphere(1, 0.2, (0.5, 0.5, 0.5))
    X, Y, Z = centres(g)
    quad = lambda x, y, z: 0.4 + 0.7 * x - 0.2 * y + 1.3 * z + 2.0 * x * x - 1.5 * y * z + 0.6 * z * z
    p = quad(X, Y, Z)
    zero = [np.zeros(orc.field_shape(g, c)) for c in range(3)]
    _, pw, _, _ = orc.loads(g, xyz, tri, *zero, p, np.zeros(p.shape, np.uint8), re=50.0)
    cen = xyz[tri].mean(axis=1)
    np.testing.assert_allclose(pw, quad(cen[:, 0], cen[:, 1], cen[:, 2]), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("sides", [1, 2])
def test_linear_shear_traction_over_a_plate(sides):
    g = orc.make_grid(32, 32, 32)
    xyz, tri = inputs.plate(8, 0.4, 0.3, 0.3, 0.51)      # normal +y for this orientation or -y
    e1, e2 = xyz[tri[0, 1]] - xyz[tri[0, 0]], xyz[tri[0, 2]] - xyz[tri[0, 0]]
    ny_sign = np.sign(np.cross(e1, e2)[1])
    gam, re = 0.8, 40.0
    X, Y, Z = faces(g, 0)
    u = gam * Y
    v, w = np.zeros(orc.field_shape(g, 1)), np.zeros(orc.field_shape(g, 2))
    p = np.zeros((g.nz, g.ny, g.nx))
    tr, pw, F, M = orc.loads(g, xyz, tri, u, v, w, p, np.zeros(p.shape, np.uint8), re=re, sides=sides)
    area = 0.4 * 0.4
    if sides == 1:
        np.testing.assert_allclose(F, [ny_sign * gam / re * area, 0.0, 0.0], atol=1e-12)
    else:
        np.testing.assert_allclose(F, 0.0, atol=1e-12)


def test_boundary_cell_pressure_from_its_probe_point():
    n = 24
    g = orc.make_grid(n, n, n)
    yw = 0.5 + 0.3 / n
    big = 1.25
    xyz = np.array([[-big, yw, -big], [1 + big, yw, -big], [-big, yw, 1 + big], [1 + big, yw, 1 + big]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    own, _ = orc.tag(g, xyz, tri)
    isb = orc.boundary_cells(g, own)
    assert isb.sum() > 0
    X, Y, Z = centres(g)
    ay = 1.7
    p = 0.3 + ay * Y
    q = orc.pressure_recon(g, p, isb, own, xyz, tri)
    h = 2.0 * np.sqrt(g.dx ** 2 + g.dy ** 2 + g.dz ** 2)
    side = np.sign(Y - yw)
    expect = p + (h - np.abs(Y - yw)) * ay * side
    B = isb == 1
    np.testing.assert_allclose(q[B], expect[B], rtol=1e-12)
    np.testing.assert_array_equal(q[~B], p[~B])
