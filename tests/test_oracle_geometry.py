"""Pins of the oracle's geometry: closest point on a triangle (Algorithm 1,
which cites Ericson 2004) and the tagging of Algorithm 1.

Pinned against brute force (dense sampling of the triangle, all nodes x all
triangles) and against the flat-plane closed form that follows from
Algorithm 1: a plane y = y_w tags exactly the nodes with 0 < |y - y_w| < dy.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2606_09799_gb300 import inputs

A = np.array([0.0, 0.0, 0.0])
B = np.array([1.0, 0.0, 0.0])
C = np.array([0.0, 1.0, 0.0])


@pytest.mark.parametrize("p,expect", [
    ((-1.0, -1.0, 0.3), (0.0, 0.0, 0.0)),      # vertex a region
    ((2.0, -0.5, -0.2), (1.0, 0.0, 0.0)),      # vertex b region
    ((-0.5, 2.0, 0.1), (0.0, 1.0, 0.0)),       # vertex c region
    ((0.5, -1.0, 0.7), (0.5, 0.0, 0.0)),       # edge ab
    ((-1.0, 0.25, 0.0), (0.0, 0.25, 0.0)),     # edge ac
    ((1.0, 1.0, 0.5), (0.5, 0.5, 0.0)),        # edge bc
    ((0.2, 0.3, 0.7), (0.2, 0.3, 0.0)),        # face
    ((0.2, 0.3, -0.7), (0.2, 0.3, 0.0)),       # face, other side
])
def test_closest_point_regions(p, expect):
    X, w = orc.closest_point(p, A, B, C)
    np.testing.assert_allclose(X, expect, atol=1e-15)
    np.testing.assert_allclose(w.sum(), 1.0, atol=1e-15)
    assert (w >= -1e-15).all()
    np.testing.assert_allclose(w[0] * A + w[1] * B + w[2] * C, X, atol=1e-15)


def test_closest_point_vs_dense_sampling():
    rng = np.random.default_rng(11)
    m = 400
    s = np.linspace(0.0, 1.0, m + 1)
    S, T = np.meshgrid(s, s)
    keep = (S + T) <= 1.0
    S, T = S[keep], T[keep]
    for _ in range(60):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        X, w = orc.closest_point(p, a, b, c)
        pts = a[None] + S[:, None] * (b - a)[None] + T[:, None] * (c - a)[None]
        dmin = np.sqrt(((pts - p) ** 2).sum(1)).min()
        d = np.linalg.norm(p - X)
        assert d <= dmin + 1e-12
        assert d >= dmin - 3.0 * np.linalg.norm(b - a + c - a) / m   # sampling resolution
        np.testing.assert_allclose(w[0] * a + w[1] * b + w[2] * c, X, atol=1e-13)
        # the residual is orthogonal to the triangle where X is interior to the face
        if (w > 1e-9).all():
            n = np.cross(b - a, c - a)
            r = p - X
            assert abs(np.dot(r, b - a)) < 1e-12 * (1 + np.linalg.norm(r))
            assert abs(np.dot(r, c - a)) < 1e-12 * (1 + np.linalg.norm(r))
            assert np.linalg.norm(np.cross(r, n)) < 1e-11 * (1 + np.linalg.norm(r) * np.linalg.norm(n))


def _tag_both(g, xyz, tri):
    o1, d1 = orc.tag(g, xyz, tri)
    o2, d2 = orc.tag(g, xyz, tri, brute=True)
    for c in range(3):
        np.testing.assert_array_equal(o1[c], o2[c])
    return o1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tagging_matches_brute_force_random(seed):
    g = orc.make_grid(12, 10, 14, 1.0, 1.0, 1.2)
    xyz, tri = inputs.random_triangles(25, seed, lo=0.25, hi=0.75, size=0.25)
    own = _tag_both(g, xyz, tri)
    assert sum(int((o >= 0).sum()) for o in own) > 50


def test_tagging_matches_brute_force_icosphere_and_plate():
    g = orc.make_grid(16, 16, 16)
    xyz, tri = inputs.icosphere(2, 0.2, (0.47, 0.52, 0.49))
    own = _tag_both(g, xyz, tri)
    assert min(int((o >= 0).sum()) for o in own) > 100
    xyz, tri = inputs.plate(8, 0.5, 0.23, 0.27, 0.51)
    _tag_both(g, xyz, tri)


def test_tagging_periodic_wrap_matches_brute_force():
    # a body straddling the periodic x and z boundaries
    g = orc.make_grid(12, 12, 12)
    xyz, tri = inputs.icosphere(1, 0.18, (0.02, 0.5, 0.97))
    own = _tag_both(g, xyz, tri)
    # tagged nodes appear on both ends of the periodic directions
    o = own[0] >= 0
    assert o[:, :, 0].any() and o[:, :, -1].any() and o[0].any() and o[-1].any()


@pytest.mark.parametrize("yw", [0.4137, 0.5 + 1e-3, 0.3711])
def test_tagging_flat_plane_closed_form(yw):
    """A plane y = yw spanning the periodic box: Algorithm 1 tags exactly the
    nodes at signed distance 0 < |y - yw| < dy (one neighbour lies across)."""
    nx, ny, nz = 8, 16, 6
    g = orc.make_grid(nx, ny, nz, 1.0, 1.0, 0.75)
    big = 0.3
    xyz = np.array([[-big, yw, -big], [1 + big, yw, -big], [-big, yw, 0.75 + big], [1 + big, yw, 0.75 + big]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    own, _ = orc.tag(g, xyz, tri)
    for c in range(3):
        nyc = ny + 1 if c == 1 else ny
        y = (np.arange(nyc) + (0.0 if c == 1 else 0.5)) * g.dy
        d = np.abs(y - yw)
        expect = (d > 0) & (d < g.dy)
        if c == 1:
            expect[0] = expect[-1] = False
        got = own[c] >= 0
        np.testing.assert_array_equal(got, np.broadcast_to(expect[None, :, None], got.shape))
        assert expect.sum() == 2


def test_tagging_order_invariance():
    """Permuting the triangle list maps owners through the permutation
    (the owner is the argmin of |N|^2, ties to the smallest index)."""
    g = orc.make_grid(16, 16, 16)
    xyz, tri = inputs.icosphere(2, 0.21, (0.5, 0.48, 0.51))
    own, d2 = orc.tag(g, xyz, tri)
    perm = np.random.default_rng(5).permutation(tri.shape[0])
    own_p, d2_p = orc.tag(g, xyz, tri[perm])
    for c in range(3):
        m = own[c] >= 0
        np.testing.assert_array_equal(m, own_p[c] >= 0)
        np.testing.assert_array_equal(d2[c][m], d2_p[c][m])
        # where the minimum is unique the owner maps through the permutation
        mapped = perm[own_p[c][m]]
        same = mapped == own[c][m]
        assert same.mean() > 0.9


def test_tagged_nodes_lie_near_the_surface_on_both_sides():
    g = orc.make_grid(24, 24, 24)
    r, cen = 0.22, np.array([0.5, 0.5, 0.5])
    xyz, tri = inputs.icosphere(3, r, cen)
    own, d2 = orc.tag(g, xyz, tri)
    diag = np.sqrt(3) * g.dx
    from helpers import node_coords
    for c in range(3):
        Z, Y, X = node_coords(g, c)
        rad = np.sqrt((X - cen[0]) ** 2 + (Y - cen[1]) ** 2 + (Z - cen[2]) ** 2)
        rad = np.broadcast_to(rad, own[c].shape)
        m = own[c] >= 0
        assert (np.sqrt(d2[c][m]) <= diag + 1e-15).all()
        assert (np.abs(rad[m] - r) < diag + 0.01).all()   # faceted sphere
        assert (rad[m] < r).sum() > 50 and (rad[m] > r).sum() > 50


@pytest.mark.parametrize("i0,ni", [(0, 12), (3, 5), (10, 2)])
def test_windowed_tagging_equals_slice_of_whole_grid(i0, ni):
    """The x-window variant of Algorithm 1 (for grids too large to tag whole)
    gives exactly the whole-grid owners of its slab, across the periodic
    boundary too (the body straddles x = 0)."""
    g = orc.make_grid(12, 10, 14, 1.0, 1.0, 1.2)
    xyz, tri = inputs.icosphere(1, 0.2, (0.05, 0.5, 0.6))
    xyz2, tri2 = inputs.random_triangles(15, 4, lo=0.3, hi=0.7, size=0.25)
    xyz = np.concatenate([xyz, xyz2])
    tri = np.concatenate([tri, tri2 + len(inputs.icosphere(1, 0.2)[0])]).astype(np.int32)
    whole, _ = orc.tag(g, xyz, tri)
    win = orc.tag_window(g, xyz, tri, i0, ni)
    for c in range(3):
        np.testing.assert_array_equal(win[c], whole[c][:, :, i0:i0 + ni])
    assert sum(int((w >= 0).sum()) for w in win) > 0


def test_large_workload_meshes_are_closed_and_clear_of_the_walls():
    """Generators of the multi-body channel and the leaflet tube: triangle
    counts, vertex indices in range, every body at least h + 2 dy from the
    walls over the first steps."""
    for wl, ntri in ((inputs.multibody_channel(steps=3), 124928), (inputs.leaflet_tube(steps=3), 182800)):
        assert wl.tri.shape == (ntri, 3)
        xyz, vel = wl.surface(0)
        assert wl.tri.min() >= 0 and wl.tri.max() < len(xyz)
        dl = np.array([wl.lx / wl.nx, wl.ly / wl.ny, wl.lz / wl.nz])
        h = 2 * np.sqrt((dl ** 2).sum())
        for s in range(3):
            xyz, _ = wl.surface(s)
            assert xyz[:, 1].min() > h + 2 * dl[1] and xyz[:, 1].max() < wl.ly - h - 2 * dl[1]
    # the closed bodies: every edge of a capped cylinder and a cube shared by two triangles
    for xyz, tri in (inputs.capped_cylinder(16, 6, 0.1, 0.4, (0.5, 0.5, 0.5), (1.0, 0.0, 0.2)),):
        e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
        _, counts = np.unique(e, axis=0, return_counts=True)
        assert (counts == 2).all()
