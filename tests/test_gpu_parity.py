"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tags must match bit for bit (they are integer decisions made in FP64 by
the same formulas); velocities and pressure after N steps must agree to
max |delta| <= 1e-10 (velocity scaled by U_ref = 1, pressure by U_ref^2).
Sizes span several tiles and ragged tails (radix-3 FFT sizes, odd ny).
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim, make_grid, tag as oracle_tag
from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def gpu_sim(wl_or_dims, **kw):
    return ibm.Simulation(*wl_or_dims, **kw)


def pair(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, **kw):
    o = OracleSim(nx, ny, nz, lx, ly, lz, **{k: v for k, v in kw.items() if k != "precision"})
    g = ibm.Simulation(nx, ny, nz, lx, ly, lz, **kw)
    return o, g


def assert_fields_close(o, g, tol=TOL, what=""):
    gu, gv, gw, gp = g.fields()
    for name, a, b in (("u", o.u, gu), ("v", o.v, gv), ("w", o.w, gw), ("p", o.p, gp)):
        err = np.abs(a - b).max()
        assert err <= tol, f"{what} {name}: max |delta| = {err:.3e}"


def assert_tags_equal(o_owners, g):
    gt = g.tags()
    for c in range(3):
        np.testing.assert_array_equal(gt[c], o_owners[c], err_msg=f"component {c}")


def run_workload(wl, nsteps, precision="fp64", use_q=True):
    o, g = pair(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, use_q=use_q, precision=precision)
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        fx, fy, fz = wl.body_force_at(s * wl.dt)
        o.set_body_force(fx, fy, fz)
        g.set_body_force(fx, fy, fz)
        o.step()
        g.step()
    return o, g


# ---------------------------------------------------------------------------
# tags
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_tags_bit_exact_random_triangles_ragged_grid(seed):
    nx, ny, nz = 24, 19, 36
    xyz, tri = inputs.random_triangles(60, seed, lo=0.38, hi=0.62, size=0.15)
    o, g = pair(nx, ny, nz, 1.0, 1.0, 1.5)
    g.set_surface(xyz, np.zeros_like(xyz), tri)
    g.step()
    own, _ = oracle_tag(o.g, xyz, tri)
    assert_tags_equal(own, g)
    d = g.diag()
    assert d["nforce"] == [int((own[c] >= 0).sum()) for c in range(3)]


def test_tags_bit_exact_periodic_wrap():
    nx, ny, nz = 32, 32, 32
    xyz, tri = inputs.icosphere(2, 0.2, (0.03, 0.5, 0.96))
    o, g = pair(nx, ny, nz)
    g.set_surface(xyz, np.zeros_like(xyz), tri)
    g.step()
    own, _ = oracle_tag(o.g, xyz, tri)
    assert_tags_equal(own, g)


@pytest.mark.parametrize("step", [0, 3, 7])
def test_tags_bit_exact_sphere64(step):
    wl = inputs.oscillating_sphere()
    o, g = pair(wl.nx, wl.ny, wl.nz)
    xyz, vel = wl.surface(step)
    g.set_surface(xyz, vel, wl.tri)
    g.step()
    own, _ = oracle_tag(o.g, xyz, wl.tri)
    assert_tags_equal(own, g)


@pytest.mark.parametrize("step", [0, 13, 61])
def test_tags_bit_exact_plate128_full_size(step):
    """The plate of the 128^3 benchmark workload, nodes exactly on the
    surface included (y = 0.5 is a v-lattice plane at step 0)."""
    wl = inputs.heaving_plate()
    o, g = pair(wl.nx, wl.ny, wl.nz)
    xyz, vel = wl.surface(step)
    g.set_surface(xyz, vel, wl.tri)
    g.step()
    own, _ = oracle_tag(o.g, xyz, wl.tri)
    assert_tags_equal(own, g)
    d = g.diag()
    assert d["nboundary"] >= 0 and sum(d["nforce"]) > 10000


# ---------------------------------------------------------------------------
# FP64 fields
# ---------------------------------------------------------------------------
def test_fp64_sphere64_ten_steps():
    """64^3 oscillating sphere, Re = 100, dt = 1e-3, 10 steps."""
    wl = inputs.oscillating_sphere()
    o, g = run_workload(wl, 10)
    assert_fields_close(o, g)
    assert_tags_equal(o.owners, g)
    d = g.diag()
    assert abs(d["slip_l1"] - o.last["slip"]) <= 1e-9 * max(1.0, o.last["slip"])
    assert abs(d["q_f"] - o.last["qF"]) <= 1e-12
    assert abs(d["sum_q_dv"]) < 1e-14
    assert d["steps"] == 10


def test_fp64_plate128_ten_steps():
    wl = inputs.heaving_plate()
    o, g = run_workload(wl, 10)
    assert_fields_close(o, g)
    d = g.diag()
    assert abs(d["slip_l1"] - o.last["slip"]) <= 1e-9 * max(1.0, o.last["slip"])


def test_fp64_ragged_sizes_radix3_and_odd_ny():
    wl = inputs.oscillating_sphere(n=48, steps=4, subdiv=2)
    o, g = pair(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3)
    for s in range(4):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    assert_fields_close(o, g)
    assert_tags_equal(o.owners, g)


@pytest.mark.parametrize("use_q", [True, False])
@pytest.mark.parametrize("scheme", ["rk2", "ab"])
def test_fp64_schemes_and_q_switch(use_q, scheme):
    wl = inputs.oscillating_sphere(n=32, steps=4, subdiv=2)
    o, g = pair(32, 32, 32, re=100.0, dt=2e-3, use_q=use_q, scheme=scheme)
    for s in range(4):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    assert_fields_close(o, g)


def test_fp64_no_body_taylor_green_free_slip():
    o, g = pair(32, 24, 4, 1.0, 1.0, 0.125, re=20.0, dt=4e-3, ybc=1)
    from helpers import sample
    PI = np.pi
    u = sample(o.g, 0, lambda X, Y, Z: np.sin(2 * PI * X) * np.cos(PI * Y))
    v = sample(o.g, 1, lambda X, Y, Z: -2 * np.cos(2 * PI * X) * np.sin(PI * Y))
    w = np.zeros_like(u)
    p = np.zeros_like(u)
    o.set_fields(u, v, w, p)
    g.set_fields(u, v, w, p)
    o.step(6)
    g.step(6)
    assert_fields_close(o, g)


def test_fp64_random_initial_field_with_body_force():
    """Random velocity and pressure (v = 0 on the walls) exercise every
    term of the explicit operator and the projection at once."""
    nx, ny, nz = 24, 20, 48
    u, v, w, p = inputs.random_fields(nx, ny, nz, seed=7, amp=0.3)
    o, g = pair(nx, ny, nz, 1.0, 1.0, 2.0, re=50.0, dt=1e-3)
    for s in (o, g):
        s.set_fields(u, v, w, p)
        s.set_body_force(0.3, -0.1, 0.2)
    xyz, tri = inputs.icosphere(2, 0.2, (0.5, 0.5, 1.0))
    vel = np.tile([0.1, -0.05, 0.2], (xyz.shape[0], 1))
    for s in (o, g):
        s.set_surface(xyz, vel, tri)
    o.step(3)
    g.step(3)
    assert_fields_close(o, g)


# ---------------------------------------------------------------------------
# API behaviour and edge cases
# ---------------------------------------------------------------------------
def test_set_get_fields_roundtrip_and_empty_surface():
    nx, ny, nz = 16, 12, 8
    u, v, w, p = inputs.random_fields(nx, ny, nz, seed=3)
    g = ibm.Simulation(nx, ny, nz)
    g.set_fields(u, v, w, p)
    gu, gv, gw, gp = g.fields()
    for a, b in ((u, gu), (v, gv), (w, gw), (p, gp)):
        np.testing.assert_array_equal(a, b)
    # no surface: a plain fractional step, no forcing nodes
    g.step(2)
    d = g.diag()
    assert d["nforce"] == [0, 0, 0] and d["nboundary"] == 0
    for t in g.tags():
        assert (t == -1).all()


def test_surface_removed_and_restored():
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    o, g = pair(32, 32, 32, re=100.0, dt=2e-3)
    xyz, vel = wl.surface(0)
    for s in (o, g):
        s.set_surface(xyz, vel, wl.tri)
    o.step()
    g.step()
    empty = np.zeros((0, 3))
    o.set_surface(empty, empty, np.zeros((0, 3), dtype=np.int32))
    ibm.ibm_set_surface(g.h, empty, empty, np.zeros((0, 3), dtype=np.int32))
    o.step()
    g.step()
    for s in (o, g):
        s.set_surface(xyz, vel, wl.tri)
    o.step()
    g.step()
    assert_fields_close(o, g)
    assert_tags_equal(o.owners, g)


def test_multi_step_replay_equals_single_steps_and_is_deterministic():
    wl = inputs.oscillating_sphere(n=32, steps=4, subdiv=2)
    xyz, vel = wl.surface(0)
    outs = []
    for mode in ("one", "many", "one"):
        g = ibm.Simulation(32, 32, 32, re=100.0, dt=2e-3)
        g.set_surface(xyz, vel, wl.tri)
        if mode == "one":
            for _ in range(4):
                g.step(1)
        else:
            g.step(4)
        outs.append(g.fields())
        g.close()
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(outs[0], outs[2]):
        np.testing.assert_array_equal(a, b)


def test_bad_surface_indices_rejected():
    g = ibm.Simulation(16, 16, 16)
    xyz = np.random.default_rng(0).uniform(0.3, 0.7, (4, 3))
    tri = np.array([[0, 1, 5]], dtype=np.int32)
    with pytest.raises(ibm.IbmError) as e:
        g.set_surface(xyz, np.zeros_like(xyz), tri)
    assert e.value.status == 1


def test_probe_leaving_domain_reports_geometry_error():
    """A body touching the wall: its probes would leave the stored planes;
    the kernel records it and the next synchronising call reports it."""
    g = ibm.Simulation(16, 16, 16)
    xyz, tri = inputs.icosphere(1, 0.15, (0.5, 0.1, 0.5))
    g.set_surface(xyz, np.zeros_like(xyz), tri)
    g.step()
    with pytest.raises(ibm.IbmError) as e:
        g.sync()
    assert e.value.status == 4
    g.sync()          # the error word is cleared once reported


def test_candidate_capacity_grows_for_large_triangles():
    g = ibm.Simulation(64, 32, 64)
    big = 0.3
    yw = 0.4137
    xyz = np.array([[-big, yw, -big], [1 + big, yw, -big], [-big, yw, 1 + big], [1 + big, yw, 1 + big]])
    tri = np.array([[0, 1, 3], [0, 3, 2]], dtype=np.int32)
    g.set_surface(xyz, np.zeros_like(xyz), tri)
    g.step()
    g.sync()
    d = g.diag()
    assert d["nforce"][0] == 2 * 64 * 64


@pytest.mark.parametrize("tune", [dict(tri_y=1, fft_plane=2), dict(tri_y=2, sweep_w=16, fft_plane=1),
                                  dict(tri_y=3, fft_lpb=2, fft_cols=2, fft_plane=1),
                                  dict(tri_y=3, sweep_zy=1, sweep_w=64, fft_lpb=8, fft_cols=16, fft_plane=2),
                                  dict(tri_y=1, sweep_zy=2, sweep_y=1, fft_plane=2),
                                  dict(tri_y=1, sweep_y=2, fft_plane=2),
                                  dict(tri_y=1, sweep_y=3, fft_plane=2),
                                  dict(tri_y=2, sweep_y=3, fft_plane=2),
                                  dict(tri_y=1, sweep_y=4, fft_plane=2),
                                  dict(tri_y=3, sweep_y=4, fft_plane=1),
                                  dict(tri_y=4, sweep_y=4, fft_plane=3),
                                  dict(tri_y=0, fft_plane=0, rhs=2, corr_check=2),
                                  dict(tri_y=0, fft_plane=0)])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_every_launch_shape_matches_oracle(tune, precision, tol):
    """Every choice the autotuner can make (Thomas variant, sweep form and
    width, streamed y sweep, bulk-copy y tiles, tabulated y rows, FFT
    tiling) computes the same step: against the oracle on a ragged grid with
    a moving sphere, 4 steps."""
    wl = inputs.oscillating_sphere(n=48, steps=4, subdiv=2)
    o = OracleSim(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3)
    g = ibm.Simulation(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision=precision)
    ibm.ibm_set_tune(g.h, **tune)
    for s in range(4):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    gu, gv, gw, gp = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= tol, err
    for c, own in enumerate(g.tags()):
        np.testing.assert_array_equal(own, o.owners[c])


@pytest.mark.parametrize("stretched", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiled_rhs_equals_the_per_cell_rhs(precision, stretched):
    """The right-hand side from z-marching tiles with shared-memory halos
    (rhs 2) and the one with two cells per thread and paired row loads
    (rhs 3, the built-in choice of the FP32 path) take every neighbour the
    per-cell kernel (rhs 1) reads from global memory and do the same
    arithmetic: fields
    equal to rounding after 3 steps with a moving sphere, on the uniform and
    on a stretched wall-normal grid, AB+CN (the previous sub-stage's H too).
    48 x 37 x 40: ragged tiles in i (48 = 32 + 16), j (37 = 9 x 4 + 1) and k
    (40 = 2 x 16 + 8), and the periodic wrap of the halo in x and z."""
    wl = inputs.oscillating_sphere(n=48, steps=3, subdiv=2)
    yf = inputs.stretched_faces(37, ly=0.9) if stretched else None
    sims = []
    for rhs in (1, 2, 3):   # 3: two cells per thread (FP32 path only; the FP64 path falls back to 1)
        g = ibm.Simulation(48, 37, 40, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, scheme="ab", precision=precision,
                           y_faces=yf)
        ibm.ibm_set_tune(g.h, rhs=rhs)
        sims.append(g)
    for s in range(3):
        xyz, vel = wl.surface(s)
        for g in sims:
            g.set_surface(xyz, vel, wl.tri)
            g.step()
    tol = 1e-14 if precision == "fp64" else 1e-6
    for other in sims[1:]:
        for a, b in zip(sims[0].fields(), other.fields()):
            assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max())
        for a, b in zip(sims[0].history(), other.history()):
            assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max())



@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cluster_plane_transforms_and_capped_thomas_equal_the_plain_forms(precision):
    """The per-plane transforms split over a cluster of 4 blocks (fft_plane 3)
    and the register-capped warp Thomas (tri_y 4) do the arithmetic of the
    one-block plane transform (fft_plane 2) and the uncapped Thomas (tri_y 1)
    element by element, only on other threads: the fields agree to rounding
    after 3 steps with a moving sphere (48 x 37 x 96: 25 kx columns split
    7/7/7/4 over the cluster; 24 rows per block)."""
    wl = inputs.oscillating_sphere(n=48, steps=3, subdiv=2)
    sims = []
    for tune in (dict(tri_y=1, fft_plane=2), dict(tri_y=4, fft_plane=3)):
        g = ibm.Simulation(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision=precision)
        ibm.ibm_set_tune(g.h, sweep_y=4, **tune)
        sims.append(g)
    for s in range(3):
        xyz, vel = wl.surface(s)
        for g in sims:
            g.set_surface(xyz, vel, wl.tri)
            g.step()
    tol = 1e-14 if precision == "fp64" else 1e-6
    for a, b in zip(sims[0].fields(), sims[1].fields()):
        assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max())
    for a, b in zip(sims[0].tags(), sims[1].tags()):
        np.testing.assert_array_equal(a, b)


def test_cluster_plane_transforms_in_chunks_match_the_plane_form():
    """A 256 x 12 x 256 mixed grid: the cluster's rows (64 per block) and
    columns (33) no longer fit its 100 KB of shared memory at once, so both
    directions go in chunks (8 lines, 7 columns).  A random divergent start,
    no body, 2 steps: fields equal to rounding to the one-block plane form."""
    rng = np.random.default_rng(7)
    nx, ny, nz = 256, 12, 256
    u0 = rng.standard_normal((nz, ny, nx))
    v0 = rng.standard_normal((nz, ny + 1, nx))
    v0[:, 0, :] = 0.0
    v0[:, ny, :] = 0.0
    w0 = rng.standard_normal((nz, ny, nx))
    out = []
    for fp in (2, 3):
        g = ibm.Simulation(nx, ny, nz, 1.0, 0.05, 1.0, re=100.0, dt=1e-5, precision="mixed")
        ibm.ibm_set_tune(g.h, fft_plane=fp)
        g.set_fields(u0, v0, w0, np.zeros((nz, ny, nx)))
        g.step(2)
        out.append(g.fields())
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-6 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tile_z_sweep_equals_streamed_to_rounding(precision):
    """The z sweep from shared-memory tiles (sweep_y = 4) runs the streamed
    z sweep's recurrences in the same order (the compiler may fuse a
    multiply-add differently): fields equal to rounding after 3 steps (FP32
    rounding of the state in the mixed path) with a moving sphere (lines
    with and without forcing rows, a partial tile of 16 lines at nx = 48;
    nz = 96, so the lines' rows move in the register batches of 8)."""
    wl = inputs.oscillating_sphere(n=48, steps=3, subdiv=2)
    for ny in (37, 48):
        sims = []
        for sy in (3, 4):
            g = ibm.Simulation(48, ny, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision=precision)
            ibm.ibm_set_tune(g.h, tri_y=1, sweep_y=sy, fft_plane=2)
            sims.append(g)
        for s in range(3):
            xyz, vel = wl.surface(s)
            for g in sims:
                g.set_surface(xyz, vel, wl.tri)
                g.step()
        # FP64: rounding of the state; mixed: once one FP32 rounding differs,
        # the FP32 arithmetic from the hi parts carries an FP32 rounding of the
        # state
        tol = 1e-14 if precision == "fp64" else 1e-6
        ref = sims[0].fields()
        for g in sims[1:]:
            for a, b in zip(ref, g.fields()):
                assert np.abs(a - b).max() <= tol * max(1.0, np.abs(a).max()), ny


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_bulk_copy_y_tiles_with_128_rows_match_oracle(precision, tol):
    """The bulk-copy y tiles where they need more than the default 48 KB of
    shared memory (128 rows; 3 tiles of 32 lines with the low parts in the
    mixed path), with a moving sphere and a random initial field."""
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    init = inputs.random_fields(32, 128, 32, seed=17, amp=0.1)
    o = OracleSim(32, 128, 32, re=150.0, dt=1e-3)
    g = ibm.Simulation(32, 128, 32, re=150.0, dt=1e-3, precision=precision)
    ibm.ibm_set_tune(g.h, tri_y=1, sweep_y=2, fft_plane=2)
    for sim in (o, g):
        sim.set_fields(*init)
    for s in range(3):
        xyz, vel = wl.surface(s)
        for sim in (o, g):
            sim.set_surface(xyz, vel, wl.tri)
            sim.step()
    gu, gv, gw, _ = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= tol, err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_energy_conserving_q_matches_oracle(precision, tol):
    """App. B's energy- and mass-conserving shape of q_F (use_q = 2) on a
    ragged grid with a moving sphere and a random initial field, 4 steps:
    fields against the oracle, sum q dV = 0 on the device."""
    wl = inputs.oscillating_sphere(n=48, steps=4, subdiv=2)
    u, v, w, p = inputs.random_fields(48, 37, 96, seed=9, amp=0.1)
    o = OracleSim(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, use_q=2)
    g = ibm.Simulation(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision=precision, use_q=2)
    o.set_fields(u, v, w, p)
    g.set_fields(u, v, w, p)
    for s in range(4):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    assert abs(o.last["q_coef"][1]) > 0
    gu, gv, gw, gp = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= tol * max(1.0, np.abs(o.u).max()), err
    d = g.diag()
    assert abs(d["q_f"] - o.last["q_coef"][0]) <= 1e-6 * max(1e-12, abs(o.last["q_coef"][0])) + tol
    assert abs(d["sum_q_dv"]) < 1e-12


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 1e-5)])
def test_radix5_grid_matches_oracle(precision, tol):
    """Grid sizes with factors of 5 (x: 100 = 4 * 5 * 5, z: 30 = 2 * 3 * 5;
    the heaving-pitching plate of Section 4.4 uses 100 x 650 x 100): the
    FFT's radix-5 butterflies against the oracle's numpy transforms."""
    nx, ny, nz = 100, 24, 30
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    u, v, w, p = inputs.random_fields(nx, ny, nz, seed=13, amp=0.1)
    o = OracleSim(nx, ny, nz, 1.0, 0.8, 1.0, re=120.0, dt=2e-3)
    g = ibm.Simulation(nx, ny, nz, 1.0, 0.8, 1.0, re=120.0, dt=2e-3, precision=precision)
    o.set_fields(u, v, w, p)
    g.set_fields(u, v, w, p)
    for s in range(3):
        xyz, vel = wl.surface(s)
        xyz = xyz * np.array([1.0, 0.8, 1.0])
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    gu, gv, gw, gp = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= tol, err
    if precision == "fp64":
        assert np.abs((o.p - o.p.mean()) - (gp - gp.mean())).max() <= 1e-10



def test_bounded_wait_gives_up_and_the_device_stays_usable():
    """The asynchronous-copy kernels never wait without bound: a wait on an
    mbarrier that cannot complete gives up after its cycle limit and
    returns, and the device context stays usable."""
    timed_out, waited = ibm.ibm_check_bounded_wait(2_000_000)
    assert timed_out == 1
    assert waited >= 2_000_000
    g = ibm.Simulation(16, 16, 16, precision="fp64")
    xyz, tri = inputs.icosphere(1, 0.2, (0.5, 0.5, 0.5))
    g.set_surface(xyz, np.zeros_like(xyz), tri)
    g.step(2)
    g.sync()
    assert g.diag()["steps"] == 2

def test_integer_path_conversions_match_hardware():
    """The mixed path's FP32 <-> FP64 conversions on the integer pipes give
    the hardware conversion's result bit for bit on 2^22 hashed cases
    (every class of binary32 input, every rounding case of the narrowing)."""
    bad, checked = ibm.ibm_check_conversions(1 << 22)
    assert checked > (1 << 22)   # most cases take the integer path
    assert bad == 0, bad


def test_alu_peak_probe_reports_plausible_rates():
    """The arithmetic roofs the benchmark reports FP64-bound kernels
    against: FMA-chain throughput of this device, FP64 far below FP32 on
    this GPU (its FP64 pipe is narrow), both within wide physical bounds."""
    fp64, fp32 = ibm.ibm_measure_alu_peaks()
    assert 0.1 < fp64 < 10.0, fp64
    assert 10.0 < fp32 < 300.0, fp32
    assert fp32 > 8 * fp64
