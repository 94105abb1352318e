"""Batched independent simulations (one launch per kernel of the step for
all instances) and the launch-shape autotuner.

Bars:
  - FP64: every instance of a batch is bit-identical to the same instance
    stepped alone (fields and tags), and matches the CPU oracle to 1e-10.
  - mixed: tags bit-identical; velocity within 1e-5 U_ref of the instance
    stepped alone (the FP32 x-sweep's scan grouping follows the batch's
    largest nx, so the rounding order differs).
  - autotuning leaves the simulation state untouched, and later steps agree
    with an untuned run to 1e-12 (FP64: the Thomas variants differ in
    rounding order only).
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu


def small_batch(count=4, steps=3, sizes=(32, 48, 64)):
    return inputs.batched_instances(count=count, seed=11, steps=steps, sizes=sizes)


def make(wl, precision):
    return ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=precision)


def run_solo(wl, nsteps, precision, **tune):
    g = make(wl, precision)
    if tune:
        ibm.ibm_set_tune(g.h, **tune)
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        g.set_surface(xyz, vel, wl.tri)
        g.step()
    return g


def run_batch(wls, nsteps, precision, one_call=False):
    sims = [make(w, precision) for w in wls]
    b = None if one_call else ibm.Batch(sims)
    for s in range(nsteps):
        for w, g in zip(wls, sims):
            xyz, vel = w.surface(s)
            g.set_surface(xyz, vel, w.tri)
        if one_call:
            ibm.ibm_step_batch([g.h for g in sims], 1)
        else:
            b.step()
    if b is not None:
        b.sync()
    return sims, b


def test_batch_fp64_bit_identical_to_solo():
    wls = small_batch()
    assert len({(w.nx, w.ny, w.nz) for w in wls}) > 1   # uneven sizes
    sims, b = run_batch(wls, 3, "fp64")
    info = b.info()
    assert info["instances"] == len(wls)
    assert info["cells"] == sum(w.cells for w in wls)
    assert info["launches_per_step"] < info["launches_per_step_solo"]
    for w, g in zip(wls, sims):
        # the batch's built-in transforms are the separate x and z kernels (a
        # cluster of blocks per plane is a one-simulation form): the same here
        ref = run_solo(w, 3, "fp64", fft_plane=1)
        for a, r in zip(g.fields(), ref.fields()):
            np.testing.assert_array_equal(a, r)
        for a, r in zip(g.tags(), ref.tags()):
            np.testing.assert_array_equal(a, r)
        assert g.diag()["steps"] == 3
    b.close()


def test_batch_instances_match_oracle():
    wls = inputs.batched_instances(count=2, seed=5, steps=3, sizes=(32, 48))
    sims, b = run_batch(wls, 3, "fp64")
    for w, g in zip(wls, sims):
        o = OracleSim(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, re=w.re, dt=w.dt)
        for s in range(3):
            xyz, vel = w.surface(s)
            o.set_surface(xyz, vel, w.tri)
            o.step()
        gt = g.tags()
        for c in range(3):
            np.testing.assert_array_equal(gt[c], o.owners[c])
        gu, gv, gw, gp = g.fields()
        err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
        assert err <= 1e-10, err
        assert np.abs((o.p - o.p.mean()) - (gp - gp.mean())).max() <= 1e-10
    b.close()


def test_batch_mixed_close_to_solo():
    wls = small_batch()
    sims, b = run_batch(wls, 3, "mixed")
    for w, g in zip(wls, sims):
        ref = run_solo(w, 3, "mixed")
        for a, r in zip(g.tags(), ref.tags()):
            np.testing.assert_array_equal(a, r)
        ga, ra = g.fields(), ref.fields()
        err = max(np.abs(ga[q] - ra[q]).max() for q in range(3))
        assert err <= 1e-5, err
    b.close()


def test_step_batch_one_call_equals_batch_object():
    wls = small_batch(count=3)
    a, b = run_batch(wls, 2, "fp64")
    c, _ = run_batch(wls, 2, "fp64", one_call=True)
    for x, y in zip(a, c):
        for p, q in zip(x.fields(), y.fields()):
            np.testing.assert_array_equal(p, q)
    b.close()
    for g in c:          # destroying a handle releases the cached batch
        g.close()


def test_batch_rebuilds_when_a_surface_changes_size():
    wls = small_batch(count=3, steps=4)
    sims = [make(w, "fp64") for w in wls]
    b = ibm.Batch(sims)
    refs = [make(w, "fp64") for w in wls]
    for r in refs:       # the batch's built-in transforms: separate x and z kernels
        ibm.ibm_set_tune(r.h, fft_plane=1)
    alt_xyz, alt_tri = inputs.icosphere(2, 0.12, (0.5, 0.5, 0.5))     # 320 triangles
    for s in range(4):
        for k, (w, g, r) in enumerate(zip(wls, sims, refs)):
            if k == 1 and s >= 2:
                xyz, tri = alt_xyz, alt_tri
                vel = np.zeros_like(xyz)
            else:
                (xyz, vel), tri = w.surface(s), w.tri
            g.set_surface(xyz, vel, tri)
            r.set_surface(xyz, vel, tri)
            r.step()
        b.step()
    b.sync()
    for g, r in zip(sims, refs):
        for p, q in zip(g.fields(), r.fields()):
            np.testing.assert_array_equal(p, q)
    b.close()


def test_autotune_leaves_state_and_agrees_with_untuned_run():
    wl = inputs.oscillating_sphere(n=48, steps=6, subdiv=2)
    a = make(wl, "fp64")
    ref = make(wl, "fp64")
    for s in range(2):
        for g in (a, ref):
            xyz, vel = wl.surface(s)
            g.set_surface(xyz, vel, wl.tri)
            g.step()
    before = a.fields()
    chosen = a.autotune(steps=2)
    assert chosen["ms_per_step"] > 0
    after = a.fields()
    for p, q in zip(before, after):
        np.testing.assert_array_equal(p, q)
    assert ibm.ibm_get_tune(a.h)["tri_y"] == chosen["tri_y"]
    for s in range(2, 4):
        for g in (a, ref):
            xyz, vel = wl.surface(s)
            g.set_surface(xyz, vel, wl.tri)
            g.step()
    for p, q in zip(a.fields(), ref.fields()):
        assert np.abs(p - q).max() <= 1e-12
    for p, q in zip(a.tags(), ref.tags()):
        np.testing.assert_array_equal(p, q)


def test_batch_autotune_leaves_state():
    wls = small_batch(count=3)
    sims, b = run_batch(wls, 2, "mixed")
    before = [g.fields() for g in sims]
    chosen = b.autotune(steps=2)
    assert chosen["ms_per_step"] > 0
    for g, bf in zip(sims, before):
        for p, q in zip(bf, g.fields()):
            np.testing.assert_array_equal(p, q)
    b.step(1)
    b.sync()
    b.close()


@pytest.mark.parametrize("tune", [dict(tri_y=1, sweep_y=2, fft_plane=2), dict(tri_y=1, sweep_y=3, fft_plane=2),
                                  dict(tri_y=2, sweep_y=3, fft_plane=2), dict(tri_y=1, sweep_y=4, fft_plane=2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_bulk_copy_y_tiles_equal_solo(precision, tune):
    """Launch-shape choices sweep_y = 2, 3 and 4 (with either Thomas
    variant) in a batch of uneven instances and alone: the same fields, bit
    for bit in FP64.  (With 2 a batch keeps the streamed y sweep: its ops
    live in global memory, not in kernel parameters where tensor maps must
    be; 3 is the mixed path's tabulated rows in both; 4 adds the z sweep
    from shared-memory tiles.)"""
    wls = small_batch()
    sims = [make(w, precision) for w in wls]
    b = ibm.Batch(sims)
    b.set_tune(**tune)
    for s in range(3):
        for w, g in zip(wls, sims):
            xyz, vel = w.surface(s)
            g.set_surface(xyz, vel, w.tri)
        b.step()
    b.sync()
    for w, g in zip(wls, sims):
        ref = make(w, precision)
        ibm.ibm_set_tune(ref.h, **tune)
        for s in range(3):
            xyz, vel = w.surface(s)
            ref.set_surface(xyz, vel, w.tri)
            ref.step()
        for a, r in zip(g.fields(), ref.fields()):
            if precision == "fp64":
                np.testing.assert_array_equal(a, r)
            else:
                np.testing.assert_allclose(a, r, rtol=0, atol=1e-5)
    b.close()


def test_tune_values_are_validated():
    g = ibm.Simulation(32, 32, 32)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_set_tune(g.h, sweep_w=24)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_set_tune(g.h, fft_cols=3)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_set_tune(g.h, sweep_y=5)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_set_tune(g.h, fft_plane=4)
    with pytest.raises(ibm.IbmError):
        ibm.ibm_set_tune(g.h, tri_y=5)
    ibm.ibm_set_tune(g.h, tri_y=2, sweep_w=16, fft_lpb=4, fft_cols=4)
    assert ibm.ibm_get_tune(g.h)["sweep_w"] == 16
