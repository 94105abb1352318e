"""Device-side state diagnostics and the saved state of a run, through the
C ABI, against the FP64 CPU oracle.

 - ibm_get_diag's max |D u - q| over C_F (Eq. mod_div), kinetic energy and
   CFL number equal the oracle's, computed from the oracle's own run and
   from the GPU's fields by the oracle's formulas;
 - the mixed paths hold D u = q to 1e-7 U/dx on the product path itself
   (the value the device reduces, not a host recomputation);
 - fields + the AB+CN history restored into a new handle continue the run
   bit for bit in FP64 (5 steps, save, restore, 5 steps = 10 steps), for
   both time schemes.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import OracleSim
from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu


def _run(wl, nsteps, precision="fp64", use_q=1, scheme="rk2", yfaces=None):
    o = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, use_q=use_q, scheme=scheme,
                  yfaces=yfaces)
    g = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, use_q=use_q,
                       precision=precision, scheme=scheme, y_faces=yfaces)
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    return o, g


def _host_diag(o, g):
    """The oracle's formulas applied to the GPU's fields, with the oracle's
    q and C_F (the tags are bit-identical)."""
    gu, gv, gw, _ = g.fields()
    if o.use_q == 2:
        q = o.last["q_field"]
    elif o.use_q:
        q = o.last["qF"]
    else:
        q = 0.0
    fluid = (o.isb == 0) if o.use_q else np.ones(o.isb.shape, dtype=bool)
    return orc.state_diagnostics(o.g, gu, gv, gw, q, fluid, o.dt)


@pytest.mark.parametrize("use_q", [0, 1, 2])
def test_fp64_diagnostics_match_oracle(use_q):
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    o, g = _run(wl, 3, use_q=use_q)
    d = g.diag()
    ud = 1.0 / o.g.dx          # U / dx
    assert d["div_max"] <= 1e-11 * ud
    assert abs(d["div_max"] - o.last["div_max"]) <= 1e-11 * ud
    assert abs(d["ke"] - o.last["ke"]) <= 1e-10 * o.last["ke"]
    assert abs(d["cfl"] - o.last["cfl"]) <= 1e-10 * o.last["cfl"]
    hd, hk, hc = _host_diag(o, g)
    assert abs(d["div_max"] - hd) <= 1e-12 * ud
    assert abs(d["ke"] - hk) <= 1e-12 * hk
    assert abs(d["cfl"] - hc) <= 1e-12 * hc


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
def test_mixed_divergence_bound_on_the_device(precision):
    """Mixed path: the device's own max |D u - q| meets 1e-7 U/dx (the
    correction solve); the single-solve form reports its larger residual."""
    wl = inputs.oscillating_sphere(n=32, steps=3, subdiv=2)
    o, g = _run(wl, 3, precision=precision)
    d = g.diag()
    ud = 1.0 / o.g.dx
    hd, hk, hc = _host_diag(o, g)
    if precision == "mixed":
        assert d["div_max"] <= 1e-7 * ud
        # pair arithmetic on the device against FP64 on the host, same state
        assert abs(d["div_max"] - hd) <= 1e-9 * ud
    else:
        assert d["div_max"] <= 1e-4 * ud
        assert abs(d["div_max"] - hd) <= 1e-3 * hd + 1e-9 * ud
    assert abs(d["ke"] - hk) <= 1e-6 * hk
    assert abs(d["cfl"] - hc) <= 1e-6 * hc
    assert abs(d["ke"] - o.last["ke"]) <= 1e-5 * o.last["ke"]
    assert abs(d["cfl"] - o.last["cfl"]) <= 1e-5 * o.last["cfl"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_diagnostics_on_the_stretched_grid(precision):
    wl = inputs.oscillating_sphere(n=32, steps=2, subdiv=2)
    yf = inputs.stretched_faces(32, 1.0, 1.4)
    o, g = _run(wl, 2, precision=precision, yfaces=yf)
    d = g.diag()
    hd, hk, hc = _host_diag(o, g)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert abs(d["ke"] - hk) <= tol * hk
    assert abs(d["cfl"] - hc) <= tol * hc
    assert d["div_max"] <= (1e-11 if precision == "fp64" else 1e-7) / float(np.min(np.diff(yf)))


@pytest.mark.parametrize("scheme", ["rk2", "ab"])
def test_save_restore_continues_bit_for_bit_fp64(scheme):
    wl = inputs.oscillating_sphere(n=32, steps=10, subdiv=2)
    ref = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, scheme=scheme)
    run = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, scheme=scheme)
    for s in range(10):
        xyz, vel = wl.surface(s)
        ref.set_surface(xyz, vel, wl.tri)
        ref.step()
    for s in range(5):
        xyz, vel = wl.surface(s)
        run.set_surface(xyz, vel, wl.tri)
        run.step()
    fields = run.fields()
    hist = run.history()
    run.close()
    new = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, scheme=scheme)
    new.set_fields(*fields)
    new.set_history(*hist)
    for s in range(5, 10):
        xyz, vel = wl.surface(s)
        new.set_surface(xyz, vel, wl.tri)
        new.step()
    for name, a, b in zip("uvwp", ref.fields(), new.fields()):
        assert np.array_equal(a, b), f"{scheme} {name}: max |delta| = {np.abs(a - b).max():.3e}"
    if scheme == "ab":
        for a, b in zip(ref.history(), new.history()):
            assert np.array_equal(a, b)


def test_without_history_ab_restart_differs():
    """The history matters for AB+CN: a restart that drops it (fields only)
    does not reproduce the run, so the test above checks something."""
    wl = inputs.oscillating_sphere(n=32, steps=10, subdiv=2)
    ref = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, scheme="ab")
    for s in range(6):
        xyz, vel = wl.surface(s)
        ref.set_surface(xyz, vel, wl.tri)
        ref.step()
        if s == 4:
            fields = ref.fields()
    new = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, scheme="ab")
    new.set_fields(*fields)
    xyz, vel = wl.surface(5)
    new.set_surface(xyz, vel, wl.tri)
    new.step()
    assert np.abs(ref.fields()[0] - new.fields()[0]).max() > 1e-12


def test_save_restore_mixed_ab_close():
    """Mixed path: the (hi, lo) state passes through FP64 on the way out and
    in.  A pair whose parts span more than 53 bits loses its lowest bits
    there, so the restored state differs from the saved one by ~1e-16.  The
    step after the restore stays within 1e-12 of the original run.  Later
    steps compute in FP32 from the hi parts; once such a difference moves an
    FP32 rounding, the runs part by an FP32 rounding of the state (~6e-8
    relative).  4 steps are held to 1e-6, and a restore that drops the
    history must land at least 10x further away."""
    wl = inputs.oscillating_sphere(n=32, steps=10, subdiv=2)
    kw = dict(re=wl.re, dt=wl.dt, scheme="ab", precision="mixed")
    ref = ibm.Simulation(32, 32, 32, **kw)
    run = ibm.Simulation(32, 32, 32, **kw)
    after = {}
    for s in range(8):
        xyz, vel = wl.surface(s)
        ref.set_surface(xyz, vel, wl.tri)
        ref.step()
        after[s] = ref.fields()
        if s < 4:
            run.set_surface(xyz, vel, wl.tri)
            run.step()
    saved = (run.fields(), run.history())
    dist = {}
    for with_history in (True, False):
        new = ibm.Simulation(32, 32, 32, **kw)
        new.set_fields(*saved[0])
        if with_history:
            new.set_history(*saved[1])
        for s in range(4, 8):
            xyz, vel = wl.surface(s)
            new.set_surface(xyz, vel, wl.tri)
            new.step()
            d = max(np.abs(a - b).max() for a, b in zip(after[s], new.fields()))
            if with_history and s == 4:
                assert d <= 1e-12, d
        dist[with_history] = d
        new.close()
    assert dist[True] <= 1e-6, dist
    assert dist[False] > 10.0 * max(dist[True], 1e-9), dist


@pytest.mark.parametrize("corr_check", [1, 2])
def test_correction_solve_runs_only_above_the_budget(corr_check):
    """IBM_MIXED: the correction solve runs in a sub-stage only when the
    first solve's max |D u' - q| over C_F exceeds the budget (Eq. mod_div);
    skipped, the step keeps the once-projected state.  corr_check 1 forms the
    residual inside the correction's forward transform, 2 in a pass of its
    own with the whole correction solve gated."""
    wl = inputs.oscillating_sphere(n=32, steps=6, subdiv=2)
    ud = 32.0                                    # U / dx of the unit box
    runs = {}
    for budget in (0.0, 1e30, None):
        g = ibm.Simulation(32, 32, 32, re=wl.re, dt=wl.dt, precision="mixed")
        ibm.ibm_set_tune(g.h, corr_check=corr_check)
        if budget is None:                       # one of the first run's residuals (an FP32 value)
            budget = sorted(runs[0.0]["first"])[2]
        g.set_div_budget(budget)
        first, taken, dmax = [], [], []
        prev = 0
        for s in range(6):
            xyz, vel = wl.surface(s)
            g.set_surface(xyz, vel, wl.tri)
            g.step()
            d = g.diag()
            first.append(d["div_first"])
            taken.append(d["corr_solves"] - prev)
            dmax.append(d["div_max"])
            prev = d["corr_solves"]
        runs[budget] = dict(first=first, taken=taken, dmax=dmax, fields=g.fields())
        g.close()
    always, never = runs[0.0], runs[1e30]
    assert all(t == 2 for t in always["taken"])  # RK2: both sub-stages
    assert all(m <= 1e-7 * ud for m in always["dmax"])
    assert all(f > 0.0 for f in always["first"])
    assert all(t == 0 for t in never["taken"])
    # without the correction the residual is that of the single FP32 solve,
    # and the device's final residual equals the first-solve residual's size
    assert all(m <= 1e-5 * ud for m in never["dmax"])
    for m, f in zip(never["dmax"], never["first"]):
        assert m <= f * (1.0 + 1e-3) + 1e-9 * ud
    mid = [v for k, v in runs.items() if k not in (0.0, 1e30)][0]
    bud = [k for k in runs if k not in (0.0, 1e30)][0]
    for f, t in zip(mid["first"], mid["taken"]):
        assert (t > 0) == (f > bud), (f, t, bud)
    # the skipped corrections stay within the velocity bar of the mixed path
    for a, b in zip(always["fields"][:3], never["fields"][:3]):
        assert np.abs(a - b).max() <= 1e-5


@pytest.mark.parametrize("budget", [0.0, 1e30, 2.0e-6])
def test_residual_pass_of_its_own_equals_the_fused_residual(budget):
    """The residual pass (corr_check 2) and the correction's forward transform
    (corr_check 1) form the same residual with the same arithmetic, so the
    decisions, the residuals and the fields agree bit for bit, with the
    correction always, never and sometimes taken (48 x 37 x 96, a moving
    sphere, 4 steps)."""
    wl = inputs.oscillating_sphere(n=48, steps=4, subdiv=2)
    out = []
    for cc in (1, 2):
        g = ibm.Simulation(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision="mixed")
        ibm.ibm_set_tune(g.h, corr_check=cc)
        g.set_div_budget(budget * 48.0)
        first, taken = [], []
        for s in range(4):
            xyz, vel = wl.surface(s)
            g.set_surface(xyz, vel, wl.tri)
            g.step()
            d = g.diag()
            first.append(d["div_first"])
            taken.append(d["corr_solves"])
        out.append((first, taken, g.fields()))
    for o in out[1:]:
        assert out[0][0] == o[0] and out[0][1] == o[1]
        for a, b in zip(out[0][2], o[2]):
            np.testing.assert_array_equal(a, b)


def test_div_budget_rejects_negative_and_nan():
    g = ibm.Simulation(16, 16, 16, re=100.0, dt=1e-3, precision="mixed")
    for bad in (-1.0, float("nan")):
        with pytest.raises(RuntimeError):
            g.set_div_budget(bad)
    g.set_div_budget(0.0)
    g.close()
