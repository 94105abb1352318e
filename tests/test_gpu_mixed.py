"""Mixed paths (FP32 bulk arithmetic; FP64 tagging, geometry, per-wavenumber
Thomas solve and reductions) against the FP64 CPU oracle and the FP64 GPU
path on the same inputs.

Error budget, written here as the bar (IBM_MIXED: velocity state as FP32
pairs plus a correction solve on the residual divergence):
  - tags bit-exact (the FP64 tagging is shared by every path);
  - velocity: max |u_mixed - u_oracle| <= 1e-5 U_ref after 10 steps;
  - discrete divergence of the projected field on the fluid cells:
    max |D u - q_F| <= 1e-7 U_ref / dx;
  - mean no-slip error ||eps||_1 within 5% of the FP64 path's;
  - pressure up to its mean: max |p_mixed - p_oracle| <= 1e-5 max(1, max |p|)
    U_ref^2 (no bar is set for it; this holds the measured 3-5e-7 with room).
IBM_MIXED_FAST (FP32 state, one solve) meets the velocity and no-slip bars;
its divergence is bounded by the FP32 solve, checked at 1e-5 U_ref / dx.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import OracleSim
from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu

VEL_TOL = 1e-5
# pressure (up to its mean) over max(1, max |p|) in units of U_ref^2: no bar
# is set for the mixed pressure; measured 2.9e-7 - 4.7e-7 on both workloads
# and both mixed forms, held here at 1e-5
PRES_TOL = 1e-5
DIV_TOL = 1e-7
DIV_TOL_FAST = 1e-5
SLIP_REL = 0.05


def run(wl, nsteps, precision):
    g = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=precision)
    slips = []
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        g.set_surface(xyz, vel, wl.tri)
        g.step()
        slips.append(g.diag()["slip_l1"])
    return g, slips


def oracle_run(wl, nsteps):
    o = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
    slips = []
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        o.step()
        slips.append(o.last["slip"])
    return o, slips


def divergence_error(g, sim_shape, lx=1.0, ly=1.0, lz=1.0):
    """max over fluid cells of |D u - q_F|, in units of U_ref / dx."""
    nx, ny, nz = sim_shape
    gr = orc.make_grid(nx, ny, nz, lx, ly, lz)
    u, v, w, p = g.fields()
    d = orc.divergence(gr, u, v, w)
    own = g.tags()
    isb = orc.boundary_cells(gr, own)
    qf = g.diag()["q_f"]
    fluid = isb == 0
    return np.abs(d - qf)[fluid].max() * gr.dx


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
@pytest.mark.parametrize("name,nsteps", [("sphere64", 10), ("plate128", 10)])
def test_mixed_vs_oracle(name, nsteps, precision):
    wl = inputs.workload(name)
    o, oslip = oracle_run(wl, nsteps)
    g, gslip = run(wl, nsteps, precision)
    gt = g.tags()
    for c in range(3):
        np.testing.assert_array_equal(gt[c], o.owners[c])
    gu, gv, gw, gp = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= VEL_TOL, f"velocity error {err:.3e}"
    perr = np.abs((o.p - o.p.mean()) - (gp - gp.mean())).max()
    assert perr <= PRES_TOL * max(1.0, np.abs(o.p).max()), f"pressure error {perr:.3e}"
    div = divergence_error(g, (wl.nx, wl.ny, wl.nz))
    tol = DIV_TOL if precision == "mixed" else DIV_TOL_FAST
    assert div <= tol, f"divergence {div:.3e} U/dx"


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
def test_mixed_slip_error_matches_fp64_path(precision):
    wl = inputs.heaving_plate()
    _, s64 = run(wl, 20, "fp64")
    _, s32 = run(wl, 20, precision)
    m64, m32 = np.mean(s64[5:]), np.mean(s32[5:])
    assert abs(m32 - m64) <= SLIP_REL * m64, (m32, m64)


@pytest.mark.parametrize("precision", ["mixed", "mixed_fast"])
def test_mixed_ragged_sizes(precision):
    wl = inputs.oscillating_sphere(n=48, steps=4, subdiv=2)
    o = OracleSim(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3)
    g = ibm.Simulation(48, 37, 96, 1.0, 0.9, 1.6, re=150.0, dt=2e-3, precision=precision)
    for s in range(4):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        g.set_surface(xyz, vel, wl.tri)
        o.step()
        g.step()
    gu, gv, gw, _ = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= VEL_TOL, f"velocity error {err:.3e}"
    div = divergence_error(g, (48, 37, 96), 1.0, 0.9, 1.6)
    assert div <= (DIV_TOL if precision == "mixed" else DIV_TOL_FAST), f"divergence {div:.3e} U/dx"


def test_mixed_set_get_fields_keep_fp64_state():
    """The mixed path stores the velocity as FP32 pairs: set/get round-trips
    an FP64 field to ~1e-14 relative."""
    u, v, w, p = inputs.random_fields(16, 12, 8, seed=4)
    g = ibm.Simulation(16, 12, 8, precision="mixed")
    g.set_fields(u, v, w, p)
    gu, gv, gw, gp = g.fields()
    for a, b in ((u, gu), (v, gv), (w, gw)):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()
    assert np.abs(p - gp).max() <= 1e-6 * np.abs(p).max()
