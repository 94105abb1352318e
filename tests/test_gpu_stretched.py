"""Non-uniform wall-normal grid (Section 2: variable cell height in the
wall-normal direction) on the GPU, FP64 path, no immersed surface.

Bars: fields within 1e-10 of the CPU oracle after several steps (RK2+CN
and AB+CN, no-slip and free-slip walls), from a random initial field with a
body force; uniform face positions through the stretched entry point give
the uniform path's fields; the projected field has no divergence (computed
here from the face positions); unsupported combinations are refused."""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu

NX, NY, NZ = 24, 20, 16


def run_pair(yf, nsteps, scheme="rk2", ybc=0, re=120.0, dt=2e-3):
    u, v, w, p = inputs.random_fields(NX, NY, NZ, seed=21, amp=0.3)
    o = OracleSim(NX, NY, NZ, re=re, dt=dt, scheme=scheme, ybc=ybc, yfaces=yf)
    g = ibm.Simulation(NX, NY, NZ, re=re, dt=dt, scheme=scheme, ybc=ybc, precision="fp64", y_faces=yf)
    for s in (o, g):
        s.set_fields(u, v, w, p)
        s.set_body_force(2.0, 0.0, 0.3)
    o.step(nsteps)
    g.step(nsteps)
    return o, g


@pytest.mark.parametrize("scheme,ybc", [("rk2", 0), ("ab", 0), ("rk2", 1)])
def test_stretched_grid_matches_oracle(scheme, ybc):
    yf = inputs.stretched_faces(NY)
    o, g = run_pair(yf, 5, scheme, ybc)
    gu, gv, gw, gp = g.fields()
    err = max(np.abs(o.u - gu).max(), np.abs(o.v - gv).max(), np.abs(o.w - gw).max())
    assert err <= 1e-10, err
    assert np.abs(o.p - gp).max() <= 1e-10 * max(1.0, np.abs(o.p).max())


def test_uniform_faces_give_the_uniform_path():
    u, v, w, p = inputs.random_fields(NX, NY, NZ, seed=22, amp=0.3)
    a = ibm.Simulation(NX, NY, NZ, re=90.0, dt=2e-3, precision="fp64")
    b = ibm.Simulation(NX, NY, NZ, re=90.0, dt=2e-3, precision="fp64", y_faces=np.linspace(0.0, 1.0, NY + 1))
    for s in (a, b):
        s.set_fields(u, v, w, p)
        s.set_body_force(1.0, 0.0, 0.0)
        s.step(4)
    for x, y in zip(a.fields(), b.fields()):
        np.testing.assert_allclose(y, x, rtol=0, atol=1e-12)


def test_projected_field_has_no_divergence():
    yf = inputs.stretched_faces(NY)
    _, g = run_pair(yf, 3)
    u, v, w, _ = g.fields()
    hc = np.diff(yf)
    div = ((np.roll(u, -1, 2) - u) * NX + (v[:, 1:, :] - v[:, :-1, :]) / hc[None, :, None]
           + (np.roll(w, -1, 0) - w) * NZ)
    assert np.abs(div).max() * hc.min() <= 1e-10


def test_unsupported_combinations_are_refused():
    yf = inputs.stretched_faces(NY)
    with pytest.raises(ibm.IbmError):
        ibm.Simulation(NX, NY, NZ, precision="mixed", y_faces=yf)
    with pytest.raises(ibm.IbmError):
        ibm.Simulation(NX, NY, NZ, precision="fp64", y_faces=yf[::-1].copy())
    g = ibm.Simulation(NX, NY, NZ, precision="fp64", y_faces=yf)
    xyz, tri = inputs.icosphere(1, 0.2, (0.5, 0.5, 0.5))
    with pytest.raises(ibm.IbmError):
        g.set_surface(xyz, np.zeros_like(xyz), tri)
    h = ibm.Simulation(NX, NY, NZ, precision="fp64")
    with pytest.raises(ibm.IbmError):
        ibm.Batch([g, h])
