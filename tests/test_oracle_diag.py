"""Pins of the oracle's state diagnostics (max |D u - q| over C_F, kinetic
energy, CFL number) against closed forms, on uniform and stretched
wall-normal grids.

 - the kinetic energy of uniform fields is 1/2 U^2 times the volume their
   nodes cover (the v nodes span the centres of the first and last rows,
   so they cover ly - h_0/2 - h_{ny-1}/2 of the wall-normal extent);
 - the CFL number of a uniform field is dt (U/dx + V/h + W/dz) at the
   interior rows, where the cell-centred mean of v is V;
 - a v field linear in y has D u equal to its slope on every cell, so the
   residual of Eq. mod_div is |slope - q|, and cells outside C_F are left
   out;
 - after a step of the method the residual is at rounding level
   (Eq. mod_div), with and without q.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from oracle.oracle import OracleSim
from helpers import sample
from paper_2606_09799_gb300 import inputs


def _grids():
    g_u = orc.make_grid(12, 10, 8, lx=1.5, ly=1.0, lz=0.75)
    yf = inputs.stretched_faces(10, 1.0, 1.6)
    g_s = orc.make_grid(12, 10, 8, lx=1.5, ly=1.0, lz=0.75, yfaces=yf)
    return [g_u, g_s]


def _fields(g, U, V, W):
    u = np.full(orc.field_shape(g, 0), U)
    v = np.full(orc.field_shape(g, 1), V)
    v[:, 0, :] = 0.0
    v[:, -1, :] = 0.0
    w = np.full(orc.field_shape(g, 2), W)
    return u, v, w


@pytest.mark.parametrize("gi", [0, 1])
def test_kinetic_energy_of_uniform_fields(gi):
    g = _grids()[gi]
    U, V, W = 0.7, -0.3, 1.1
    u, v, w = _fields(g, U, V, W)
    hc, _ = orc.row_heights(g)
    lx, ly, lz = g.nx * g.dx, float(np.sum(hc)), g.nz * g.dz
    fluid = np.ones((g.nz, g.ny, g.nx), dtype=bool)
    _, ke, _ = orc.state_diagnostics(g, u, v, w, 0.0, fluid, 1e-3)
    exact = 0.5 * (U * U + W * W) * lx * ly * lz + 0.5 * V * V * lx * lz * (ly - 0.5 * hc[0] - 0.5 * hc[-1])
    assert abs(ke - exact) <= 1e-13 * exact


@pytest.mark.parametrize("gi", [0, 1])
def test_cfl_of_uniform_fields(gi):
    g = _grids()[gi]
    U, V, W, dt = 0.7, -0.3, 1.1, 2e-3
    u, v, w = _fields(g, U, V, W)
    hc, _ = orc.row_heights(g)
    fluid = np.ones((g.nz, g.ny, g.nx), dtype=bool)
    _, _, cfl = orc.state_diagnostics(g, u, v, w, 0.0, fluid, dt)
    # interior rows see the full V; the wall rows half of it
    per_row = [U / g.dx + (abs(V) if 0 < j < g.ny - 1 else 0.5 * abs(V)) / hc[j] + W / g.dz for j in range(g.ny)]
    assert abs(cfl - dt * max(per_row)) <= 1e-13 * cfl
    # one field at a time reduces to the one-dimensional Courant number
    u2, v2, w2 = _fields(g, U, 0.0, 0.0)
    _, _, c1 = orc.state_diagnostics(g, u2, v2, w2, 0.0, fluid, dt)
    assert abs(c1 - dt * U / g.dx) <= 1e-15


def test_divergence_residual_of_a_linear_field():
    g = _grids()[0]
    a = 0.37
    u = np.zeros(orc.field_shape(g, 0))
    w = np.zeros(orc.field_shape(g, 2))
    v = sample(g, 1, lambda X, Y, Z: a * Y + 0 * X + 0 * Z).copy()
    fluid = np.ones((g.nz, g.ny, g.nx), dtype=bool)
    d0, _, _ = orc.state_diagnostics(g, u, v, w, 0.0, fluid, 1e-3)
    assert abs(d0 - a) <= 1e-13
    d1, _, _ = orc.state_diagnostics(g, u, v, w, a, fluid, 1e-3)
    assert d1 <= 1e-13
    # a cell outside C_F does not count, however large its residual
    v[3, 4, 5] += 10.0
    d2, _, _ = orc.state_diagnostics(g, u, v, w, a, fluid, 1e-3)
    assert abs(d2 - 10.0 / g.dy) <= 1e-11
    mask = fluid.copy()
    mask[3, 4, 5] = False
    mask[3, 3, 5] = False   # the cell below shares the moved face
    d3, _, _ = orc.state_diagnostics(g, u, v, w, a, mask, 1e-3)
    assert d3 <= 1e-12
    # per-cell q (the shape of App. B) is subtracted cell by cell
    q = np.full((g.nz, g.ny, g.nx), a)
    d4, _, _ = orc.state_diagnostics(g, u, v, w, q, mask, 1e-3)
    assert d4 == d3


@pytest.mark.parametrize("use_q", [0, 1, 2])
def test_residual_after_a_step_is_rounding(use_q):
    wl = inputs.oscillating_sphere(n=16, steps=2, subdiv=1)
    o = OracleSim(16, 16, 16, re=wl.re, dt=2e-3, use_q=use_q)
    for s in range(2):
        xyz, vel = wl.surface(s)
        o.set_surface(xyz, vel, wl.tri)
        o.step()
    assert o.last["div_max"] <= 1e-11 / o.g.dx
    assert o.last["ke"] > 0.0 and o.last["cfl"] > 0.0
    if use_q:
        # the boundary cells are excluded: their divergence is q_B = D uhat, not q_F
        assert np.any(o.isb)
