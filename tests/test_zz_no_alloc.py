"""Tagging for callers that must not allocate device memory.

ibm_tag_noalloc serves code that cannot call cudaMalloc when it needs the
tags (memory reserved once at start-up, another allocator's callback, a loop
that may not block on allocation); it keeps its working memory in a fixed
array inside the library.  Its owners must equal, bit for bit, those the
allocating path produces (ibm_step then ibm_get_tags) on the same grid and
surface -- checked on two calls in a row, since every call reuses the same
array and must not see the previous call's contents.  This file is collected
last so that a run stopping at the first failure has already run every other
test.
"""
import numpy as np
import pytest

from paper_2606_09799_gb300 import ibm, inputs

pytestmark = pytest.mark.gpu


def _owners_like(torch, nx, ny, nz):
    dev = torch.device("cuda", 0)
    return (torch.empty((nz, ny, nx), dtype=torch.int32, device=dev),
            torch.empty((nz, ny + 1, nx), dtype=torch.int32, device=dev),
            torch.empty((nz, ny, nx), dtype=torch.int32, device=dev))


def test_tag_noalloc_equals_allocating_path_on_two_calls():
    torch = pytest.importorskip("torch")
    wl = inputs.oscillating_sphere()           # 64^3: 790,528 nodes, inside the fixed array
    nx, ny, nz = wl.nx, wl.ny, wl.nz
    assert 3 * nx * ny * nz + nx * nz <= ibm.IBM_NOALLOC_MAX_NODES
    dev = torch.device("cuda", 0)
    tri = torch.from_numpy(wl.tri).to(dev)
    owners = _owners_like(torch, nx, ny, nz)
    sim = ibm.Simulation(nx, ny, nz, re=wl.re, dt=wl.dt)
    stream = torch.cuda.current_stream().cuda_stream
    for step in (0, 6):                          # two calls in a row, different surfaces
        xyz, vel = wl.surface(step)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
        ref = sim.tags()
        st = ibm.ibm_tag_noalloc(nx, ny, nz, torch.from_numpy(xyz).to(dev), tri, owners, stream=stream)
        assert st == 0, ibm.STATUS.get(st, st)
        for c in range(3):
            np.testing.assert_array_equal(owners[c].cpu().numpy(), ref[c])
        assert sum(int((o >= 0).sum()) for o in owners) > 1000
    sim.close()


def test_tag_noalloc_free_slip_walls_and_a_non_unit_box():
    """Other sizes, box lengths and wall condition than the 64^3 cube: the
    owners still equal those of a handle made by ibm_create_grid with the
    same description, on two calls in a row."""
    torch = pytest.importorskip("torch")
    nx, ny, nz, lx, ly, lz = 48, 40, 60, 1.2, 1.0, 1.5
    assert 3 * nx * ny * nz + nx * nz <= ibm.IBM_NOALLOC_MAX_NODES
    dev = torch.device("cuda", 0)
    owners = _owners_like(torch, nx, ny, nz)
    sim = ibm.Simulation(nx, ny, nz, lx, ly, lz, re=100.0, dt=1e-3, ybc=ibm.IBM_FREESLIP)
    stream = torch.cuda.current_stream().cuda_stream
    for seed, centre in ((3, (0.6, 0.5, 0.75)), (4, (0.05, 0.45, 1.45))):   # the second wraps in x and z
        xyz, tri = inputs.icosphere(2, 0.22, centre)
        xyz = xyz + 0.01 * np.random.default_rng(seed).standard_normal(xyz.shape)
        sim.set_surface(xyz, np.zeros_like(xyz), tri)
        sim.step()
        ref = sim.tags()
        st = ibm.ibm_tag_noalloc(nx, ny, nz, torch.from_numpy(xyz).to(dev), torch.from_numpy(tri).to(dev), owners,
                                 lx=lx, ly=ly, lz=lz, ybc=ibm.IBM_FREESLIP, stream=stream)
        assert st == 0, ibm.STATUS.get(st, st)
        for c in range(3):
            np.testing.assert_array_equal(owners[c].cpu().numpy(), ref[c])
        assert sum(int((o >= 0).sum()) for o in owners) > 1000
    sim.close()


def test_tag_noalloc_rejects_oversized_grid_and_bad_indices():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    xyz, tri = inputs.icosphere(1, 0.2, (0.5, 0.5, 0.5))
    x = torch.from_numpy(xyz).to(dev)
    # 128^3 holds 6.3 million nodes, beyond the fixed array
    big = _owners_like(torch, 128, 128, 128)
    assert ibm.ibm_tag_noalloc(128, 128, 128, x, torch.from_numpy(tri).to(dev), big) == 8   # IBM_ERR_CAPACITY
    small = _owners_like(torch, 16, 16, 16)
    bad = tri.copy()
    bad[3, 1] = xyz.shape[0] + 5
    assert ibm.ibm_tag_noalloc(16, 16, 16, x, torch.from_numpy(bad).to(dev), small) == 1    # IBM_ERR_ARG
    assert ibm.ibm_tag_noalloc(16, 16, 16, x, torch.from_numpy(tri).to(dev), small) == 0
