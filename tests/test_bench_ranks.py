"""The multi-rank bookkeeping of bench.py (replicas, no collective on the
data path): every rank times its own replica, the job time is the slowest
rank's and the value counts all ranks' cell updates.  Two gloo ranks on CPU
(the GPU launch uses NCCL with the same calls)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [12.5, 20.0][rank]
    dist.barrier()
    ms = bench.max_over_ranks(ms_local, torch.device("cpu"), world)
    value = bench.whole_job_gcups(2_097_152, 10, world, ms)
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_max_time_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 20.0                                   # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 2_097_152 * 10 / 0.020 / 1e9)


def test_single_rank_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.0, torch.device("cpu"), 1) == 7.0
    assert bench.whole_job_gcups(100, 10, 1, 1.0) == pytest.approx(100 * 10 / 1e-3 / 1e9)
