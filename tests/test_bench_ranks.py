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


def test_traffic_lookup_follows_the_kernel_source(tmp_path):
    """The roofline's DRAM traffic comes from the committed ncu summary only
    while the kernel's source file is the one the counters were taken on."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel source v1\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    summary = tmp_path / "traffic.md"
    summary.write_text("| stage | kernel | source | sha256 | launches | MB per launch |\n|---|---|---|---|---|---|\n"
                       f"| sweep_y | `SweepYStream<float>` | k.cu | {sha} | 2 | 80.5 |\n")
    assert bench.ncu_traffic("sweep_y", "SweepYStream<float>", str(summary), str(tmp_path)) == 80.5e6
    assert bench.ncu_traffic("sweep_y", "SweepZY<float>", str(summary), str(tmp_path)) is None
    assert bench.ncu_traffic("tri_y", "SweepYStream<float>", str(summary), str(tmp_path)) is None
    src.write_text("kernel source v2\n")
    assert bench.ncu_traffic("sweep_y", "SweepYStream<float>", str(summary), str(tmp_path)) is None
    assert bench.stage_kernel("sweep_y", {"sweep_y": 1}, "mixed") == "SweepYStream<float>"
    assert bench.stage_kernel("tri_y", {"tri_y": 3}, "fp64") == "TriYSmem<double>"
    assert bench.stage_kernel("tri_y", {"tri_y": 0}, "mixed", 128) == "TriYWarp<float, 16, 7>"
    assert bench.stage_kernel("tri_y", {"tri_y": 1}, "mixed", 128) == "TriYWarp<float, 16, 1>"
    assert bench.stage_kernel("fft_x_fwd", {}, "mixed") == "FftPlaneFwd<float>"
    assert bench.stage_kernel("fft_x_fwd", {"fft_plane": 3}, "mixed") == "FftPlaneFwdCl<float, 4>"
    assert bench.stage_kernel("fft_x_fwd", {"fft_plane": 2}, "fp64") == "FftPlaneFwd<double>"
    assert bench.stage_kernel("fft_x_fwd", {"fft_plane": 1}, "mixed") == "FftXFwd<float>"
    # the 256 x 192 x 256 channel: its plane does not fit one block, a cluster of 4 takes it
    assert bench.fft_form({}, 256, 256, 4) == "cluster"
    assert bench.fft_form({}, 256, 256, 8) == "split"
    assert bench.fft_form({}, 48, 60, 4) == "plane"
