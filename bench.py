#!/usr/bin/env python
"""Throughput of the sharp-interface IBM fractional step on GB300.

Metric: fractional-step cell updates per second (GCUPS): one update = one
cell through a whole time step (Algorithm 1 tagging of the three grids and
both RK2+CN sub-stages: IB forcing, explicit terms, factorised implicit
sweeps, consistent mass correction q, FFT/Thomas Poisson solve, projection),
plus the no-slip error diagnostic.

Workload (one step): the 128^3 zero-thickness plate -- staggered grid on the
unit cube, periodic x and z, walls at y = 0, 1; square plate of side 0.4
triangulated 64 x 64 (8,192 triangles) heaving 0.05 sin(2 pi t) with the
bending mode 0.02 sin(pi s) sin(2 pi t); Re = 200, dt = 5e-4, fluid at rest.
The surface of every step is prescribed (moved between steps).

Arms
  default            the CUDA library through its C ABI; the mixed
                     (FP32 bulk / FP64 tagging, tridiagonal, geometry) and the
                     FP64 paths run on the same inputs, `value` is the
                     headline path (--precision), the other is reported beside
                     it with its no-slip error.
  --impl reference   the plain FP64 CPU oracle on the host cores, same
                     workload and metric (one whole oracle step per step).

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torchrun, one rank per GPU, each advancing its own replica (no collective
on the data path), the barrier-bracketed time taken as the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fractional-step cell updates/s (GCUPS), mixed vs FP64 at equal slip error"
UNIT = "GCUPS"
WORKLOAD = ("plate128: 128^3 staggered grid on the unit cube (x, z periodic, no-slip walls in y), "
            "zero-thickness square plate of side 0.4 triangulated 64x64 (8192 triangles) heaving "
            "0.05 sin(2 pi t) plus bending 0.02 sin(pi s) sin(2 pi t); Re=200, dt=5e-4, RK2+CN, fluid at rest")
L2_FLUSH_BYTES = 256 << 20


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("IBM_BENCH_OUT", os.path.join(ROOT, "bench_out")),
                                 f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic bytes (FP32/mixed) and FP64 flops per cell
# ---------------------------------------------------------------------------
def algorithmic_bytes_per_cell(stage: str, word: int, pairs: bool = False) -> float:
    """Compulsory words per cell of each kernel group and sub-stage: one read
    of every input field, one write of every output field (the sparse IB
    part is counted per forcing node elsewhere).  pairs: the mixed path's
    velocity state is an FP32 (hi, lo) pair, two words per velocity node
    where a kernel reads or writes the state."""
    reads_writes = {
        "rhs": (5.5, 4.5),          # u, v, w, p (+ H^{s-1} on sub-stage 2, averaged) -> R x3 (+ H x3 on sub-stage 1)
        "sweep_x": (3, 3),
        "sweep_z": (3, 3),
        "sweep_y": (6, 3),          # du x3 and u^s x3 -> uhat x3
        "fft_x_fwd": (3, 1),        # uhat x3 -> half spectrum (2 words x (nx/2+1)/nx)
        "correction": (3, 1),       # the correction's forward transform: projected state x3 -> half spectrum
        "fft_z_fwd": (1, 1),
        "tri_y": (1, 1),
        "fft_z_inv": (1, 1),
        "fft_x_inv": (1, 1),
        "project": (5, 4),          # uhat x3, phi, p -> u x3, p
    }
    if pairs:
        reads_writes.update({
            "sweep_y": (9, 6),      # du x3 and u^s x3 as (hi, lo) -> uhat x3 as (hi, lo)
            "project": (9, 7),      # uhat x3 (hi, lo), p, phi, phi2 -> u x3 (hi, lo), p
            "correction": (7, 1),   # uhat x3 (hi, lo), phi -> half spectrum of the residual divergence
        })
    r, w = reads_writes.get(stage, (0, 0))
    return (r + w) * word


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "traffic_plate128.md")


def fft_form(tune: dict | None, nx: int = 128, nz: int = 128, word: int = 4) -> str:
    """How the launch shapes run the x and z transforms of one simulation:
    "plane" (fused per y-plane in one block: fft_plane 2, and the built-in
    choice where the plane and its work buffers fit 200 KB of shared memory),
    "cluster" (fused per y-plane over a cluster of 4 blocks, each within
    100 KB: fft_plane 3, and the built-in choice where the plane does not
    fit) or "split" (separate x and z kernels)."""
    v = (tune or {}).get("fft_plane", 0)
    nkx, c = nx // 2 + 1, 2 * word          # complex word
    plane_b = nz * nkx * c
    wmax = (200 * 1024 - plane_b) // (2 * c)
    lcp, cmax = min(nz // 2, wmax // (nx + 1)), max(1, min(nkx, wmax // nz))   # x lines padded to nx + 1
    czp = -(-nkx // -(-nkx // cmax))
    plane_fits = lcp >= 1 and czp * nz <= wmax and plane_b + 2 * max(lcp * (nx + 1), czp * nz) * c <= 200 * 1024
    if v in (0, 2) and plane_fits:
        return "plane"
    if v in (0, 3) and nz % 8 == 0 and nkx >= 4:
        nzc, cw = nz // 4, -(-nkx // 4)
        wm = (100 * 1024 - nzc * nkx * c) // (2 * c)
        if min(nzc // 2, wm // (nx + 1)) >= 1 and min(cw, wm // nz) >= 1:
            return "cluster"
    return "split"


def stage_kernel(stage: str, tune: dict | None, precision: str, ny: int = 128, nz: int = 128) -> str | None:
    """Kernel that the given launch shapes run for a stage of the 128^3 step
    (the name the ncu summaries use), or None when it is not recorded."""
    t = tune or {}
    T = "float" if precision == "mixed" else "double"
    if stage in ("sweep_y", "sweep_z"):
        sy = t.get("sweep_y", 0)
        if sy in (1, 2, 3, 4):
            if stage == "sweep_z":
                return f"SweepZTile<{T}>" if sy == 4 else f"SweepZStream<{T}>"
            if sy in (3, 4) and precision == "mixed":
                return f"SweepYStretched<{T}>"
            if sy == 2:
                return f"SweepYTma<{T}>"
            return f"SweepYStream<{T}>"
        if precision == "mixed" and t.get("sweep_zy", 0) != 1:
            return f"SweepLanes<{T}, 16, 8>"
        return f"SweepZY<{T}>"
    if stage == "tri_y":
        v = t.get("tri_y", 0)
        lanes = 8 if ny <= 64 else (16 if ny <= 128 else 32)     # 8 rows per lane
        warp = f"TriYWarp<{T}, {lanes}, 7>" if ny <= 256 else f"TriY<{T}>"
        uncapped = f"TriYWarp<{T}, {lanes}, 1>" if ny <= 256 else f"TriY<{T}>"
        return {0: warp, 4: warp, 1: uncapped, 2: f"TriY<{T}>", 3: f"TriYSmem<{T}>"}[v]
    if stage == "fft_x_fwd":
        form = fft_form(t, nz=nz, word=4 if precision == "mixed" else 8)
        return {"cluster": f"FftPlaneFwdCl<{T}, 4>", "plane": f"FftPlaneFwd<{T}>"}.get(form, f"FftXFwd<{T}>")
    if stage == "rhs":
        v = t.get("rhs", 0)
        if v == 2:
            return f"RhsTile<{T}, 0>"
        if precision == "mixed" and v in (0, 3):
            return "RhsVec<0>"
        return f"Rhs<{T}, 0, int>"
    if stage == "project":
        return f"Project<{T}>"
    return None


def ncu_traffic(stage: str, kernel: str | None, summary: str = TRAFFIC_SUMMARY, root: str = ROOT) -> float | None:
    """DRAM bytes (read + write) per launch of `kernel` in `stage` from the
    committed ncu summary, or None when it has no row for it or the kernel's
    source file has changed since the counters were taken (its SHA-256 is
    recorded beside the figure)."""
    import hashlib
    if kernel is None or not os.path.exists(summary):
        return None
    for line in open(summary):
        cells = [c.strip().strip("`") for c in line.strip().strip("|").split("|")]
        if len(cells) < 6 or cells[0] != stage or cells[1] != kernel:
            continue
        path = os.path.join(root, cells[2])
        if not os.path.exists(path):
            return None
        with open(path, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != cells[3]:
                return None
        try:
            return float(cells[5]) * 1e6
        except ValueError:
            return None
    return None


def group_traffic(stages, kernel: str | None) -> float | None:
    """DRAM bytes per launch of a kernel group (stages that run the same
    kernel, launched alike often): the mean of its stages' recorded figures,
    or None when any of them is missing or stale."""
    tr = [ncu_traffic(s2, kernel) for s2 in stages]
    return sum(tr) / len(tr) if tr and all(t is not None for t in tr) else None


TAG_FLOPS_PER_PAIR = 100.0   # closest point ~73, N and |N|^2 8, neighbour tests up to ~36 (FP64, counted from source)


def tag_pairs(wl, step: int) -> int:
    """Algorithmic work of Algorithm 1 for one step: (node, triangle) pairs
    with the node strictly inside the triangle's box min - d < x < max + d,
    summed over the three staggered grids (nodes holding unknowns only)."""
    import numpy as np
    xyz, _ = wl.surface(step)
    V = xyz[wl.tri]                                   # (nt, 3 vertices, 3 coords)
    lo, hi = V.min(axis=1), V.max(axis=1)
    d = np.array([wl.lx / wl.nx, wl.ly / wl.ny, wl.lz / wl.nz])
    n = np.array([wl.nx, wl.ny, wl.nz])
    total = 0
    for c in range(3):
        cnt = np.ones(len(V), dtype=np.int64)
        for a in range(3):
            off = 0.0 if a == c else 0.5
            l = (lo[:, a] - d[a]) / d[a] - off
            h = (hi[:, a] + d[a]) / d[a] - off
            i0 = np.floor(l).astype(np.int64) + 1      # first index with coordinate > lo - d
            i1 = np.ceil(h).astype(np.int64) - 1       # last index with coordinate < hi + d
            if a == 1:
                jlo = 1 if c == 1 else 0
                i0 = np.maximum(i0, jlo)
                i1 = np.minimum(i1, n[1] - 1)
            cnt *= np.maximum(0, i1 - i0 + 1)
        total += int(cnt.sum())
    return total


# Plain Thomas per wavenumber (Eq. elliptic after the x and z transforms):
# forward y_j = (r_j - a y_{j-1}) / d_j, one multiply-add and one multiply
# (3 flops), backward x_j = y_j - c'_j x_{j+1}, one multiply-add (2 flops),
# for the real and the imaginary part of every (kx, kz, j).
TRI_FLOPS_PER_ROW = 10.0
# Algorithmic bytes of the Thomas pass per (kx, kz, j): read and write the
# complex spectrum (FP32 pairs in the mixed path, FP64 in the FP64 path).
TRI_BYTES_PER_ROW = {"mixed": 16.0, "fp64": 32.0}
# Algorithmic bytes per cell of one whole step (two RK2 sub-stages), the
# planned compulsory traffic of every stage: 224 B per sub-stage in the
# mixed path (FP32 words, FP64 Thomas), 432 B in the FP64 path.
STEP_BYTES_PER_CELL = {"mixed": 448.0, "fp64": 864.0}


def fp64_flops_per_cell(stage: str) -> float:
    """FP64 floating-point operations per cell of each kernel group in the
    FP64 path (adds, multiplies and FMAs counted as executed instructions x
    flops: an FMA counts 2), counted from the kernel source."""
    return {"rhs": 150.0, "sweep_x": 15.0, "sweep_z": 15.0, "sweep_y": 15.0, "fft_x_fwd": 45.0,
            "fft_z_fwd": 40.0, "tri_y": 8.0, "fft_z_inv": 40.0, "fft_x_inv": 40.0, "project": 30.0}.get(stage, 0.0)


def set_budget(sim, args, dx):
    """Divergence budget of the mixed path's correction solve: the solve runs
    in a sub-stage only when the first solve leaves max |D u - q| over the
    fluid cells above it (U_ref = 1, so the budget is a multiple of 1/dx)."""
    if sim.precision == "mixed" and args.div_budget > 0.0:
        sim.set_div_budget(args.div_budget / dx)


def correction_record(args, diag, substages, dx):
    """How many of the timed sub-stages took the correction solve."""
    return {"budget_U_per_dx": args.div_budget, "taken": int(diag.get("corr_timed", diag["corr_solves"])),
            "substages": int(substages), "last_first_solve_residual_U_per_dx": diag["div_first"] * dx}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def gpu_arm(args):
    import numpy as np
    import torch
    from paper_2606_09799_gb300 import ibm, inputs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.fp64_peak_tflops <= 0:
        args.fp64_peak_tflops, args.fp32_peak_tflops = ibm.ibm_measure_alu_peaks()
    wl = inputs.heaving_plate()
    K, W = args.steps, args.warmup
    nsteps_total = W + K
    tri = wl.tri
    # every step's surface, resident on the device before timing
    surf = [wl.surface(s) for s in range(nsteps_total + 1)]
    dxyz = [torch.from_numpy(x).to(dev) for x, _ in surf]
    dvel = [torch.from_numpy(v).to(dev) for _, v in surf]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    results = {}
    order = [args.precision] + [p for p in ("mixed", "fp64") if p != args.precision]
    if args.only_headline:
        order = order[:1]
    for prec in order:
        sim = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=prec,
                             stream=stream.cuda_stream)
        set_budget(sim, args, wl.lx / wl.nx)
        sim.set_surface(surf[0][0], surf[0][1], tri)
        for s in range(W):
            sim.set_surface(dxyz[s], dvel[s])
            sim.step(1)
        sim.sync()
        if args.tune:
            sim.set_tune(**args.tune)                                  # fixed launch shapes
            tune = ibm.ibm_get_tune(sim.h)
        else:
            tune = sim.autotune(steps=3) if args.autotune else None   # launch shapes (state restored)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        corr0 = sim.diag()["corr_solves"]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            for n in range(K):
                flush.fill_(n & 0xFF)                        # L2 flush between timed steps (outside the events)
                ev[n][0].record(stream)
                sim.set_surface(dxyz[W + n], dvel[W + n])    # this step's prescribed surface (device resident)
                sim.step(1)
                ev[n][1].record(stream)
            torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = sum(a.elapsed_time(b) for a, b in ev)
        diag = sim.diag()
        diag["corr_timed"] = diag["corr_solves"] - corr0
        sim.sync()
        ms = max_over_ranks(ms, dev, world)
        # stage profile of the same workload (CUDA events recorded on the launching stream)
        prof = ibm.ibm_profile_stages(sim.h, args.profile_steps)
        # end-to-end: host surface in pinned memory -> device, step, diagnostics read back
        hx = torch.from_numpy(surf[0][0]).pin_memory()
        hv = torch.from_numpy(surf[0][1]).pin_memory()
        e2e_ms = 0.0
        d2h = 0
        torch.cuda.synchronize()
        ke = max(3, min(K, 20))
        for n in range(ke):
            hx.copy_(torch.from_numpy(surf[(W + n) % len(surf)][0]))
            hv.copy_(torch.from_numpy(surf[(W + n) % len(surf)][1]))
            flush.fill_(n & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ibm.ibm_set_surface(sim.h, hx, hv, None, tri.shape[0])
            ibm.ibm_step(sim.h, 1)
            dd = ibm.ibm_get_diag(sim.h)
            e2e_ms += (time.perf_counter() - t0) * 1e3
            d2h = dd["d2h_bytes"]
        results[prec] = dict(ms=ms, diag=diag, prof=prof, e2e_ms=e2e_ms, e2e_steps=ke, d2h=d2h,
                             clocks=clk.summary(), tune=tune)
        sim.close()
    batched = None if (args.only_headline or args.no_batch) else batched_leg(args, dev, stream, flush, world)
    ab = None
    if not (args.only_headline or args.no_ab):
        ab = ab_leg(args, wl, dxyz, dvel, surf, dev, stream, flush, world, results[args.precision]["tune"])
    stretched = None
    if not (args.only_headline or args.no_stretched):
        stretched = stretched_leg(args, dev, stream, flush, world)
    if rank != 0:
        return None
    head = results[args.precision]
    cells = wl.cells
    value = whole_job_gcups(cells, K, world, head["ms"])
    e2e_value = world * cells * head["e2e_steps"] / (head["e2e_ms"] / 1e3) / 1e9
    h2d = 2 * surf[0][0].nbytes
    peaks = measured_peaks()
    prof = head["prof"]
    # roofline of every kernel group of the headline path; the kernel with the
    # most device time per step is reported (stages that run the same kernel,
    # such as the Thomas passes of the first and the correction solve, summed)
    fp64_peak = args.fp64_peak_tflops
    pairs = tag_pairs(wl, W)
    nrows = (wl.nx // 2 + 1) * wl.nz * wl.ny
    hbm = peaks.get("hbm_gbs", 6800.0)
    groups = {}
    tune_h = head["tune"] or {}
    plane = fft_form(tune_h, wl.nx, wl.nz, 4 if args.precision == "mixed" else 8) != "split"
    # the correction solve's Thomas and inverse transforms are gated: a launch
    # whose sub-stage met the divergence budget returns at entry, so their
    # per-launch rates would count launches that did no work; they are left
    # out here (their time is in stages_ms_per_step), and the Thomas and the
    # inverse transforms are rated on the first solve's launches alone
    merged = {}
    fused_check = tune_h.get("corr_check", 0) != 2   # else a residual pass shares the correction's stage
    if plane and fused_check:
        merged["fft_x_fwd"] = ("fft_x_fwd", "correction")
    skip = {s2 for k, v in merged.items() for s2 in v if s2 != k} | {"correction_tri", "correction_inv"}
    if not fused_check:   # the residual pass and the gated forward transform share a stage
        skip.add("correction")
    for name, (tot_ms, ngroups) in prof.items():
        if name in ("other",) or name in skip or ngroups == 0 or tot_ms <= 0:
            continue
        stages = merged.get(name, (name,))
        tot = sum(prof[s2][0] for s2 in stages if s2 in prof)
        launches = sum(prof[s2][1] for s2 in stages if s2 in prof) * args.profile_steps
        avg_ms = tot / launches
        per_step_ms = tot / args.profile_steps
        if name == "tagging":
            work = pairs * TAG_FLOPS_PER_PAIR
            g = dict(bound="alu", achieved=work / (avg_ms / 1e3) / 1e12, peak=fp64_peak, unit="TFLOP/s")
        elif name == "tri_y":
            fl = TRI_FLOPS_PER_ROW * nrows / (avg_ms / 1e3) / 1e12
            by = TRI_BYTES_PER_ROW[args.precision] * nrows / (avg_ms / 1e3) / 1e9
            g = dict(bound="alu", achieved=fl, peak=fp64_peak, unit="TFLOP/s",
                     hbm={"achieved": by, "peak": hbm, "frac": by / hbm})
            if by / hbm > fl / fp64_peak:
                g = dict(bound="hbm", achieved=by, peak=hbm, unit="GB/s", alu={"achieved": fl, "peak": fp64_peak,
                                                                               "frac": fl / fp64_peak})
        elif args.precision == "fp64" and fp64_flops_per_cell(name) > 0:
            work = fp64_flops_per_cell(name) * cells
            g = dict(bound="alu", achieved=work / (avg_ms / 1e3) / 1e12, peak=fp64_peak, unit="TFLOP/s")
        elif algorithmic_bytes_per_cell(name, 4) > 0:
            # bytes of an average launch of the group (the correction's forward
            # transform reads more than the first solve's)
            nl = [prof[s2][1] for s2 in stages if s2 in prof]
            work = sum(algorithmic_bytes_per_cell(s2, 4, pairs=args.precision == "mixed") * prof[s2][1]
                       for s2 in stages if s2 in prof) / sum(nl) * cells
            g = dict(bound="hbm", achieved=work / (avg_ms / 1e3) / 1e9, peak=hbm, unit="GB/s")
        else:
            continue
        g.update(avg_ms=avg_ms, ms_per_step=per_step_ms, launches_per_step=launches / args.profile_steps,
                 stages=list(stages))
        g["frac"] = g["achieved"] / g["peak"] if g["peak"] else None
        groups[name] = g
    tot_all = sum(g["ms_per_step"] for g in groups.values())
    for g in groups.values():
        g["share"] = g["ms_per_step"] / tot_all
    top = max(groups, key=lambda k: groups[k]["ms_per_step"])
    tg = groups[top]
    kname = stage_kernel(top, head["tune"], args.precision, wl.ny, wl.nz)
    roof = {"bound": tg["bound"], "achieved": tg["achieved"], "peak": tg["peak"], "unit": tg["unit"],
            "frac": tg["frac"], "traffic": group_traffic(tg["stages"], kname), "kernel": top, "kernel_name": kname,
            "ms_per_step": tg["ms_per_step"], "launches_per_step": tg["launches_per_step"],
            "peak_source": ("FP64 FMA-chain probe ibm_measure_alu_peaks, this run (of measured)"
                            if tg["bound"] == "alu" else "MEASURED_PEAKS.json hbm_gbs (of measured)")}
    for k in ("hbm", "alu"):
        if k in tg:
            roof[k] = tg[k]
    step_bytes = STEP_BYTES_PER_CELL[args.precision] * cells
    step_ach = step_bytes / (head["ms"] / K / 1e3) / 1e9
    step_roof = {"bound": "hbm", "bytes_per_cell": STEP_BYTES_PER_CELL[args.precision], "achieved": step_ach,
                 "peak": hbm, "unit": "GB/s", "frac": step_ach / hbm,
                 "roof_gcups": hbm * 1e9 / STEP_BYTES_PER_CELL[args.precision] / 1e9}
    kernels_per_step = head["diag"]["kernels_per_step"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": head["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": cells, "triangles": int(tri.shape[0]),
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MiB write outside the events)"},
        "roofline": roof,
        "step_roofline": step_roof,
        "alu_peaks": {"fp64_tflops": args.fp64_peak_tflops, "fp32_tflops": args.fp32_peak_tflops,
                      "source": "ibm_measure_alu_peaks (FMA chains, CUDA events), this run"},
        "gpu_launches": (kernels_per_step + 2) * K,
        "clocks": head["clocks"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": head["d2h"]},
        "slip_l1": head["diag"]["slip_l1"],
        "stages_ms_per_step": {k: v[0] / args.profile_steps for k, v in prof.items() if v[1] > 0},
        "stage_roofline": {k: {kk: (round(vv, 4) if isinstance(vv, float) else vv) for kk, vv in g.items()}
                           for k, g in groups.items()},
        "tag_pairs_per_step": pairs,
    }
    for prec, r in results.items():
        dg = r["diag"]
        line[prec] = {"value": world * cells * K / (r["ms"] / 1e3) / 1e9, "ms_per_step": r["ms"] / K,
                      "slip_l1": dg["slip_l1"], "clocks": r["clocks"], "tune": r["tune"],
                      "div_max_U_per_dx": dg["div_max"] * wl.lx / wl.nx, "ke": dg["ke"], "cfl": dg["cfl"]}
        if prec == "mixed":
            line[prec]["correction"] = correction_record(args, dg, 2 * K, wl.lx / wl.nx)
    if batched is not None:
        line["batched"] = batched
    if ab is not None:
        line["ab_cn"] = ab
    if stretched is not None:
        line["stretched"] = stretched
    if not args.no_large and world == 1:
        line["large"] = large_leg(args, dev, stream, flush)
    if args.e5_steps > 0:
        line["e5_heaving_pitching_plate"] = e5_leg(args, dev, stream)
    if "mixed" in results and "fp64" in results:
        sm, sf = results["mixed"]["diag"]["slip_l1"], results["fp64"]["diag"]["slip_l1"]
        line["slip_rel_diff_mixed_vs_fp64"] = abs(sm - sf) / sf if sf else None
        line["speedup_mixed_vs_fp64"] = line["mixed"]["value"] / line["fp64"]["value"]
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_steps)
        if not args.no_large:
            line["cpu_baseline_extra"] = cpu_baseline_extra()
    return line


def ab_leg(args, wl, dxyz, dvel, surf, dev, stream, flush, world, tune):
    """The same workload and protocol with the AB+CN scheme (one sub-stage
    per step, Section 2) in the headline precision, launch shapes as tuned
    for RK2+CN."""
    import torch
    from paper_2606_09799_gb300 import ibm

    K, W = args.steps, args.warmup
    sim = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=args.precision,
                         scheme="ab", stream=stream.cuda_stream)
    set_budget(sim, args, wl.lx / wl.nx)
    if tune:
        sim.set_tune(**{k: v for k, v in tune.items() if k != "ms_per_step"})
    sim.set_surface(surf[0][0], surf[0][1], wl.tri)
    for s in range(W):
        sim.set_surface(dxyz[s], dvel[s])
        sim.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for n in range(K):
        flush.fill_(n & 0xFF)
        ev[n][0].record(stream)
        sim.set_surface(dxyz[W + n], dvel[W + n])
        sim.step(1)
        ev[n][1].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev, world)
    diag = sim.diag()
    sim.close()
    return {"scheme": "AB+CN", "precision": args.precision, "value": whole_job_gcups(wl.cells, K, world, ms),
            "unit": UNIT, "ms_per_step": ms / K, "slip_l1": diag["slip_l1"]}


def stretched_leg(args, dev, stream, flush, world):
    """The non-uniform wall-normal grid leg: the channel alone and with an
    immersed wall across it (the channel cases of Section 4)."""
    from paper_2606_09799_gb300 import inputs

    wl = inputs.immersed_wall_channel(nx=128, ny=128, nz=128, y_wall=0.1213, nq=32)
    wall = (wl.surface(0)[0], wl.tri)
    out = stretched_run(args, dev, stream, flush, world, None, "fp64")
    out["with_immersed_wall"] = stretched_run(args, dev, stream, flush, world, wall, "fp64")
    out["mixed"] = stretched_run(args, dev, stream, flush, world, None, "mixed")
    out["mixed"]["with_immersed_wall"] = stretched_run(args, dev, stream, flush, world, wall, "mixed")
    return out


def stretched_run(args, dev, stream, flush, world, wall, precision):
    """One path on a non-uniform wall-normal grid: the 128^3 channel with
    cells clustered at both walls (tanh stretching, 3x taller at mid-channel),
    with the immersed wall `wall` = (xyz, tri) or none, driven by a uniform
    body force from a seeded random field; same timing protocol as the
    headline."""
    import numpy as np
    import torch
    from paper_2606_09799_gb300 import ibm, inputs

    n = 128
    K, W = max(3, min(args.steps, 20)), max(3, args.warmup)
    yf = inputs.stretched_faces(n)
    sim = ibm.Simulation(n, n, n, re=200.0, dt=5e-4, precision=precision, stream=stream.cuda_stream, y_faces=yf)
    sim.set_fields(*inputs.random_fields(n, n, n, seed=31, amp=0.1))
    sim.set_body_force(8.0 / 200.0, 0.0, 0.0)
    hmin = float(np.min(np.diff(yf)))
    set_budget(sim, args, hmin)
    if wall is not None:
        sim.set_surface(wall[0], np.zeros_like(wall[0]), wall[1])
    for _ in range(W):
        sim.step(1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    corr0 = sim.diag()["corr_solves"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for m in range(K):
        flush.fill_(m & 0xFF)
        ev[m][0].record(stream)
        sim.step(1)
        ev[m][1].record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dev, world)
    dg = sim.diag()
    slip = dg["slip_l1"]
    dg["corr_timed"] = dg["corr_solves"] - corr0
    prof = ibm.ibm_profile_stages(sim.h, 2)
    sim.close()
    # mixed path: every HBM-bound kernel group against the measured copy rate,
    # with the algorithmic bytes per cell of the uniform grid's groups (the
    # same fields; the wall-normal tables add under 1 MB)
    roof = {}
    if precision == "mixed":
        peak = measured_peaks().get("hbm_gbs", 6800.0)
        for name, (tot_ms, ngroups) in prof.items():
            b = algorithmic_bytes_per_cell(name, 4, pairs=True)
            if ngroups == 0 or tot_ms <= 0 or b <= 0:
                continue
            avg_ms = tot_ms / (ngroups * 2)
            ach = b * n ** 3 / (avg_ms / 1e3) / 1e9
            roof[name] = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                          "avg_ms": round(avg_ms, 4), "frac": round(ach / peak, 4)}
    what = ("no surface" if wall is None else
            "an immersed rigid wall across the box at y = 0.1213 (plate of 2,048 triangles)")
    return {"workload": "stretched128: 128^3 channel, tanh-stretched wall-normal cells (beta 1.8), " + what + ", "
                        "body-force driven from a seeded random field; Re=200, dt=5e-4, RK2+CN, "
                        + ("FP64" if precision == "fp64" else "mixed (FP32 bulk, (hi, lo) velocity, correction solve)"),
            "cells": n ** 3, "steps": K, "value": whole_job_gcups(n ** 3, K, world, ms), "unit": UNIT,
            "ms_per_step": ms / K, "slip_l1": slip if wall is not None else None,
            "stages_ms_per_step": {k: v[0] / 2 for k, v in prof.items() if v[1] > 0},
            "div_max_U_per_hmin": dg["div_max"] * hmin,
            **({"correction": correction_record(args, dg, 2 * K, hmin)} if precision == "mixed" else {}),
            **({"stage_roofline": roof} if roof else {})}


def large_leg(args, dev, stream, flush):
    """The two large synthetic workloads of the metric's family -- the
    256x192x256 channel with 16 moving bodies and the 512x384x512 tube with
    three hinged leaflets -- on the mixed path, same protocol as the headline
    (device-resident surfaces, L2 flushed between timed steps, autotuned
    launch shapes), with the stage times and the device's own divergence
    residual.  The tube also runs the FP64 path on the same inputs and steps,
    and reports the largest difference of the mixed fields from it (velocity
    over U_ref, pressure over U_ref^2).  The tube's pulsatile body force is
    held at its t = 0 value (the rate does not depend on it)."""
    import torch
    from paper_2606_09799_gb300 import ibm, inputs

    out = {}
    W, K = 3, max(3, min(args.steps, 6))
    for name in ("channel256", "leaflet512"):
        wl = inputs.workload(name)
        surf = [wl.surface(s) for s in range(W + K)]
        dx = [torch.from_numpy(x).to(dev) for x, _ in surf]
        dv = [torch.from_numpy(v).to(dev) for _, v in surf]
        cells = wl.nx * wl.ny * wl.nz
        precs = ("mixed", "fp64") if name == "leaflet512" else ("mixed",)
        res = {}
        fields = {}
        for prec in precs:
            sim = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=prec,
                                 stream=stream.cuda_stream)
            if wl.initial is not None:
                sim.set_fields(*wl.initial())
            ibm.ibm_set_body_force(sim.h, *wl.body_force_at(0.0))
            set_budget(sim, args, wl.lx / wl.nx)
            sim.set_surface(surf[0][0], surf[0][1], wl.tri)
            for s in range(W):
                sim.set_surface(dx[s], dv[s])
                sim.step(1)
            sim.sync()
            tune = sim.autotune(steps=2) if prec == "mixed" else None   # state saved and restored
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            corr0 = sim.diag()["corr_solves"]
            torch.cuda.synchronize()
            for n in range(K):
                flush.fill_(n & 0xFF)
                ev[n][0].record(stream)
                sim.set_surface(dx[W + n], dv[W + n])
                sim.step(1)
                ev[n][1].record(stream)
            torch.cuda.synchronize()
            ms = sum(a.elapsed_time(b) for a, b in ev) / K
            d = sim.diag()
            r = {"precision": prec, "cells": cells, "triangles": int(wl.tri.shape[0]), "steps": K, "warmup": W,
                 "ms_per_step": ms, "value": cells / (ms / 1e3) / 1e9, "unit": UNIT, "slip_l1": d["slip_l1"],
                 "div_max_U_per_dx": d["div_max"] * wl.lx / wl.nx, "cfl": d["cfl"]}
            if prec == "mixed":
                d["corr_timed"] = d["corr_solves"] - corr0
                r["correction"] = correction_record(args, d, 2 * K, wl.lx / wl.nx)
            if len(precs) > 1:
                # the state after the same W + K steps on both paths
                shp = [(wl.nz, wl.ny, wl.nx), (wl.nz, wl.ny + 1, wl.nx), (wl.nz, wl.ny, wl.nx), (wl.nz, wl.ny, wl.nx)]
                f = tuple(torch.empty(sh, dtype=torch.float64, device=dev) for sh in shp)
                ibm.ibm_get_fields(sim.h, wl.nx, wl.ny, wl.nz, out=f)
                fields[prec] = f
            if prec == "mixed":
                prof = ibm.ibm_profile_stages(sim.h, 2)   # two more steps, after the fields were taken
                r["tune"] = tune
                r["stages_ms_per_step"] = {k: v[0] / 2 for k, v in prof.items() if v[1] > 0}
            sim.close()
            res[prec] = r
        entry = dict(res["mixed"])
        if "fp64" in res:
            fm, ff = fields["mixed"], fields["fp64"]
            entry["fp64_gpu"] = res["fp64"]
            entry["vs_fp64_gpu"] = {
                "max_abs_du": max(float((a - b).abs().max()) for a, b in zip(fm[:3], ff[:3])),
                "max_abs_dp": float((fm[3] - ff[3]).abs().max()),
                "max_abs_u": max(float(b.abs().max()) for b in ff[:3]),
                "after_steps": W + K,
                "slip_rel_diff": (abs(res["mixed"]["slip_l1"] - res["fp64"]["slip_l1"]) / res["fp64"]["slip_l1"]
                                  if res["fp64"]["slip_l1"] else None)}
            del fm, ff
        fields.clear()
        out[name] = entry
        del dx, dv
        torch.cuda.empty_cache()
    return out


def cpu_baseline_extra():
    """The oracle's other timings: one thread on the 64^3 oscillating sphere
    (all 10 steps), and all host cores on the 256x192x256 channel with 16
    bodies (2 whole steps) and on the 512x384x512 leaflet tube (1 whole
    step), reported as cell updates/s."""
    from oracle import oracle as orc
    from oracle.oracle import OracleSim
    from paper_2606_09799_gb300 import inputs
    out = {}
    wl = inputs.oscillating_sphere()
    ncores = orc.threads()
    orc.set_threads(1)
    try:
        sim = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
        t0 = time.perf_counter()
        for s in range(10):
            xyz, vel = wl.surface(s)
            sim.set_surface(xyz, vel, wl.tri)
            sim.step()
        dt = time.perf_counter() - t0
    finally:
        orc.set_threads(ncores)
    out["sphere64_one_thread"] = {"value": wl.cells * 10 / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                  "sample": "10 whole time steps of the 64^3 oscillating sphere (FP64)",
                                  "seconds": dt}
    wl = inputs.workload("channel256")
    sim = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
    if wl.initial is not None:
        sim.set_fields(*wl.initial())
    sim.set_body_force(*wl.body_force_at(0.0))
    t0 = time.perf_counter()
    for s in range(2):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
    dt = time.perf_counter() - t0
    cells = wl.nx * wl.ny * wl.nz
    out["channel256"] = {"value": cells * 2 / dt / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": "2 whole time steps of the 256x192x256 channel with 16 moving bodies (FP64)",
                         "seconds_per_step": dt / 2}
    del sim
    # the 512x384x512 tube: one whole step (about 18 GB of host memory and
    # half a minute on 16 cores)
    wl = inputs.workload("leaflet512")
    sim = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
    if wl.initial is not None:
        sim.set_fields(*wl.initial())
    sim.set_body_force(*wl.body_force_at(0.0))
    t0 = time.perf_counter()
    xyz, vel = wl.surface(0)
    sim.set_surface(xyz, vel, wl.tri)
    sim.step()
    dt = time.perf_counter() - t0
    cells = wl.nx * wl.ny * wl.nz
    out["leaflet512"] = {"value": cells / dt / 1e9, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": "1 whole time step of the 512x384x512 tube with three leaflets (FP64)",
                         "seconds_per_step": dt}
    del sim
    return out


def max_over_ranks(ms: float, device, world: int) -> float:
    """The slowest rank's time (every rank gets it): the whole job's timed
    region ends when the last replica finishes."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gcups(cells_per_rank: int, steps: int, world: int, ms_max: float) -> float:
    """Cell updates of all ranks' replicas over the slowest rank's time (weak
    scaling: every rank advances its own copy of the workload)."""
    return world * cells_per_rank * steps / (ms_max / 1e3) / 1e9


def batched_leg(args, dev, stream, flush, world):
    """The uneven batch (32 instances, sizes from {32, 48, 64, 96}^3, FP32
    bulk): GCUPS of the batched step (one launch per kernel for all
    instances, one graph per step) against the same instances stepped one
    by one; each step's surfaces are uploaded from device-resident arrays
    inside the timed region in both cases."""
    import torch
    from paper_2606_09799_gb300 import ibm, inputs

    K, W = max(3, min(args.steps, args.batch_steps)), max(3, args.warmup)
    wls = inputs.batched_instances(steps=W + K)
    cells = sum(w.cells for w in wls)
    surf = [[w.surface(s) for s in range(W + K)] for w in wls]
    dsurf = [[(torch.from_numpy(x).to(dev), torch.from_numpy(v).to(dev)) for x, v in ss] for ss in surf]

    def make():
        sims = []
        for w, ss in zip(wls, surf):
            g = ibm.Simulation(w.nx, w.ny, w.nz, w.lx, w.ly, w.lz, re=w.re, dt=w.dt, precision="mixed",
                               stream=stream.cuda_stream)
            set_budget(g, args, w.lx / w.nx)
            g.set_surface(ss[0][0], ss[0][1], w.tri)
            sims.append(g)
        return sims

    def timed(sims, step_all):
        for s in range(W):
            for g, ds in zip(sims, dsurf):
                g.set_surface(*ds[s])
            step_all()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        with ClockSampler(dist_env()[2]) as clk:
            for n in range(K):
                flush.fill_(n & 0xFF)
                ev[n][0].record(stream)
                for g, ds in zip(sims, dsurf):
                    g.set_surface(*ds[W + n])
                step_all()
                ev[n][1].record(stream)
            torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev), clk.summary()

    sims = make()
    b = ibm.Batch(sims, stream=stream.cuda_stream)
    for g, ds in zip(sims, dsurf):
        g.set_surface(*ds[0])
    tune = b.autotune(steps=2) if args.autotune else None
    ms_b, clk_b = timed(sims, lambda: b.step(1))
    b.sync()
    info = b.info()
    prof = b.profile_stages(1)
    slip = sum(g.diag()["slip_l1"] for g in sims) / len(sims)
    b.close()
    for g in sims:
        g.close()
    sims = make()
    ms_s, clk_s = timed(sims, lambda: [g.step(1) for g in sims])
    for g in sims:
        g.sync()
        g.close()
    return {"workload": f"batch32: {len(wls)} instances, nx, ny, nz each from {{32,48,64,96}} (seed 4), "
                        f"one sphere/cube/disc each (500-5000 triangles) translating sinusoidally; "
                        f"Re in [50,500]; FP32 bulk", "instances": len(wls), "cells": cells,
            "steps": K, "warmup": W, "value": world * cells * K / (ms_b / 1e3) / 1e9, "unit": UNIT,
            "ms_per_step": ms_b / K, "solo_value": world * cells * K / (ms_s / 1e3) / 1e9,
            "solo_ms_per_step": ms_s / K, "speedup_vs_solo": ms_s / ms_b,
            "launches_per_step": info["launches_per_step"], "launches_per_step_solo": info["launches_per_step_solo"],
            "tune": tune, "slip_l1_mean": slip, "clocks": clk_b, "clocks_solo": clk_s,
            "stages_ms_per_step": {k: v[0] for k, v in prof.items() if v[1] > 0}}


def e5_leg(args, dev, stream):
    """No-slip error time series of the heaving and pitching plate (Section
    4.4 geometry, 100 x 650 x 100): ||eps||_1 every step on the mixed and
    the FP64 paths, for context beside the paper's ~1e-4 U_ref over one
    period.  Opt-in (--e5-steps N)."""
    from paper_2606_09799_gb300 import ibm, inputs

    wl = inputs.heaving_pitching_plate(steps=args.e5_steps)
    out = {"workload": "heaving/pitching plate of Section 4.4: 100x650x100 cells on 2x13x2, plate side 1 "
                       "(50x50 quads), B=6, w=1/6, theta=(pi/6) sin(2wt), Re=100, dt=%g" % wl.dt,
           "paper": "||eps||_1 of order 1e-4 U over one period (Fig. heaving_plate)"}
    for prec, nsteps in (("mixed", args.e5_steps), ("fp64", min(args.e5_steps, 500))):
        g = ibm.Simulation(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt, precision=prec,
                           stream=stream.cuda_stream)
        series = []
        t0 = time.perf_counter()
        for s in range(nsteps):
            xyz, vel = wl.surface(s)
            g.set_surface(xyz, vel, wl.tri if s == 0 else None)
            g.step()
            series.append(g.diag()["slip_l1"])
        wall = time.perf_counter() - t0
        g.close()
        arr = [x for x in series[10:]] or series
        out[prec] = {"steps": nsteps, "t_end": nsteps * wl.dt, "slip_mean": sum(arr) / len(arr),
                     "slip_max": max(arr), "series_every_10": series[::10], "wall_s": wall}
    return out


def cpu_baseline(nsteps: int):
    """The FP64 CPU oracle as it stands, on a bounded sample of the same
    workload: its first `nsteps` whole time steps."""
    from oracle.oracle import OracleSim, threads
    from paper_2606_09799_gb300 import inputs
    wl = inputs.heaving_plate()
    sim = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
    t0 = time.perf_counter()
    for s in range(nsteps):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
    dt = time.perf_counter() - t0
    return {"value": wl.cells * nsteps / dt / 1e9, "unit": UNIT, "cores": threads(), "kind": "oracle",
            "sample": f"first {nsteps} whole time steps of the 128^3 plate workload (FP64, OpenMP loops)",
            "seconds": dt}


def reference_arm(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    from oracle.oracle import OracleSim, threads
    from paper_2606_09799_gb300 import inputs
    wl = inputs.heaving_plate()
    sim = OracleSim(wl.nx, wl.ny, wl.nz, wl.lx, wl.ly, wl.lz, re=wl.re, dt=wl.dt)
    for s in range(args.warmup):
        xyz, vel = wl.surface(s)
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
    times = []
    for n in range(args.steps):
        xyz, vel = wl.surface(args.warmup + n)
        t0 = time.perf_counter()
        sim.set_surface(xyz, vel, wl.tri)
        sim.step()
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = wl.cells * args.steps / total / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": wl.cells, "triangles": int(wl.tri.shape[0]),
                   "precision": "fp64", "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads(), "kind": "oracle",
                         "sample": f"{args.steps} whole time steps of the 128^3 plate workload after "
                                   f"{args.warmup} warm-up steps"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "slip_l1": sim.last.get("slip"),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"],
                    help="headline path: mixed (FP32 bulk, FP64 tagging, tridiagonal and correction) or fp64")
    ap.add_argument("--only-headline", action="store_true", help="skip the other precision's run")
    ap.add_argument("--profile-steps", type=int, default=5)
    ap.add_argument("--cpu-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the built-in launch shapes (no autotuning before timing)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances leg")
    ap.add_argument("--no-ab", action="store_true", help="skip the AB+CN leg")
    ap.add_argument("--no-stretched", action="store_true", help="skip the non-uniform wall-normal grid leg")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 256x192x256 channel and 512x384x512 tube leg (and the oracle's extra timings)")
    ap.add_argument("--e5-steps", type=int, default=0,
                    help="also record the no-slip error series of the heaving/pitching plate (opt-in)")
    ap.add_argument("--tune", default="", help="fixed launch shapes instead of autotuning, e.g. tri_y=3,sweep_zy=2")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--div-budget", type=float, default=1e-7,
                    help="mixed path: correction-solve budget on max |D u - q| in U_ref/dx, by default the "
                         "1e-7 bound the mixed path must meet (0: always correct)")
    ap.add_argument("--fp64-peak-tflops", type=float, default=0.0,
                    help="FP64 roof in TFLOP/s; 0 (default) measures it on the device (ibm_measure_alu_peaks)")
    args = ap.parse_args()
    args.tune = {k: int(v) for k, v in (kv.split("=") for kv in args.tune.split(",") if kv)}
    args.fp32_peak_tflops = None
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    line = reference_arm(args) if args.impl == "reference" else gpu_arm(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
