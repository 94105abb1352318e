"""Thin ctypes binding of the C ABI in include/ibm.h.

Every function below has the name of the C entry point it calls and does
argument marshalling only (numpy arrays or torch tensors in, status codes to
exceptions out).  All computation runs in the CUDA library
libibm_gb300.so; there is no Python or CPU fallback: if the library cannot
be loaded, every call raises.

Fields are FP64 arrays in C order [k][j][i]: u, w, p of shape (nz, ny, nx),
v of shape (nz, ny + 1, nx).  Surfaces are (nv, 3) FP64 vertex positions and
velocities and (nt, 3) int32 triangles.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

from . import build as _build

_LIB = None
_LOCK = threading.Lock()

IBM_RK2_CN, IBM_AB_CN = 0, 1
IBM_NOSLIP, IBM_FREESLIP = 0, 1
IBM_FP64, IBM_MIXED, IBM_MIXED_FAST = 0, 1, 2

STATUS = {0: "IBM_OK", 1: "IBM_ERR_ARG", 2: "IBM_ERR_CUDA", 3: "IBM_ERR_OOM", 4: "IBM_ERR_GEOMETRY",
          5: "IBM_ERR_DIVERGED", 6: "IBM_ERR_TIMEOUT", 7: "IBM_ERR_STATE", 8: "IBM_ERR_CAPACITY"}


class IbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ibm_grid_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("re", ctypes.c_double), ("dt", ctypes.c_double),
                ("scheme", ctypes.c_int), ("ybc", ctypes.c_int), ("precision", ctypes.c_int),
                ("use_q", ctypes.c_int)]


class ibm_diag(ctypes.Structure):
    _fields_ = [("slip_l1", ctypes.c_double), ("slip_comp", ctypes.c_double * 3),
                ("nforce", ctypes.c_int64 * 3), ("nboundary", ctypes.c_int64),
                ("q_f", ctypes.c_double), ("sum_q_dv", ctypes.c_double), ("steps", ctypes.c_int64),
                ("ncandidates", ctypes.c_int64), ("kernels_per_step", ctypes.c_int64),
                ("d2h_bytes", ctypes.c_int64), ("div_max", ctypes.c_double), ("ke", ctypes.c_double),
                ("cfl", ctypes.c_double), ("div_first", ctypes.c_double), ("corr_solves", ctypes.c_int64)]

IBM_NSTAGES = 19


class ibm_tune(ctypes.Structure):
    _fields_ = [("tri_y", ctypes.c_int), ("sweep_w", ctypes.c_int), ("fft_lpb", ctypes.c_int),
                ("fft_cols", ctypes.c_int), ("sweep_zy", ctypes.c_int), ("fft_plane", ctypes.c_int),
                ("sweep_y", ctypes.c_int), ("rhs", ctypes.c_int), ("corr_check", ctypes.c_int),
                ("ms_per_step", ctypes.c_double)]


class ibm_batch_info(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int64), ("cells", ctypes.c_int64), ("launches_per_step", ctypes.c_int64),
                ("launches_per_step_solo", ctypes.c_int64), ("shape", ctypes.c_int32 * 3)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

EXPORTS = ("ibm_create_grid", "ibm_destroy", "ibm_set_surface", "ibm_set_body_force", "ibm_set_fields",
           "ibm_step", "ibm_get_fields", "ibm_get_tags", "ibm_get_diag", "ibm_sync", "ibm_last_error",
           "ibm_set_allocator", "ibm_version", "ibm_profile_stages", "ibm_stage_name", "ibm_tag_noalloc",
           "ibm_set_tune", "ibm_get_tune", "ibm_autotune", "ibm_batch_create", "ibm_batch_destroy",
           "ibm_batch_step", "ibm_batch_sync", "ibm_batch_get_info", "ibm_batch_profile_stages",
           "ibm_batch_set_tune", "ibm_batch_autotune", "ibm_batch_last_error", "ibm_step_batch",
           "ibm_get_loads", "ibm_get_pressure_recon", "ibm_check_conversions", "ibm_create_grid_stretched", "ibm_check_bounded_wait",
           "ibm_get_history", "ibm_set_history", "ibm_measure_alu_peaks", "ibm_set_div_budget")


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libibm_gb300.so (building it in-tree first when it is missing
    or stale).  Raises if it cannot be built or loaded."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        if build_if_needed and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"CUDA library {_build.LIB} is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(_build.LIB)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.ibm_create_grid.argtypes = [ctypes.POINTER(ibm_grid_desc), P, ctypes.POINTER(P)]
        L.ibm_destroy.argtypes = [P]
        L.ibm_set_surface.argtypes = [P, I, P, P, I, P, I]
        L.ibm_set_body_force.argtypes = [P, D, D, D]
        L.ibm_set_div_budget.argtypes = [P, D]
        L.ibm_set_fields.argtypes = [P, P, P, P, P, I]
        L.ibm_step.argtypes = [P, I]
        L.ibm_get_fields.argtypes = [P, P, P, P, P, I]
        L.ibm_get_history.argtypes = [P, P, P, P, I]
        L.ibm_set_history.argtypes = [P, P, P, P, I]
        L.ibm_get_tags.argtypes = [P, I, P, I]
        L.ibm_get_diag.argtypes = [P, ctypes.POINTER(ibm_diag)]
        L.ibm_sync.argtypes = [P]
        L.ibm_last_error.argtypes = [P]
        L.ibm_last_error.restype = ctypes.c_char_p
        L.ibm_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
        L.ibm_version.restype = ctypes.c_char_p
        L.ibm_profile_stages.argtypes = [P, I, P, P]
        L.ibm_stage_name.argtypes = [I]
        L.ibm_tag_noalloc.argtypes = [ctypes.POINTER(ibm_grid_desc), I, P, I, P, P, P, P, P]
        L.ibm_stage_name.restype = ctypes.c_char_p
        L.ibm_set_tune.argtypes = [P, ctypes.POINTER(ibm_tune)]
        L.ibm_get_tune.argtypes = [P, ctypes.POINTER(ibm_tune)]
        L.ibm_autotune.argtypes = [P, I, ctypes.POINTER(ibm_tune)]
        L.ibm_batch_create.argtypes = [P, I, P, ctypes.POINTER(P)]
        L.ibm_batch_destroy.argtypes = [P]
        L.ibm_batch_step.argtypes = [P, I]
        L.ibm_batch_sync.argtypes = [P]
        L.ibm_batch_get_info.argtypes = [P, ctypes.POINTER(ibm_batch_info)]
        L.ibm_batch_profile_stages.argtypes = [P, I, P, P]
        L.ibm_batch_set_tune.argtypes = [P, ctypes.POINTER(ibm_tune)]
        L.ibm_batch_autotune.argtypes = [P, I, ctypes.POINTER(ibm_tune)]
        L.ibm_batch_last_error.argtypes = [P]
        L.ibm_batch_last_error.restype = ctypes.c_char_p
        L.ibm_step_batch.argtypes = [P, I, I]
        L.ibm_get_loads.argtypes = [P, I, P, P, P, P, P]
        L.ibm_get_pressure_recon.argtypes = [P, P, I]
        L.ibm_create_grid_stretched.argtypes = [ctypes.POINTER(ibm_grid_desc), P, P, ctypes.POINTER(P)]
        L.ibm_check_bounded_wait.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_longlong)]
        L.ibm_check_bounded_wait.restype = ctypes.c_int
        L.ibm_measure_alu_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.ibm_check_conversions.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong),
                                            ctypes.POINTER(ctypes.c_longlong)]
        for name in EXPORTS:
            if name not in ("ibm_last_error", "ibm_version", "ibm_stage_name", "ibm_batch_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(h, status: int):
    if status != 0:
        msg = load().ibm_last_error(h).decode() if h else ""
        raise IbmError(status, msg)


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return 0


# ---------------------------------------------------------------------------
# C entry points
# ---------------------------------------------------------------------------
def ibm_create_grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, re=100.0, dt=1e-3, scheme=IBM_RK2_CN, ybc=IBM_NOSLIP,
                    precision=IBM_FP64, use_q=1, stream=None, y_faces=None):
    """y_faces: None (uniform wall-normal spacing) or ny + 1 face positions
    (ibm_create_grid_stretched)."""
    L = load()
    d = ibm_grid_desc(nx, ny, nz, lx, ly, lz, re, dt, scheme, ybc, precision, int(use_q))
    h = ctypes.c_void_p()
    if y_faces is None:
        _check(None, L.ibm_create_grid(ctypes.byref(d), _stream_handle(stream), ctypes.byref(h)))
    else:
        yf = np.ascontiguousarray(y_faces, dtype=np.float64)
        if yf.shape != (ny + 1,):
            raise ValueError("y_faces: ny + 1 face positions")
        _check(None, L.ibm_create_grid_stretched(ctypes.byref(d), yf.ctypes.data_as(ctypes.c_void_p),
                                                 _stream_handle(stream), ctypes.byref(h)))
    return h.value


def ibm_destroy(h):
    _check(h, load().ibm_destroy(h))


def ibm_set_surface(h, xyz, vel, tri=None, ntris=None):
    """xyz, vel: (nv, 3) FP64; tri: (nt, 3) int32, or None to keep the
    previous connectivity (then ntris must be given)."""
    xp, xd = _ptr(xyz)
    vp, vd = _ptr(vel)
    tp, td = _ptr(tri)
    if xd != vd or (tri is not None and td != xd):
        raise ValueError("xyz, vel and tri must all live on the host or all on the device")
    nt = int(tri.shape[0]) if tri is not None else int(ntris)
    _check(h, load().ibm_set_surface(h, int(xyz.shape[0]), xp, vp, nt, tp, xd))


def ibm_set_surface_raw(h, nverts, xyz_ptr, vel_ptr, ntris, tri_ptr, on_device):
    _check(h, load().ibm_set_surface(h, int(nverts), xyz_ptr, vel_ptr, int(ntris), tri_ptr, int(on_device)))


def ibm_set_body_force(h, fx, fy, fz):
    _check(h, load().ibm_set_body_force(h, float(fx), float(fy), float(fz)))


def ibm_set_div_budget(h, budget):
    _check(h, load().ibm_set_div_budget(h, float(budget)))


def ibm_set_fields(h, u=None, v=None, w=None, p=None):
    ptrs = [_ptr(a) for a in (u, v, w, p)]
    dev = {d for (q, d) in ptrs if q is not None}
    if len(dev) > 1:
        raise ValueError("fields must all live on the host or all on the device")
    _check(h, load().ibm_set_fields(h, *[q for q, _ in ptrs], dev.pop() if dev else 0))


def ibm_step(h, nsteps=1):
    _check(h, load().ibm_step(h, int(nsteps)))


def ibm_get_fields(h, nx, ny, nz, out=None):
    """Returns (u, v, w, p) as FP64 numpy arrays (or fills `out`, a tuple of
    four contiguous FP64 arrays or device tensors)."""
    if out is None:
        out = (np.empty((nz, ny, nx)), np.empty((nz, ny + 1, nx)), np.empty((nz, ny, nx)), np.empty((nz, ny, nx)))
    ptrs = [_ptr(a) for a in out]
    _check(h, load().ibm_get_fields(h, *[q for q, _ in ptrs], ptrs[0][1]))
    return out


def ibm_get_history(h, nx, ny, nz, out=None):
    """Returns the non-linear history (hu, hv, hw) of AB+CN as FP64 arrays
    (or fills `out`, three contiguous FP64 arrays or device tensors)."""
    if out is None:
        out = (np.empty((nz, ny, nx)), np.empty((nz, ny + 1, nx)), np.empty((nz, ny, nx)))
    ptrs = [_ptr(a) for a in out]
    _check(h, load().ibm_get_history(h, *[q for q, _ in ptrs], ptrs[0][1]))
    return out


def ibm_set_history(h, hu=None, hv=None, hw=None):
    ptrs = [_ptr(a) for a in (hu, hv, hw)]
    dev = {d for (q, d) in ptrs if q is not None}
    if len(dev) > 1:
        raise ValueError("history arrays must all live on the host or all on the device")
    _check(h, load().ibm_set_history(h, *[q for q, _ in ptrs], dev.pop() if dev else 0))


def ibm_get_tags(h, comp, shape):
    owner = np.empty(shape, dtype=np.int32)
    _check(h, load().ibm_get_tags(h, int(comp), owner.ctypes.data, 0))
    return owner


def ibm_get_diag(h) -> dict:
    d = ibm_diag()
    _check(h, load().ibm_get_diag(h, ctypes.byref(d)))
    return {"slip_l1": d.slip_l1, "slip_comp": list(d.slip_comp), "nforce": list(d.nforce),
            "nboundary": d.nboundary, "q_f": d.q_f, "sum_q_dv": d.sum_q_dv, "steps": d.steps,
            "ncandidates": d.ncandidates, "kernels_per_step": d.kernels_per_step, "d2h_bytes": d.d2h_bytes,
            "div_max": d.div_max, "ke": d.ke, "cfl": d.cfl, "div_first": d.div_first,
            "corr_solves": d.corr_solves}


def ibm_profile_stages(h, nsteps=1) -> dict:
    """{stage name: (device ms summed over nsteps, kernels per step)}."""
    ms = (ctypes.c_double * IBM_NSTAGES)()
    kn = (ctypes.c_int64 * IBM_NSTAGES)()
    _check(h, load().ibm_profile_stages(h, int(nsteps), ms, kn))
    return {ibm_stage_name(i): (ms[i], kn[i]) for i in range(IBM_NSTAGES)}


IBM_NOALLOC_MAX_NODES = 1048576


def ibm_tag_noalloc(nx, ny, nz, xyz, tri, owners, lx=1.0, ly=1.0, lz=1.0, ybc=IBM_NOSLIP, stream=None):
    """Tags of one surface without any device allocation by the library (for
    callers that must not allocate at that point).  xyz: (nv, 3) FP64 and
    tri: (nt, 3) int32 device tensors; owners: three int32 device tensors of
    the u, v, w field shapes, overwritten.  Returns the status code."""
    d = ibm_grid_desc(nx, ny, nz, lx, ly, lz, 1.0, 1.0, IBM_RK2_CN, ybc, IBM_FP64, 1)
    ptrs = [_ptr(a) for a in (xyz, tri) + tuple(owners)]
    if any(dev != 1 for _, dev in ptrs):
        raise ValueError("ibm_tag_noalloc takes device arrays only")
    return load().ibm_tag_noalloc(ctypes.byref(d), int(xyz.shape[0]), ptrs[0][0], int(tri.shape[0]), ptrs[1][0],
                                  ptrs[2][0], ptrs[3][0], ptrs[4][0], _stream_handle(stream))


def _tune_dict(t: ibm_tune) -> dict:
    return {"tri_y": t.tri_y, "sweep_w": t.sweep_w, "fft_lpb": t.fft_lpb, "fft_cols": t.fft_cols,
            "sweep_zy": t.sweep_zy, "fft_plane": t.fft_plane, "sweep_y": t.sweep_y, "rhs": t.rhs,
            "corr_check": t.corr_check, "ms_per_step": t.ms_per_step}


def ibm_set_tune(h, tri_y=0, sweep_w=0, fft_lpb=0, fft_cols=0, sweep_zy=0, fft_plane=0, sweep_y=0, rhs=0,
                 corr_check=0):
    _check(h, load().ibm_set_tune(h, ctypes.byref(ibm_tune(tri_y, sweep_w, fft_lpb, fft_cols, sweep_zy, fft_plane,
                                                           sweep_y, rhs, corr_check, 0.0))))


def ibm_get_tune(h) -> dict:
    t = ibm_tune()
    _check(h, load().ibm_get_tune(h, ctypes.byref(t)))
    return _tune_dict(t)


def ibm_autotune(h, steps=3) -> dict:
    t = ibm_tune()
    _check(h, load().ibm_autotune(h, int(steps), ctypes.byref(t)))
    return _tune_dict(t)


def _bcheck(b, status: int):
    if status != 0:
        msg = load().ibm_batch_last_error(b).decode() if b else ""
        raise IbmError(status, msg)


def _handles(hs):
    arr = (ctypes.c_void_p * len(hs))(*hs)
    return arr


def ibm_batch_create(hs, stream=None):
    b = ctypes.c_void_p()
    _check(hs[0] if hs else None, load().ibm_batch_create(_handles(hs), len(hs), _stream_handle(stream),
                                                          ctypes.byref(b)))
    return b.value


def ibm_batch_destroy(b):
    _bcheck(b, load().ibm_batch_destroy(b))


def ibm_batch_step(b, nsteps=1):
    _bcheck(b, load().ibm_batch_step(b, int(nsteps)))


def ibm_batch_sync(b):
    _bcheck(b, load().ibm_batch_sync(b))


def ibm_batch_get_info(b) -> dict:
    i = ibm_batch_info()
    _bcheck(b, load().ibm_batch_get_info(b, ctypes.byref(i)))
    return {"instances": i.instances, "cells": i.cells, "launches_per_step": i.launches_per_step,
            "launches_per_step_solo": i.launches_per_step_solo, "shape": list(i.shape)}


def ibm_batch_profile_stages(b, nsteps=1) -> dict:
    ms = (ctypes.c_double * IBM_NSTAGES)()
    kn = (ctypes.c_int64 * IBM_NSTAGES)()
    _bcheck(b, load().ibm_batch_profile_stages(b, int(nsteps), ms, kn))
    return {ibm_stage_name(i): (ms[i], kn[i]) for i in range(IBM_NSTAGES)}


def ibm_batch_set_tune(b, tri_y=0, sweep_w=0, fft_lpb=0, fft_cols=0, sweep_zy=0, fft_plane=0, sweep_y=0, rhs=0,
                       corr_check=0):
    _bcheck(b, load().ibm_batch_set_tune(b, ctypes.byref(ibm_tune(tri_y, sweep_w, fft_lpb, fft_cols, sweep_zy,
                                                                   fft_plane, sweep_y, rhs, corr_check, 0.0))))


def ibm_batch_autotune(b, steps=3) -> dict:
    t = ibm_tune()
    _bcheck(b, load().ibm_batch_autotune(b, int(steps), ctypes.byref(t)))
    return _tune_dict(t)


def ibm_batch_last_error(b) -> str:
    return load().ibm_batch_last_error(b).decode()


def ibm_step_batch(hs, nsteps=1):
    _check(hs[0], load().ibm_step_batch(_handles(hs), len(hs), int(nsteps)))


def ibm_get_loads(h, nt, sides=1, pole=(0.0, 0.0, 0.0)):
    """(force (3,), torque (3,), per-triangle force and torque (nt, 6),
    wall pressure (nt,)) from the current step (Section 3.3)."""
    F, M = np.zeros(3), np.zeros(3)
    tr, pw = np.zeros((nt, 6)), np.zeros(nt)
    pl = np.ascontiguousarray(pole, dtype=np.float64)
    _check(h, load().ibm_get_loads(h, int(sides), pl.ctypes.data, F.ctypes.data, M.ctypes.data,
                                   tr.ctypes.data, pw.ctypes.data))
    return F, M, tr, pw


def ibm_measure_alu_peaks() -> tuple:
    """(FP64, FP32) fused multiply-add throughput of the current device in
    TFLOP/s (FMA = 2 flops)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    st = load().ibm_measure_alu_peaks(ctypes.byref(a), ctypes.byref(b))
    if st != 0:
        raise IbmError(st, "ibm_measure_alu_peaks failed")
    return a.value, b.value


def ibm_check_conversions(n: int) -> tuple:
    """(mismatches, checked) of the integer-path FP32 <-> FP64 conversions
    against the hardware conversions on n hashed cases."""
    bad, fast = ctypes.c_longlong(0), ctypes.c_longlong(0)
    st = load().ibm_check_conversions(int(n), ctypes.byref(bad), ctypes.byref(fast))
    if st != 0:
        raise IbmError(st, "ibm_check_conversions failed")
    return bad.value, fast.value


def ibm_check_bounded_wait(limit_cycles: int) -> tuple:
    """(timed_out, waited_cycles) of a bounded mbarrier wait that cannot
    complete (ibm_check_bounded_wait)."""
    t, c = ctypes.c_int(0), ctypes.c_longlong(0)
    st = load().ibm_check_bounded_wait(int(limit_cycles), ctypes.byref(t), ctypes.byref(c))
    if st != 0:
        raise IbmError(st, "ibm_check_bounded_wait failed")
    return t.value, c.value


def ibm_get_pressure_recon(h, nx, ny, nz):
    p = np.empty((nz, ny, nx))
    _check(h, load().ibm_get_pressure_recon(h, p.ctypes.data, 0))
    return p


def ibm_stage_name(i) -> str:
    return load().ibm_stage_name(int(i)).decode()


def ibm_sync(h):
    _check(h, load().ibm_sync(h))


def ibm_last_error(h) -> str:
    return load().ibm_last_error(h).decode()


def ibm_version() -> str:
    return load().ibm_version().decode()


_TORCH_HOOK = None


def ibm_set_allocator_torch():
    """Route the library's device allocations through PyTorch's caching
    allocator (on the current device and stream)."""
    global _TORCH_HOOK
    import torch

    def _alloc(nbytes, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes)))
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _TORCH_HOOK = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(None, load().ibm_set_allocator(_TORCH_HOOK[0], _TORCH_HOOK[1], None))


def ibm_reset_allocator():
    global _TORCH_HOOK
    _check(None, load().ibm_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _TORCH_HOOK = None


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Simulation:
    """One simulation instance (a handle) with numpy-friendly accessors."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, re=100.0, dt=1e-3, scheme="rk2", ybc=0,
                 precision="fp64", use_q=True, stream=None, y_faces=None):
        self.shape = (nx, ny, nz)
        self.precision = precision
        sch = IBM_AB_CN if scheme == "ab" else IBM_RK2_CN
        prec = {"fp64": IBM_FP64, "mixed": IBM_MIXED, "mixed_fast": IBM_MIXED_FAST}[precision]
        self.h = ibm_create_grid(nx, ny, nz, lx, ly, lz, re, dt, sch, ybc, prec, int(use_q), stream, y_faces)
        self.nt = 0

    def close(self):
        if self.h:
            ibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_surface(self, xyz, vel, tri=None):
        if tri is not None:
            self.nt = int(tri.shape[0])
            ibm_set_surface(self.h, xyz, vel, tri)
        else:
            ibm_set_surface(self.h, xyz, vel, None, self.nt)

    def set_body_force(self, fx, fy, fz):
        ibm_set_body_force(self.h, fx, fy, fz)

    def set_div_budget(self, budget):
        ibm_set_div_budget(self.h, budget)

    def set_fields(self, u=None, v=None, w=None, p=None):
        ibm_set_fields(self.h, u, v, w, p)

    def step(self, n=1):
        ibm_step(self.h, n)

    def fields(self):
        nx, ny, nz = self.shape
        return ibm_get_fields(self.h, nx, ny, nz)

    def history(self):
        nx, ny, nz = self.shape
        return ibm_get_history(self.h, nx, ny, nz)

    def set_history(self, hu=None, hv=None, hw=None):
        ibm_set_history(self.h, hu, hv, hw)

    def tags(self):
        nx, ny, nz = self.shape
        return [ibm_get_tags(self.h, c, (nz, ny + 1 if c == 1 else ny, nx)) for c in range(3)]

    def diag(self):
        return ibm_get_diag(self.h)

    def sync(self):
        ibm_sync(self.h)

    def autotune(self, steps=3):
        return ibm_autotune(self.h, steps)

    def loads(self, sides=1, pole=(0.0, 0.0, 0.0)):
        return ibm_get_loads(self.h, self.nt, sides, pole)

    def pressure_recon(self):
        nx, ny, nz = self.shape
        return ibm_get_pressure_recon(self.h, nx, ny, nz)

    def set_tune(self, **kw):
        ibm_set_tune(self.h, **kw)


class Batch:
    """Independent simulations advanced together: one launch per kernel of
    the step for all of them (ibm_batch_*)."""

    def __init__(self, sims, stream=None):
        self.sims = list(sims)
        self.b = ibm_batch_create([s.h for s in self.sims], stream)

    def close(self):
        if self.b:
            ibm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        ibm_batch_step(self.b, n)

    def sync(self):
        ibm_batch_sync(self.b)

    def info(self):
        return ibm_batch_get_info(self.b)

    def profile_stages(self, nsteps=1):
        return ibm_batch_profile_stages(self.b, nsteps)

    def autotune(self, steps=3):
        return ibm_batch_autotune(self.b, steps)

    def set_tune(self, **kw):
        ibm_batch_set_tune(self.b, **kw)
