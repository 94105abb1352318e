"""Plain FP64 CPU oracle of the sharp-interface IBM fractional step.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the product path.  It
shares no code with the CUDA library; the two meet only through the data
format (arrays [k][j][i], i fastest) and the seeded input generators.

The time step follows the paper's order (Section 2 and Section 3):

  once per step   Algorithm 1 tagging of the three staggered grids
  per sub-stage   IB step on the forcing nodes (Eqs. IB_step, probe, new_IB)
                  explicit right-hand side of Eq. NS_prov
                  approximate factorisation: x, then z, then y sweeps
                  divergence, boundary cells and q (Eqs. q_boundary, q_F)
                  Poisson solve of Eq. elliptic_mod: FFT in x and z
                  (numpy.fft, the one library step), Thomas in y
                  projection (Eq. projection), pressure (Eq. update_pressure)
  after the step  no-slip error on the forcing points (Section 4.4)

The C kernels live in ibm_oracle.c; this module compiles it on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ibm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libibm_oracle.so")
_LIB = None
_LOCK = threading.Lock()

RK2_CN = "rk2"
AB_CN = "ab"
# (gamma, rho, alpha) per sub-stage, Section 2 after Eq. NS_prov
SCHEMES = {
    RK2_CN: ((0.5, 0.0, 0.5), (1.0, -0.5, 0.5)),
    AB_CN: ((1.5, -0.5, 1.0),),
}


def build(force: bool = False) -> str:
    """Compile ibm_oracle.c into a shared library (no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ybc", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("yf", ctypes.c_void_p)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_GP = ctypes.POINTER(Grid)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = ctypes.CDLL(_SO)
            L.orc_threads.restype = _I
            L.orc_set_threads.argtypes = [_I]
            L.orc_grid_init.argtypes = [_GP, _I, _I, _I, _D, _D, _D, _I]
            L.orc_closest_point.argtypes = [_P] * 6
            L.orc_tag_alg1.argtypes = [_GP, _I, _P, _I, _P, _P, _P]
            L.orc_tag_brute.argtypes = [_GP, _I, _P, _I, _P, _P, _P]
            L.orc_tag_alg1_window.argtypes = [_GP, _I, _P, _I, _P, ctypes.c_long, ctypes.c_long, _P, _P]
            L.orc_q_energy.argtypes = [_GP, _P, _P, _P, _P, _P, _P, _P, _P]
            L.orc_loads.argtypes = [_GP, _P, _I, _P, _P, _P, _P, _P, _P, _D, _I, _P, _P, _P, _P, _P]
            L.orc_pressure_recon.argtypes = [_GP, _P, _P, _P, _P, _P, _P]
            L.orc_force.argtypes = [_GP, _I, _P, _P, _P, _P, _P, _P, _D]
            L.orc_force.restype = _I
            L.orc_slip.argtypes = [_GP, _I, _P, _P, _P, _P, _P, _D, _P, _P]
            L.orc_slip.restype = _I
            L.orc_rhs.argtypes = [_GP] + [_P] * 10 + [_D] * 5 + [_P] * 7
            L.orc_sweep.argtypes = [_GP, _I, _I, _P, _P, _D]
            L.orc_divergence.argtypes = [_GP, _P, _P, _P, _P]
            L.orc_boundary_cells.argtypes = [_GP, _P, _P, _P, _P]
            L.orc_rhs_poisson.argtypes = [_GP, _P, _P, _I, _D, _P, _P, _P]
            L.orc_rhs_poisson.restype = _D
            L.orc_poisson_y.argtypes = [_GP, _P]
            L.orc_lap_c.argtypes = [_GP, _P, _P]
            L.orc_project.argtypes = [_GP, _P, _P, _P, _P, _P, _P, _D, _D]
            _LIB = L
    return _LIB


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on."""
    lib().orc_set_threads(int(n))


def make_grid(nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, ybc=0, yfaces=None) -> Grid:
    """yfaces: ny + 1 increasing wall-normal face positions from 0 to ly
    (Section 2: variable cell size in the wall-normal direction), or None
    for uniform spacing."""
    g = Grid()
    lib().orc_grid_init(ctypes.byref(g), nx, ny, nz, lx, ly, lz, ybc)
    if yfaces is not None:
        yf = np.ascontiguousarray(yfaces, dtype=np.float64)
        if yf.shape != (ny + 1,) or yf[0] != 0.0 or not np.all(np.diff(yf) > 0) or abs(yf[-1] - ly) > 1e-12 * ly:
            raise ValueError("yfaces: ny + 1 increasing positions from 0 to ly")
        g._yf_array = yf          # the grid holds the array its pointer refers to
        g.yf = yf.ctypes.data
    return g


def field_shape(g: Grid, c: int):
    return (g.nz, g.ny + 1 if c == 1 else g.ny, g.nx)


def closest_point(p, a, b, c):
    """Closest point X on triangle (a,b,c) to p and its barycentric weights."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (p, a, b, c)]
    X = np.zeros(3)
    w = np.zeros(3)
    lib().orc_closest_point(*[_p(x) for x in arrs], _p(X), _p(w))
    return X, w


def tag(g: Grid, xyz: np.ndarray, tri: np.ndarray, brute: bool = False):
    """Algorithm 1 on the three staggered grids.  Returns (owner, d2) lists;
    owner = -1 on fluid nodes, else the owning triangle index."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    owners, d2s = [], []
    fn = lib().orc_tag_brute if brute else lib().orc_tag_alg1
    for c in range(3):
        own = np.full(field_shape(g, c), -1, dtype=np.int32)
        d2 = np.full(field_shape(g, c), np.inf)
        fn(ctypes.byref(g), c, _p(xyz), int(tri.shape[0]), _p(tri), _p(own), _p(d2))
        owners.append(own)
        d2s.append(d2)
    return owners, d2s


def tag_window(g: Grid, xyz: np.ndarray, tri: np.ndarray, i0: int, ni: int):
    """Algorithm 1 owners of the nodes with x index in [i0, i0 + ni), per
    component, as arrays [k][j][i - i0] (for grids too large to tag whole)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    owners = []
    for c in range(3):
        shape = (g.nz, g.ny + 1 if c == 1 else g.ny, ni)
        own = np.full(shape, -1, dtype=np.int32)
        d2 = np.full(shape, np.inf)
        lib().orc_tag_alg1_window(ctypes.byref(g), c, _p(xyz), int(tri.shape[0]), _p(tri), int(i0), int(ni),
                                  _p(own), _p(d2))
        owners.append(own)
    return owners


def boundary_cells(g: Grid, owners):
    isb = np.zeros((g.nz, g.ny, g.nx), dtype=np.uint8)
    lib().orc_boundary_cells(ctypes.byref(g), _p(owners[0]), _p(owners[1]), _p(owners[2]), _p(isb))
    return isb


def divergence(g: Grid, u, v, w):
    d = np.zeros((g.nz, g.ny, g.nx))
    lib().orc_divergence(ctypes.byref(g), _p(u), _p(v), _p(w), _p(d))
    return d


def lap_c(g: Grid, phi):
    out = np.zeros_like(phi)
    lib().orc_lap_c(ctypes.byref(g), _p(phi), _p(out))
    return out


def poisson(g: Grid, rhs: np.ndarray) -> np.ndarray:
    """Solve L_c phi = rhs (Eq. elliptic): FFT in x and z, Thomas in y per
    mode, zero-mean gauge."""
    spec = np.ascontiguousarray(np.fft.rfft2(rhs, axes=(0, 2)))
    buf = spec.view(np.float64)
    lib().orc_poisson_y(ctypes.byref(g), _p(buf))
    return np.ascontiguousarray(np.fft.irfft2(spec, s=(g.nz, g.nx), axes=(0, 2)))


def sweep(g: Grid, c: int, direction: int, f: np.ndarray, owner: np.ndarray, beta: float):
    lib().orc_sweep(ctypes.byref(g), c, direction, _p(f), _p(owner), beta)


def no_tags(g: Grid):
    return [np.full(field_shape(g, c), -1, dtype=np.int32) for c in range(3)]


def rhs(g: Grid, u, v, w, p, owners, gam, rho, alp, dt, re, fb=(0.0, 0.0, 0.0), Hprev=None):
    """Explicit right-hand side of Eq. NS_prov; returns (R, H) lists."""
    if Hprev is None:
        Hprev = [np.zeros(field_shape(g, c)) for c in range(3)]
    fb = np.ascontiguousarray(fb, dtype=np.float64)
    R = [np.zeros(field_shape(g, c)) for c in range(3)]
    H = [np.zeros(field_shape(g, c)) for c in range(3)]
    lib().orc_rhs(ctypes.byref(g), _p(u), _p(v), _p(w), _p(p), _p(Hprev[0]), _p(Hprev[1]), _p(Hprev[2]),
                  _p(owners[0]), _p(owners[1]), _p(owners[2]), gam, rho, alp, dt, re, _p(fb),
                  _p(R[0]), _p(R[1]), _p(R[2]), _p(H[0]), _p(H[1]), _p(H[2]))
    return R, H


def force(g: Grid, c, src, dst, owner, xyz, vel, tri, h):
    """Eq. new_IB on the forcing nodes of component c (dst updated in place)."""
    bad = lib().orc_force(ctypes.byref(g), c, _p(src), _p(dst), _p(owner),
                          _p(np.ascontiguousarray(xyz, dtype=np.float64)),
                          _p(np.ascontiguousarray(vel, dtype=np.float64)),
                          _p(np.ascontiguousarray(tri, dtype=np.int32)), h)
    return int(bad)


def rhs_poisson(g: Grid, div, isb, use_q, adt):
    out = np.zeros_like(div)
    A = ctypes.c_double()
    VF = ctypes.c_double()
    qF = lib().orc_rhs_poisson(ctypes.byref(g), _p(div), _p(isb), int(use_q), adt, _p(out),
                               ctypes.byref(A), ctypes.byref(VF))
    return out, qF, A.value, VF.value


def q_energy(g: Grid, div, isb, p, u, v, w):
    """Energy- and mass-conserving q (App. B): (q field, (alpha, beta, A, B,
    S0, S1, S2))."""
    q = np.zeros_like(div)
    coef = np.zeros(7)
    lib().orc_q_energy(ctypes.byref(g), _p(div), _p(isb), _p(p), _p(u), _p(v), _p(w), _p(q), _p(coef))
    return q, coef


def loads(g: Grid, xyz, tri, u, v, w, p, isb, re, sides=1, pole=(0.0, 0.0, 0.0)):
    """Hydrodynamic loads of Section 3.3 (MLS probes at the centroids):
    (per-triangle force and torque (nt, 6), wall pressure (nt,), F, M)."""
    if g.yf:
        raise ValueError("loads: the MLS probes are written for a uniform grid")
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    isb = np.ascontiguousarray(isb, dtype=np.uint8)
    tr = np.zeros((tri.shape[0], 6))
    pw = np.zeros(tri.shape[0])
    F, M = np.zeros(3), np.zeros(3)
    pole = np.ascontiguousarray(pole, dtype=np.float64)
    lib().orc_loads(ctypes.byref(g), _p(xyz), int(tri.shape[0]), _p(tri), _p(u), _p(v), _p(w), _p(p), _p(isb),
                    float(re), int(sides), _p(pole), _p(tr), _p(pw), _p(F), _p(M))
    return tr, pw, F, M


def pressure_recon(g: Grid, p, isb, owners, xyz, tri):
    """p with the boundary cells given the value at their probe point
    (Section 3.2, post-processing)."""
    if g.yf:
        raise ValueError("pressure_recon: the probes are written for a uniform grid")
    q = np.zeros_like(p)
    lib().orc_pressure_recon(ctypes.byref(g), _p(p), _p(np.ascontiguousarray(isb, dtype=np.uint8)),
                             _p(np.ascontiguousarray(owners[0], dtype=np.int32)),
                             _p(np.ascontiguousarray(xyz, dtype=np.float64)),
                             _p(np.ascontiguousarray(tri, dtype=np.int32)), _p(q))
    return q


def row_heights(g: Grid):
    """Wall-normal cell heights h_c(j) (ny) and centre distances across the
    faces h_f(j) (ny; face j = 0 is the wall, measured to the mirror image of
    the first centre) of the grid, uniform or not."""
    if g.yf:
        yf = g._yf_array
        hc = np.diff(yf)
        yc = 0.5 * (yf[:-1] + yf[1:])
        hf = np.empty(g.ny)
        hf[0] = 2.0 * yc[0]
        hf[1:] = np.diff(yc)
        return hc, hf
    return np.full(g.ny, g.dy), np.full(g.ny, g.dy)


def state_diagnostics(g: Grid, u, v, w, q, fluid, dt):
    """Diagnostics of a velocity state (no counterpart in the method's
    steps; they measure its result):
      div_max = max over the cells where `fluid` holds of |D u - q|, the
                residual of Eq. mod_div (the projected field has D u = q);
      ke      = 1/2 sum over the velocity nodes of the three grids of
                u^2 dV, dV the node's control volume (dx h dz, h the cell
                height for u and w, the distance of the centres for v; the
                wall planes of v hold no unknown and are left out);
      cfl     = dt max over the cells of |u_c|/dx + |v_c|/h + |w_c|/dz with
                u_c the mean of the cell's two faces of each component.
    q: scalar or per-cell array; fluid: boolean mask of the cells (nz, ny, nx)."""
    hc, hf = row_heights(g)
    div = divergence(g, u, v, w)
    r = np.abs(div - q)
    div_max = float(r[fluid].max()) if np.any(fluid) else 0.0
    hcb = hc[None, :, None]
    ke = 0.5 * g.dx * g.dz * (np.sum(u * u * hcb) + np.sum(v[:, :g.ny, :] ** 2 * hf[None, :, None])
                               + np.sum(w * w * hcb))
    uc = 0.5 * np.abs(u + np.roll(u, -1, axis=2))
    vc = 0.5 * np.abs(v[:, :-1, :] + v[:, 1:, :])
    wc = 0.5 * np.abs(w + np.roll(w, -1, axis=0))
    cfl = dt * float(np.max(uc / g.dx + vc / hcb + wc / g.dz))
    return div_max, float(ke), cfl


def project(g: Grid, u, v, w, p, phi, adt, re):
    lp = lap_c(g, phi)
    lib().orc_project(ctypes.byref(g), _p(u), _p(v), _p(w), _p(p), _p(phi), _p(lp), adt, re)


class OracleSim:
    """One simulation instance advanced by the plain FP64 oracle."""

    def __init__(self, nx, ny, nz, lx=1.0, ly=1.0, lz=1.0, re=100.0, dt=1e-3, scheme=RK2_CN, ybc=0,
                 use_q=True, yfaces=None):
        self.g = make_grid(nx, ny, nz, lx, ly, lz, ybc, yfaces)
        self.nonuniform = yfaces is not None
        # use_q: 0 none, 1 uniform q_F (Eq. for q_F, mass only), 2 energy- and mass-conserving shape (App. B)
        self.re, self.dt, self.scheme, self.use_q = float(re), float(dt), scheme, int(use_q)
        g = self.g
        self.u = np.zeros(field_shape(g, 0))
        self.v = np.zeros(field_shape(g, 1))
        self.w = np.zeros(field_shape(g, 2))
        self.p = np.zeros((nz, ny, nx))
        self.H = [np.zeros(field_shape(g, c)) for c in range(3)]
        self.fb = np.zeros(3)
        self.xyz = np.zeros((0, 3))
        self.vel = np.zeros((0, 3))
        self.tri = np.zeros((0, 3), dtype=np.int32)
        diag = np.sqrt((g.dx * g.dx + g.dy * g.dy) + g.dz * g.dz)
        self.h = 2.0 * diag                     # probe length, Section 3.1
        self.owners = None
        self.last = {}
        self.nsteps = 0

    # -- inputs ----------------------------------------------------------
    def set_fields(self, u, v, w, p):
        self.u[...] = u
        self.v[...] = v
        self.w[...] = w
        self.p[...] = p

    def set_surface(self, xyz, vel, tri):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        self.vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
        self.tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)

    def set_body_force(self, fx, fy, fz):
        self.fb = np.array([fx, fy, fz], dtype=np.float64)

    def fields(self):
        return self.u, self.v, self.w, self.p

    # -- stages ----------------------------------------------------------
    def _tag(self):
        if self.tri.shape[0] == 0:
            self.owners = [np.full(field_shape(self.g, c), -1, dtype=np.int32) for c in range(3)]
        else:
            self.owners, _ = tag(self.g, self.xyz, self.tri)
        self.isb = boundary_cells(self.g, self.owners)

    def _force(self):
        L, g = lib(), self.g
        flds = [self.u, self.v, self.w]
        snaps = [f.copy() for f in flds]          # u^e always from the snapshot of u^s
        for c in range(3):
            bad = L.orc_force(ctypes.byref(g), c, _p(snaps[c]), _p(flds[c]), _p(self.owners[c]),
                              _p(self.xyz), _p(self.vel), _p(self.tri), self.h)
            if bad:
                raise RuntimeError(f"{bad} IB probes of component {c} left the domain")

    def _substage(self, gam, rho, alp):
        L, g = lib(), self.g
        dt, re = self.dt, self.re
        if self.tri.shape[0]:
            self._force()
        R = [np.zeros(field_shape(g, c)) for c in range(3)]
        Hn = [np.zeros(field_shape(g, c)) for c in range(3)]
        L.orc_rhs(ctypes.byref(g), _p(self.u), _p(self.v), _p(self.w), _p(self.p),
                  _p(self.H[0]), _p(self.H[1]), _p(self.H[2]),
                  _p(self.owners[0]), _p(self.owners[1]), _p(self.owners[2]),
                  gam, rho, alp, dt, re, _p(self.fb), _p(R[0]), _p(R[1]), _p(R[2]),
                  _p(Hn[0]), _p(Hn[1]), _p(Hn[2]))
        beta = alp * dt / (2.0 * re)
        for c in range(3):
            for d in (0, 2, 1):
                sweep(g, c, d, R[c], self.owners[c], beta)
        self.u += R[0]
        self.v += R[1]
        self.w += R[2]
        adt = alp * dt
        div = divergence(g, self.u, self.v, self.w)
        rhs = np.zeros_like(div)
        A = ctypes.c_double()
        VF = ctypes.c_double()
        qF = L.orc_rhs_poisson(ctypes.byref(g), _p(div), _p(self.isb), min(self.use_q, 1), adt, _p(rhs),
                               ctypes.byref(A), ctypes.byref(VF))
        if self.use_q == 2:
            qk, coef = q_energy(g, div, self.isb, self.p, self.u, self.v, self.w)
            rhs = (div - qk) / adt
            qF = coef[0]
            self.last.update(q_field=qk, q_coef=coef)
        phi = poisson(g, rhs)
        lp = lap_c(g, phi)
        L.orc_project(ctypes.byref(g), _p(self.u), _p(self.v), _p(self.w), _p(self.p), _p(phi), _p(lp), adt, re)
        self.H = Hn
        self.last.update(qF=qF, A=A.value, VF=VF.value, phi=phi, rhs=rhs, div_hat=div)

    def slip(self):
        """||eps||_1 = sum_i ||eps_i||_1 / 3, ||eps_i||_1 = mean |eps_i| over
        the forcing points of component i (Section 4.4)."""
        L, g = lib(), self.g
        tot, per = 0.0, []
        for c, f in enumerate((self.u, self.v, self.w)):
            s = ctypes.c_double()
            n = ctypes.c_long()
            bad = L.orc_slip(ctypes.byref(g), c, _p(f), _p(self.owners[c]), _p(self.xyz), _p(self.vel),
                             _p(self.tri), self.h, ctypes.byref(s), ctypes.byref(n))
            if bad:
                raise RuntimeError("slip probe left the domain")
            m = s.value / n.value if n.value else 0.0
            per.append((m, n.value))
            tot += m
        return tot / 3.0, per

    def diagnostics(self):
        """(max |D u - q| over C_F, kinetic energy, CFL) of the current state
        with the last sub-stage's q: q_F (uniform shape) or the per-cell
        shape of App. B on the fluid cells; without q, D u = 0 on every cell."""
        if self.use_q == 2:
            q = self.last["q_field"]
        elif self.use_q:
            q = self.last.get("qF", 0.0)
        else:
            q = 0.0
        fluid = (self.isb == 0) if self.use_q else np.ones((self.g.nz, self.g.ny, self.g.nx), dtype=bool)
        return state_diagnostics(self.g, self.u, self.v, self.w, q, fluid, self.dt)

    def step(self, n: int = 1):
        for _ in range(n):
            self._tag()
            for (gam, rho, alp) in SCHEMES[self.scheme]:
                self._substage(gam, rho, alp)
            self.nsteps += 1
            self.last["div_max"], self.last["ke"], self.last["cfl"] = self.diagnostics()
            if self.tri.shape[0]:
                self.last["slip"], self.last["slip_per_comp"] = self.slip()
        return self
