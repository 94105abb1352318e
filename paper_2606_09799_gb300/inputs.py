"""Seeded synthetic inputs: triangulated bodies, prescribed kinematics and
initial fields for the sharp-interface IBM fractional step.

This module holds none of the method's arithmetic: it only builds surfaces,
their vertex velocities and starting fields.  It is the one module shared by
the CUDA path's tests and benchmark and the CPU oracle's tests, so both see
bit-identical inputs.

Workloads (x and z periodic, walls at y = 0 and y = ly, U_ref = L_ref = 1):

  sphere64  64^3 cells on the unit cube; rigid icosphere (golden-ratio
            icosahedron, 3 midpoint subdivisions, 1,280 triangles) of
            diameter 0.25 centred mid-box, x_c = 0.5 + 0.1 sin(2 pi t);
            Re = 100, dt = 1e-3, 10 steps, fluid at rest.
  plate128  128^3 cells on the unit cube; zero-thickness square plate of
            side 0.4 in the x-z plane at y = 0.5, 64 x 64 quads split into
            8,192 triangles, heaving 0.05 sin(2 pi t) plus the bending mode
            0.02 sin(pi s) sin(2 pi t), s = (x - 0.3)/0.4; Re = 200,
            dt = 5e-4, 100 steps, fluid at rest.
  batch32   32 independent instances advanced together: each of nx, ny, nz
            drawn from {32, 48, 64, 96} (PCG64 seed 4), unit cube; one body
            per instance -- icosphere (1,280 triangles), cube (12 n^2
            triangles, n in 7..20) or zero-thickness disc (500-5,000
            triangles) of size 0.24-0.4 centred mid-box -- translating with
            a seeded sinusoid per axis (amplitude <= 0.05, frequency
            0.5-2); Re uniform in [50, 500], dt = 0.2 dx_min / (1 + U_max),
            200 steps, fluid at rest.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional, Tuple

import numpy as np

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# surface generators
# ---------------------------------------------------------------------------
def icosphere(subdiv: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> Tuple[np.ndarray, np.ndarray]:
    """Golden-ratio icosahedron refined `subdiv` times by edge midpoints,
    every vertex pushed onto the sphere.  20 * 4**subdiv triangles, outward
    counter-clockwise orientation."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    V = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    xyz = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(np.array(faces, dtype=np.int32))


def plate(nq: int, side: float, x0: float, z0: float, y0: float) -> Tuple[np.ndarray, np.ndarray]:
    """Zero-thickness square plate in the x-z plane at height y0, corner at
    (x0, y0, z0), nq x nq quads, each split into two triangles."""
    s = np.linspace(0.0, 1.0, nq + 1)
    X, Z = np.meshgrid(x0 + side * s, z0 + side * s, indexing="xy")    # [iz][ix]
    xyz = np.stack([X.ravel(), np.full(X.size, y0), Z.ravel()], axis=1)
    tris = []
    for iz in range(nq):
        for ix in range(nq):
            a = iz * (nq + 1) + ix
            b, c, d = a + 1, a + (nq + 1), a + (nq + 1) + 1
            tris.append((a, b, d))
            tris.append((a, d, c))
    return np.ascontiguousarray(xyz), np.ascontiguousarray(np.array(tris, dtype=np.int32))


def cube(n: int, side: float, center) -> Tuple[np.ndarray, np.ndarray]:
    """Closed cube surface, each face n x n quads split into two triangles
    (12 n^2 triangles; vertices on shared edges are duplicated per face,
    which Algorithm 1 does not mind)."""
    s = np.linspace(-0.5, 0.5, n + 1) * side
    A, B = np.meshgrid(s, s, indexing="ij")
    a, b = A.ravel(), B.ravel()
    h = np.full(a.size, 0.5 * side)
    faces = [np.stack([h, a, b], 1), np.stack([-h, a, b], 1), np.stack([a, h, b], 1),
             np.stack([a, -h, b], 1), np.stack([a, b, h], 1), np.stack([a, b, -h], 1)]
    xyz, tris = [], []
    for f, pts in enumerate(faces):
        base = f * (n + 1) ** 2
        xyz.append(pts)
        for i in range(n):
            for j in range(n):
                q = base + i * (n + 1) + j
                tris.append((q, q + n + 1, q + n + 2))
                tris.append((q, q + n + 2, q + 1))
    xyz = np.concatenate(xyz) + np.asarray(center, dtype=np.float64)
    return np.ascontiguousarray(xyz), np.ascontiguousarray(np.array(tris, dtype=np.int32))


def disc(nr: int, nth: int, radius: float, center) -> Tuple[np.ndarray, np.ndarray]:
    """Zero-thickness disc in the x-z plane through `center`: nr rings of nth
    vertices around the centre vertex (nth + 2 nth (nr - 1) triangles)."""
    cx, cy, cz = center
    pts = [(cx, cy, cz)]
    for r in range(1, nr + 1):
        rad = radius * r / nr
        for k in range(nth):
            th = TWO_PI * k / nth
            pts.append((cx + rad * math.cos(th), cy, cz + rad * math.sin(th)))
    tris = []
    for k in range(nth):
        tris.append((0, 1 + k, 1 + (k + 1) % nth))
    for r in range(1, nr):
        i0, i1 = 1 + (r - 1) * nth, 1 + r * nth
        for k in range(nth):
            k1 = (k + 1) % nth
            tris.append((i0 + k, i1 + k, i1 + k1))
            tris.append((i0 + k, i1 + k1, i0 + k1))
    return np.ascontiguousarray(np.array(pts, dtype=np.float64)), np.ascontiguousarray(np.array(tris, dtype=np.int32))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    lx: float
    ly: float
    lz: float
    re: float
    dt: float
    steps: int
    tri: np.ndarray                                            # (nt, 3) int32
    surface_at: Callable[[float], Tuple[np.ndarray, np.ndarray]]  # t -> (xyz, vel)
    body_force_at: Callable[[float], Tuple[float, float, float]] = lambda t: (0.0, 0.0, 0.0)
    initial: Optional[Callable[[], Tuple[np.ndarray, ...]]] = None
    scheme: str = "rk2"

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def surface(self, step: int):
        return self.surface_at(step * self.dt)

    def initial_fields(self):
        if self.initial is not None:
            return self.initial()
        nx, ny, nz = self.nx, self.ny, self.nz
        return (np.zeros((nz, ny, nx)), np.zeros((nz, ny + 1, nx)), np.zeros((nz, ny, nx)),
                np.zeros((nz, ny, nx)))


def oscillating_sphere(n: int = 64, steps: int = 10, subdiv: int = 3) -> Workload:
    """Rigid sphere d = 0.25 oscillating in x with amplitude 0.1, period 1."""
    xyz0, tri = icosphere(subdiv, 0.125, (0.5, 0.5, 0.5))

    def surface_at(t):
        dx = 0.1 * math.sin(TWO_PI * t)
        ux = 0.1 * TWO_PI * math.cos(TWO_PI * t)
        xyz = xyz0.copy()
        xyz[:, 0] += dx
        vel = np.zeros_like(xyz)
        vel[:, 0] = ux
        return xyz, vel

    return Workload(f"sphere{n}", n, n, n, 1.0, 1.0, 1.0, 100.0, 1e-3, steps, tri, surface_at)


def heaving_plate(n: int = 128, steps: int = 100, nq: int = 64) -> Workload:
    """Zero-thickness plate (side 0.4) heaving 0.05 sin(2 pi t) with the
    bending mode 0.02 sin(pi s) sin(2 pi t), s = (x - 0.3)/0.4."""
    xyz0, tri = plate(nq, 0.4, 0.3, 0.3, 0.5)
    s = (xyz0[:, 0] - 0.3) / 0.4
    bend = np.sin(math.pi * s)

    def surface_at(t):
        st, ct = math.sin(TWO_PI * t), math.cos(TWO_PI * t)
        xyz = xyz0.copy()
        xyz[:, 1] = 0.5 + 0.05 * st + 0.02 * bend * st
        vel = np.zeros_like(xyz)
        vel[:, 1] = 0.05 * TWO_PI * ct + 0.02 * TWO_PI * bend * ct
        return xyz, vel

    return Workload(f"plate{n}", n, n, n, 1.0, 1.0, 1.0, 200.0, 5e-4, steps, tri, surface_at)


def translating(name, nx, ny, nz, re, dt, steps, xyz0, tri, amp, freq, phase) -> Workload:
    """Rigid body translating with x_c(t) = x_c0 + amp sin(2 pi freq t + phase)
    per axis (vertex velocity = the translation velocity)."""
    amp, freq, phase = (np.asarray(v, dtype=np.float64) for v in (amp, freq, phase))

    def surface_at(t):
        arg = TWO_PI * freq * t + phase
        xyz = xyz0 + (amp * (np.sin(arg) - np.sin(phase)))[None, :]
        vel = np.broadcast_to(amp * TWO_PI * freq * np.cos(arg), xyz0.shape).copy()
        return np.ascontiguousarray(xyz), np.ascontiguousarray(vel)

    return Workload(name, nx, ny, nz, 1.0, 1.0, 1.0, re, dt, steps, tri, surface_at)


def batched_instances(count: int = 32, seed: int = 4, steps: int = 200,
                      sizes=(32, 48, 64, 96)) -> List[Workload]:
    """The uneven batch: per instance nx, ny, nz from `sizes`, one body
    (sphere, cube or thin disc, 500-5,000 triangles) on seeded sinusoidal
    translation, Re in [50, 500], dt = 0.2 dx_min / (1 + U_max)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny, nz = (int(v) for v in rng.choice(sizes, size=3))
        kind = int(rng.integers(0, 3))
        size = float(rng.uniform(0.24, 0.4))
        c = (0.5, 0.5, 0.5)
        if kind == 0:
            xyz, tri = icosphere(3, size / 2, c)
        elif kind == 1:
            xyz, tri = cube(int(rng.integers(7, 21)), size, c)
        else:
            nth = int(rng.integers(24, 65))
            nr = int(rng.integers(max(2, 260 // nth + 1), 2500 // nth + 1))
            xyz, tri = disc(nr, nth, size / 2, c)
        amp = rng.uniform(0.0, 0.05, 3)
        freq = rng.uniform(0.5, 2.0, 3)
        phase = rng.uniform(0.0, TWO_PI, 3)
        re = float(rng.uniform(50.0, 500.0))
        umax = float(np.linalg.norm(amp * TWO_PI * freq))
        dt = 0.2 * (1.0 / max(nx, ny, nz)) / (1.0 + umax)
        out.append(translating(f"batch{i}", nx, ny, nz, re, dt, steps, xyz, tri, amp, freq, phase))
    return out


def random_fields(nx: int, ny: int, nz: int, seed: int, amp: float = 1.0):
    """Seeded smooth-ish random velocity and pressure fields (v = 0 on the
    walls) for stage-level parity tests."""
    rng = np.random.default_rng(seed)
    u = amp * rng.standard_normal((nz, ny, nx))
    v = amp * rng.standard_normal((nz, ny + 1, nx))
    v[:, 0, :] = 0.0
    v[:, ny, :] = 0.0
    w = amp * rng.standard_normal((nz, ny, nx))
    p = amp * rng.standard_normal((nz, ny, nx))
    return u, v, w, p


def random_triangles(n: int, seed: int, lo=0.3, hi=0.7, size: float = 0.15):
    """Seeded random (disjoint-vertex) triangles inside [lo, hi]^3."""
    rng = np.random.default_rng(seed)
    cen = rng.uniform(lo, hi, size=(n, 3))
    xyz = (cen[:, None, :] + rng.uniform(-size / 2, size / 2, size=(n, 3, 3))).reshape(-1, 3)
    tri = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return np.ascontiguousarray(xyz), tri


WORKLOADS = {
    "sphere64": oscillating_sphere,
    "plate128": heaving_plate,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
