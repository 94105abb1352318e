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
  channel256  256 x 192 x 256 cells on 4/3 x 1 x 4/3, 16 moving bodies of
            mixed thickness (spheres, capped cylinders, zero-thickness
            plates; ~125,000 triangles) in a perturbed Poiseuille flow,
            Re_b = 5600 (see multibody_channel).
  leaflet512  512 x 384 x 512 cells (~100M), a finite-thickness tube with
            three zero-thickness leaflets opening and closing periodically,
            182,800 triangles, pulsatile forcing, Re = 1000 (see
            leaflet_tube).
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


def capped_cylinder(n_around, n_along, radius, length, center, axis):
    """Closed cylinder (hemispherical caps) of the given axis direction."""
    axis = np.asarray(axis, float)
    axis /= np.linalg.norm(axis)
    # orthonormal frame
    t = np.array([1.0, 0, 0]) if abs(axis[0]) < 0.9 else np.array([0, 1.0, 0])
    e1 = np.cross(axis, t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    pts, tris = [], []
    th = TWO_PI * np.arange(n_around) / n_around
    ring = np.stack([np.cos(th), np.sin(th)], 1)
    ncap = max(2, n_around // 8)
    # rings: cap A (from pole), body, cap B
    rings = []
    for k in range(1, ncap + 1):
        phi = (math.pi / 2) * k / ncap
        rings.append((-length / 2 - radius * math.cos(phi), radius * math.sin(phi)))
    for k in range(1, n_along):
        rings.append((-length / 2 + length * k / n_along, radius))
    for k in range(ncap, 0, -1):
        phi = (math.pi / 2) * k / ncap
        rings.append((length / 2 + radius * math.cos(phi), radius * math.sin(phi)))
    c = np.asarray(center, float)
    pts.append(c + axis * (-length / 2 - radius))
    for (s, r) in rings:
        for q in range(n_around):
            pts.append(c + axis * s + r * (ring[q, 0] * e1 + ring[q, 1] * e2))
    pts.append(c + axis * (length / 2 + radius))
    nr = len(rings)
    for q in range(n_around):
        tris.append((0, 1 + (q + 1) % n_around, 1 + q))
    for k in range(nr - 1):
        a0, b0 = 1 + k * n_around, 1 + (k + 1) * n_around
        for q in range(n_around):
            q1 = (q + 1) % n_around
            tris.append((a0 + q, a0 + q1, b0 + q1))
            tris.append((a0 + q, b0 + q1, b0 + q))
    last = len(pts) - 1
    a0 = 1 + (nr - 1) * n_around
    for q in range(n_around):
        tris.append((a0 + q, a0 + (q + 1) % n_around, last))
    return np.ascontiguousarray(np.array(pts, dtype=np.float64)), np.ascontiguousarray(np.array(tris, dtype=np.int32))


def rot_matrix(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def rigid(xyz0, center, tamp, tfreq, tphase, raxis, ramp, rfreq, rphase):
    """Rigid motion: translation c(t) = c0 + tamp sin(2 pi tfreq t + tphase) - tamp sin(tphase)
    per axis, rotation about raxis through the centre by ramp sin(2 pi rfreq t + rphase)."""
    rel = xyz0 - center
    k = np.asarray(raxis, float) / np.linalg.norm(raxis)

    def at(t):
        arg = TWO_PI * tfreq * t + tphase
        dc = tamp * (np.sin(arg) - np.sin(tphase))
        vc = tamp * TWO_PI * tfreq * np.cos(arg)
        th = ramp * (math.sin(TWO_PI * rfreq * t + rphase) - math.sin(rphase))
        om = ramp * TWO_PI * rfreq * math.cos(TWO_PI * rfreq * t + rphase)
        Rm = rot_matrix(k, th)
        r = rel @ Rm.T
        xyz = center + dc + r
        vel = vc + om * np.cross(k, r)
        return np.ascontiguousarray(xyz), np.ascontiguousarray(vel)
    return at


def tube_surface(radius, nx_rings, n_around, lx, yc, zc, outward=True):
    """Open cylinder along x spanning the periodic length lx: rings at
    x = k lx / nx_rings, k = 0..nx_rings (the last ring is the first one
    shifted by the period, so the surface is continuous across x = 0)."""
    th = TWO_PI * np.arange(n_around) / n_around
    pts = []
    for k in range(nx_rings + 1):
        x = lx * k / nx_rings
        for q in range(n_around):
            pts.append((x, yc + radius * math.cos(th[q]), zc + radius * math.sin(th[q])))
    tris = []
    for k in range(nx_rings):
        a0, b0 = k * n_around, (k + 1) * n_around
        for q in range(n_around):
            q1 = (q + 1) % n_around
            if outward:
                tris.append((a0 + q, a0 + q1, b0 + q1)); tris.append((a0 + q, b0 + q1, b0 + q))
            else:
                tris.append((a0 + q, b0 + q1, a0 + q1)); tris.append((a0 + q, b0 + q, b0 + q1))
    return np.ascontiguousarray(np.array(pts, dtype=np.float64)), np.ascontiguousarray(np.array(tris, dtype=np.int32))


def leaflets(r_in, x0, yc, zc, nr, nphi, theta_max):
    """Three zero-thickness leaflets, each a 120-degree sector of the cross
    section at x0 hinged on the circle r = r_in.  A material point at
    distance s = r_in - rho from its hinge moves to x = x0 + s sin(theta),
    r = r_in - s cos(theta); theta(t) = theta_max (1 - cos 2 pi t) / 2."""
    rho_s, phi_s, tris = [], [], []
    for k in range(3):
        base = len(rho_s)
        rho_s.append(0.0); phi_s.append(0.0)     # apex of this leaflet
        for r in range(1, nr + 1):
            for q in range(nphi + 1):
                rho_s.append(r_in * r / nr)
                phi_s.append(TWO_PI * (k + q / nphi) / 3)
        for q in range(nphi):
            tris.append((base, base + 1 + q, base + 1 + q + 1))
        for r in range(1, nr):
            i0, i1 = base + 1 + (r - 1) * (nphi + 1), base + 1 + r * (nphi + 1)
            for q in range(nphi):
                tris.append((i0 + q, i1 + q, i1 + q + 1)); tris.append((i0 + q, i1 + q + 1, i0 + q + 1))
    rho = np.array(rho_s); phi = np.array(phi_s)
    s = r_in - rho

    def at(t):
        th = theta_max * (1 - math.cos(TWO_PI * t)) / 2
        dth = theta_max * math.pi * math.sin(TWO_PI * t)
        r = r_in - s * math.cos(th)
        xyz = np.stack([x0 + s * math.sin(th), yc + r * np.cos(phi), zc + r * np.sin(phi)], 1)
        dr = s * math.sin(th) * dth
        vel = np.stack([s * math.cos(th) * dth, dr * np.cos(phi), dr * np.sin(phi)], 1)
        return xyz, vel
    return at, np.array(tris, dtype=np.int32)


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


def _concat(parts):
    """Concatenate bodies (surface functions of t and connectivities) into
    one surface; triangle indices are global in body order."""
    tris, offs, off = [], [], 0
    for at, tri in parts:
        n = at(0.0)[0].shape[0]
        tris.append(tri + off)
        offs.append(off)
        off += n
    tri = np.ascontiguousarray(np.concatenate(tris).astype(np.int32))

    def surface_at(t):
        xs, vs = zip(*(at(t) for at, _ in parts))
        return np.ascontiguousarray(np.concatenate(xs)), np.ascontiguousarray(np.concatenate(vs))
    return tri, surface_at


def multibody_channel(steps: int = 100, seed: int = 3) -> Workload:
    """256 x 192 x 256 cells on 4/3 x 1 x 4/3 (cubic cells, dx = 1/192):
    8 icospheres d = 0.1 (4 subdivisions), 4 capped cylinders d = 0.05 of
    length 0.5 (horizontal axes), 4 plates 0.2 x 0.2 (56 x 56 quads) in
    random planes -- about 125,000 triangles -- placed by PCG64 seed 3 with
    their boxes, grown by their motion and by h + 2 dx, disjoint from each
    other (periodic images included) and from the walls; each translating
    (amplitude U[0, 0.02] per axis) and rotating about a random axis
    (amplitude U[0, pi/12]) at one frequency U[0.5, 2].  Flow: Poiseuille
    6y(1-y) plus 5% seeded smooth noise, body force f_x = 12/Re_b,
    Re_b = 5600, dt = 2e-4."""
    nx, ny, nz = 256, 192, 256
    lx = lz = 4.0 / 3.0
    L = np.array([lx, 1.0, lz])
    dl = L / np.array([nx, ny, nz])
    clear = 2 * math.sqrt((dl ** 2).sum()) + 2 * dl.max()
    rng = np.random.default_rng(seed)
    boxes, parts = [], []
    for kind in ["cylinder"] * 4 + ["plate"] * 4 + ["sphere"] * 8:
        if kind == "sphere":
            xyz, tri = icosphere(4, 0.05, (0.0, 0.0, 0.0))
        elif kind == "cylinder":
            ang = rng.uniform(0, math.pi)
            xyz, tri = capped_cylinder(64, 100, 0.025, 0.5, (0.0, 0.0, 0.0), (math.cos(ang), 0.0, math.sin(ang)))
        else:
            xyz, tri = plate(56, 0.2, -0.1, -0.1, 0.0)
            xyz = xyz @ rot_matrix(rng.normal(size=3), rng.uniform(0, math.pi)).T
        tamp = rng.uniform(0, 0.02, 3)
        ramp = rng.uniform(0, math.pi / 12)
        f = rng.uniform(0.5, 2.0)
        raxis = rng.normal(size=3)
        rad = np.linalg.norm(xyz, axis=1).max()
        grow = 2 * tamp + 2 * rad * math.sin(ramp) + clear
        lo0, hi0 = xyz.min(0) - grow, xyz.max(0) + grow
        for _ in range(20000):
            c = rng.uniform(0, 1, 3) * L
            lo, hi = c + lo0, c + hi0
            if lo[1] < 0 or hi[1] > 1:
                continue
            ok = True
            for (l2, h2) in boxes:
                sep = hi[1] <= l2[1] or h2[1] <= lo[1]
                for d in (0, 2):
                    sep = sep or all(hi[d] <= l2[d] + sh or h2[d] + sh <= lo[d] for sh in (-L[d], 0.0, L[d]))
                if not sep:
                    ok = False
                    break
            if ok:
                break
        else:
            raise RuntimeError("body placement failed")
        boxes.append((lo, hi))
        parts.append((rigid(xyz + c, c, tamp, f, rng.uniform(0, TWO_PI, 3), raxis, ramp, f, rng.uniform(0, TWO_PI)),
                      tri))
    tri, surface_at = _concat(parts)
    re_b = 5600.0

    def initial():
        r2 = np.random.default_rng(seed + 100)
        y = (np.arange(ny) + 0.5) / ny
        yv = np.arange(ny + 1) / ny
        xs, zs = (np.arange(nx) + 0.5) / nx * lx, (np.arange(nz) + 0.5) / nz * lz
        Z, Y, X = np.meshgrid(zs, y, xs, indexing="ij")
        noise = np.zeros((3, nz, ny, nx))
        for q in range(3):
            for _ in range(4):
                kx, kz = r2.integers(1, 4, 2)
                ph = r2.uniform(0, TWO_PI, 2)
                noise[q] += (0.05 / 4) * np.sin(math.pi * Y) * np.sin(TWO_PI * kx * X / lx + ph[0]) * \
                    np.cos(TWO_PI * kz * Z / lz + ph[1])
        u = 6.0 * Y * (1.0 - Y) + noise[0]
        w = noise[2]
        v = np.zeros((nz, ny + 1, nx))
        v[:, 1:ny, :] = 0.5 * (noise[1][:, 1:, :] + noise[1][:, :-1, :])
        return u, v, w, np.zeros((nz, ny, nx))

    return Workload("channel256", nx, ny, nz, lx, 1.0, lz, re_b, 2e-4, steps, tri, surface_at,
                    body_force_at=lambda t: (12.0 / re_b, 0.0, 0.0), initial=initial)


def leaflet_tube(steps: int = 50) -> Workload:
    """512 x 384 x 512 cells on 4/3 x 1 x 4/3 (~100M cells): a tube along x
    (inner radius 0.3, wall 0.02: inner and outer surfaces, 160 x 256 quads
    each, continuous across the periodic x boundary) through (y, z) =
    (0.5, 2/3), and three zero-thickness leaflets (120-degree sectors,
    40 x 80 each) at x = 2/3 hinged on the inner radius, opening to
    theta_max (1 - cos 2 pi t)/2 with theta_max = pi/3, period 1: 182,800
    triangles.  Fluid at rest driven by f_x(t) = U'(t) + 8 U(t)/(Re r^2),
    U(t) = 1 + 0.5 sin 2 pi t (the periodic-x reading of a pulsatile
    inflow); Re = 1000, dt = 1e-4."""
    nx, ny, nz = 512, 384, 512
    lx = lz = 4.0 / 3.0
    yc, zc, r_in = 0.5, 2.0 / 3.0, 0.3
    ti, tti = tube_surface(r_in, 160, 256, lx, yc, zc, outward=False)
    to, tto = tube_surface(r_in + 0.02, 160, 256, lx, yc, zc, outward=True)
    lat, ltri = leaflets(r_in, 2.0 / 3.0, yc, zc, 40, 80, math.pi / 3)
    still = lambda xyz: (lambda t: (xyz, np.zeros_like(xyz)))
    tri, surface_at = _concat([(still(ti), tti), (still(to), tto), (lat, ltri)])
    re = 1000.0

    def force(t):
        U = 1.0 + 0.5 * math.sin(TWO_PI * t)
        dU = 0.5 * TWO_PI * math.cos(TWO_PI * t)
        return (dU + 8.0 * U / (re * r_in * r_in), 0.0, 0.0)

    return Workload("leaflet512", nx, ny, nz, lx, 1.0, lz, re, 1e-4, steps, tri, surface_at, body_force_at=force)


def heaving_pitching_plate(steps: int = 2500, dt: float = 2e-3, nq: int = 50) -> Workload:
    """Section 4.4's moving-plate case at the paper's geometry: a square
    zero-thickness plate of side L = 1 in quiescent fluid heaving along the
    wall-normal axis, b(t) = B sin(w t), B = 6, and pitching about the
    spanwise axis, theta(t) = (pi/6) sin(2 w t); U_ref = B w = 1, Re = 100;
    box 2 x 13 x 2 (the paper's [-L, L] x [-L, L] x [-6.5L, 6.5L] with the
    heave axis wall-normal, shifted to start at 0), 100 x 650 x 100 cells,
    dx = 0.02; the plate (nq x nq quads) centred at (1, 6.5, 1) at t = 0.
    dt = 2e-3 (CFL ~0.1): the printed step, 1e-5, would need ~4M steps
    per period."""
    B, om, th0 = 6.0, 1.0 / 6.0, math.pi / 6.0
    xyz0, tri = plate(nq, 1.0, 0.5, 0.5, 6.5)
    X1 = xyz0[:, 0] - 1.0

    def surface_at(t):
        th, dth = th0 * math.sin(2 * om * t), th0 * 2 * om * math.cos(2 * om * t)
        b, db = B * math.sin(om * t), B * om * math.cos(om * t)
        xyz = xyz0.copy()
        xyz[:, 0] = 1.0 + X1 * math.cos(th)
        xyz[:, 1] = 6.5 + b - X1 * math.sin(th)
        vel = np.zeros_like(xyz)
        vel[:, 0] = -X1 * math.sin(th) * dth
        vel[:, 1] = db - X1 * math.cos(th) * dth
        return np.ascontiguousarray(xyz), np.ascontiguousarray(vel)

    return Workload("heaving_plate_e5", 100, 650, 100, 2.0, 13.0, 2.0, 100.0, dt, steps, tri, surface_at)


def stretched_faces(ny: int, ly: float = 1.0, beta: float = 1.8) -> np.ndarray:
    """ny + 1 wall-normal face positions clustered at both walls,
    y = ly/2 (1 + tanh(beta (2 s - 1)) / tanh(beta)), s = j / ny: a smooth
    stretching (cells about 3x taller at mid-channel than at the walls for
    beta = 1.8), for the non-uniform grid of Section 2."""
    s = np.arange(ny + 1) / ny
    y = 0.5 * ly * (1.0 + np.tanh(beta * (2.0 * s - 1.0)) / np.tanh(beta))
    y[0], y[-1] = 0.0, ly
    return y


def immersed_wall_channel(nx: int = 64, ny: int = 96, nz: int = 64, y_wall: float = 0.1213, steps: int = 10,
                          re: float = 100.0, dt: float = 1e-3, force: float = 2.0, nq: int = 1) -> Workload:
    """Channel with an immersed rigid wall across the whole periodic box at
    y = y_wall (the lower wall of the channel cases of Section 4) and a body
    force along x.  The wall is a plate wider than the box (0.3 beyond it on
    every side; nq x nq quads, two triangles each); it is meant for a
    stretched wall-normal grid (stretched_faces) with no node on the wall."""
    big = 0.3
    xyz, tri = plate(nq, 1.0 + 2.0 * big, -big, -big, y_wall)

    def surface_at(t):
        return xyz.copy(), np.zeros_like(xyz)

    return Workload(f"wallchannel{nx}x{ny}x{nz}", nx, ny, nz, 1.0, 1.0, 1.0, re, dt, steps, tri, surface_at,
                    lambda t: (force, 0.0, 0.0))


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
    "channel256": multibody_channel,
    "leaflet512": leaflet_tube,
}


def workload(name: str, **kw) -> Workload:
    return WORKLOADS[name](**kw)
