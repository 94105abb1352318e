// geometry.cuh -- exact-rounding FP64 geometry shared by the tagging,
// forcing and no-slip-error kernels: lattice positions of the staggered
// nodes and the closest point of a triangle (Algorithm 1 of arXiv
// 2606.09799, which cites Ericson 2004).
#pragma once

#include "common.cuh"

namespace ibm {

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double ddot(const double x[3], const double y[3]) {
  return dadd(dadd(dmul(x[0], y[0]), dmul(x[1], y[1])), dmul(x[2], y[2]));
}

// Wall-normal coordinate of lattice row j: faces (half = 0) or cell centres
// (half = 1).  On the non-uniform grid it comes from the row tables, one row
// beyond either wall included.
__device__ __forceinline__ double ylat(const Geo& g, long long j, int half) {
  if (g.yt.yc) return half ? g.yt.yc[j + 1] : g.yt.yv[j + 1];
  return half ? dmul(dadd((double)j, 0.5), g.dy) : dmul((double)j, g.dy);
}

// Squared diagonal of the local Eulerian cell of component c's node in row
// j (Algorithm 1): on the non-uniform grid its wall-normal side is the cell
// height for u and w (centres) and the distance of the centres for v (faces).
__device__ __forceinline__ double yspan(const Geo& g, int c, long long j) {
  return c == 1 ? g.yt.hf[j] : g.yt.hc[j];
}
__device__ __forceinline__ double diag2_at(const Geo& g, int c, long long j) {
  if (!g.yt.yc) return g.diag2;
  const double hy = yspan(g, c, j);
  return dadd(dadd(dmul(g.dx, g.dx), dmul(hy, hy)), dmul(g.dz, g.dz));
}

// Lattice position of component c's node with (possibly unwrapped) indices.
__device__ __forceinline__ void node_pos(const Geo& g, int c, long long i, long long j, long long k, double x[3]) {
  x[0] = (c == 0) ? dmul((double)i, g.dx) : dmul(dadd((double)i, 0.5), g.dx);
  x[1] = ylat(g, j, c != 1);
  x[2] = (c == 2) ? dmul((double)k, g.dz) : dmul(dadd((double)k, 0.5), g.dz);
}

// Per-triangle data of the closest-point classification: the vertices and
// edge vectors (each edge formed as the same difference of vertices as in
// the per-point formulas, so reusing them changes no rounding).
struct TriConst {
  double a[3], b[3], c[3], ab[3], ac[3], bc[3];
};

__device__ inline void tri_const(const double a[3], const double b[3], const double c[3], TriConst& T) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    T.a[d] = a[d];
    T.b[d] = b[d];
    T.c[d] = c[d];
    T.ab[d] = dsub(b[d], a[d]);
    T.ac[d] = dsub(c[d], a[d]);
    T.bc[d] = dsub(c[d], b[d]);
  }
}

// FP32 copy of a triangle's constants for the tagging pre-screen, in
// coordinates relative to the first vertex: position of lattice point i
// along axis d is (i - ia[d][half]) * del[d] - fr[d][half].
struct TriF32 {
  float ab[3], ac[3], bc[3];
  float aa, abac, cc, iaa, icc, ibc, iden;
  int ia[3][2];     // lattice index of the first vertex (32-bit: no 64-bit conversions in the screen)
  float fr[3][2];
  float del[3], diag2;
  float ay;         // y of the first vertex (non-uniform rows: positions from the row table)
  float ymn, ymx;   // the triangle's y extent
};

// Everything the kernels of one step derive from a triangle alone, formed
// once per step by one thread per triangle: the closest-point constants,
// the centroid (periodic image of a node), the lattice box of Algorithm 1
// per velocity component (first index and extent per axis, pair counts)
// and the FP32 screen constants (screen = 0 where the screen's error bound
// does not hold).
struct TriRec {
  TriConst tc;
  double cen[3];
  TriF32 f;
  int n0[3][3];
  int ext[3][3];
  long long cnt[3];
  int screen;
};

// Closest point X on the triangle to p with barycentric weights (Ericson
// 2004, cited by Algorithm 1; Voronoi regions: three vertex regions, three
// edge regions, the face).  The textbook quantities in the textbook order:
// the six scalar products of the edge vectors with p - a, p - b and p - c,
// each from its own difference vector, and the edge and face parameters as
// quotients of those products.  Exact-rounding FP64 (no contraction), so the
// result is the IEEE-754 value of these formulas bit for bit.
__device__ inline void closest_point_exact(const double p[3], const TriConst& T, double X[3], double w[3]) {
  double ap[3], bp[3], cp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) ap[d] = dsub(p[d], T.a[d]);
  const double d1 = ddot(T.ab, ap), d2 = ddot(T.ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = T.a[d];
    w[0] = 1.0; w[1] = 0.0; w[2] = 0.0;
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) bp[d] = dsub(p[d], T.b[d]);
  const double d3 = ddot(T.ab, bp), d4 = ddot(T.ac, bp);
  if (d3 >= 0.0 && d4 <= d3) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = T.b[d];
    w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
    return;
  }
  const double vc = dsub(dmul(d1, d4), dmul(d3, d2));
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double t = ddiv(d1, dsub(d1, d3));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(T.a[d], dmul(t, T.ab[d]));
    w[0] = dsub(1.0, t); w[1] = t; w[2] = 0.0;
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) cp[d] = dsub(p[d], T.c[d]);
  const double d5 = ddot(T.ab, cp), d6 = ddot(T.ac, cp);
  if (d6 >= 0.0 && d5 <= d6) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = T.c[d];
    w[0] = 0.0; w[1] = 0.0; w[2] = 1.0;
    return;
  }
  const double vb = dsub(dmul(d5, d2), dmul(d1, d6));
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double t = ddiv(d2, dsub(d2, d6));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(T.a[d], dmul(t, T.ac[d]));
    w[0] = dsub(1.0, t); w[1] = 0.0; w[2] = t;
    return;
  }
  const double va = dsub(dmul(d3, d6), dmul(d5, d4));
  const double e43 = dsub(d4, d3), e56 = dsub(d5, d6);
  if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) {
    const double t = ddiv(e43, dadd(e43, e56));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(T.b[d], dmul(t, T.bc[d]));
    w[0] = 0.0; w[1] = dsub(1.0, t); w[2] = t;
    return;
  }
  const double s = ddiv(1.0, dadd(dadd(va, vb), vc));
  const double v = dmul(vb, s), u = dmul(vc, s);
#pragma unroll
  for (int d = 0; d < 3; ++d) X[d] = dadd(dadd(T.a[d], dmul(T.ab[d], v)), dmul(T.ac[d], u));
  w[0] = dsub(dsub(1.0, v), u); w[1] = v; w[2] = u;
}

// Coordinate of lattice index i along axis a for a node offset of 0 (face)
// or half a cell; the same formula as node_pos.
__device__ __forceinline__ double lat(long long i, double del, int half) {
  return half ? dmul(dadd((double)i, 0.5), del) : dmul((double)i, del);
}

// Exact index range of the lattice points strictly inside (lo, hi): start
// from a conservative range and shrink it with the predicate itself (the
// coordinate is monotone in the index), so the set equals that of testing
// every point.
__device__ __forceinline__ void exact_range(double lo, double hi, double del, double idel, int half,
                                            long long& i0, long long& i1) {
  const double off = half ? 0.5 : 0.0;
  // conservative start (one index of margin absorbs the rounding of lo / del)
  i0 = (long long)floor(lo * idel - off) - 1;
  i1 = (long long)ceil(hi * idel - off) + 1;
  while (i0 <= i1 && !(lo < lat(i0, del, half))) ++i0;
  while (i1 >= i0 && !(lat(i1, del, half) < hi)) --i1;
}

// Whether row j of component c's lattice lies inside the box of Algorithm 1
// in y, the margin being that node's own cell size (non-uniform grid).
__device__ __forceinline__ bool row_inside(const Geo& g, int c, long long j, double ymn, double ymx) {
  const double y = ylat(g, j, c != 1), hy = yspan(g, c, j);
  return dsub(ymn, hy) < y && y < dadd(ymx, hy);
}

// First and last row of component c's lattice (j in [jlo, jhi]) inside that
// box on the non-uniform grid: bisection to the rows within the largest cell
// size of [ymn, ymx] (a superset, since every margin is at most hmax), then
// the exact predicate inwards.  Rows between the two may still fail it; the
// pair test checks every row again.
__device__ inline void nu_row_range(const Geo& g, int c, long long jlo, long long jhi, double ymn, double ymx,
                                    long long& j0, long long& j1) {
  const int half = c != 1;
  const double lo = dsub(ymn, g.yt.hmax), hi = dadd(ymx, g.yt.hmax);
  long long a = jlo, b = jhi + 1;   // first row above lo
  while (a < b) {
    const long long m = (a + b) >> 1;
    if (ylat(g, m, half) > lo) b = m; else a = m + 1;
  }
  j0 = a;
  a = jlo - 1;
  b = jhi;   // last row below hi
  while (a < b) {
    const long long m = (a + b + 1) >> 1;
    if (ylat(g, m, half) < hi) a = m; else b = m - 1;
  }
  j1 = a;
  while (j0 <= j1 && !row_inside(g, c, j0, ymn, ymx)) ++j0;
  while (j1 >= j0 && !row_inside(g, c, j1, ymn, ymx)) --j1;
}

__device__ __forceinline__ void load_vertex(const Surf& s, int v, double out[3]) {
  out[0] = __ldg(s.x + v);
  out[1] = __ldg(s.x + s.nv + v);
  out[2] = __ldg(s.x + 2 * (long long)s.nv + v);
}

__device__ __forceinline__ void load_triangle(const Surf& s, int t, double a[3], double b[3], double c[3]) {
  load_vertex(s, __ldg(s.t + t), a);
  load_vertex(s, __ldg(s.t + s.nt + t), b);
  load_vertex(s, __ldg(s.t + 2 * (long long)s.nt + t), c);
}

}  // namespace ibm
