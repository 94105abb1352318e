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

// Lattice position of component c's node with (possibly unwrapped) indices.
__device__ __forceinline__ void node_pos(const Geo& g, int c, long long i, long long j, long long k, double x[3]) {
  x[0] = (c == 0) ? dmul((double)i, g.dx) : dmul(dadd((double)i, 0.5), g.dx);
  x[1] = (c == 1) ? dmul((double)j, g.dy) : dmul(dadd((double)j, 0.5), g.dy);
  x[2] = (c == 2) ? dmul((double)k, g.dz) : dmul(dadd((double)k, 0.5), g.dz);
}

// Closest point X on triangle (a,b,c) to p with barycentric weights
// (Ericson 2004, Voronoi regions: three vertex regions, three edge regions,
// the face).  Exact-rounding FP64.
__device__ inline void closest_point_exact(const double p[3], const double a[3], const double b[3], const double c[3],
                                    double X[3], double w[3]) {
  double ab[3], ac[3], ap[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ab[d] = dsub(b[d], a[d]);
    ac[d] = dsub(c[d], a[d]);
    ap[d] = dsub(p[d], a[d]);
  }
  const double d1 = ddot(ab, ap), d2 = ddot(ac, ap);
  if (d1 <= 0.0 && d2 <= 0.0) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = a[d];
    w[0] = 1.0; w[1] = 0.0; w[2] = 0.0;
    return;
  }
  double bp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) bp[d] = dsub(p[d], b[d]);
  const double d3 = ddot(ab, bp), d4 = ddot(ac, bp);
  if (d3 >= 0.0 && d4 <= d3) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = b[d];
    w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
    return;
  }
  const double vc = dsub(dmul(d1, d4), dmul(d3, d2));
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double t = ddiv(d1, dsub(d1, d3));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(a[d], dmul(t, ab[d]));
    w[0] = dsub(1.0, t); w[1] = t; w[2] = 0.0;
    return;
  }
  double cp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) cp[d] = dsub(p[d], c[d]);
  const double d5 = ddot(ab, cp), d6 = ddot(ac, cp);
  if (d6 >= 0.0 && d5 <= d6) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = c[d];
    w[0] = 0.0; w[1] = 0.0; w[2] = 1.0;
    return;
  }
  const double vb = dsub(dmul(d5, d2), dmul(d1, d6));
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double t = ddiv(d2, dsub(d2, d6));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(a[d], dmul(t, ac[d]));
    w[0] = dsub(1.0, t); w[1] = 0.0; w[2] = t;
    return;
  }
  const double va = dsub(dmul(d3, d6), dmul(d5, d4));
  const double e43 = dsub(d4, d3), e56 = dsub(d5, d6);
  if (va <= 0.0 && e43 >= 0.0 && e56 >= 0.0) {
    const double t = ddiv(e43, dadd(e43, e56));
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = dadd(b[d], dmul(t, dsub(c[d], b[d])));
    w[0] = 0.0; w[1] = dsub(1.0, t); w[2] = t;
    return;
  }
  const double s = ddiv(1.0, dadd(dadd(va, vb), vc));
  const double v = dmul(vb, s), u = dmul(vc, s);
#pragma unroll
  for (int d = 0; d < 3; ++d) X[d] = dadd(dadd(a[d], dmul(ab[d], v)), dmul(ac[d], u));
  w[0] = dsub(dsub(1.0, v), u); w[1] = v; w[2] = u;
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
