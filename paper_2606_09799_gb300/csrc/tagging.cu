// tagging.cu -- Algorithm 1 of arXiv 2606.09799 (fast tagging of the forcing
// nodes) on the three staggered velocity grids, with deterministic
// compaction of the forcing nodes and boundary cells (Section 3.2).
//
// Work shape: one warp per (triangle, velocity component); the lanes stride
// over the Eulerian points inside the triangle's Cartesian box.  A point that
// passes the test of Algorithm 1 becomes a candidate: |N|^2 is folded into a
// per-node atomicMin, and the pair is appended to a candidate list with a
// warp-aggregated atomic.  A second pass keeps, per node, the candidate of
// smallest |N|^2 (ties: smallest triangle index), and a third marks the node
// in the per-cell flag bytes.  A dense, deterministic scan of those bytes then
// emits the forcing list and the boundary-cell list sorted by cell index.
//
// Every geometric predicate is evaluated in FP64 with explicit
// round-to-nearest operations (no contraction into FMA), in the same order
// as the textual definition of each quantity, so tags are reproducible
// bit for bit by any IEEE-754 implementation of the same formulas.
#include <algorithm>

#include "common.cuh"
#include "exec.cuh"
#include "geometry.cuh"
#include "launch.h"

namespace ibm {

// ---------------------------------------------------------------------------
// sparse reset of the per-node state touched by the previous step
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tag_reset(const Blk& bk, const Geo& g, const Cand* __restrict__ cand, unsigned cap, DevState* ds,
                            unsigned long long* d2min, unsigned* owner, unsigned* flags32, unsigned* ub,
                            const unsigned* __restrict__ ublist) {
  const unsigned n = min(ds->ncand, cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const Cand cd = cand[e];
    const int c = (int)(cd.key >> 30);
    const long long node = cd.key & KEY_MASK;
    d2min[comp_off(g, c) + node] = ~0ull;
    owner[comp_off(g, c) + node] = 0xFFFFFFFFu;
    const int pl = planes(g, c);
    long long i, j, k;
    split3(node, g.nx, pl, i, j, k);
    const long long cell = cidx(g, i, j, k);
    atomicAnd(flags32 + (cell >> 2), ~(0xFFu << (8 * (cell & 3))));
  }
  const unsigned nu = min(ds->nub, cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < nu; e += bk.gx * blockDim.x) ub[ublist[e]] = 0xFFFFFFFFu;
}
struct TagReset {
  static constexpr int kThreads = 256;
  Geo g;
  const Cand* cand;
  unsigned cap;
  DevState* ds;
  unsigned long long* d2min;
  unsigned* owner;
  unsigned* flags32;
  unsigned* ub;
  const unsigned* ublist;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    tag_reset(bk, g, cand, cap, ds, d2min, owner, flags32, ub, ublist);
  }
};

// ---------------------------------------------------------------------------
// Per-triangle set-up, one thread per triangle: closest-point constants,
// centroid, the exact lattice box of Algorithm 1 per component and the FP32
// screen constants.  Every kernel of the step that needs a triangle's
// constants reads them here, so they are formed once (FP64 is scarce on
// this GPU: a warp-wide FP64 instruction costs about 20 SM cycles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_setup(const Blk& bk, const Geo& g, const Surf& s) {
  const int t = bk.x * blockDim.x + threadIdx.x;
  if (t >= s.nt) return;
  double A[3], B[3], C[3];
  load_triangle(s, t, A, B, C);
  TriRec R;
  tri_const(A, B, C, R.tc);
  const TriConst& TC = R.tc;
  // (the centroid only picks a node's periodic image: any rounding serves)
#pragma unroll
  for (int d = 0; d < 3; ++d) R.cen[d] = (A[d] + B[d] + C[d]) * (1.0 / 3.0);
  const double del[3] = {g.dx, g.dy, g.dz};
  const double idel[3] = {g.idx, g.idy, g.idz};
  double lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = dsub(fmin(A[d], fmin(B[d], C[d])), del[d]);
    hi[d] = dadd(fmax(A[d], fmax(B[d], C[d])), del[d]);
  }
  // ranges per axis for face (half = 0) and half-offset (half = 1) lattices
  long long r0[3][2], r1[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) exact_range(lo[d], hi[d], del[d], idel[d], hf, r0[d][hf], r1[d][hf]);
  long long total = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    long long prod = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int hf = (d == c) ? 0 : 1;
      long long a0 = r0[d][hf], a1 = r1[d][hf];
      if (d == 1) {
        const long long jlo = c == 1 ? 1 : 0;
        if (g.yt.yc)   // non-uniform rows: each node's own cell size is its margin
          nu_row_range(g, c, jlo, g.ny - 1, fmin(A[1], fmin(B[1], C[1])), fmax(A[1], fmax(B[1], C[1])), a0, a1);
        a0 = a0 < jlo ? jlo : a0;
        a1 = a1 > g.ny - 1 ? g.ny - 1 : a1;
      }
      const long long e = a1 - a0 + 1 > 0 ? a1 - a0 + 1 : 0;
      R.n0[c][d] = (int)a0;
      R.ext[c][d] = (int)e;
      prod *= e;
    }
    R.cnt[c] = prod;
    total += prod;
  }
  // FP32 screen: skinny or large triangles and strongly anisotropic cells
  // (where its error bound does not hold) skip it
  // (the screen's constants: scalar products of the edge vectors and the
  // reciprocal denominators of its edge and face parameters)
  const double aa = ddot(TC.ab, TC.ab), abac = ddot(TC.ab, TC.ac), cc = ddot(TC.ac, TC.ac);
  const double bcbc = ddot(TC.bc, TC.bc);
  const double den = dsub(dmul(aa, cc), dmul(abac, abac));
  double dmin = fmin(del[0], fmin(del[1], del[2])), dmax = fmax(del[0], fmax(del[1], del[2]));
  bool rows_ok = true;
  if (g.yt.yc) {
    // non-uniform rows: the local cells of the rows in the triangle's box
    // (and one beyond), from the row table, decide the scale
    dmin = fmin(del[0], del[2]);
    dmax = fmax(del[0], del[2]);
    const int ny = g.ny;
    for (int half = 0; half < 2 && rows_ok; ++half) {
      const int c = half ? 0 : 1;
      const int j0 = R.n0[c][1] - 1, j1 = R.n0[c][1] + R.ext[c][1];
      if (R.ext[c][1] > 64) rows_ok = false;
      for (int j = max(j0, half ? 0 : 1); j <= min(j1, half ? ny - 1 : ny - 1) && rows_ok; ++j) {
        const float4 r = g.yt.rowf[half * (ny + 1) + j];
        dmin = fmin(dmin, (double)fmin(r.y, fmin(r.z, r.w)));
        dmax = fmax(dmax, (double)fmax(r.y, fmax(r.z, r.w)));
      }
    }
  }
  const double lmax2 = fmax(aa, fmax(cc, bcbc));
  R.screen = rows_ok && den > 0.05 * aa * cc && lmax2 <= 256.0 * dmin * dmin && dmax <= 4.0 * dmin &&
             total < (1ll << 30);
  TriF32& F = R.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    F.ab[d] = (float)TC.ab[d];
    F.ac[d] = (float)TC.ac[d];
    F.bc[d] = (float)TC.bc[d];
    F.del[d] = (float)del[d];
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const double off = hf ? 0.5 : 0.0;
      const double q = floor(A[d] * idel[d] - off);
      F.ia[d][hf] = (int)q;
      F.fr[d][hf] = (float)(A[d] - (q + off) * del[d]);
    }
  }
  // (FP32 reciprocals: the screen's margins are far wider than their error,
  // and an FP64 division is costly on this GPU)
  F.aa = (float)aa;
  F.abac = (float)abac;
  F.cc = (float)cc;
  F.iaa = 1.0f / F.aa;
  F.icc = 1.0f / F.cc;
  F.ibc = 1.0f / (float)bcbc;
  F.iden = 1.0f / (float)den;
  F.diag2 = (float)g.diag2;
  F.ay = (float)A[1];
  F.ymn = (float)fmin(A[1], fmin(B[1], C[1]));
  F.ymx = (float)fmax(A[1], fmax(B[1], C[1]));
  s.rec[t] = R;
}
struct TriSetup {
  static constexpr int kThreads = 128;
  Geo g;
  Surf s;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_setup(bk, g, s); }
};

// ---------------------------------------------------------------------------
// Algorithm 1: one warp per triangle, its lanes spread over the Eulerian
// points of all three staggered grids inside the triangle's box
// ---------------------------------------------------------------------------

// Cheap FP32 screen of one (node, triangle) pair, in coordinates relative to
// the triangle's first vertex (so every quantity is of the cell's size).  It
// returns false only when the exact FP64 test certainly fails: |N|^2 above
// diag^2 by a margin, or every neighbour's scalar product clearly positive.
// Near the decision boundary |N| is at least del_min / sqrt(3), so the
// margins (0.4% of |N|^2 + del |N_d|) bound the FP32 error of N relative to
// the cell.  That error is about eps_32 * L / sin^2(theta) for a triangle of
// edge L and smallest angle theta; the screen is used only where this stays
// below 1e-3 of the margin's scale (sin^2 > 0.05, edges within 16 cells, cell
// aspect ratio within 4), else every pair goes to the exact test.  On the
// non-uniform wall-normal grid the cell is the node's own (its row's
// spacing, the rows bracketing it for the neighbour test), and the row's
// position is its FP32 table value less the vertex's (an error of about
// 1e-7 of the box, well inside the margins).  Tags are decided by the FP64
// test alone.
__device__ __forceinline__ void screen_eval(const TriF32& F, const Geo& g, int c, const int idx3[3], float& n2,
                                            float& lowest, float& scale, float& diag2) {
  float p[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // static indices only (a runtime index would put F in local memory)
    const float pf = (float)(idx3[d] - F.ia[d][0]) * F.del[d] - F.fr[d][0];
    const float ph = (float)(idx3[d] - F.ia[d][1]) * F.del[d] - F.fr[d][1];
    p[d] = d == c ? pf : ph;
  }
  float dlo = F.del[1], dhi = F.del[1];
  diag2 = F.diag2;
  if (g.yt.rowf) {
    const float4 r = g.yt.rowf[(c != 1) * (g.ny + 1) + idx3[1]];
    p[1] = r.x - F.ay;
    dlo = r.z;
    dhi = r.w;
    diag2 = (F.del[0] * F.del[0] + r.y * r.y) + F.del[2] * F.del[2];
  }
  const float d1 = F.ab[0] * p[0] + F.ab[1] * p[1] + F.ab[2] * p[2];
  const float d2 = F.ac[0] * p[0] + F.ac[1] * p[1] + F.ac[2] * p[2];
  float X[3];
  const float d3 = d1 - F.aa, d4 = d2 - F.abac, d5 = d1 - F.abac, d6 = d2 - F.cc;
  const float vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
  if (d1 <= 0.f && d2 <= 0.f) {
    X[0] = X[1] = X[2] = 0.f;
  } else if (d3 >= 0.f && d4 <= d3) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = F.ab[d];
  } else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
    const float t = d1 * F.iaa;
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = t * F.ab[d];
  } else if (d6 >= 0.f && d5 <= d6) {
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = F.ac[d];
  } else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
    const float t = d2 * F.icc;
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = t * F.ac[d];
  } else if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
    const float t = (d4 - d3) * F.ibc;
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = F.ab[d] + t * F.bc[d];
  } else {
    const float v = vb * F.iden, w = vc * F.iden;
#pragma unroll
    for (int d = 0; d < 3; ++d) X[d] = F.ab[d] * v + F.ac[d] * w;
  }
  float N[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) N[d] = p[d] - X[d];
  n2 = N[0] * N[0] + N[1] * N[1] + N[2] * N[2];
  // N . (neighbour - X) = |N|^2 -+ del_d N_d: the smallest over the six (in
  // y the neighbour on N's side: the row below if N_y > 0, else above)
  lowest = 3.4e38f;
  scale = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float dd = d == 1 ? (N[1] > 0.f ? dlo : dhi) : F.del[d];
    const float t = dd * fabsf(N[d]);
    lowest = fminf(lowest, n2 - t);
    scale = fmaxf(scale, d == 1 ? fmaxf(dlo, dhi) * fabsf(N[1]) : t);
  }
}

// The pair may pass the exact test (false: it certainly fails).
__device__ __forceinline__ bool screen_maybe(float diag2, float n2, float lowest, float scale) {
  return !(n2 > diag2 * 1.004f) && lowest < 4e-3f * (n2 + scale) + 1e-9f * diag2;
}
// The pair certainly passes the exact test (the same margins, other side).
__device__ __forceinline__ bool screen_certain(float diag2, float n2, float lowest, float scale) {
  return n2 <= diag2 * 0.996f && lowest < -(4e-3f * (n2 + scale) + 1e-9f * diag2);
}
// Bounds of the exact |N|^2 from the FP32 one: the FP32 error of |N|^2 is
// below 1e-4 diag^2 wherever the screen runs (see above); the bounds leave
// 4e-3 relative plus 1e-3 diag^2.
__device__ __forceinline__ float n2_upper(float diag2, float n2) { return n2 * 1.004f + 1e-3f * diag2; }
__device__ __forceinline__ float n2_lower(float diag2, float n2) { return n2 * 0.996f - 1e-3f * diag2; }


// Non-uniform rows: row j of component c's lattice lies inside the box of
// Algorithm 1 (margin: the node's own cell), with a margin of 1e-3 of the
// cell over the FP32 errors (about 1e-7 of the box) -- a pair the screen
// calls certain must pass the exact test, box included.
__device__ __forceinline__ bool row_inside_f(const Geo& g, const TriF32& F, int c, int j) {
  const float4 r = g.yt.rowf[(c != 1) * (g.ny + 1) + j];
  const float m = 1e-3f * r.y;
  return r.x > F.ymn - r.y + m && r.x < F.ymx + r.y - m;
}

// pair n of a triangle's box -> (component, unwrapped lattice indices)
__device__ __forceinline__ void decode_pair(const TriRec* __restrict__ rec, long long n, int& c, long long idx3[3]) {
  const long long cnt0 = rec->cnt[0], cnt1 = rec->cnt[1], total = cnt0 + cnt1 + rec->cnt[2];
  c = n < cnt0 ? 0 : (n < cnt0 + cnt1 ? 1 : 2);
  const long long q = n - (c == 0 ? 0 : (c == 1 ? cnt0 : cnt0 + cnt1));
  // selects instead of runtime indices (keeps the record's fields in registers)
  const int ni = max(c == 0 ? rec->ext[0][0] : (c == 1 ? rec->ext[1][0] : rec->ext[2][0]), 1);
  const int nj = max(c == 0 ? rec->ext[0][1] : (c == 1 ? rec->ext[1][1] : rec->ext[2][1]), 1);
  long long qj, ri, rj;
  if (total < (1ll << 30)) {
    const unsigned q32 = (unsigned)q, qi32 = q32 / (unsigned)ni, qj32 = qi32 / (unsigned)nj;
    qj = qj32;
    ri = q32 - qi32 * (unsigned)ni;
    rj = qi32 - qj32 * (unsigned)nj;
  } else {
    const long long qi = q / ni;
    qj = qi / nj;
    ri = q - qi * ni;
    rj = qi - qj * nj;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int b0 = c == 0 ? rec->n0[0][d] : (c == 1 ? rec->n0[1][d] : rec->n0[2][d]);
    idx3[d] = b0 + (d == 0 ? ri : (d == 1 ? rj : qj));
  }
}

// The owner of a node is the qualifying pair of smallest |N|^2, so a pair
// whose |N|^2 certainly exceeds that of a pair that certainly qualifies
// can neither own the node nor change whether it is tagged.  Phase 0 folds
// an upper bound of |N|^2 of every certainly-qualifying pair (FP32 screen)
// into a per-node word `ub` (first touches listed in `ublist` for the sparse
// reset); phase 1 lists the pairs that may qualify and whose lower bound
// does not exceed the node's `ub` -- the owner and every pair tied with it
// always among them -- for the exact FP64 test (TagExact), which takes
// them one per lane, so its warps are full whatever the survivors per
// triangle.  One warp per triangle, lanes over the pairs of its box.
template <int PHASE>
__device__ __forceinline__ void tag_pairs(const Blk& bk, const Geo& g, const Surf& s, unsigned cap,
                                          unsigned* __restrict__ ub, unsigned* __restrict__ ublist,
                                          unsigned long long* __restrict__ surv, DevState* ds) {
  const int lane = threadIdx.x & 31;
  const long long t = ((long long)bk.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= s.nt) return;
  const TriRec* __restrict__ rec = s.rec + t;
  const long long total = rec->cnt[0] + rec->cnt[1] + rec->cnt[2];
  if (total == 0) return;
  const bool screen = rec->screen != 0;
  if (PHASE == 0 && !screen) return;   // no FP32 bound without the screen
  TriF32 F;
  if (screen) F = rec->f;
  // index of a lattice point in the comp_off layout of the three grids
  auto node_of = [&](int c, const long long i3[3]) -> unsigned {
    int i = (int)i3[0], k = (int)i3[2];
    i = i < 0 ? i + g.nx : (i >= g.nx ? i - g.nx : i);   // a box is narrower than the domain
    k = k < 0 ? k + g.nz : (k >= g.nz ? k - g.nz : k);
    const unsigned pl = c == 1 ? (unsigned)g.ny + 1u : (unsigned)g.ny;
    const unsigned off = c == 0 ? 0u : (c == 1 ? (unsigned)g.ncell : (unsigned)(g.ncell + g.nvf));
    return off + ((unsigned)k * pl + (unsigned)i3[1]) * (unsigned)g.nx + (unsigned)i;
  };
  // warp-aggregated append of this lane's item (if `has`) to a list
  auto append = [&](bool has, unsigned* counter, auto store) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, has);
    if (!m) return;
    unsigned pos = 0;
    const int leader = __ffs(m) - 1;
    if (lane == leader) pos = atomicAdd(counter, (unsigned)__popc(m));
    pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
    if (has) {
      const unsigned slot = pos + __popc(m & ((1u << lane) - 1u));
      if (slot < cap) store(slot);
      else atomicOr(&ds->err, ERR_CAND_OVERFLOW);
    }
  };
  for (long long base = 0; base < total; base += 32) {
    const long long n = base + lane;
    bool hit = false;
    unsigned ni = 0;
    if (n < total) {
      if (screen) {
        int c;
        long long i3[3];
        decode_pair(rec, n, c, i3);
        const int idx3[3] = {(int)i3[0], (int)i3[1], (int)i3[2]};
        float n2, lowest, scale, d2;
        screen_eval(F, g, c, idx3, n2, lowest, scale, d2);
        // (non-uniform rows: a row outside the box of Algorithm 1, whose
        // margin is the node's own cell, is left to the exact test)
        if (PHASE == 0) {
          if (screen_certain(d2, n2, lowest, scale) && !(g.yt.rowf && !row_inside_f(g, F, c, idx3[1]))) {
            ni = node_of(c, i3);
            hit = atomicMin(ub + ni, __float_as_uint(n2_upper(d2, n2))) == 0xFFFFFFFFu;   // first touch
          }
        } else if (screen_maybe(d2, n2, lowest, scale)) {
          const unsigned u = __ldcg(ub + node_of(c, i3));
          hit = u == 0xFFFFFFFFu || n2_lower(d2, n2) <= __uint_as_float(u);
        }
      } else {
        hit = true;   // phase 1 only: every pair of an unscreened triangle is tested exactly
      }
    }
    if (PHASE == 0) append(hit, &ds->nub, [&](unsigned slot) { ublist[slot] = ni; });
    else append(hit, &ds->nsurv, [&](unsigned slot) { surv[slot] = ((unsigned long long)t << 32) | (unsigned)n; });
  }
}
template <int PHASE>
struct TagPairs {
  static constexpr int kThreads = 128;
  Geo g;
  Surf s;
  unsigned cap;
  unsigned* ub;
  unsigned* ublist;
  unsigned long long* surv;
  DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tag_pairs<PHASE>(bk, g, s, cap, ub, ublist, surv, ds); }
};

// The exact test of Algorithm 1, FP64 with explicit rounding, one listed
// (triangle, pair) per thread: |N|^2 <= diag^2 and a scalar product
// N . (x^{k,n} - X) < 0 for one of the six lattice neighbours (or N = 0).
// A pair that passes folds |N|^2 into the node's minimum and joins the
// candidate list.
__device__ __forceinline__ void tag_exact(const Blk& bk, const Geo& g, const Surf& s, Cand* __restrict__ cand,
                                          unsigned cap, unsigned long long* d2min,
                                          const unsigned long long* __restrict__ surv, DevState* ds) {
  const unsigned ns = min(ds->nsurv, cap);
  const int lane = threadIdx.x & 31;
  const double del[3] = {g.dx, g.dy, g.dz};
  const unsigned stride = bk.gx * blockDim.x;
  // whole warps iterate together (the candidate append is warp-aggregated)
  for (unsigned e0 = bk.x * blockDim.x + (threadIdx.x & ~31u); e0 < ns; e0 += stride) {
    const unsigned e = e0 + lane;
    bool tagged = false;
    unsigned key = 0, tri = 0;
    unsigned long long d2bits = 0;
    if (e < ns) {
      const unsigned long long sv = surv[e];
      tri = (unsigned)(sv >> 32);
      const TriRec* __restrict__ rec = s.rec + tri;
      int c;
      long long idx3[3];
      decode_pair(rec, (long long)(unsigned)sv, c, idx3);
      const TriConst TC = rec->tc;
      double x[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) x[d] = lat(idx3[d], del[d], d == c ? 0 : 1);
      double diag2 = g.diag2;
      bool inbox = true;
      if (g.yt.yc) {
        // non-uniform rows: the node's own cell gives the box margin in y
        // and the diagonal
        x[1] = ylat(g, idx3[1], c != 1);
        inbox = row_inside(g, c, idx3[1], fmin(TC.a[1], fmin(TC.b[1], TC.c[1])), fmax(TC.a[1], fmax(TC.b[1], TC.c[1])));
        diag2 = diag2_at(g, c, idx3[1]);
      }
      double X[3], wb[3], N[3], P[3];
      closest_point_exact(x, TC, X, wb);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        N[d] = dsub(x[d], X[d]);
        P[d] = dmul(N[d], N[d]);
      }
      const double n2 = dadd(dadd(P[0], P[1]), P[2]);
      if (inbox && n2 <= diag2) {
        if (n2 == 0.0) {
          tagged = true;   // a node on the surface: alpha = 0 in Eq. new_IB
        } else {
          // only the neighbour's own axis differs from N; the other two
          // products are the P[] already formed (same operands and rounding)
#pragma unroll
          for (int d = 0; d < 3 && !tagged; ++d) {
#pragma unroll
            for (int sg = -1; sg <= 1 && !tagged; sg += 2) {
              const double xn = d == 1 ? ylat(g, idx3[1] + sg, c != 1) : lat(idx3[d] + sg, del[d], d == c ? 0 : 1);
              const double vd = dsub(xn, X[d]);
              const double Q = dmul(N[d], vd);
              const double dot = d == 0 ? dadd(dadd(Q, P[1]), P[2])
                                        : (d == 1 ? dadd(dadd(P[0], Q), P[2]) : dadd(dadd(P[0], P[1]), Q));
              if (dot < 0.0) tagged = true;
            }
          }
        }
        if (tagged) {
          const long long node = fidx(g, c, wrapi(idx3[0], g.nx), idx3[1], wrapi(idx3[2], g.nz));
          key = ((unsigned)c << 30) | (unsigned)node;
          d2bits = (unsigned long long)__double_as_longlong(n2);
          atomicMin(d2min + comp_off(g, c) + node, d2bits);
        }
      }
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, tagged);
    if (mask) {
      unsigned pos = 0;
      const int leader = __ffs(mask) - 1;
      if (lane == leader) pos = atomicAdd(&ds->ncand, (unsigned)__popc(mask));
      pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
      if (tagged) {
        const unsigned slot = pos + __popc(mask & ((1u << lane) - 1u));
        if (slot < cap) {
          Cand cd;
          cd.key = key;
          cd.tri = tri;
          cd.d2 = d2bits;
          cand[slot] = cd;
        } else {
          atomicOr(&ds->err, ERR_CAND_OVERFLOW);
        }
      }
    }
  }
}
struct TagExact {
  static constexpr int kThreads = 128;
  Geo g;
  Surf s;
  Cand* cand;
  unsigned cap;
  unsigned long long* d2min;
  const unsigned long long* surv;
  DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tag_exact(bk, g, s, cand, cap, d2min, surv, ds); }
};

// Per node keep the smallest triangle index among the candidates of minimum |N|^2.
__device__ __forceinline__ void tag_resolve(const Blk& bk, const Geo& g, const Cand* __restrict__ cand, unsigned cap, const DevState* ds,
                              const unsigned long long* __restrict__ d2min, unsigned* owner) {
  const unsigned n = min(ds->ncand, cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const Cand cd = cand[e];
    const long long o = comp_off(g, (int)(cd.key >> 30)) + (cd.key & KEY_MASK);
    if (cd.d2 == d2min[o]) atomicMin(owner + o, cd.tri);
  }
}
struct TagResolve {
  static constexpr int kThreads = 256;
  Geo g;
  const Cand* cand;
  unsigned cap;
  const DevState* ds;
  const unsigned long long* d2min;
  unsigned* owner;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tag_resolve(bk, g, cand, cap, ds, d2min, owner); }
};

// Mark the winning (node, owner) pairs in the per-cell flag bytes, and in
// the per-line records the sweeps use: the first forcing index of every x-
// and z-line and of every y-line, per component.
__device__ __forceinline__ void tag_mark(const Blk& bk, const Geo& g, const Cand* __restrict__ cand, unsigned cap, const DevState* ds,
                           const unsigned long long* __restrict__ d2min, const unsigned* __restrict__ owner,
                           unsigned* flags32, const LineInfo& li) {
  const unsigned n = min(ds->ncand, cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const Cand cd = cand[e];
    const int c = (int)(cd.key >> 30);
    const long long node = cd.key & KEY_MASK;
    const long long o = comp_off(g, c) + node;
    if (cd.d2 == d2min[o] && cd.tri == owner[o]) {
      const int pl = planes(g, c);
      long long i, j, k;
      split3(node, g.nx, pl, i, j, k);
      const long long cell = cidx(g, i, j, k);
      atomicOr(flags32 + (cell >> 2), (unsigned)(1u << c) << (8 * (cell & 3)));
      atomicMin(li.x + line_x(g, c, j, k), (int)i);
      atomicMin(li.z + line_z(g, c, i, j), (int)k);
      atomicMin(li.y + line_y(g, c, i, k), (int)j);
    }
  }
}
struct TagMark {
  static constexpr int kThreads = 256;
  Geo g;
  const Cand* cand;
  unsigned cap;
  const DevState* ds;
  const unsigned long long* d2min;
  const unsigned* owner;
  unsigned* flags32;
  LineInfo li;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tag_mark(bk, g, cand, cap, ds, d2min, owner, flags32, li); }
};

__device__ __forceinline__ unsigned flag_of(const unsigned* flags32, long long cell) {
  return (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
}

// Boundary cells (Section 3.2): all six faces hold forcing nodes.  Checked
// once per cell, from the candidate that won the cell's lower x-face.
__device__ __forceinline__ void tag_boundary(const Blk& bk, const Geo& g, const Cand* __restrict__ cand, unsigned cap, const DevState* ds,
                               const unsigned long long* __restrict__ d2min, const unsigned* __restrict__ owner,
                               unsigned* flags32) {
  const unsigned n = min(ds->ncand, cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const Cand cd = cand[e];
    if ((cd.key >> 30) != 0) continue;
    const long long node = cd.key & KEY_MASK;
    if (!(cd.d2 == d2min[node] && cd.tri == owner[node])) continue;
    long long i, j, k;
    split3(node, g.nx, g.ny, i, j, k);
    const long long ip = (i + 1 == g.nx) ? 0 : i + 1, kp = (k + 1 == g.nz) ? 0 : k + 1;
    const long long cell = cidx(g, i, j, k);
    const unsigned f0 = flag_of(flags32, cell);
    bool all = (f0 & FLAG_U) && (f0 & FLAG_V) && (f0 & FLAG_W);
    all = all && (flag_of(flags32, cidx(g, ip, j, k)) & FLAG_U);
    all = all && (j + 1 < g.ny) && (flag_of(flags32, cidx(g, i, j + 1, k)) & FLAG_V);
    all = all && (flag_of(flags32, cidx(g, i, j, kp)) & FLAG_W);
    if (all) atomicOr(flags32 + (cell >> 2), (unsigned)FLAG_B << (8 * (cell & 3)));
  }
}
struct TagBoundary {
  static constexpr int kThreads = 256;
  Geo g;
  const Cand* cand;
  unsigned cap;
  const DevState* ds;
  const unsigned long long* d2min;
  const unsigned* owner;
  unsigned* flags32;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tag_boundary(bk, g, cand, cap, ds, d2min, owner, flags32); }
};

// ---------------------------------------------------------------------------
// deterministic compaction of the flag bytes: count, scan, write
// ---------------------------------------------------------------------------
constexpr int CMP_THREADS = 256;
constexpr int CMP_PER_THREAD = 16;   // one uint4 of flag bytes
constexpr int CMP_CHUNK = CMP_THREADS * CMP_PER_THREAD;

__device__ __forceinline__ void load16(const unsigned* flags32, long long ncell, long long cell0, uint8_t out[16]) {
  if (cell0 + 16 <= ncell) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(flags32 + (cell0 >> 2)));
    const unsigned wv[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int m = 0; m < 16; ++m) out[m] = (uint8_t)(wv[m >> 2] >> (8 * (m & 3)));
  } else {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const long long cell = cell0 + m;
      out[m] = cell < ncell ? (uint8_t)flag_of(flags32, cell) : 0;
    }
  }
}

__device__ __forceinline__ void cmp_count(const Blk& bk, const Geo& g, const unsigned* __restrict__ flags32,
                                                           unsigned* __restrict__ blk) {
  __shared__ unsigned red[4][CMP_THREADS / 32];
  const long long cell0 = (long long)bk.x * CMP_CHUNK + (long long)threadIdx.x * CMP_PER_THREAD;
  uint8_t f[16];
  load16(flags32, g.ncell, cell0, f);
  unsigned cnt[4] = {0, 0, 0, 0};
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    cnt[0] += f[m] & 1;
    cnt[1] += (f[m] >> 1) & 1;
    cnt[2] += (f[m] >> 2) & 1;
    cnt[3] += (f[m] >> 3) & 1;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned v = cnt[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned v = 0;
    for (int w = 0; w < CMP_THREADS / 32; ++w) v += red[threadIdx.x][w];
    blk[(long long)bk.x * 4 + threadIdx.x] = v;
  }
}
struct CmpCount {
  static constexpr int kThreads = CMP_THREADS;
  Geo g;
  const unsigned* flags32;
  unsigned* blk;
  __device__ __forceinline__ void operator()(const Blk& bk) const { cmp_count(bk, g, flags32, blk); }
};

// single block: exclusive scan of the per-block counts (in place), totals to ds
__device__ __forceinline__ void cmp_scan(const Blk& bk, unsigned* blk, int nblk, DevState* ds, unsigned fcap) {
  // block-wide exclusive scan of the per-block counts (integers: exact in any
  // order): per-thread runs of `per` blocks, warp shuffles, warp totals
  __shared__ unsigned wsum[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (nblk + 1023) / 1024;
  const int b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
  unsigned loc[4] = {0, 0, 0, 0}, inc[4];
  for (int b = b0; b < b1; ++b)
    for (int q = 0; q < 4; ++q) loc[q] += blk[4 * b + q];
  for (int q = 0; q < 4; ++q) {
    unsigned v = loc[q];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned nb = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += nb;
    }
    inc[q] = v;
    if (lane == 31) wsum[q][wid] = v;
  }
  __syncthreads();
  if (wid == 0) {
    for (int q = 0; q < 4; ++q) {
      unsigned v = wsum[q][lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned nb = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += nb;
      }
      wsum[q][lane] = v;   // inclusive over warps
    }
  }
  __syncthreads();
  unsigned run[4];
  for (int q = 0; q < 4; ++q) run[q] = inc[q] - loc[q] + (wid > 0 ? wsum[q][wid - 1] : 0u);
  for (int b = b0; b < b1; ++b)
    for (int q = 0; q < 4; ++q) {
      const unsigned v = blk[4 * b + q];
      blk[4 * b + q] = run[q];
      run[q] += v;
    }
  if (threadIdx.x == 0) {
    const unsigned n0 = wsum[0][31], n1 = wsum[1][31], n2 = wsum[2][31];
    ds->nforce_c[0] = n0;
    ds->nforce_c[1] = n1;
    ds->nforce_c[2] = n2;
    ds->nbound = wsum[3][31];
    ds->force_base[0] = 0;
    ds->force_base[1] = n0;
    ds->force_base[2] = n0 + n1;
    if ((unsigned long long)n0 + n1 + n2 > fcap || wsum[3][31] > fcap) atomicOr(&ds->err, ERR_LIST_OVERFLOW);
  }
}
struct CmpScan {
  static constexpr int kThreads = 1024;
  unsigned* blk;
  int nblk;
  DevState* ds;
  unsigned fcap;
  __device__ __forceinline__ void operator()(const Blk& bk) const { cmp_scan(bk, blk, nblk, ds, fcap); }
};

__device__ __forceinline__ void cmp_write(const Blk& bk, const Geo& g, const unsigned* __restrict__ flags32,
                                                           const unsigned* __restrict__ blk,
                                                           const unsigned* __restrict__ owner, const DevState* ds,
                                                           ForceNode* flist, unsigned* blist, unsigned fcap) {
  __shared__ unsigned wsum[4][CMP_THREADS / 32];
  const long long cell0 = (long long)bk.x * CMP_CHUNK + (long long)threadIdx.x * CMP_PER_THREAD;
  uint8_t f[16];
  load16(flags32, g.ncell, cell0, f);
  unsigned cnt[4] = {0, 0, 0, 0};
#pragma unroll
  for (int m = 0; m < 16; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) cnt[q] += (f[m] >> q) & 1;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  unsigned excl[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned v = cnt[q];
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += y;
    }
    excl[q] = v - cnt[q];
    if (lane == 31) wsum[q][wrp] = v;
  }
  __syncthreads();
  unsigned pos[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned before = 0;
    for (int w = 0; w < wrp; ++w) before += wsum[q][w];
    pos[q] = blk[(long long)bk.x * 4 + q] + before + excl[q];
  }
  const unsigned base[3] = {ds->force_base[0], ds->force_base[1], ds->force_base[2]};
  // (i, j, k) of the thread's first cell by one 32-bit division (node keys
  // hold 30 bits), then stepped along its 16 consecutive cells
  const unsigned nxu = (unsigned)g.nx, nyu = (unsigned)g.ny;
  unsigned ci = 0, cj = 0, ck = 0;
  if (cell0 < g.ncell) {
    const unsigned c0 = (unsigned)cell0, row = c0 / nxu;
    ci = c0 - row * nxu;
    cj = row % nyu;
    ck = row / nyu;
  }
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    if (f[m]) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if ((f[m] >> c) & 1) {
          const unsigned slot = base[c] + pos[c]++;
          const long long node = fidx(g, c, ci, cj, ck);
          if (slot < fcap) {
            ForceNode fn;
            fn.key = ((unsigned)c << 30) | (unsigned)node;
            fn.tri = owner[comp_off(g, c) + node];
            flist[slot] = fn;
          }
        }
      }
      if (f[m] & FLAG_B) {
        const unsigned slot = pos[3]++;
        if (slot < fcap) blist[slot] = (unsigned)(cell0 + m);
      }
    }
    if (++ci == nxu) {
      ci = 0;
      if (++cj == nyu) {
        cj = 0;
        ++ck;
      }
    }
  }
}
struct CmpWrite {
  static constexpr int kThreads = CMP_THREADS;
  Geo g;
  const unsigned* flags32;
  const unsigned* blk;
  const unsigned* owner;
  const DevState* ds;
  ForceNode* flist;
  unsigned* blist;
  unsigned fcap;
  __device__ __forceinline__ void operator()(const Blk& bk) const { cmp_write(bk, g, flags32, blk, owner, ds, flist, blist, fcap); }
};

// move this step's candidate count to "previous", zero the current one
__device__ __forceinline__ void copy_count(const Blk& bk, DevState* ds) {
  ds->ncand_prev = ds->ncand;
  ds->ncand = 0;
  ds->nub = 0;
  ds->nsurv = 0;
}
struct CopyCount {
  static constexpr int kThreads = 32;
  DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { copy_count(bk, ds); }
};

// ---------------------------------------------------------------------------
// host launcher: the whole tagging stage of one step
// ---------------------------------------------------------------------------
// Fill `n` words with `value` (the per-line records are reset every step;
// a kernel rather than a memset so that batches merge it like the rest).
__device__ __forceinline__ void fill32(const Blk& bk, unsigned* p, long long n, unsigned value) {
  const long long stride = (long long)bk.gx * blockDim.x;
  for (long long e = (long long)bk.x * blockDim.x + threadIdx.x; e < n; e += stride) p[e] = value;
}
struct Fill32 {
  static constexpr int kThreads = 256;
  unsigned* p;
  long long n;
  unsigned value;
  __device__ __forceinline__ void operator()(const Blk& bk) const { fill32(bk, p, n, value); }
};

void launch_tagging(const Geo& g, const Surf& s, const TagBuffers& b, DevState* ds, Exec& ex) {
  ex.mark(ST_TAG);
  const long long words = (long long)(b.lines.bytes / 4);
  // every line: "no forcing node" (0x7F7F7F7F exceeds any index)
  ex.launch(dim3((unsigned)std::min<long long>((words + 255) / 256, num_sms() * 4ll)), dim3(256), 0,
            Fill32{reinterpret_cast<unsigned*>(b.lines.x), words, 0x7F7F7F7Fu});
  // previous step's candidates reset their nodes, then the counters restart
  ex.launch(dim3(scaled_blocks(g, 8192, 4, num_sms() * 4)), dim3(256), 0,
            TagReset{g, b.cand, b.cap, ds, b.d2min, b.owner, b.flags32, b.ub, b.ublist});
  ex.launch(dim3(1), dim3(1), 0, CopyCount{ds});
  const bool live = s.nt > 0;
  ex.launch(grid_if(live, dim3((unsigned)((s.nt + 31) / 32))), dim3(32), 0, TriSetup{g, s});
  const long long blocks = ((long long)s.nt * 32 + 127) / 128;   // one warp per triangle
  ex.launch(grid_if(live, dim3((unsigned)blocks)), dim3(128), 0, TagPairs<0>{g, s, b.cap, b.ub, b.ublist, b.surv, ds});
  ex.launch(grid_if(live, dim3((unsigned)blocks)), dim3(128), 0, TagPairs<1>{g, s, b.cap, b.ub, b.ublist, b.surv, ds});
  // about one survivor per thread: the FP64 test is a latency chain
  ex.launch(grid_if(live, dim3(scaled_blocks(g, 2048, 8, num_sms() * 8))), dim3(128), 0,
            TagExact{g, s, b.cand, b.cap, b.d2min, b.surv, ds});
  const dim3 gb = grid_if(live, dim3(scaled_blocks(g, 4096, 8, num_sms() * 8)));
  ex.launch(gb, dim3(256), 0, TagResolve{g, b.cand, b.cap, ds, b.d2min, b.owner});
  ex.launch(gb, dim3(256), 0, TagMark{g, b.cand, b.cap, ds, b.d2min, b.owner, b.flags32, b.lines});
  ex.launch(gb, dim3(256), 0, TagBoundary{g, b.cand, b.cap, ds, b.d2min, b.owner, b.flags32});
  const int nblk = (int)((g.ncell + CMP_CHUNK - 1) / CMP_CHUNK);
  ex.launch(dim3(nblk), dim3(CMP_THREADS), 0, CmpCount{g, b.flags32, b.blk});
  ex.launch(dim3(1), dim3(1024), 0, CmpScan{b.blk, nblk, ds, b.cap});
  ex.launch(dim3(nblk), dim3(CMP_THREADS), 0, CmpWrite{g, b.flags32, b.blk, b.owner, ds, b.flist, b.blist, b.cap});
}

int compaction_blocks(const Geo& g) { return (int)((g.ncell + CMP_CHUNK - 1) / CMP_CHUNK); }

}  // namespace ibm
