// common.cuh -- device-side definitions shared by the kernels of the GB300
// sharp-interface IBM fractional step (arXiv 2606.09799).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ibm {

// Device error word bits (reported to the host at the next synchronising call).
constexpr unsigned ERR_PROBE = 1u;           // IB probe stencil left the stored planes
constexpr unsigned ERR_CAND_OVERFLOW = 2u;   // tagging candidate list overflowed
constexpr unsigned ERR_LIST_OVERFLOW = 4u;   // forcing / boundary list overflowed
constexpr unsigned ERR_NONFINITE = 8u;       // NaN/Inf met in a reduction
constexpr unsigned ERR_DEGENERATE = 16u;     // a triangle of zero area
constexpr unsigned ERR_WAIT = 32u;           // a bounded wait on an asynchronous copy ran out

// Per-cell flag bits: the velocity nodes of the cell's lower faces that are
// forcing nodes, and whether the cell is a boundary cell (Section 3.2).
constexpr uint8_t FLAG_U = 1, FLAG_V = 2, FLAG_W = 4, FLAG_B = 8;

// Wall-normal spacings of a non-uniform grid (Section 2: variable cell size
// in the wall-normal direction), device FP64 tables: ihc[j] = 1 / height of
// cell j (ny); ihf[j] = 1 / distance of the centres across face j (ny + 1;
// the wall faces measure to the mirror image of the first / last centre);
// hc[j] = height of cell j; hf[j] = distance of the centres across face j
// (ny + 1); yc[j + 1] = centre of row j for j in [-1, ny] and yv[j + 1] =
// face j for j in [-1, ny + 1], rows beyond a wall being mirror images;
// hmax = the largest of hc and hf.  ysw: the y sweep's rows for lines
// without forcing nodes (tangential components: a, 1/pivot, c' over ny rows;
// then v: the same over ny - 1 rows).  ysw2: for lines with forcing nodes,
// 1/pivot and c' of a segment that starts at row s, at [s][m] (tangential
// components: two ny x ny arrays; then v: two (ny-1) x (ny-1)); null when ny
// is above 1024.  yswf, ysw2f: their FP32 copies for the mixed path.  All
// null (0) on a uniform grid.
struct YTab {
  const double* ihc;
  const double* ihf;
  const double* hc;
  const double* hf;
  const double* yc;
  const double* yv;
  const double* ysw;
  const double* ysw2;
  const float* yswf;    // FP32 copies of ysw and ysw2 (mixed path), else null
  const float* ysw2f;
  // rows of the tagging pre-screen, FP32: for the face rows (v, [0][j]) and
  // the centre rows (u and w, [1][j]), j = 0..ny, at [half * (ny + 1) + j]:
  // (y_j, the wall-normal side of the node's local cell, y_j - y_{j-1},
  // y_{j+1} - y_j)
  const float4* rowf;
  double hmax;
};

// Grid as seen by every kernel (passed by value).
struct Geo {
  int nx, ny, nz, nkx;
  int ybc;                       // 0 no-slip, 1 free-slip on the y walls
  double lx, ly, lz;
  double dx, dy, dz;
  double idx, idy, idz;          // reciprocal spacings
  double diag2;                  // squared diagonal of a cell (Algorithm 1)
  double h;                      // probe length, twice the cell diagonal (Section 3.1)
  long long ncell;               // nx*ny*nz: size of u, w, p
  long long nvf;                 // nx*(ny+1)*nz: size of v
  YTab yt;                       // non-uniform wall-normal spacing, or null pointers
};

__host__ __device__ inline int planes(const Geo& g, int c) { return c == 1 ? g.ny + 1 : g.ny; }
__host__ __device__ inline long long comp_size(const Geo& g, int c) { return c == 1 ? g.nvf : g.ncell; }
// offset of component c inside arrays that hold the three grids back to back
__host__ __device__ inline long long comp_off(const Geo& g, int c) {
  return c == 0 ? 0 : (c == 1 ? g.ncell : g.ncell + g.nvf);
}
__host__ __device__ inline long long cidx(const Geo& g, long long i, long long j, long long k) {
  return (k * g.ny + j) * g.nx + i;
}
__host__ __device__ inline long long fidx(const Geo& g, int c, long long i, long long j, long long k) {
  return (k * planes(g, c) + j) * g.nx + i;
}
// Lattice indices of linear index `node` (< 2^30, the width of the node
// keys) on a grid of nx x pl x nz points, by 32-bit division.
__host__ __device__ inline void split3(long long node, int nx, int pl, long long& i, long long& j, long long& k) {
  const unsigned nu = (unsigned)node, row = nu / (unsigned)nx;
  i = (long long)(nu - row * (unsigned)nx);
  j = (long long)(row % (unsigned)pl);
  k = (long long)(row / (unsigned)pl);
}
__host__ __device__ inline int wrapi(long long i, int n) {
  long long r = i % n;
  return (int)(r < 0 ? r + n : r);
}

// Device-resident scalars of a handle: inputs refreshed between steps and
// reduction results, so a captured graph never bakes values in.
struct DevState {
  double fb[3];                  // uniform body force
  float fbf[3];                  // the same in FP32 (the FP32 kernels read it without a conversion)
  double qf[2];                  // q_F of each sub-stage
  float qf_hi[2], qf_lo[2];      // q_F as an unevaluated FP32 pair (mixed correction)
  double sum_a[2];               // sum over C_B of D uhat dV per sub-stage
  double qa[2], qb[2];           // energy-conserving shape: q_F^k = qa + qb (p^k - e^k) (App. B)
  double sum_qdv[2];             // sum over all cells of q dV
  double slip_sum[3];            // sum |eps_i| of the last step
  double div_max;                // max over C_F of |D u - q| after the last projection of the step
  double ke;                     // kinetic energy 1/2 sum u^2 dV of the step's result
  double cfl;                    // CFL number of the step's result
  unsigned int res1[2];          // mixed path: bits of max over C_F of |D u' - q| (FP32) after the first solve
                                 // of each sub-stage, u' the once-projected state
  float div_budget;              // the correction solve runs when that residual exceeds it (NaN: runs)
  unsigned long long ncorr;      // correction solves taken
  unsigned int err;              // ERR_* bits
  unsigned int ncand;            // candidates of the current step
  unsigned int ncand_prev;       // candidates of the previous step (sparse reset)
  unsigned int nub;              // nodes with an |N|^2 bound this step (sparse reset)
  unsigned int nsurv;            // pairs listed for the exact tagging test this step
  unsigned int nbound;           // boundary cells
  unsigned int nforce_c[3];      // forcing nodes per component
  unsigned int force_base[3];    // start of each component's forcing sub-list
  unsigned long long steps;
};

// One (node, triangle) pair that passed Algorithm 1.
struct Cand {
  unsigned int key;              // comp << 30 | node index inside the component's array
  unsigned int tri;
  unsigned long long d2;         // bit pattern of |N|^2 (monotone for d2 >= 0)
};

// One forcing node with its owning triangle.
struct ForceNode {
  unsigned int key;
  unsigned int tri;
};

constexpr unsigned KEY_MASK = (1u << 30) - 1u;

struct TriRec;

// Surface as stored on the device (structure of arrays).
struct Surf {
  const double* x;               // x[nv], then y[nv], then z[nv]
  const double* u;               // vertex velocities, same layout
  const int* t;                  // vertex a of every triangle, then b, then c
  TriRec* rec;                   // per-triangle constants of the current step (nt)
  int nv, nt;
};

// Scheme coefficients of one sub-stage (Section 2 after Eq. NS_prov).
struct Stage {
  double gam, rho, alp;
  int s;                          // sub-stage index
};

// ---- FP32 <-> FP64 conversions on the integer pipes ------------------------
// On this GPU a hardware FP32 <-> FP64 conversion occupies the narrow FP64
// pipe for about as long as two FP64 FMAs.  Both directions are written here
// from the IEEE 754 binary32 / binary64 encodings: widening moves the sign,
// exponent and mantissa fields (exact); narrowing truncates the mantissa to
// 23 bits and rounds to nearest, ties to even, from the round and sticky
// bits.  Zero and every normal result take this path; subnormal, infinite
// or NaN operands set `special`, and the caller redoes the batch with the
// hardware conversions (a warp-uniform branch that ordinary data never
// takes), so the results are those of the hardware conversions bit for bit.
__device__ __forceinline__ double f2d_int(float f, bool& special) {
  const unsigned b = __float_as_uint(f);
  const unsigned e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  special |= (e == 0u && m != 0u) || e == 0xFFu;
  const unsigned hi = (b & 0x80000000u) | (e ? (((e + 896u) << 20) | (m >> 3)) : 0u);
  return __hiloint2double((int)hi, (int)(m << 29));
}
__device__ __forceinline__ float d2f_int(double d, bool& special) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ah = hi & 0x7FFFFFFFu, e = ah >> 20;
  const bool zero = ah == 0u && lo == 0u;
  special |= !zero && (e < 897u || e > 1150u);   // outside the normal binary32 exponents
  unsigned fb = ((e - 896u) << 23) | ((ah & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned rnd = (lo >> 28) & 1u, sticky = (lo & 0x0FFFFFFFu) != 0u, lsb = (lo >> 29) & 1u;
  fb += rnd & (sticky | lsb);                      // a carry moves into the exponent, as it should
  return __uint_as_float((hi & 0x80000000u) | (zero ? 0u : fb));
}

// Sum of n partial values p[b * stride + off] by one warp in a fixed order:
// lane l adds b = l, l + 32, ... in turn, then a butterfly of pairwise sums.
// Every lane returns the same value (each pairwise add is commutative), and
// the result depends only on n and the data.
__device__ __forceinline__ double warp_sum_fixed(const double* __restrict__ p, int n, int stride, int off) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
#pragma unroll 4
  for (int b = lane; b < n; b += 32) s += p[(long long)b * stride + off];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  return s;
}

// ---- unevaluated FP32 pairs (hi + lo): error-free transformations ----------
// s + e == a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// p + e == a * b exactly (fused multiply-add residual)
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);   // rounded product, never contracted into a later add
  e = fmaf(a, b, -p);
}
// (hi, lo) <- (hi, lo) + d, renormalised
__device__ __forceinline__ void ff_add(float& hi, float& lo, float d) {
  float s, e;
  two_sum(hi, d, s, e);
  const float t = lo + e;
  const float h2 = s + t;
  lo = t - (h2 - s);
  hi = h2;
}

}  // namespace ibm
