// noalloc.cu -- tagging of the forcing nodes (Algorithm 1) for callers that
// must not allocate device memory.  The result is identical, bit for bit, to
// the tags a simulation handle on a uniform grid (ibm_create_grid) computes
// (ibm_step followed by ibm_get_tags);
// the working memory lives in a fixed, file-scope device array instead of
// buffers allocated per handle.
#include "../../include/ibm.h"
#include "common.cuh"
#include "geometry.cuh"

namespace ibm {

// Working memory of ibm_tag_noalloc: the smallest |N|^2 seen so far at every
// node of the three grids (bit pattern of the FP64 value), plus one word
// that records a triangle with a vertex index out of range.  It belongs to
// the library and is held on every GPU that loads it until the process ends.
static __device__ __align__(256) unsigned long long g_noalloc_d2[IBM_NOALLOC_MAX_NODES];
static __device__ __align__(256) unsigned g_noalloc_bad[64];

namespace {

// Device addresses of the working memory on the current device.  Host code
// cannot use the symbols' addresses directly; they are looked up on every
// call (a host-side query once the library's device code is loaded), so a
// device reset or a new primary context never leaves a stale address.
cudaError_t noalloc_setup(unsigned long long** d2, unsigned** bad) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_d2);
  if (e != cudaSuccess) return e;
  *d2 = static_cast<unsigned long long*>(p);
  e = cudaGetSymbolAddress(&p, g_noalloc_bad);
  if (e != cudaSuccess) return e;
  *bad = static_cast<unsigned*>(p);
  return cudaSuccess;
}

__global__ void k_na_init(unsigned long long* d2, long long nall, unsigned* own, long long nown, unsigned* bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nall; i += stride) d2[i] = ~0ull;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nown; i += stride) own[i] = 0xFFFFFFFFu;
  if (blockIdx.x == 0 && threadIdx.x == 0) bad[0] = 0u;
}

struct Owners {
  unsigned* o[3];
};

// One warp per triangle, lanes over the Eulerian points of the three grids
// inside its box, the test of Algorithm 1 per point (same arithmetic as the
// handle's tagging).  phase 0: fold |N|^2 into the per-node minimum;
// phase 1: among the pairs achieving it, keep the smallest triangle index.
__global__ void __launch_bounds__(128) k_na_tag(Geo g, const double* __restrict__ xyz, int nv,
                                                const int* __restrict__ tri, int nt, unsigned long long* d2,
                                                Owners own, unsigned* bad, int phase) {
  const int lane = threadIdx.x & 31;
  const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (t >= nt) return;
  const int va = tri[3 * t], vb = tri[3 * t + 1], vc = tri[3 * t + 2];
  if (va < 0 || va >= nv || vb < 0 || vb >= nv || vc < 0 || vc >= nv) {
    if (lane == 0) atomicOr(bad, 1u);
    return;
  }
  double A[3], B[3], C[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    A[d] = xyz[3ll * va + d];
    B[d] = xyz[3ll * vb + d];
    C[d] = xyz[3ll * vc + d];
  }
  TriConst TC;
  tri_const(A, B, C, TC);
  const double del[3] = {g.dx, g.dy, g.dz};
  const double idel[3] = {g.idx, g.idy, g.idz};
  double lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = dsub(fmin(A[d], fmin(B[d], C[d])), del[d]);
    hi[d] = dadd(fmax(A[d], fmax(B[d], C[d])), del[d]);
  }
  long long r0[3][2], r1[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) exact_range(lo[d], hi[d], del[d], idel[d], hf, r0[d][hf], r1[d][hf]);
  long long n0[3][3], ext[3][3], cnt[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    long long prod = 1;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int hf = (d == c) ? 0 : 1;
      long long a0 = r0[d][hf], a1 = r1[d][hf];
      if (d == 1) {
        const long long jlo = c == 1 ? 1 : 0;
        a0 = a0 < jlo ? jlo : a0;
        a1 = a1 > g.ny - 1 ? g.ny - 1 : a1;
      }
      n0[c][d] = a0;
      ext[c][d] = a1 - a0 + 1;
      prod *= ext[c][d] > 0 ? ext[c][d] : 0;
    }
    cnt[c] = prod;
  }
  const long long total = cnt[0] + cnt[1] + cnt[2];
  for (long long n = lane; n < total; n += 32) {
    const int c = n < cnt[0] ? 0 : (n < cnt[0] + cnt[1] ? 1 : 2);
    const long long q = n - (c == 0 ? 0 : (c == 1 ? cnt[0] : cnt[0] + cnt[1]));
    const long long ni = ext[c][0], nj = ext[c][1];
    const long long idx3[3] = {n0[c][0] + q % ni, n0[c][1] + (q / ni) % nj, n0[c][2] + q / (ni * nj)};
    double x[3], X[3], wb[3], N[3], P[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) x[d] = lat(idx3[d], del[d], d == c ? 0 : 1);
    closest_point_exact(x, TC, X, wb);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      N[d] = dsub(x[d], X[d]);
      P[d] = dmul(N[d], N[d]);
    }
    const double n2 = dadd(dadd(P[0], P[1]), P[2]);
    if (!(n2 <= g.diag2)) continue;
    bool tagged = n2 == 0.0;
#pragma unroll
    for (int d = 0; d < 3 && !tagged; ++d) {
#pragma unroll
      for (int sg = -1; sg <= 1 && !tagged; sg += 2) {
        const double vd = dsub(lat(idx3[d] + sg, del[d], d == c ? 0 : 1), X[d]);
        const double Q = dmul(N[d], vd);
        const double dot = d == 0 ? dadd(dadd(Q, P[1]), P[2])
                                  : (d == 1 ? dadd(dadd(P[0], Q), P[2]) : dadd(dadd(P[0], P[1]), Q));
        if (dot < 0.0) tagged = true;
      }
    }
    if (!tagged) continue;
    const long long node = fidx(g, c, wrapi(idx3[0], g.nx), idx3[1], wrapi(idx3[2], g.nz));
    const unsigned long long bits = (unsigned long long)__double_as_longlong(n2);
    if (phase == 0) atomicMin(d2 + comp_off(g, c) + node, bits);
    else if (bits == d2[comp_off(g, c) + node]) atomicMin(own.o[c] + node, (unsigned)t);
  }
}

}  // namespace
}  // namespace ibm

using namespace ibm;

extern "C" ibm_status ibm_tag_noalloc(const ibm_grid_desc* desc, int nverts, const double* xyz, int ntris,
                                      const int32_t* tri, int32_t* owner_u, int32_t* owner_v, int32_t* owner_w,
                                      void* stream) {
  if (!desc || nverts < 0 || ntris < 0 || !owner_u || !owner_v || !owner_w) return IBM_ERR_ARG;
  if (ntris > 0 && (!xyz || !tri)) return IBM_ERR_ARG;
  const ibm_grid_desc d = *desc;
  if (d.nx < 1 || d.ny < 2 || d.nz < 1 || !(d.lx > 0 && d.ly > 0 && d.lz > 0)) return IBM_ERR_ARG;
  if (d.ybc != IBM_NOSLIP && d.ybc != IBM_FREESLIP) return IBM_ERR_ARG;
  // the grid as the simulation handles see it (same formulas, same rounding)
  Geo g{};
  g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.nkx = d.nx / 2 + 1;
  g.ybc = d.ybc;
  g.lx = d.lx; g.ly = d.ly; g.lz = d.lz;
  g.dx = d.lx / (double)d.nx;
  g.dy = d.ly / (double)d.ny;
  g.dz = d.lz / (double)d.nz;
  g.idx = 1.0 / g.dx; g.idy = 1.0 / g.dy; g.idz = 1.0 / g.dz;
  {
    volatile double sx = g.dx * g.dx, sy = g.dy * g.dy, sz = g.dz * g.dz;
    volatile double sxy = sx + sy;
    g.diag2 = sxy + sz;
  }
  g.ncell = (long long)d.nx * d.ny * d.nz;
  g.nvf = (long long)d.nx * (d.ny + 1) * d.nz;
  const long long nall = 2 * g.ncell + g.nvf;
  if (nall > IBM_NOALLOC_MAX_NODES) return IBM_ERR_CAPACITY;
  unsigned long long* d2 = nullptr;
  unsigned* bad = nullptr;
  if (noalloc_setup(&d2, &bad) != cudaSuccess) return IBM_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // the three owner arrays are cleared one after the other (they need not
  // be contiguous)
  k_na_init<<<256, 256, 0, st>>>(d2, nall, reinterpret_cast<unsigned*>(owner_u), g.ncell, bad);
  k_na_init<<<256, 256, 0, st>>>(d2, 0, reinterpret_cast<unsigned*>(owner_v), g.nvf, bad);
  k_na_init<<<256, 256, 0, st>>>(d2, 0, reinterpret_cast<unsigned*>(owner_w), g.ncell, bad);
  if (ntris > 0) {
    Owners own{{reinterpret_cast<unsigned*>(owner_u), reinterpret_cast<unsigned*>(owner_v),
                reinterpret_cast<unsigned*>(owner_w)}};
    const unsigned blocks = (unsigned)(((long long)ntris * 32 + 127) / 128);
    k_na_tag<<<blocks, 128, 0, st>>>(g, xyz, nverts, tri, ntris, d2, own, bad, 0);
    k_na_tag<<<blocks, 128, 0, st>>>(g, xyz, nverts, tri, ntris, d2, own, bad, 1);
  }
  if (cudaGetLastError() != cudaSuccess) return IBM_ERR_CUDA;
  unsigned hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) return IBM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return IBM_ERR_CUDA;
  return hbad ? IBM_ERR_ARG : IBM_OK;
}
