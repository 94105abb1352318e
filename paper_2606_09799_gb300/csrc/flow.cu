// flow.cu -- provisional velocity of the fractional step (Section 2 and
// Section 3.1 of arXiv 2606.09799):
//   IB step on the forcing nodes (Eqs. IB_step, probe, new_IB),
//   explicit right-hand side of Eq. NS_prov on the fluid nodes,
//   approximate factorisation of the CN operator, solved direction by
//   direction (x, then z, then y) with the Thomas algorithm,
//   and the no-slip error of Section 4.4 on the forcing points.
// Bulk arithmetic is templated on T (double: FP64 path, float: mixed path);
// geometry is always FP64.
#include <math.h>

#include "common.cuh"
#include "geometry.cuh"
#include <cuda.h>
#include <mutex>
#include "launch.h"
#include "mbar.cuh"

namespace ibm {

template <typename T>
__device__ __forceinline__ T* comp_ptr(const Fields<T>& f, int c) {
  return c == 0 ? f.u : (c == 1 ? f.v : f.w);
}

// Trilinear interpolation of component c at P from the 8 surrounding nodes
// of the same staggered lattice.  x and z wrap; in y the stencil must lie
// in the stored planes (u, w: 0..ny-1; v: 0..ny with the wall planes).
// On the non-uniform wall-normal grid the bracketing rows come from a
// bisection over the row table and the y weight from their coordinates.
template <typename T>
__device__ bool trilinear(const Geo& g, int c, const T* __restrict__ f, const double P[3], double* out) {
  const double sx = P[0] * g.idx - (c == 0 ? 0.0 : 0.5);
  const double sy = P[1] * g.idy - (c == 1 ? 0.0 : 0.5);
  const double sz = P[2] * g.idz - (c == 2 ? 0.0 : 0.5);
  const double fx = floor(sx), fy = floor(sy), fz = floor(sz);
  const long long i0 = (long long)fx, k0 = (long long)fz;
  long long j0 = (long long)fy;
  double ty = sy - fy;
  if (g.yt.yc) {
    const int half = c != 1;
    const long long jmax = planes(g, c) - 1;
    if (!(ylat(g, 0, half) <= P[1] && P[1] < ylat(g, jmax, half))) return false;
    long long a = 0, b = jmax;   // ylat(a) <= P[1] < ylat(b)
    while (b - a > 1) {
      const long long m = (a + b) >> 1;
      if (ylat(g, m, half) <= P[1]) a = m; else b = m;
    }
    j0 = a;
    const double ya = ylat(g, a, half);
    ty = (P[1] - ya) / (ylat(g, a + 1, half) - ya);
  }
  if (j0 < 0 || j0 + 1 > planes(g, c) - 1) return false;
  const double tx = sx - fx, tz = sz - fz;
  const int ia = wrapi(i0, g.nx), ib = wrapi(i0 + 1, g.nx);
  const int ka = wrapi(k0, g.nz), kb = wrapi(k0 + 1, g.nz);
  const int pl = planes(g, c);
  auto at = [&](int i, long long j, int k) { return (double)f[((long long)k * pl + j) * g.nx + i]; };
  const double c00 = (1.0 - tx) * at(ia, j0, ka) + tx * at(ib, j0, ka);
  const double c10 = (1.0 - tx) * at(ia, j0 + 1, ka) + tx * at(ib, j0 + 1, ka);
  const double c01 = (1.0 - tx) * at(ia, j0, kb) + tx * at(ib, j0, kb);
  const double c11 = (1.0 - tx) * at(ia, j0 + 1, kb) + tx * at(ib, j0 + 1, kb);
  const double c0 = (1.0 - ty) * c00 + ty * c10;
  const double c1 = (1.0 - ty) * c01 + ty * c11;
  *out = (1.0 - tz) * c0 + tz * c1;
  return true;
}

// Geometry of one forcing node: position (periodic image nearest to the
// owning triangle), closest point, normal vector and the wall velocity U.
struct NodeGeom {
  double x[3], X[3], N[3], n2, U;
  double h;   // probe length: twice the diagonal of the node's local cell (Section 3.1)
};

__device__ inline void forcing_geometry(const Geo& g, const Surf& s, unsigned key, unsigned tri, NodeGeom& ng) {
  const int c = (int)(key >> 30);
  const long long node = key & KEY_MASK;
  const int pl = planes(g, c);
  long long i, j, k;
  split3(node, g.nx, pl, i, j, k);
  const int va = __ldg(s.t + tri), vb = __ldg(s.t + s.nt + tri), vc = __ldg(s.t + 2 * (long long)s.nt + tri);
  // the triangle's constants of this step (formed by the tagging set-up)
  const TriRec* __restrict__ R = s.rec + tri;
  node_pos(g, c, i, j, k, ng.x);
  const long long mi = llround((R->cen[0] - ng.x[0]) / g.lx);
  const long long mk = llround((R->cen[2] - ng.x[2]) / g.lz);
  if (mi != 0 || mk != 0) node_pos(g, c, i + mi * g.nx, j, k + mk * g.nz, ng.x);
  double wb[3];
  const TriConst TC = R->tc;
  closest_point_exact(ng.x, TC, ng.X, wb);
#pragma unroll
  for (int d = 0; d < 3; ++d) ng.N[d] = dsub(ng.x[d], ng.X[d]);
  ng.n2 = ddot(ng.N, ng.N);
  const long long nv = s.nv;
  ng.U = wb[0] * __ldg(s.u + c * nv + va) + wb[1] * __ldg(s.u + c * nv + vb) + wb[2] * __ldg(s.u + c * nv + vc);
  ng.h = g.yt.yc ? 2.0 * sqrt(diag2_at(g, c, j)) : g.h;
}

// Probe of one forcing node (Eq. probe): point x^e = X + h N/|N|,
// alpha = |N| / h (0 for a node on the surface, which takes U) and the wall
// velocity U.  The surface is that of step n in every sub-stage, so the
// step's first forcing launch computes it (geom) and stores it; the second
// sub-stage and the no-slip error read it back.
__device__ __forceinline__ void forcing_probe(const Geo& g, const Surf& s, const ForceNode& fn, double* __restrict__ rec,
                                              bool geom, double xe[3], double& alpha, double& U) {
  if (geom) {
    NodeGeom ng;
    forcing_geometry(g, s, fn.key, fn.tri, ng);
    U = ng.U;
    alpha = 0.0;
    for (int d = 0; d < 3; ++d) xe[d] = ng.X[d];
    if (ng.n2 != 0.0) {
      const double nl = sqrt(ng.n2);
#pragma unroll
      for (int d = 0; d < 3; ++d) xe[d] = ng.X[d] + ng.h * (ng.N[d] / nl);
      alpha = nl / ng.h;
    }
    rec[0] = xe[0];
    rec[1] = xe[1];
    rec[2] = xe[2];
    rec[3] = alpha;
    rec[4] = U;
  } else {
    xe[0] = rec[0];
    xe[1] = rec[1];
    xe[2] = rec[2];
    alpha = rec[3];
    U = rec[4];
  }
}

// Eq. new_IB for every forcing node, reading u^e from the unmodified state
// (a snapshot: the values are written by a second kernel).
template <typename T>
__device__ __forceinline__ void ib_force(const Blk& bk, const Geo& g, const Surf& s, const Fields<T>& f, const ForceNode* __restrict__ flist, unsigned cap,
                           DevState* ds, double* __restrict__ probe, bool geom) {
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const ForceNode fn = flist[e];
    const int c = (int)(fn.key >> 30);
    double xe[3], alpha, U;
    forcing_probe(g, s, fn, probe + 5ull * e, geom, xe, alpha, U);
    double uf = U;
    if (alpha != 0.0) {
      double ue;
      if (!trilinear<T>(g, c, comp_ptr(f, c), xe, &ue)) {
        atomicOr(&ds->err, ERR_PROBE);
        ue = 0.0;
      }
      uf = (1.0 - alpha) * U + alpha * ue;
    }
    f.uf[e] = (T)uf;
  }
}
template <typename T>
struct IbForce {
  static constexpr int kThreads = 128;
  Geo g;
  Surf s;
  Fields<T> f;
  const ForceNode* flist;
  unsigned cap;
  DevState* ds;
  double* probe;
  int geom;
  __device__ __forceinline__ void operator()(const Blk& bk) const { ib_force<T>(bk, g, s, f, flist, cap, ds, probe, geom != 0); }
};

template <typename T>
__device__ __forceinline__ void ib_scatter(const Blk& bk, const Fields<T>& f, const ForceNode* __restrict__ flist, unsigned cap, const DevState* ds) {
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  for (unsigned e = bk.x * blockDim.x + threadIdx.x; e < n; e += bk.gx * blockDim.x) {
    const ForceNode fn = flist[e];
    const int c = (int)(fn.key >> 30);
    comp_ptr(f, c)[fn.key & KEY_MASK] = f.uf[e];
    if (f.lo[c]) f.lo[c][fn.key & KEY_MASK] = (T)0;
  }
}
template <typename T>
struct IbScatter {
  static constexpr int kThreads = 256;
  Fields<T> f;
  const ForceNode* flist;
  unsigned cap;
  const DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { ib_scatter<T>(bk, f, flist, cap, ds); }
};

template <typename T>
void launch_ib_force(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds, bool geom,
                     Exec& ex) {
  const dim3 gb = grid_if(s.nt > 0, dim3(scaled_blocks(g, 4096, 8, num_sms() * 4)));
  ex.mark(ST_FORCE);
  ex.launch(gb, dim3(128), 0, IbForce<T>{g, s, f, b.flist, b.cap, ds, b.probe, geom ? 1 : 0});
  ex.launch(gb, dim3(256), 0, IbScatter<T>{f, b.flist, b.cap, ds});
}

// ---------------------------------------------------------------------------
// Explicit right-hand side of Eq. NS_prov in delta form:
//   R = dt [gamma H^s + rho H^{s-1} - alpha G p^s + alpha/Re L u^s + alpha f]
// on fluid nodes, R = 0 on forcing nodes.  H = -div(u u) in conservative
// form with arithmetic averages of neighbouring nodes onto cell centres
// (normal fluxes) and cell edges (cross fluxes); v = 0 on the walls; the
// tangential components see the ghost value u_{-1} = gs u_0 beyond a wall
// (gs = -1 no-slip at rest, +1 free-slip).
// ---------------------------------------------------------------------------
// Scalar coefficients of one sub-stage in the bulk type, formed once on the
// host (no per-thread FP64 arithmetic in the FP32 path).
template <typename T>
struct RhsCoef {
  T idx, idy, idz, idx2, idy2, idz2;
  T gs;                 // wall ghost sign of the tangential components
  T cg, cr, ca, cv;     // gamma, rho, alpha, alpha / Re
  T dt;
  T fba;                // alpha, multiplying the body force read from the device state
};

// I: the index type -- int where every field has fewer than 2^31 entries
// (the 64-bit address arithmetic would otherwise take a large share of this
// issue-bound kernel's instructions), else long long.
template <typename T, bool NU, typename I>
__device__ __forceinline__ void rhs(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32, const RhsCoef<T>& cf,
                                             int use_hp, int write_h, const DevState* ds) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const T idx = cf.idx, idy = cf.idy, idz = cf.idz;
  const T idx2 = cf.idx2, idy2 = cf.idy2, idz2 = cf.idz2;
  const T gs = cf.gs;
  const T q = (T)0.25;
  const T cg = cf.cg, cr = cf.cr, ca = cf.ca, cv = cf.cv, tdt = cf.dt;
  // (the FP32 path reads the force's FP32 copy: a conversion would occupy
  // the narrow FP64 pipe once per thread)
  T fbx, fby, fbz;
  if constexpr (sizeof(T) == 4) {
    fbx = cf.fba * ds->fbf[0];
    fby = cf.fba * ds->fbf[1];
    fbz = cf.fba * ds->fbf[2];
  } else {
    fbx = cf.fba * (T)ds->fb[0];
    fby = cf.fba * (T)ds->fb[1];
    fbz = cf.fba * (T)ds->fb[2];
  }
  const I pv = (I)(ny + 1) * nx;   // v plane stride (k)
  const I pu = (I)ny * nx;         // u, w, p plane stride
  const T* __restrict__ U = f.u;
  const T* __restrict__ V = f.v;
  const T* __restrict__ W = f.w;
  const T* __restrict__ P = f.p;
  {
    const int i = bk.x * blockDim.x + threadIdx.x;
    const int j = bk.y * blockDim.y + threadIdx.y;
    const int k = bk.z;
    if (i >= nx || j >= ny) return;
    const I cell = (I)k * pu + (I)j * nx + i;
    const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
    const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
    const I r0 = (I)k * pu + (I)j * nx;      // row (j,k) of u, w, p
    const I rkp = (I)kp * pu + (I)j * nx, rkm = (I)km * pu + (I)j * nx;
    const I v0 = (I)k * pv + (I)j * nx;      // row (j,k) of v
    const I v1 = v0 + nx;                    // row (j+1,k) of v
    const I vkm0 = (I)km * pv + (I)j * nx, vkp0 = (I)kp * pv + (I)j * nx;
    const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
    const bool jlo = j == 0, jhi = j + 1 == ny;
    const T pc = P[r0 + i];
    // non-uniform wall-normal spacing: this row's inverse cell height and
    // centre distances below / above (the wall ghosts at mirrored distances)
    constexpr bool nun = NU;
    const T ihc = nun ? (T)g.yt.ihc[j] : idy, ihs = nun ? (T)g.yt.ihf[j] : idy, ihn = nun ? (T)g.yt.ihf[j + 1] : idy;
    // ---------------- u at (i dx, (j+1/2) dy, (k+1/2) dz) ----------------
    {
      const T uc = U[r0 + i], ue = U[r0 + ip], uw = U[r0 + im];
      const T un = jhi ? gs * uc : U[r0 + nx + i];
      const T us = jlo ? gs * uc : U[r0 - nx + i];
      const T uf = U[rkp + i], ub = U[rkm + i];
      const T adx = ((uc + ue) * (uc + ue) - (uw + uc) * (uw + uc)) * q * idx;
      const T vt = jhi ? (T)0 : (V[v1 + im] + V[v1 + i]) * (uc + un);
      const T vb = jlo ? (T)0 : (V[v0 + im] + V[v0 + i]) * (us + uc);
      const T ady = (vt - vb) * q * ihc;
      const T wf = (W[rkp + im] + W[rkp + i]) * (uc + uf);
      const T wb = (W[r0 + im] + W[r0 + i]) * (ub + uc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((un - uc) * ihn - (uc - us) * ihs) * ihc : (un - (T)2 * uc + us) * idy2;
      const T lap = (ue - (T)2 * uc + uw) * idx2 + lapy + (uf - (T)2 * uc + ub) * idz2;
      const T G = (pc - P[r0 + im]) * idx;
      T r = cg * H - ca * G + cv * lap + fbx;
      if (use_hp) r += cr * f.Hp[0][r0 + i];
      if (write_h) f.H[0][r0 + i] = H;
      f.R[0][r0 + i] = (fl & FLAG_U) ? (T)0 : tdt * r;
    }
    // ---------------- w at ((i+1/2) dx, (j+1/2) dy, k dz) ----------------
    {
      const T wc = W[r0 + i], we = W[r0 + ip], ww = W[r0 + im];
      const T wn = jhi ? gs * wc : W[r0 + nx + i];
      const T ws = jlo ? gs * wc : W[r0 - nx + i];
      const T wf = W[rkp + i], wb = W[rkm + i];
      const T ue = (U[rkm + ip] + U[r0 + ip]) * (wc + we);
      const T uw = (U[rkm + i] + U[r0 + i]) * (ww + wc);
      const T adx = (ue - uw) * q * idx;
      const T vt = jhi ? (T)0 : (V[vkm0 + nx + i] + V[v1 + i]) * (wc + wn);
      const T vb = jlo ? (T)0 : (V[vkm0 + i] + V[v0 + i]) * (ws + wc);
      const T ady = (vt - vb) * q * ihc;
      const T adz = ((wc + wf) * (wc + wf) - (wb + wc) * (wb + wc)) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((wn - wc) * ihn - (wc - ws) * ihs) * ihc : (wn - (T)2 * wc + ws) * idy2;
      const T lap = (we - (T)2 * wc + ww) * idx2 + lapy + (wf - (T)2 * wc + wb) * idz2;
      const T G = (pc - P[rkm + i]) * idz;
      T r = cg * H - ca * G + cv * lap + fbz;
      if (use_hp) r += cr * f.Hp[2][r0 + i];
      if (write_h) f.H[2][r0 + i] = H;
      f.R[2][r0 + i] = (fl & FLAG_W) ? (T)0 : tdt * r;
    }
    // ---------------- v at ((i+1/2) dx, j dy, (k+1/2) dz), 1 <= j <= ny-1 ----------------
    if (j >= 1) {
      const T vc = V[v0 + i], ve = V[v0 + ip], vw = V[v0 + im];
      const T vn = V[v1 + i], vs = V[v0 - nx + i];
      const T vf = V[vkp0 + i], vbk = V[vkm0 + i];
      const T ue = (U[r0 - nx + ip] + U[r0 + ip]) * (vc + ve);
      const T uw = (U[r0 - nx + i] + U[r0 + i]) * (vw + vc);
      const T adx = (ue - uw) * q * idx;
      const T ady = ((vc + vn) * (vc + vn) - (vs + vc) * (vs + vc)) * q * ihs;
      const T wf = (W[rkp - nx + i] + W[rkp + i]) * (vc + vf);
      const T wb = (W[r0 - nx + i] + W[r0 + i]) * (vbk + vc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((vn - vc) * ihc - (vc - vs) * (T)g.yt.ihc[j - 1]) * ihs : (vn - (T)2 * vc + vs) * idy2;
      const T lap = (ve - (T)2 * vc + vw) * idx2 + lapy + (vf - (T)2 * vc + vbk) * idz2;
      const T G = (pc - P[r0 - nx + i]) * ihs;
      T r = cg * H - ca * G + cv * lap + fby;
      if (use_hp) r += cr * f.Hp[1][v0 + i];
      if (write_h) f.H[1][v0 + i] = H;
      f.R[1][v0 + i] = (fl & FLAG_V) ? (T)0 : tdt * r;
    } else {
      // wall planes of v carry no unknown
      f.R[1][v0 + i] = (T)0;
      f.R[1][(I)k * pv + (I)ny * nx + i] = (T)0;
      if (write_h) {
        f.H[1][v0 + i] = (T)0;
        f.H[1][(I)k * pv + (I)ny * nx + i] = (T)0;
      }
    }
  }
}
template <typename T, bool NU, typename I = long long>
struct Rhs {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  RhsCoef<T> cf;
  int use_hp;
  int write_h;
  const DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { rhs<T, NU, I>(bk, g, f, flags32, cf, use_hp, write_h, ds); }
};

// Tiled form of the same right-hand side: a block of 32 x 4 threads takes a
// tile of 32 x 4 cells in (i, j) and marches through RT_KC planes of k.  The
// planes k-1, k, k+1 of u, v, w and k-1, k of p, each with a one-cell halo in
// i and j, sit in shared memory rings, so a step loads one new plane per
// field (its own cell plus a share of the halo) and every neighbour the
// stencil takes comes from shared memory.  The arithmetic is the per-cell
// kernel's, term by term, so both give the same values.
constexpr int RT_TI = 32, RT_TJ = 4, RT_KC = 16;
constexpr int RT_W = RT_TI + 2, RT_H = RT_TJ + 2, RT_P = RT_W * RT_H;   // one staged plane

template <typename T, bool NU>
__device__ __forceinline__ void rhs_tile(const Blk& bk, const Geo& g, const Fields<T>& f,
                                         const unsigned* __restrict__ flags32, const RhsCoef<T>& cf, int use_hp,
                                         int write_h, const DevState* ds) {
  __shared__ T su[3][RT_P], sv[3][RT_P], sw[3][RT_P], sp[2][RT_P];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const T idx = cf.idx, idy = cf.idy, idz = cf.idz;
  const T idx2 = cf.idx2, idy2 = cf.idy2, idz2 = cf.idz2;
  const T gs = cf.gs;
  const T q = (T)0.25;
  const T cg = cf.cg, cr = cf.cr, ca = cf.ca, cv = cf.cv, tdt = cf.dt;
  T fbx, fby, fbz;
  if constexpr (sizeof(T) == 4) {
    fbx = cf.fba * ds->fbf[0];
    fby = cf.fba * ds->fbf[1];
    fbz = cf.fba * ds->fbf[2];
  } else {
    fbx = cf.fba * (T)ds->fb[0];
    fby = cf.fba * (T)ds->fb[1];
    fbz = cf.fba * (T)ds->fb[2];
  }
  const long long pv = (long long)(ny + 1) * nx;
  const long long pu = (long long)ny * nx;
  const int i0 = bk.x * RT_TI, j0 = bk.y * RT_TJ, k0 = bk.z * RT_KC;
  const int k1 = min(nz, k0 + RT_KC);
  const int tid = threadIdx.y * RT_TI + threadIdx.x;
  // the (at most two) staged elements this thread loads per plane: tile
  // column c (-1 .. RT_TI, periodic in x) and row r (-1 .. RT_TJ); rows
  // outside a field's grid are never read by the stencil and not loaded
  long long ou[2], ov[2];
  bool lu[2], lv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = tid + h * RT_TI * RT_TJ;
    const int r = e / RT_W, c = e - r * RT_W;
    const int gi = ((i0 + c - 1) % nx + nx) % nx;
    const int gj = j0 + r - 1;
    lu[h] = e < RT_P && gj >= 0 && gj < ny;
    lv[h] = e < RT_P && gj >= 0 && gj <= ny;
    ou[h] = (long long)gj * nx + gi;
    ov[h] = ou[h];
  }
  auto stage = [&](T (*dst)[RT_P], const T* __restrict__ src, int slot, int k, long long pstride, const bool* live,
                   const long long* off) {
    const long long base = (long long)k * pstride;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = tid + h * RT_TI * RT_TJ;
      if (live[h]) dst[slot][e] = src[base + off[h]];
    }
  };
  // the next plane's elements travel in registers while a step computes
  T nu[2], nv[2], nw[2], np[2];
  auto fetch = [&](T* reg, const T* __restrict__ src, int k, long long pstride, const bool* live,
                   const long long* off) {
    const long long base = (long long)k * pstride;
#pragma unroll
    for (int h = 0; h < 2; ++h) reg[h] = live[h] ? src[base + off[h]] : (T)0;
  };
  auto put = [&](T (*dst)[RT_P], int slot, const T* reg, const bool* live) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (live[h]) dst[slot][tid + h * RT_TI * RT_TJ] = reg[h];
  };
  const T* __restrict__ U = f.u;
  const T* __restrict__ V = f.v;
  const T* __restrict__ W = f.w;
  const T* __restrict__ P = f.p;
  auto wrapk = [&](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
  // planes k0 - 1 and k0 of u, v, w, and k0 - 1 of p staged; plane k0 + 1
  // of u, v, w and plane k0 of p in registers
  {
    const int km = wrapk(k0 - 1);
    stage(su, U, (k0 + 2) % 3, km, pu, lu, ou);
    stage(sv, V, (k0 + 2) % 3, km, pv, lv, ov);
    stage(sw, W, (k0 + 2) % 3, km, pu, lu, ou);
    stage(sp, P, (k0 + 1) % 2, km, pu, lu, ou);
    stage(su, U, k0 % 3, k0, pu, lu, ou);
    stage(sv, V, k0 % 3, k0, pv, lv, ov);
    stage(sw, W, k0 % 3, k0, pu, lu, ou);
    const int kp = wrapk(k0 + 1);
    fetch(nu, U, kp, pu, lu, ou);
    fetch(nv, V, kp, pv, lv, ov);
    fetch(nw, W, kp, pu, lu, ou);
    fetch(np, P, k0, pu, lu, ou);
  }
  const int ti = threadIdx.x, tj = threadIdx.y;
  const int i = i0 + ti, j = j0 + tj;
  const bool live = i < nx && j < ny;
  const bool jlo = j == 0, jhi = j + 1 == ny;
  constexpr bool nun = NU;
  T ihc = idy, ihs = idy, ihn = idy, ihcm = idy;
  if (nun && live) {
    ihc = (T)g.yt.ihc[j];
    ihs = (T)g.yt.ihf[j];
    ihn = (T)g.yt.ihf[j + 1];
    if (j >= 1) ihcm = (T)g.yt.ihc[j - 1];
  }
  const int s0 = (tj + 1) * RT_W + (ti + 1);   // this cell in a staged plane
  for (int k = k0; k < k1; ++k) {
    const int sm = (k + 2) % 3, sc = k % 3, sf = (k + 1) % 3;   // planes k - 1, k, k + 1
    const int pm = (k + 1) % 2, pc0 = k % 2;                     // p planes k - 1, k
    __syncthreads();   // the ring slots about to be refilled are no longer read
    put(su, sf, nu, lu);
    put(sv, sf, nv, lv);
    put(sw, sf, nw, lu);
    put(sp, pc0, np, lu);
    if (k + 1 < k1) {   // the following plane, in flight during this step
      const int kq = wrapk(k + 2);
      fetch(nu, U, kq, pu, lu, ou);
      fetch(nv, V, kq, pv, lv, ov);
      fetch(nw, W, kq, pu, lu, ou);
      fetch(np, P, k + 1, pu, lu, ou);
    }
    __syncthreads();
    if (!live) continue;
    // neighbour (di, dj) of this cell in a staged plane
    auto at = [&](const T* pl, int di, int dj) { return pl[s0 + dj * RT_W + di]; };
    const T* um = su[sm]; const T* uk = su[sc]; const T* uq = su[sf];
    const T* vm = sv[sm]; const T* vk = sv[sc]; const T* vq = sv[sf];
    const T* wm = sw[sm]; const T* wk = sw[sc]; const T* wq = sw[sf];
    const T* pm_ = sp[pm]; const T* pk = sp[pc0];
    const long long r0 = (long long)k * pu + (long long)j * nx;
    const long long v0 = (long long)k * pv + (long long)j * nx;
    const long long cell = r0 + i;
    const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
    const T pcv = at(pk, 0, 0);
    // ---------------- u ----------------
    {
      const T uc = at(uk, 0, 0), ue = at(uk, 1, 0), uw = at(uk, -1, 0);
      const T un = jhi ? gs * uc : at(uk, 0, 1);
      const T us = jlo ? gs * uc : at(uk, 0, -1);
      const T uf = at(uq, 0, 0), ub = at(um, 0, 0);
      const T adx = ((uc + ue) * (uc + ue) - (uw + uc) * (uw + uc)) * q * idx;
      const T vt = jhi ? (T)0 : (at(vk, -1, 1) + at(vk, 0, 1)) * (uc + un);
      const T vb = jlo ? (T)0 : (at(vk, -1, 0) + at(vk, 0, 0)) * (us + uc);
      const T ady = (vt - vb) * q * ihc;
      const T wf = (at(wq, -1, 0) + at(wq, 0, 0)) * (uc + uf);
      const T wb = (at(wk, -1, 0) + at(wk, 0, 0)) * (ub + uc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((un - uc) * ihn - (uc - us) * ihs) * ihc : (un - (T)2 * uc + us) * idy2;
      const T lap = (ue - (T)2 * uc + uw) * idx2 + lapy + (uf - (T)2 * uc + ub) * idz2;
      const T G = (pcv - at(pk, -1, 0)) * idx;
      T r = cg * H - ca * G + cv * lap + fbx;
      if (use_hp) r += cr * f.Hp[0][cell];
      if (write_h) f.H[0][cell] = H;
      f.R[0][cell] = (fl & FLAG_U) ? (T)0 : tdt * r;
    }
    // ---------------- w ----------------
    {
      const T wc = at(wk, 0, 0), we = at(wk, 1, 0), ww = at(wk, -1, 0);
      const T wn = jhi ? gs * wc : at(wk, 0, 1);
      const T ws = jlo ? gs * wc : at(wk, 0, -1);
      const T wf = at(wq, 0, 0), wb = at(wm, 0, 0);
      const T ue = (at(um, 1, 0) + at(uk, 1, 0)) * (wc + we);
      const T uw = (at(um, 0, 0) + at(uk, 0, 0)) * (ww + wc);
      const T adx = (ue - uw) * q * idx;
      const T vt = jhi ? (T)0 : (at(vm, 0, 1) + at(vk, 0, 1)) * (wc + wn);
      const T vb = jlo ? (T)0 : (at(vm, 0, 0) + at(vk, 0, 0)) * (ws + wc);
      const T ady = (vt - vb) * q * ihc;
      const T adz = ((wc + wf) * (wc + wf) - (wb + wc) * (wb + wc)) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((wn - wc) * ihn - (wc - ws) * ihs) * ihc : (wn - (T)2 * wc + ws) * idy2;
      const T lap = (we - (T)2 * wc + ww) * idx2 + lapy + (wf - (T)2 * wc + wb) * idz2;
      const T G = (pcv - at(pm_, 0, 0)) * idz;
      T r = cg * H - ca * G + cv * lap + fbz;
      if (use_hp) r += cr * f.Hp[2][cell];
      if (write_h) f.H[2][cell] = H;
      f.R[2][cell] = (fl & FLAG_W) ? (T)0 : tdt * r;
    }
    // ---------------- v, 1 <= j <= ny-1 ----------------
    if (j >= 1) {
      const T vc = at(vk, 0, 0), ve = at(vk, 1, 0), vw = at(vk, -1, 0);
      const T vn = at(vk, 0, 1), vs = at(vk, 0, -1);
      const T vf = at(vq, 0, 0), vbk = at(vm, 0, 0);
      const T ue = (at(uk, 1, -1) + at(uk, 1, 0)) * (vc + ve);
      const T uw = (at(uk, 0, -1) + at(uk, 0, 0)) * (vw + vc);
      const T adx = (ue - uw) * q * idx;
      const T ady = ((vc + vn) * (vc + vn) - (vs + vc) * (vs + vc)) * q * ihs;
      const T wf = (at(wq, 0, -1) + at(wq, 0, 0)) * (vc + vf);
      const T wb = (at(wk, 0, -1) + at(wk, 0, 0)) * (vbk + vc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lapy = nun ? ((vn - vc) * ihc - (vc - vs) * ihcm) * ihs : (vn - (T)2 * vc + vs) * idy2;
      const T lap = (ve - (T)2 * vc + vw) * idx2 + lapy + (vf - (T)2 * vc + vbk) * idz2;
      const T G = (pcv - at(pk, 0, -1)) * ihs;
      T r = cg * H - ca * G + cv * lap + fby;
      if (use_hp) r += cr * f.Hp[1][v0 + i];
      if (write_h) f.H[1][v0 + i] = H;
      f.R[1][v0 + i] = (fl & FLAG_V) ? (T)0 : tdt * r;
    } else {
      f.R[1][v0 + i] = (T)0;
      f.R[1][(long long)k * pv + (long long)ny * nx + i] = (T)0;
      if (write_h) {
        f.H[1][v0 + i] = (T)0;
        f.H[1][(long long)k * pv + (long long)ny * nx + i] = (T)0;
      }
    }
  }
}
template <typename T, bool NU>
struct RhsTile {
  static constexpr int kThreads = RT_TI * RT_TJ;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  RhsCoef<T> cf;
  int use_hp;
  int write_h;
  const DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    rhs_tile<T, NU>(bk, g, f, flags32, cf, use_hp, write_h, ds);
  }
};

// Two cells per thread along x (launch shape rhs = 3, FP32 path; nx is even
// on every grid): every row the stencil reads is loaded as one float2 for
// the thread's cells i0, i0 + 1 plus a scalar on either side where an
// x-neighbour is needed, so the loads, their address arithmetic and the
// stores are shared by the two cells.  Each cell's arithmetic is the
// per-cell kernel's, term by term.
template <bool NU>
__device__ __forceinline__ void rhs_vec(const Blk& bk, const Geo& g, const Fields<float>& f,
                                        const unsigned* __restrict__ flags32, const RhsCoef<float>& cf, int use_hp,
                                        int write_h, const DevState* ds) {
  using T = float;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const T idx = cf.idx, idy = cf.idy, idz = cf.idz;
  const T idx2 = cf.idx2, idy2 = cf.idy2, idz2 = cf.idz2;
  const T gs = cf.gs;
  const T q = (T)0.25;
  const T cg = cf.cg, cr = cf.cr, ca = cf.ca, cv = cf.cv, tdt = cf.dt;
  const T fbx = cf.fba * ds->fbf[0], fby = cf.fba * ds->fbf[1], fbz = cf.fba * ds->fbf[2];
  const int i0 = 2 * (int)(bk.x * blockDim.x + threadIdx.x);
  const int j = bk.y * blockDim.y + threadIdx.y;
  const int k = bk.z;
  if (i0 >= nx || j >= ny) return;
  const int pv = (ny + 1) * nx, pu = ny * nx;
  const int im = i0 == 0 ? nx - 1 : i0 - 1;        // left of cell a = i0
  const int ip2 = i0 + 2 == nx ? 0 : i0 + 2;       // right of cell b = i0 + 1
  const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
  const int r0 = k * pu + j * nx, rkp = kp * pu + j * nx, rkm = km * pu + j * nx;
  const int v0 = k * pv + j * nx, v1 = v0 + nx;
  const int vkm0 = km * pv + j * nx, vkp0 = kp * pv + j * nx;
  const bool jlo = j == 0, jhi = j + 1 == ny;
  const T* __restrict__ U = f.u;
  const T* __restrict__ V = f.v;
  const T* __restrict__ W = f.w;
  const T* __restrict__ P = f.p;
  auto ld2 = [](const T* p, int o) { return *reinterpret_cast<const float2*>(p + o); };
  const float2 zero2 = make_float2(0.0f, 0.0f);
  // rows of u
  const float2 Ur = ld2(U, r0 + i0);
  const T Ur_m = U[r0 + im], Ur_p = U[r0 + ip2];
  const float2 Un2 = jhi ? zero2 : ld2(U, r0 + nx + i0);
  const float2 Us2 = jlo ? zero2 : ld2(U, r0 - nx + i0);
  const T Us_p = jlo ? (T)0 : U[r0 - nx + ip2];
  const float2 Uf2 = ld2(U, rkp + i0), Ub2 = ld2(U, rkm + i0);
  const T Ub_p = U[rkm + ip2];
  // rows of v
  const float2 V1 = ld2(V, v1 + i0);
  const T V1_m = V[v1 + im];
  const float2 V0 = ld2(V, v0 + i0);
  const T V0_m = V[v0 + im], V0_p = V[v0 + ip2];
  const float2 Vs2 = jlo ? zero2 : ld2(V, v0 - nx + i0);
  const float2 Vf2 = ld2(V, vkp0 + i0), Vb2 = ld2(V, vkm0 + i0), Vbn2 = ld2(V, vkm0 + nx + i0);
  // rows of w
  const float2 W0 = ld2(W, r0 + i0);
  const T W0_m = W[r0 + im], W0_p = W[r0 + ip2];
  const float2 Wn2 = jhi ? zero2 : ld2(W, r0 + nx + i0);
  const float2 Ws2 = jlo ? zero2 : ld2(W, r0 - nx + i0);
  const float2 Wf2 = ld2(W, rkp + i0), Wb2 = ld2(W, rkm + i0);
  const T Wf_m = W[rkp + im];
  const float2 Wfs2 = jlo ? zero2 : ld2(W, rkp - nx + i0);
  // rows of p
  const float2 P0 = ld2(P, r0 + i0), Pb2 = ld2(P, rkm + i0);
  const T P0_m = P[r0 + im];
  const float2 Ps2 = jlo ? zero2 : ld2(P, r0 - nx + i0);
  // flags of both cells (one word: i0 even)
  const unsigned fw = flags32[(r0 + i0) >> 2];
  const unsigned sh = 8u * (unsigned)((r0 + i0) & 3);
  const unsigned fla = (fw >> sh) & 0xFFu, flb = (fw >> (sh + 8u)) & 0xFFu;
  constexpr bool nun = NU;
  const T ihc = nun ? (T)g.yt.ihc[j] : idy, ihs = nun ? (T)g.yt.ihf[j] : idy, ihn = nun ? (T)g.yt.ihf[j + 1] : idy;
  const T ihcm = (nun && j >= 1) ? (T)g.yt.ihc[j - 1] : idy;
  // ---------------- u ----------------
  auto ucomp = [&](T uc, T ue, T uw, T unr, T usr, T uf, T ub, T v1m, T v1c, T v0m, T v0c, T wpm, T wpc, T w0m,
                   T w0c, T pc, T pm, T& H) {
    const T un = jhi ? gs * uc : unr;
    const T us = jlo ? gs * uc : usr;
    const T adx = ((uc + ue) * (uc + ue) - (uw + uc) * (uw + uc)) * q * idx;
    const T vt = jhi ? (T)0 : (v1m + v1c) * (uc + un);
    const T vb = jlo ? (T)0 : (v0m + v0c) * (us + uc);
    const T ady = (vt - vb) * q * ihc;
    const T wf = (wpm + wpc) * (uc + uf);
    const T wb = (w0m + w0c) * (ub + uc);
    const T adz = (wf - wb) * q * idz;
    H = -(adx + ady + adz);
    const T lapy = nun ? ((un - uc) * ihn - (uc - us) * ihs) * ihc : (un - (T)2 * uc + us) * idy2;
    const T lap = (ue - (T)2 * uc + uw) * idx2 + lapy + (uf - (T)2 * uc + ub) * idz2;
    const T G = (pc - pm) * idx;
    return cg * H - ca * G + cv * lap + fbx;
  };
  {
    T Ha, Hb;
    T ra = ucomp(Ur.x, Ur.y, Ur_m, Un2.x, Us2.x, Uf2.x, Ub2.x, V1_m, V1.x, V0_m, V0.x, Wf_m, Wf2.x, W0_m, W0.x, P0.x,
                 P0_m, Ha);
    T rb = ucomp(Ur.y, Ur_p, Ur.x, Un2.y, Us2.y, Uf2.y, Ub2.y, V1.x, V1.y, V0.x, V0.y, Wf2.x, Wf2.y, W0.x, W0.y, P0.y,
                 P0.x, Hb);
    if (use_hp) {
      const float2 hp = ld2(f.Hp[0], r0 + i0);
      ra += cr * hp.x;
      rb += cr * hp.y;
    }
    if (write_h) *reinterpret_cast<float2*>(f.H[0] + r0 + i0) = make_float2(Ha, Hb);
    *reinterpret_cast<float2*>(f.R[0] + r0 + i0) =
        make_float2((fla & FLAG_U) ? (T)0 : tdt * ra, (flb & FLAG_U) ? (T)0 : tdt * rb);
  }
  // ---------------- w ----------------
  auto wcomp = [&](T wc, T we, T ww, T wnr, T wsr, T wf, T wb, T ukmp, T u0p, T ukm, T u0, T vkmn, T v1c, T vkm, T v0c,
                   T pc, T pkm, T& H) {
    const T wn = jhi ? gs * wc : wnr;
    const T ws = jlo ? gs * wc : wsr;
    const T ue = (ukmp + u0p) * (wc + we);
    const T uw = (ukm + u0) * (ww + wc);
    const T adx = (ue - uw) * q * idx;
    const T vt = jhi ? (T)0 : (vkmn + v1c) * (wc + wn);
    const T vb = jlo ? (T)0 : (vkm + v0c) * (ws + wc);
    const T ady = (vt - vb) * q * ihc;
    const T adz = ((wc + wf) * (wc + wf) - (wb + wc) * (wb + wc)) * q * idz;
    H = -(adx + ady + adz);
    const T lapy = nun ? ((wn - wc) * ihn - (wc - ws) * ihs) * ihc : (wn - (T)2 * wc + ws) * idy2;
    const T lap = (we - (T)2 * wc + ww) * idx2 + lapy + (wf - (T)2 * wc + wb) * idz2;
    const T G = (pc - pkm) * idz;
    return cg * H - ca * G + cv * lap + fbz;
  };
  {
    T Ha, Hb;
    T ra = wcomp(W0.x, W0.y, W0_m, Wn2.x, Ws2.x, Wf2.x, Wb2.x, Ub2.y, Ur.y, Ub2.x, Ur.x, Vbn2.x, V1.x, Vb2.x, V0.x,
                 P0.x, Pb2.x, Ha);
    T rb = wcomp(W0.y, W0_p, W0.x, Wn2.y, Ws2.y, Wf2.y, Wb2.y, Ub_p, Ur_p, Ub2.y, Ur.y, Vbn2.y, V1.y, Vb2.y, V0.y,
                 P0.y, Pb2.y, Hb);
    if (use_hp) {
      const float2 hp = ld2(f.Hp[2], r0 + i0);
      ra += cr * hp.x;
      rb += cr * hp.y;
    }
    if (write_h) *reinterpret_cast<float2*>(f.H[2] + r0 + i0) = make_float2(Ha, Hb);
    *reinterpret_cast<float2*>(f.R[2] + r0 + i0) =
        make_float2((fla & FLAG_W) ? (T)0 : tdt * ra, (flb & FLAG_W) ? (T)0 : tdt * rb);
  }
  // ---------------- v, 1 <= j <= ny-1 ----------------
  if (j >= 1) {
    auto vcomp = [&](T vc, T ve, T vw, T vn, T vs, T vf, T vbk, T usp, T u0p, T us, T u0, T wps, T wp0, T w0s, T w00,
                     T pc, T ps, T& H) {
      const T ue = (usp + u0p) * (vc + ve);
      const T uw = (us + u0) * (vw + vc);
      const T adx = (ue - uw) * q * idx;
      const T ady = ((vc + vn) * (vc + vn) - (vs + vc) * (vs + vc)) * q * ihs;
      const T wf = (wps + wp0) * (vc + vf);
      const T wb = (w0s + w00) * (vbk + vc);
      const T adz = (wf - wb) * q * idz;
      H = -(adx + ady + adz);
      const T lapy = nun ? ((vn - vc) * ihc - (vc - vs) * ihcm) * ihs : (vn - (T)2 * vc + vs) * idy2;
      const T lap = (ve - (T)2 * vc + vw) * idx2 + lapy + (vf - (T)2 * vc + vbk) * idz2;
      const T G = (pc - ps) * ihs;
      return cg * H - ca * G + cv * lap + fby;
    };
    T Ha, Hb;
    T ra = vcomp(V0.x, V0.y, V0_m, V1.x, Vs2.x, Vf2.x, Vb2.x, Us2.y, Ur.y, Us2.x, Ur.x, Wfs2.x, Wf2.x, Ws2.x, W0.x,
                 P0.x, Ps2.x, Ha);
    T rb = vcomp(V0.y, V0_p, V0.x, V1.y, Vs2.y, Vf2.y, Vb2.y, Us_p, Ur_p, Us2.y, Ur.y, Wfs2.y, Wf2.y, Ws2.y, W0.y,
                 P0.y, Ps2.y, Hb);
    if (use_hp) {
      const float2 hp = ld2(f.Hp[1], v0 + i0);
      ra += cr * hp.x;
      rb += cr * hp.y;
    }
    if (write_h) *reinterpret_cast<float2*>(f.H[1] + v0 + i0) = make_float2(Ha, Hb);
    *reinterpret_cast<float2*>(f.R[1] + v0 + i0) =
        make_float2((fla & FLAG_V) ? (T)0 : tdt * ra, (flb & FLAG_V) ? (T)0 : tdt * rb);
  } else {
    // wall planes of v carry no unknown
    *reinterpret_cast<float2*>(f.R[1] + v0 + i0) = zero2;
    *reinterpret_cast<float2*>(f.R[1] + k * pv + ny * nx + i0) = zero2;
    if (write_h) {
      *reinterpret_cast<float2*>(f.H[1] + v0 + i0) = zero2;
      *reinterpret_cast<float2*>(f.H[1] + k * pv + ny * nx + i0) = zero2;
    }
  }
}
template <bool NU>
struct RhsVec {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<float> f;
  const unsigned* flags32;
  RhsCoef<float> cf;
  int use_hp;
  int write_h;
  const DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    rhs_vec<NU>(bk, g, f, flags32, cf, use_hp, write_h, ds);
  }
};

template <typename T>
void launch_rhs(const Geo& g, const Fields<T>& f, const TagBuffers& b, const Stage& sg, double dt, double re,
                bool use_hp, bool write_h, DevState* ds, Exec& ex) {
  RhsCoef<T> cf;
  cf.idx = (T)g.idx; cf.idy = (T)g.idy; cf.idz = (T)g.idz;
  cf.idx2 = (T)(g.idx * g.idx); cf.idy2 = (T)(g.idy * g.idy); cf.idz2 = (T)(g.idz * g.idz);
  cf.gs = g.ybc == 0 ? (T)-1 : (T)1;
  cf.cg = (T)sg.gam; cf.cr = (T)sg.rho; cf.ca = (T)sg.alp; cf.cv = (T)(sg.alp / re);
  cf.dt = (T)dt;
  cf.fba = (T)sg.alp;
  ex.mark(ST_RHS);
  const int hp = use_hp ? 1 : 0, wh = write_h ? 1 : 0;
  if (ex.tune.rhs == 2) {   // tiles marching in z (measured slower than one thread per cell at 128^3)
    const dim3 grid((g.nx + RT_TI - 1) / RT_TI, (g.ny + RT_TJ - 1) / RT_TJ, (g.nz + RT_KC - 1) / RT_KC),
        blk(RT_TI, RT_TJ);
    if (g.yt.ihc)
      ex.launch(grid, blk, 0, RhsTile<T, true>{g, f, b.flags32, cf, hp, wh, ds});
    else
      ex.launch(grid, blk, 0, RhsTile<T, false>{g, f, b.flags32, cf, hp, wh, ds});
    return;
  }
  const dim3 grid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz), blk(32, 4);
  // 32-bit indices when every field (the largest: v, with ny + 1 planes)
  // has fewer than 2^31 entries; a batch decides by its largest instance
  const bool i32 = (long long)(ex.shape.ny + 1) * ex.shape.nx * ex.shape.nz < (1ll << 31);
  if constexpr (sizeof(T) == 4) {
    // two cells per thread along x (FP32; the built-in choice there)
    if ((ex.tune.rhs == 3 || ex.tune.rhs == 0) && i32 && g.nx % 2 == 0 && ex.shape.nx % 2 == 0) {
      const dim3 gv((g.nx / 2 + 31) / 32, (g.ny + 3) / 4, g.nz);
      if (g.yt.ihc)
        ex.launch(gv, blk, 0, RhsVec<true>{g, f, b.flags32, cf, hp, wh, ds});
      else
        ex.launch(gv, blk, 0, RhsVec<false>{g, f, b.flags32, cf, hp, wh, ds});
      return;
    }
  }
  if (g.yt.ihc) {   // non-uniform wall-normal spacing
    if (i32) ex.launch(grid, blk, 0, Rhs<T, true, int>{g, f, b.flags32, cf, hp, wh, ds});
    else ex.launch(grid, blk, 0, Rhs<T, true>{g, f, b.flags32, cf, hp, wh, ds});
  } else {
    if (i32) ex.launch(grid, blk, 0, Rhs<T, false, int>{g, f, b.flags32, cf, hp, wh, ds});
    else ex.launch(grid, blk, 0, Rhs<T, false>{g, f, b.flags32, cf, hp, wh, ds});
  }
}

// ---------------------------------------------------------------------------
// Approximate factorisation: (1 - beta L_x)(1 - beta L_z)(1 - beta L_y) du = R
// Each factor is a tridiagonal system per grid line; forcing nodes are
// identity rows (the provisional equation is not solved there).  Every
// pivot depends only on the row's position m inside its segment (from the
// line start or from the row after an identity row), so all lines run on
// tabulated recurrences: no division, no scratch.  Lines without forcing
// nodes (known from the per-line records written by the tagging) take a
// branch-free path with batched loads.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_forcing(const unsigned* flags32, long long cell, int c) {
  return (flags32[cell >> 2] >> (8 * (cell & 3) + c)) & 1u;
}

// Line solvers.  `E(m)` is a reference to row m of this thread's line in
// shared memory, `F(m)` the flag byte of its cell; rows are solved in place.

// periodic line (x or z) of component c; f0 = first forcing row or >= n
template <typename T, class Elem, class Flag>
__device__ __forceinline__ void solve_periodic(int n, int c, int f0, int d, T a, const SweepTables<T>& tb, Elem E,
                                               Flag F) {
  auto forcing = [&](int r) { return (F(r) >> c) & 1; };
  if (f0 >= n) {
    // Sherman-Morrison: y = T^-1 r by tabulated Thomas, y_0 = g0 . r, then
    // x = y - (v.y / (1 + v.z)) z
    const T* __restrict__ inv = tb.inv[d];
    const T* __restrict__ cp = tb.cp[d];
    const T* __restrict__ zv = tb.zv[d];
    const T* __restrict__ g0 = tb.g0[d];
    T prev = (T)0, acc = (T)0;
    for (int m = 0; m < n; ++m) {
      const T dm = E(m);
      acc += __ldg(g0 + m) * dm;
      prev = (dm - a * prev) * __ldg(inv + m);
      E(m) = prev;
    }
    const T fact = (acc + (a / tb.gam[d]) * prev) / tb.smden[d];
    T y = prev;
    E(n - 1) = y - fact * __ldg(zv + n - 1);
    for (int m = n - 2; m >= 0; --m) {
      y = E(m) - __ldg(cp + m) * y;
      E(m) = y - fact * __ldg(zv + m);
    }
    return;
  }
  // rotated to start at the first forcing row: row 0 of the rotated system
  // is an identity row; the periodic coupling of the last row to it moves
  // to the right-hand side
  const T* __restrict__ invR = tb.invR[d];
  const T* __restrict__ cpR = tb.cpR[d];
  auto rot = [&](int q) { const int r = f0 + q; return r >= n ? r - n : r; };
  const T x0 = E(f0);
  T prev = x0;
  int m = 0;
  for (int q = 1; q < n; ++q) {
    const int r = rot(q);
    if (forcing(r)) { prev = E(r); m = 0; continue; }
    T dq = E(r);
    if (q == n - 1) dq -= a * x0;
    prev = (dq - a * prev) * __ldg(invR + m);
    E(r) = prev;
    ++m;
  }
  T x = prev;
  int mq = -1;
  if (!forcing(rot(n - 1))) {
    int lo = n - 2;
    while (lo > 0 && !forcing(rot(lo))) --lo;
    mq = (n - 1) - lo - 1;
  }
  for (int q = n - 2; q >= 1; --q) {
    const int r = rot(q);
    if (forcing(r)) { x = E(r); mq = -1; continue; }
    if (mq < 0) {
      int lo = q - 1;
      while (lo > 0 && !forcing(rot(lo))) --lo;
      mq = q - lo - 1;
    } else {
      --mq;
    }
    x = E(r) - __ldg(cpR + mq) * x;
    E(r) = x;
  }
}

// wall-normal line of component c (n rows); any = line holds forcing rows
template <typename T, class Elem, class Flag>
__device__ __forceinline__ void solve_wall(int n, int c, bool any, T a, const SweepTables<T>& tb, Elem E, Flag F) {
  const bool tang = c != 1;
  auto forcing = [&](int r) { return (F(r) >> c) & 1; };
  if (!any) {
    const T* __restrict__ inv = tang ? tb.yinvW : tb.vinvR;
    const T* __restrict__ cp = tang ? tb.ycpW : tb.vcpR;
    const T invlast = tang ? tb.yinvLW[n - 1] : inv[n - 1];
    T prev = (T)0;
    for (int m = 0; m < n; ++m) {
      prev = (E(m) - a * prev) * (m == n - 1 ? invlast : __ldg(inv + m));
      E(m) = prev;
    }
    T x = prev;
    for (int m = n - 2; m >= 0; --m) {
      x = E(m) - __ldg(cp + m) * x;
      E(m) = x;
    }
    return;
  }
  // W segments start at a wall (tangential components), R segments after
  // an identity row; a tangential last row carries the wall diagonal
  T prev = (T)0;
  int m = 0;
  bool segW = tang;
  for (int j = 0; j < n; ++j) {
    if (forcing(j)) { prev = E(j); m = 0; segW = false; continue; }
    T iv;
    if (!tang) iv = __ldg(tb.vinvR + m);
    else if (j == n - 1) iv = segW ? __ldg(tb.yinvLW + m) : __ldg(tb.yinvLR + m);
    else iv = segW ? __ldg(tb.yinvW + m) : __ldg(tb.yinvR + m);
    prev = (E(j) - a * prev) * iv;
    E(j) = prev;
    ++m;
  }
  T x = prev;
  int mq = -1;
  bool qW = false;
  auto seg_of = [&](int q, int& mpos, bool& w) {
    int lo = q - 1;
    while (lo >= 0 && !forcing(lo)) --lo;
    mpos = q - lo - 1;
    w = tang && lo < 0;
  };
  if (!forcing(n - 1)) seg_of(n - 1, mq, qW);
  for (int j = n - 2; j >= 0; --j) {
    if (forcing(j)) { x = E(j); mq = -1; continue; }
    if (mq < 0) seg_of(j, mq, qW);
    else --mq;
    const T cpj = !tang ? __ldg(tb.vcpR + mq) : (qW ? __ldg(tb.ycpW + mq) : __ldg(tb.ycpR + mq));
    x = E(j) - cpj * x;
    E(j) = x;
  }
}

// Asynchronous global -> shared copies (cp.async): every load of a tile is
// issued up front and waited for once, instead of one memory latency per
// element.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// x-sweep: a block holds W complete x-lines (rows (j, k) of component
// blockIdx.y) in shared memory, loaded and stored row by row (coalesced);
// thread t solves line t.  Tile [W][nx+1] of T, then [W][nx] flag bytes.
template <typename T>
__device__ __forceinline__ void sweep_x(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32,
                                                const SweepTables<T>& tb, const int* __restrict__ lfirst) {
  extern __shared__ unsigned char smem_raw[];
  const int W = blockDim.x, t = threadIdx.x;
  const int c = bk.y;
  const int n = g.nx, ld = n + 1;
  const int j0 = c == 1 ? 1 : 0, nj = c == 1 ? g.ny - 1 : g.ny;
  const int nlines = nj * g.nz;
  const int l0 = bk.x * W;
  T* tile = reinterpret_cast<T*>(smem_raw);
  unsigned char* fl = reinterpret_cast<unsigned char*>(tile + (size_t)W * ld);
  T* __restrict__ R = f.R[c];
  const unsigned char* fbytes = reinterpret_cast<const unsigned char*>(flags32);
  const bool words = (n & 3) == 0;   // flag bytes of a row copied four at a time
  for (int r = 0; r < W; ++r) {
    const int l = l0 + r;
    if (l >= nlines) break;
    const int j = j0 + l % nj, k = l / nj;
    const long long base = fidx(g, c, 0, j, k), fb = cidx(g, 0, j, k);
    for (int i = t; i < n; i += W) cp_async<sizeof(T)>(tile + r * ld + i, R + base + i);
    if (words) {
      for (int q = t; q < n / 4; q += W) cp_async<4>(fl + r * n + 4 * q, fbytes + fb + 4 * q);
    } else {
      for (int i = t; i < n; i += W) fl[r * n + i] = fbytes[fb + i];
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int l = l0 + t;
  if (l < nlines) {
    const int j = j0 + l % nj, k = l / nj;
    T* row = tile + t * ld;
    const unsigned char* frow = fl + t * n;
    solve_periodic<T>(n, c, lfirst[line_x(g, c, j, k)], 0, -tb.off[0], tb, [&](int m) -> T& { return row[m]; },
                      [&](int m) { return (int)frow[m]; });
  }
  __syncthreads();
  for (int r = 0; r < W; ++r) {
    const int l2 = l0 + r;
    if (l2 >= nlines) break;
    const int j = j0 + l2 % nj, k = l2 / nj;
    const long long base = fidx(g, c, 0, j, k);
    for (int i = t; i < n; i += W) R[base + i] = tile[r * ld + i];
  }
}
template <typename T>
struct SweepX {
  static constexpr int kThreads = 64;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_x<T>(bk, g, f, flags32, tb, lfirst); }
};

// x-sweep, one warp per line: lane l holds rows [l K, l K + K) of the line
// (K = ceil(nx/32)) in registers, loaded coalesced.  Both Thomas passes are
// affine recurrences y_m = A_m y_{m-1} + B_m (forward) and y_m = A_m y_{m+1}
// + B_m (backward); each lane composes the maps of its rows, a warp shuffle
// scan composes the lanes, and each lane then finishes its rows.  Identity
// rows (forcing nodes) are the maps (0, d).  Used for the FP32 bulk type.
template <typename T>
struct AffMap {
  T A, B;
};
// the map of `later` applied after `earlier`
template <typename T>
__device__ __forceinline__ AffMap<T> aff_then(AffMap<T> earlier, AffMap<T> later) {
  return AffMap<T>{later.A * earlier.A, later.A * earlier.B + later.B};
}
// exclusive scan of lane maps in increasing lane order (lane 0: identity)
template <typename T>
__device__ __forceinline__ AffMap<T> scan_up_excl(AffMap<T> m, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const T a = __shfl_up_sync(0xFFFFFFFFu, m.A, o), b = __shfl_up_sync(0xFFFFFFFFu, m.B, o);
    if (lane >= o) m = aff_then(AffMap<T>{a, b}, m);
  }
  const T a = __shfl_up_sync(0xFFFFFFFFu, m.A, 1), b = __shfl_up_sync(0xFFFFFFFFu, m.B, 1);
  return lane == 0 ? AffMap<T>{(T)1, (T)0} : AffMap<T>{a, b};
}
// exclusive scan in decreasing lane order (lane 31: identity)
template <typename T>
__device__ __forceinline__ AffMap<T> scan_down_excl(AffMap<T> m, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const T a = __shfl_down_sync(0xFFFFFFFFu, m.A, o), b = __shfl_down_sync(0xFFFFFFFFu, m.B, o);
    if (lane + o < 32) m = aff_then(AffMap<T>{a, b}, m);
  }
  const T a = __shfl_down_sync(0xFFFFFFFFu, m.A, 1), b = __shfl_down_sync(0xFFFFFFFFu, m.B, 1);
  return lane == 31 ? AffMap<T>{(T)1, (T)0} : AffMap<T>{a, b};
}

// K consecutive rows q0 .. q0+K-1 of a line (rows >= n read as 0): four at
// a time as aligned 16-byte vectors when the line and n allow (FP32, K a
// multiple of 4), so a warp's load covers a contiguous span instead of 32
// strided words.
template <typename T, int K>
__device__ __forceinline__ void load_rows(const T* __restrict__ p, int q0, int n, T (&v)[K]) {
  if constexpr (sizeof(T) == 4 && K % 4 == 0) {
    if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
      for (int u4 = 0; u4 < K / 4; ++u4) {
        const int q = q0 + 4 * u4;
        const float4 x = q < n ? *reinterpret_cast<const float4*>(p + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * u4] = x.x;
        v[4 * u4 + 1] = x.y;
        v[4 * u4 + 2] = x.z;
        v[4 * u4 + 3] = x.w;
      }
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < K; ++u) v[u] = q0 + u < n ? p[q0 + u] : (T)0;
}
template <typename T, int K>
__device__ __forceinline__ void store_rows(T* __restrict__ p, int q0, int n, const T (&v)[K]) {
  if constexpr (sizeof(T) == 4 && K % 4 == 0) {
    if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
      for (int u4 = 0; u4 < K / 4; ++u4) {
        const int q = q0 + 4 * u4;
        if (q < n) *reinterpret_cast<float4*>(p + q) = make_float4(v[4 * u4], v[4 * u4 + 1], v[4 * u4 + 2], v[4 * u4 + 3]);
      }
      return;
    }
  }
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (q0 + u < n) p[q0 + u] = v[u];
}

template <typename T, int K>
__device__ __forceinline__ void sweep_x_warp(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32,
                                                      const SweepTables<T>& tb, const int* __restrict__ lfirst) {
  const int lane = threadIdx.x & 31;
  const int c = bk.y;
  const int n = g.nx;
  const int j0 = c == 1 ? 1 : 0, nj = c == 1 ? g.ny - 1 : g.ny;
  const int l = bk.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (l >= nj * g.nz) return;
  const int j = j0 + l % nj, k = l / nj;
  const long long base = fidx(g, c, 0, j, k);
  T* __restrict__ R = f.R[c];
  const T a = -tb.off[0];
  const int f0 = lfirst[line_x(g, c, j, k)];
  const int q0 = lane * K;
  T v[K];
  if (f0 >= n) {
    // ------------- no forcing node: Sherman-Morrison on the periodic line
    const T* __restrict__ inv = tb.inv[0];
    const T* __restrict__ cp = tb.cp[0];
    const T* __restrict__ zv = tb.zv[0];
    const T* __restrict__ g0 = tb.g0[0];
    T ivr[K], g0r[K], cpr[K], zvr[K];
    load_rows<T, K>(R + base, q0, n, v);
    load_rows<T, K>(inv, q0, n, ivr);
    load_rows<T, K>(g0, q0, n, g0r);
    load_rows<T, K>(cp, q0, n, cpr);
    load_rows<T, K>(zv, q0, n, zvr);
    T acc = (T)0;
    AffMap<T> mp{(T)1, (T)0};
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (q0 + u < n) {
        const T iv = ivr[u];
        acc += g0r[u] * v[u];
        mp = aff_then(mp, AffMap<T>{-a * iv, v[u] * iv});
      }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    const AffMap<T> pre = scan_up_excl(mp, lane);
    T y = pre.B;   // y'_{q0 - 1}
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (q0 + u < n) {
        y = (v[u] - a * y) * ivr[u];
        v[u] = y;
      }
    const T ylast = __shfl_sync(0xFFFFFFFFu, y, (n - 1) / K);
    const T fact = (acc + (a / tb.gam[0]) * ylast) / tb.smden[0];
    // backward: y_m = -cp_m y_{m+1} + y'_m, row n-1: y = y'_{n-1}
    mp = AffMap<T>{(T)1, (T)0};
#pragma unroll
    for (int u = K - 1; u >= 0; --u)
      if (q0 + u < n) {
        const AffMap<T> rm = (q0 + u == n - 1) ? AffMap<T>{(T)0, v[u]} : AffMap<T>{-cpr[u], v[u]};
        mp = aff_then(mp, rm);
      }
    const AffMap<T> suf = scan_down_excl(mp, lane);
    T yn = suf.B;  // y_{q0 + K}
#pragma unroll
    for (int u = K - 1; u >= 0; --u)
      if (q0 + u < n) {
        yn = (q0 + u == n - 1) ? v[u] : v[u] - cpr[u] * yn;
        v[u] = yn - fact * zvr[u];
      }
    store_rows<T, K>(R + base, q0, n, v);
    return;
  }
  // ------------- forcing rows: the line rotated to start at f0 (identity)
  const T* __restrict__ invR = tb.invR[0];
  const T* __restrict__ cpR = tb.cpR[0];
  const long long fb = cidx(g, 0, j, k);
  const unsigned char* fbytes = reinterpret_cast<const unsigned char*>(flags32);
  int rr[K];
  bool idn[K];
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    int r = f0 + q;
    if (r >= n) r -= n;
    rr[u] = r;
    if (q < n) {
      v[u] = R[base + r];
      idn[u] = (fbytes[fb + r] >> c) & 1;
    } else {
      v[u] = (T)0;
      idn[u] = true;
    }
  }
  const T x0 = __shfl_sync(0xFFFFFFFFu, v[0], 0);   // row q = 0 is an identity row
  // segment positions: distance from the last identity row before each row
  int lastid = -1;
#pragma unroll
  for (int u = 0; u < K; ++u)
    if (q0 + u < n && idn[u]) lastid = q0 + u;
  int before = lastid;
  for (int o = 1; o < 32; o <<= 1) {
    const int t2 = __shfl_up_sync(0xFFFFFFFFu, before, o);
    if (lane >= o && t2 > before) before = t2;
  }
  before = __shfl_up_sync(0xFFFFFFFFu, before, 1);
  if (lane == 0) before = -1;
  int mseg[K];
  {
    int last = before;
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int q = q0 + u;
      mseg[u] = q - last - 1;
      if (q < n && idn[u]) last = q;
    }
  }
  AffMap<T> mp{(T)1, (T)0};
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if (idn[u]) { mp = AffMap<T>{(T)0, v[u]}; continue; }
    const T iv = __ldg(invR + mseg[u]);
    const T dq = (q == n - 1) ? v[u] - a * x0 : v[u];
    mp = aff_then(mp, AffMap<T>{-a * iv, dq * iv});
  }
  const AffMap<T> pre = scan_up_excl(mp, lane);
  T y = pre.B;
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if (idn[u]) { y = v[u]; continue; }
    const T dq = (q == n - 1) ? v[u] - a * x0 : v[u];
    y = (dq - a * y) * __ldg(invR + mseg[u]);
    v[u] = y;
  }
  // backward: fluid rows y_q = -cp_q y_{q+1} + y'_q; identity rows and the
  // last row keep their value
  mp = AffMap<T>{(T)1, (T)0};
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = idn[u] || q == n - 1;
    mp = aff_then(mp, keep ? AffMap<T>{(T)0, v[u]} : AffMap<T>{-__ldg(cpR + mseg[u]), v[u]});
  }
  const AffMap<T> suf = scan_down_excl(mp, lane);
  T yn = suf.B;
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = idn[u] || q == n - 1;
    yn = keep ? v[u] : v[u] - __ldg(cpR + mseg[u]) * yn;
    if (!idn[u]) R[base + rr[u]] = yn;
  }
}
template <typename T, int K>
struct SweepXWarp {
  static constexpr int kThreads = 256;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_x_warp<T, K>(bk, g, f, flags32, tb, lfirst); }
};

// ---------------------------------------------------------------------------
// Warp-cooperative z and y sweeps (FP32 path).  A warp holds G = 32/L lines
// (consecutive i), L lanes per line, lane s holding rows [s K, s K + K) of
// its line in registers, so a warp load of one row offset touches L rows of
// G consecutive floats (whole 32-byte sectors for G = 8), and 32/L times as
// many lanes work on the recurrences as with one thread per line.  The
// Thomas recurrences are composed as affine maps per lane and across the L
// lanes of a line by shuffle scans restricted to the line's lanes (the
// lines of one warp take different branches).
// ---------------------------------------------------------------------------
template <typename T, int L>
__device__ __forceinline__ AffMap<T> gscan_up_excl(AffMap<T> m, int s, unsigned mask) {
  for (int o = 1; o < L; o <<= 1) {
    const T a = __shfl_up_sync(mask, m.A, o, L), b = __shfl_up_sync(mask, m.B, o, L);
    if (s >= o) m = aff_then(AffMap<T>{a, b}, m);
  }
  const T a = __shfl_up_sync(mask, m.A, 1, L), b = __shfl_up_sync(mask, m.B, 1, L);
  return s == 0 ? AffMap<T>{(T)1, (T)0} : AffMap<T>{a, b};
}
template <typename T, int L>
__device__ __forceinline__ AffMap<T> gscan_down_excl(AffMap<T> m, int s, unsigned mask) {
  for (int o = 1; o < L; o <<= 1) {
    const T a = __shfl_down_sync(mask, m.A, o, L), b = __shfl_down_sync(mask, m.B, o, L);
    if (s + o < L) m = aff_then(AffMap<T>{a, b}, m);
  }
  const T a = __shfl_down_sync(mask, m.A, 1, L), b = __shfl_down_sync(mask, m.B, 1, L);
  return s == L - 1 ? AffMap<T>{(T)1, (T)0} : AffMap<T>{a, b};
}
// index of the last identity row before this lane's rows (-1: none), from
// the lane's own last identity row `mine`
template <int L>
__device__ __forceinline__ int last_identity_before(int mine, int s, unsigned mask) {
  int before = mine;
  for (int o = 1; o < L; o <<= 1) {
    const int t2 = __shfl_up_sync(mask, before, o, L);
    if (s >= o && t2 > before) before = t2;
  }
  before = __shfl_up_sync(mask, before, 1, L);
  return s == 0 ? -1 : before;
}

// One periodic line (z direction, table slot d = 1) of n rows at elements
// R[base + r * stride]; f0 = first forcing row or >= n.  Same recurrences
// as solve_periodic: Sherman-Morrison without forcing rows, else the line
// rotated to start at f0 (an identity row) with segment tables.
template <typename T, int K, int L>
__device__ __forceinline__ void periodic_line_lanes(int n, int f0, int c, int d, T a, const SweepTables<T>& tb, int s,
                                                    unsigned mask, T* __restrict__ R, long long base,
                                                    long long stride, const unsigned char* __restrict__ fbytes,
                                                    long long fbase, long long fstride) {
  const int q0 = s * K;
  T v[K];
  if (f0 >= n) {
    const T* __restrict__ inv = tb.inv[d];
    const T* __restrict__ cp = tb.cp[d];
    const T* __restrict__ zv = tb.zv[d];
    const T* __restrict__ g0 = tb.g0[d];
#pragma unroll
    for (int u = 0; u < K; ++u) v[u] = q0 + u < n ? R[base + (q0 + u) * stride] : (T)0;
    T acc = (T)0;
    AffMap<T> mp{(T)1, (T)0};
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (q0 + u < n) {
        const T iv = __ldg(inv + q0 + u);
        acc += __ldg(g0 + q0 + u) * v[u];
        mp = aff_then(mp, AffMap<T>{-a * iv, v[u] * iv});
      }
    for (int o = 1; o < L; o <<= 1) acc += __shfl_xor_sync(mask, acc, o, L);
    const AffMap<T> pre = gscan_up_excl<T, L>(mp, s, mask);
    T y = pre.B;
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (q0 + u < n) {
        y = (v[u] - a * y) * __ldg(inv + q0 + u);
        v[u] = y;
      }
    const T ylast = __shfl_sync(mask, y, (n - 1) / K, L);
    const T fact = (acc + (a / tb.gam[d]) * ylast) / tb.smden[d];
    mp = AffMap<T>{(T)1, (T)0};
#pragma unroll
    for (int u = K - 1; u >= 0; --u)
      if (q0 + u < n) {
        const AffMap<T> rm = (q0 + u == n - 1) ? AffMap<T>{(T)0, v[u]} : AffMap<T>{-__ldg(cp + q0 + u), v[u]};
        mp = aff_then(mp, rm);
      }
    const AffMap<T> suf = gscan_down_excl<T, L>(mp, s, mask);
    T yn = suf.B;
#pragma unroll
    for (int u = K - 1; u >= 0; --u)
      if (q0 + u < n) {
        yn = (q0 + u == n - 1) ? v[u] : v[u] - __ldg(cp + q0 + u) * yn;
        R[base + (q0 + u) * stride] = yn - fact * __ldg(zv + q0 + u);
      }
    return;
  }
  // forcing rows: the line rotated to start at f0 (an identity row)
  const T* __restrict__ invR = tb.invR[d];
  const T* __restrict__ cpR = tb.cpR[d];
  auto rot = [&](int q) { const int r = f0 + q; return r >= n ? r - n : r; };
  unsigned idm = 0;   // bit u: row q0 + u is an identity row (or past the end)
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q < n) {
      const int r = rot(q);
      v[u] = R[base + r * stride];
      if ((fbytes[fbase + r * fstride] >> c) & 1) idm |= 1u << u;
    } else {
      v[u] = (T)0;
      idm |= 1u << u;
    }
  }
  const T x0 = __shfl_sync(mask, v[0], 0, L);   // row q = 0 is an identity row
  const int before = last_identity_before<L>(idm == 0 ? -1 : q0 + 31 - __clz(idm & (q0 + K <= n ? ~0u : ((1u << (n - q0 > 0 ? n - q0 : 0)) - 1u))), s, mask);
  // position of row q0 + u in its segment (rows since the last identity row)
  auto mseg = [&](int u) {
    const unsigned below = idm & ((1u << u) - 1u);
    const int last = below ? q0 + 31 - __clz(below) : before;
    return q0 + u - last - 1;
  };
  AffMap<T> mp{(T)1, (T)0};
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if ((idm >> u) & 1) { mp = AffMap<T>{(T)0, v[u]}; continue; }
    const T iv = __ldg(invR + mseg(u));
    const T dq = (q == n - 1) ? v[u] - a * x0 : v[u];
    mp = aff_then(mp, AffMap<T>{-a * iv, dq * iv});
  }
  const AffMap<T> pre = gscan_up_excl<T, L>(mp, s, mask);
  T y = pre.B;
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if ((idm >> u) & 1) { y = v[u]; continue; }
    const T dq = (q == n - 1) ? v[u] - a * x0 : v[u];
    y = (dq - a * y) * __ldg(invR + mseg(u));
    v[u] = y;
  }
  mp = AffMap<T>{(T)1, (T)0};
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = ((idm >> u) & 1) || q == n - 1;
    mp = aff_then(mp, keep ? AffMap<T>{(T)0, v[u]} : AffMap<T>{-__ldg(cpR + mseg(u)), v[u]});
  }
  const AffMap<T> suf = gscan_down_excl<T, L>(mp, s, mask);
  T yn = suf.B;
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = ((idm >> u) & 1) || q == n - 1;
    yn = keep ? v[u] : v[u] - __ldg(cpR + mseg(u)) * yn;
    if (!((idm >> u) & 1)) R[base + rot(q) * stride] = yn;
  }
}

// One wall-normal line of component c (n rows at R[base + q * stride]):
// the recurrences of solve_wall (segments from the wall (W) or after an
// identity row (R), the wall diagonal in a tangential last row, Dirichlet
// walls for v); the solution du is added to the state u^s on output
// (uhat = u^s + du), as an error-free pair update when Lc holds low parts.
template <typename T, int K, int L>
__device__ __forceinline__ void wall_line_lanes(int n, int c, bool any, T a, const SweepTables<T>& tb, int s,
                                                unsigned mask, const T* __restrict__ R, T* __restrict__ Uc,
                                                T* __restrict__ Lc, long long base, long long stride,
                                                const unsigned char* __restrict__ fbytes, long long fbase,
                                                long long fstride) {
  const bool tang = c != 1;
  const int q0 = s * K;
  T v[K], us[K], ul[K];
  unsigned idm = 0;
  // every load up front: the state (and its low parts) is read here, not in
  // the output loop, where stores to the same arrays would serialise them
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    v[u] = us[u] = ul[u] = (T)0;
    if (q < n) {
      const long long id = base + q * stride;
      v[u] = R[id];
      us[u] = Uc[id];
      if (Lc) ul[u] = Lc[id];
      if (any && ((fbytes[fbase + q * fstride] >> c) & 1)) idm |= 1u << u;
    }
  }
  const int before = last_identity_before<L>(idm ? q0 + 31 - __clz(idm) : -1, s, mask);
  // position of row q0 + u in its segment, and whether the segment starts at
  // the wall (tangential components, no identity row before it)
  auto last_of = [&](int u) {
    const unsigned below = idm & ((1u << u) - 1u);
    return below ? q0 + 31 - __clz(below) : before;
  };
  auto inv_of = [&](int u, int q) -> T {
    const int last = last_of(u), m = q - last - 1;
    if (!tang) return __ldg(tb.vinvR + m);
    const bool w = last < 0;
    if (q == n - 1) return w ? __ldg(tb.yinvLW + m) : __ldg(tb.yinvLR + m);
    return w ? __ldg(tb.yinvW + m) : __ldg(tb.yinvR + m);
  };
  auto cp_of = [&](int u) -> T {
    const int last = last_of(u), m = q0 + u - last - 1;
    if (!tang) return __ldg(tb.vcpR + m);
    return last < 0 ? __ldg(tb.ycpW + m) : __ldg(tb.ycpR + m);
  };
  AffMap<T> mp{(T)1, (T)0};
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if ((idm >> u) & 1) { mp = AffMap<T>{(T)0, v[u]}; continue; }
    const T iv = inv_of(u, q);
    mp = aff_then(mp, AffMap<T>{-a * iv, v[u] * iv});
  }
  const AffMap<T> pre = gscan_up_excl<T, L>(mp, s, mask);
  T y = pre.B;
#pragma unroll
  for (int u = 0; u < K; ++u) {
    const int q = q0 + u;
    if (q >= n) break;
    if ((idm >> u) & 1) { y = v[u]; continue; }
    y = (v[u] - a * y) * inv_of(u, q);
    v[u] = y;
  }
  mp = AffMap<T>{(T)1, (T)0};
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = ((idm >> u) & 1) || q == n - 1;
    mp = aff_then(mp, keep ? AffMap<T>{(T)0, v[u]} : AffMap<T>{-cp_of(u), v[u]});
  }
  const AffMap<T> suf = gscan_down_excl<T, L>(mp, s, mask);
  T yn = suf.B;
#pragma unroll
  for (int u = K - 1; u >= 0; --u) {
    const int q = q0 + u;
    if (q >= n) continue;
    const bool keep = ((idm >> u) & 1) || q == n - 1;
    yn = keep ? v[u] : v[u] - cp_of(u) * yn;
    const long long id = base + q * stride;
    if (Lc) {
      float hi = (float)us[u], lo = (float)ul[u];
      ff_add(hi, lo, (float)yn);
      Uc[id] = (T)hi;
      Lc[id] = (T)lo;
    } else {
      Uc[id] = us[u] + yn;
    }
  }
}

// dir 2: z-lines at fixed j (bk.z); dir 1: y-lines at fixed k (bk.z).
// Block: 256 threads, 8 warps x G lines = 64 consecutive i of component bk.y.
template <typename T, int K, int L>
__device__ __forceinline__ void sweep_lanes(const Blk& bk, const Geo& g, const Fields<T>& f,
                                            const unsigned* __restrict__ flags32, const SweepTables<T>& tb,
                                            const int* __restrict__ lfirst, int dir) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane / L, s = lane % L;
  const unsigned mask = (L == 32) ? 0xFFFFFFFFu : (((1u << L) - 1u) << (grp * L));
  const int c = bk.y;
  const int i = bk.x * (8 * G) + wid * G + grp;
  if (i >= g.nx) return;   // whole line groups only (their lanes share i)
  const int pl = planes(g, c);
  const unsigned char* fbytes = reinterpret_cast<const unsigned char*>(flags32);
  T* __restrict__ R = f.R[c];
  if (dir == 2) {
    if (c == 1 && (int)bk.z >= g.ny - 1) return;   // v has ny-1 interior planes
    const int j = (c == 1 ? 1 : 0) + bk.z;
    const long long base = fidx(g, c, i, j, 0), stride = (long long)pl * g.nx;
    const long long fbase = cidx(g, i, j, 0), fstride = (long long)g.ny * g.nx;
    periodic_line_lanes<T, K, L>(g.nz, lfirst[line_z(g, c, i, j)], c, 1, -tb.off[2], tb, s, mask, R, base, stride,
                                 fbytes, fbase, fstride);
  } else {
    const int k = bk.z;
    const int jj0 = c == 1 ? 1 : 0;
    const int n = c == 1 ? g.ny - 1 : g.ny;
    const long long base = fidx(g, c, i, jj0, k), fbase = cidx(g, i, jj0, k);
    T* __restrict__ Uc = c == 0 ? f.u : (c == 1 ? f.v : f.w);
    wall_line_lanes<T, K, L>(n, c, lfirst[line_y(g, c, i, k)] < g.ny, -tb.off[1], tb, s, mask, R, Uc, f.lo[c], base,
                             g.nx, fbytes, fbase, g.nx);
  }
}
template <typename T, int K, int L>
struct SweepLanes {
  static constexpr int kThreads = 256;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  int dir;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_lanes<T, K, L>(bk, g, f, flags32, tb, lfirst, dir); }
};

// z- and y-sweeps: a block holds the lines of W consecutive i (one plane
// position each) for all n rows, tile [n][W] (row m of line t at m*W + t);
// rows are loaded and stored coalesced.  dir 2: z-lines at fixed j
// (blockIdx.z); dir 1: y-lines at fixed k (blockIdx.z), and the solution du
// is added to the state (uhat = u^s + du) on the way out.
template <typename T>
__device__ __forceinline__ void sweep_zy(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32,
                                                 const SweepTables<T>& tb, const int* __restrict__ lfirst, int dir) {
  extern __shared__ unsigned char smem_raw[];
  const int W = blockDim.x, t = threadIdx.x;
  const int c = bk.y;
  const int i0 = bk.x * W;
  const int pl = planes(g, c);
  int n;
  long long base, stride, fbase, fstride;
  if (dir == 2) {
    if (c == 1 && (int)bk.z >= g.ny - 1) return;   // v has ny-1 interior planes
    const int j = (c == 1 ? 1 : 0) + bk.z;     // fixed j of these z-lines
    n = g.nz;
    base = fidx(g, c, i0, j, 0);
    stride = (long long)pl * g.nx;
    fbase = cidx(g, i0, j, 0);
    fstride = (long long)g.ny * g.nx;
  } else {
    const int k = bk.z;
    const int jj0 = c == 1 ? 1 : 0;
    n = c == 1 ? g.ny - 1 : g.ny;
    base = fidx(g, c, i0, jj0, k);
    stride = g.nx;
    fbase = cidx(g, i0, jj0, k);
    fstride = g.nx;
  }
  const int w = min(W, g.nx - i0);
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* ust = tile + (size_t)n * W;                        // y-sweep: the state u^s of the same lines
  const bool pair = dir == 1 && f.lo[c] != nullptr;     // y-sweep on a (hi, lo) velocity state
  T* ulo = ust + (size_t)n * W;                         // ... and its low parts
  unsigned char* fl = reinterpret_cast<unsigned char*>(tile + (size_t)(dir == 1 ? (pair ? 3 : 2) : 1) * n * W);
  T* __restrict__ R = f.R[c];
  T* __restrict__ Uc = comp_ptr(f, c);
  const unsigned char* fbytes = reinterpret_cast<const unsigned char*>(flags32);
  const bool words = (w & 3) == 0 && (fstride & 3) == 0 && (fbase & 3) == 0;
  if (t < w) {
    for (int m = 0; m < n; ++m) {
      cp_async<sizeof(T)>(tile + m * W + t, R + base + m * stride + t);
      if (dir == 1) cp_async<sizeof(T)>(ust + m * W + t, Uc + base + m * stride + t);
      if (pair) cp_async<sizeof(T)>(ulo + m * W + t, f.lo[c] + base + m * stride + t);
    }
  }
  if (words) {
    for (int e = t; e < n * (w / 4); e += W) {
      const int m = e / (w / 4), q = e - m * (w / 4);
      cp_async<4>(fl + m * W + 4 * q, fbytes + fbase + m * fstride + 4 * q);
    }
  } else if (t < w) {
    for (int m = 0; m < n; ++m) fl[m * W + t] = fbytes[fbase + m * fstride + t];
  }
  cp_async_wait_all();
  __syncthreads();
  if (t < w) {
    const int i = i0 + t;
    auto E = [&](int m) -> T& { return tile[m * W + t]; };
    auto F = [&](int m) { return (int)fl[m * W + t]; };
    if (dir == 2) {
      const int j = (c == 1 ? 1 : 0) + bk.z;
      solve_periodic<T>(n, c, lfirst[line_z(g, c, i, j)], 1, -tb.off[2], tb, E, F);
      for (int m = 0; m < n; ++m) R[base + m * stride + t] = tile[m * W + t];
    } else {
      const int k = bk.z;
      solve_wall<T>(n, c, lfirst[line_y(g, c, i, k)] < g.ny, -tb.off[1], tb, E, F);
      if (f.lo[c]) {
        // velocity state as a (hi, lo) pair: add du without rounding it away
        T* __restrict__ Lc = f.lo[c];
        for (int m = 0; m < n; ++m) {
          const long long id = base + m * stride + t;
          float hi = (float)ust[m * W + t], lo = (float)ulo[m * W + t];
          ff_add(hi, lo, (float)tile[m * W + t]);
          Uc[id] = (T)hi;
          Lc[id] = (T)lo;
        }
      } else {
        for (int m = 0; m < n; ++m) Uc[base + m * stride + t] = ust[m * W + t] + tile[m * W + t];
      }
    }
  }
}
template <typename T>
struct SweepZY {
  static constexpr int kThreads = 64;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  int dir;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_zy<T>(bk, g, f, flags32, tb, lfirst, dir); }
};

// y-sweep streamed through registers, one thread per line (component bk.y,
// line t = i + nx k, so a warp reads each row of 32 neighbouring lines as
// one coalesced segment).  Rows are read SYB at a time ahead of the
// recurrence.  The forward pass writes its values over R and the backward
// multiplier c' of every row into the scratch array (0 on identity rows),
// so the backward pass is the same branch-free recurrence for every line,
// x_j = p_j - c'_j x_{j+1}, adding du to the state on its way out.  Same
// recurrences, tables and operation order as solve_wall: a forcing row is
// a forward step with multiplier 0 and pivot 1, which leaves its value.
constexpr int SYB = 16;

template <typename T>
__device__ __forceinline__ void sweep_y_stream(const Blk& bk, const Geo& g, const Fields<T>& f,
                                               const unsigned* __restrict__ flags32, const SweepTables<T>& tb,
                                               const int* __restrict__ lfirst) {
  const int c = bk.y;
  const long long t = (long long)bk.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nx * g.nz) return;
  const int i = (int)(t % g.nx), k = (int)(t / g.nx);
  const int jj0 = c == 1 ? 1 : 0;
  const int n = c == 1 ? g.ny - 1 : g.ny;
  const int sn = g.nx;   // row stride of both the field and the flag bytes
  const long long base = fidx(g, c, i, jj0, k);
  T* __restrict__ Rl = f.R[c] + base;
  T* __restrict__ Sl = f.scr + comp_off(g, c) + base;
  T* __restrict__ Ul = comp_ptr(f, c) + base;
  T* __restrict__ Ll = f.lo[c] ? f.lo[c] + base : nullptr;
  const unsigned char* __restrict__ Fl = reinterpret_cast<const unsigned char*>(flags32) + cidx(g, i, jj0, k);
  const T a = -tb.off[1];
  const bool tang = c != 1;
  const bool any = lfirst[line_y(g, c, i, k)] < g.ny;
  // ---- forward: p_j = (r_j - a_j p_{j-1}) iv_j; c'_j to the scratch
  T prev = (T)0;
  int m = 0;
  bool segW = tang;
  for (int j0 = 0; j0 < n; j0 += SYB) {
    T e[SYB];
    unsigned char fl[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int j = j0 + u;
      e[u] = (T)0;
      fl[u] = 0;
      if (j < n) {
        e[u] = Rl[j * sn];
        if (any) fl[u] = Fl[j * sn];
      }
    }
    // segment positions and table entries of the batch (flags only)
    T iv[SYB], cq[SYB], am[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int j = j0 + u;
      const bool frc = (fl[u] >> c) & 1;
      const bool last = j == n - 1;
      const T* ivt = !tang ? tb.vinvR : (last ? (segW ? tb.yinvLW : tb.yinvLR) : (segW ? tb.yinvW : tb.yinvR));
      const T* cpt = !tang ? tb.vcpR : (segW ? tb.ycpW : tb.ycpR);
      iv[u] = (T)1;
      cq[u] = (T)0;
      am[u] = (T)0;
      if (j < n && !frc) {
        iv[u] = __ldg(ivt + m);
        if (!last) cq[u] = __ldg(cpt + m);
        am[u] = a;
      }
      m = frc ? 0 : m + 1;
      segW = segW && !frc;
    }
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int j = j0 + u;
      if (j < n) {
        prev = (e[u] - am[u] * prev) * iv[u];
        Rl[j * sn] = prev;
        if (any) Sl[j * sn] = cq[u];   // a line without forcing rows reads c' from the table
      }
    }
  }
  // ---- backward: x_j = p_j - c'_j x_{j+1}; uhat = u^s + x
  const T* __restrict__ cpw = tang ? tb.ycpW : tb.vcpR;   // c' of one wall segment
  T x = (T)0;
  for (int j1 = n - 1; j1 >= 0; j1 -= SYB) {
    T pv[SYB], cv[SYB], uh[SYB], ul[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int j = j1 - u;
      pv[u] = cv[u] = uh[u] = ul[u] = (T)0;
      if (j >= 0) {
        pv[u] = Rl[j * sn];
        cv[u] = any ? Sl[j * sn] : (j < n - 1 ? __ldg(cpw + j) : (T)0);
        uh[u] = Ul[j * sn];
        if (Ll) ul[u] = Ll[j * sn];
      }
    }
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int j = j1 - u;
      if (j < 0) break;
      x = pv[u] - cv[u] * x;
      if (Ll) {
        // velocity state as a (hi, lo) pair: add du without rounding it away
        float hi = (float)uh[u], lo = (float)ul[u];
        ff_add(hi, lo, (float)x);
        Ul[j * sn] = (T)hi;
        Ll[j * sn] = (T)lo;
      } else {
        Ul[j * sn] = uh[u] + x;
      }
    }
  }
}
// z-sweep streamed the same way, one thread per periodic line (component
// bk.y, line t = i + nx l at plane j = l (+1 for v)).  A line without
// forcing rows is solved by Sherman-Morrison (tabulated Thomas of the
// modified matrix, first-row dot product g0, correction along zv); a line
// with forcing rows runs rotated to start at its first forcing row (an
// identity row), its last row's periodic coupling moved to the right-hand
// side.  Both share the forward step p_q = (d_q - a_q p_{q-1}) iv_q with c'_q
// stored in the scratch array, and the backward step x_q = p_q - c'_q x_{q+1}
// (minus fact zv_q for Sherman-Morrison); same operation order as
// solve_periodic.
template <typename T>
__device__ __forceinline__ void sweep_z_stream(const Blk& bk, const Geo& g, const Fields<T>& f,
                                               const unsigned* __restrict__ flags32, const SweepTables<T>& tb,
                                               const int* __restrict__ lfirst) {
  const int c = bk.y;
  const int nplanes = c == 1 ? g.ny - 1 : g.ny;    // v: interior planes j = 1 .. ny-1
  const long long t = (long long)bk.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nx * nplanes) return;
  const int i = (int)(t % g.nx), l = (int)(t / g.nx);
  const int j = (c == 1 ? 1 : 0) + l;
  const int n = g.nz;
  const int sn = planes(g, c) * g.nx;              // row stride along z
  const int fs = g.ny * g.nx;                      // flag-byte stride along z
  const long long base = fidx(g, c, i, j, 0);
  T* __restrict__ Rl = f.R[c] + base;
  T* __restrict__ Sl = f.scr + comp_off(g, c) + base;
  const unsigned char* __restrict__ Fl = reinterpret_cast<const unsigned char*>(flags32) + cidx(g, i, j, 0);
  const T a = -tb.off[2];
  const int f0 = lfirst[line_z(g, c, i, j)];
  const bool any = f0 < n;
  const int r0 = any ? f0 : 0;
  const T x0 = any ? Rl[f0 * sn] : (T)0;
  auto rot = [&](int q) { const int r = r0 + q; return r >= n ? r - n : r; };
  // ---- forward
  T prev = (T)0, acc = (T)0;
  int m = 0;
  for (int q0 = 0; q0 < n; q0 += SYB) {
    T e[SYB];
    unsigned char fl[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int q = q0 + u;
      e[u] = (T)0;
      fl[u] = 0;
      if (q < n) {
        const int r = rot(q);
        e[u] = Rl[r * sn];
        if (any) fl[u] = Fl[r * fs];
      }
    }
    T iv[SYB], cq[SYB], am[SYB], gq[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int q = q0 + u;
      const bool frc = (fl[u] >> c) & 1;
      iv[u] = (T)1;
      cq[u] = (T)0;
      am[u] = (T)0;
      gq[u] = (T)0;
      if (q < n && !frc) {
        if (any) {
          iv[u] = __ldg(tb.invR[1] + m);
          if (q < n - 1) cq[u] = __ldg(tb.cpR[1] + m);
        } else {
          iv[u] = __ldg(tb.inv[1] + q);
          if (q < n - 1) cq[u] = __ldg(tb.cp[1] + q);
          gq[u] = __ldg(tb.g0[1] + q);
        }
        am[u] = a;
      }
      m = frc ? 0 : m + 1;
    }
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int q = q0 + u;
      if (q < n) {
        T dq = e[u];
        if (any && q == n - 1 && am[u] != (T)0) dq -= a * x0;
        if (!any) acc += gq[u] * dq;
        prev = (dq - am[u] * prev) * iv[u];
        const int r = rot(q);
        Rl[r * sn] = prev;
        Sl[r * sn] = cq[u];
      }
    }
  }
  const T fact = any ? (T)0 : (acc + (a / tb.gam[1]) * prev) / tb.smden[1];
  // ---- backward
  T x = (T)0;
  for (int q1 = n - 1; q1 >= 0; q1 -= SYB) {
    T pv[SYB], cv[SYB], zq[SYB];
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int q = q1 - u;
      pv[u] = cv[u] = zq[u] = (T)0;
      if (q >= 0) {
        const int r = rot(q);
        pv[u] = Rl[r * sn];
        cv[u] = Sl[r * sn];
        if (!any) zq[u] = __ldg(tb.zv[1] + q);
      }
    }
#pragma unroll
    for (int u = 0; u < SYB; ++u) {
      const int q = q1 - u;
      if (q < 0) break;
      x = pv[u] - cv[u] * x;
      Rl[rot(q) * sn] = any ? x : x - fact * zq[u];
    }
  }
}
template <typename T>
struct SweepZStream {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_z_stream<T>(bk, g, f, flags32, tb, lfirst); }
};

// z-sweep from a shared-memory tile: a block of ZT_THREADS threads stages the
// ZT_W z-lines of ZT_W consecutive i at one plane (component bk.z, plane
// bk.y) -- all n rows, one coalesced 128-byte row segment each, every copy
// issued before the first wait -- together with the rows' flag bytes (when
// a line of the tile crosses a body) and the z tables.  One warp then runs
// the same recurrences as the streamed z-sweep (same operations in the same
// order; a multiply-add may be fused differently) from shared memory, one
// lane per line; lane t reads row r at r * ZT_W + t, so the lanes never share a bank
// whatever rotation their lines take.  The block writes the tile back
// coalesced.  The forward pass keeps each row's position in its segment in
// the flag byte (0 on a forcing row), from which the backward pass reads c'.
constexpr int ZT_W = 32, ZT_THREADS = 128;
template <typename T>
__host__ __device__ inline size_t sweep_z_tile_smem(int n) {
  return (size_t)n * ZT_W * sizeof(T) + (size_t)6 * n * sizeof(T) + (size_t)n * ZT_W;
}
template <typename T>
__device__ __forceinline__ void sweep_z_tile(const Blk& bk, const Geo& g, const Fields<T>& f,
                                             const unsigned* __restrict__ flags32, const SweepTables<T>& tb,
                                             const int* __restrict__ lfirst) {
  extern __shared__ unsigned char smem_raw[];
  const int c = bk.z;
  const int nplanes = c == 1 ? g.ny - 1 : g.ny;    // v: interior planes j = 1 .. ny-1
  if ((int)bk.y >= nplanes) return;
  const int j = (c == 1 ? 1 : 0) + bk.y;
  const int i0 = bk.x * ZT_W;
  const int w = min(ZT_W, g.nx - i0);
  const int n = g.nz;
  const long long sn = (long long)planes(g, c) * g.nx;   // row stride along z
  const long long fs = (long long)g.ny * g.nx;           // flag-byte stride along z
  T* tile = reinterpret_cast<T*>(smem_raw);               // [n][ZT_W]
  T* tabs = tile + (size_t)n * ZT_W;                      // inv, cp, g0, zv, invR, cpR (n each)
  unsigned char* fl = reinterpret_cast<unsigned char*>(tabs + (size_t)6 * n);   // [n][ZT_W]
  T* __restrict__ Rl = f.R[c] + fidx(g, c, i0, j, 0);
  const unsigned char* __restrict__ Fl = reinterpret_cast<const unsigned char*>(flags32) + cidx(g, i0, j, 0);
  const int tid = threadIdx.x;
  __shared__ int any_s;
  if (tid == 0) any_s = 0;
  __syncthreads();
  int f0 = n;
  if (tid < w) {
    f0 = lfirst[line_z(g, c, i0 + tid, j)];
    if (f0 < n) atomicOr(&any_s, 1);
  }
  // every row of the tile, then the tables
  for (int e = tid; e < n * ZT_W; e += ZT_THREADS) {
    const int r = e / ZT_W, t = e - r * ZT_W;
    if (t < w) cp_async<sizeof(T)>(tile + e, Rl + r * sn + t);
  }
  for (int e = tid; e < n; e += ZT_THREADS) {
    tabs[e] = tb.inv[1][e];
    tabs[n + e] = e < n - 1 ? tb.cp[1][e] : (T)0;
    tabs[2 * n + e] = tb.g0[1][e];
    tabs[3 * n + e] = tb.zv[1][e];
    tabs[4 * n + e] = tb.invR[1][e];
    tabs[5 * n + e] = tb.cpR[1][e];
  }
  __syncthreads();   // any_s
  const bool tile_any = any_s != 0;
  if (tile_any) {
    for (int e = tid; e < n * ZT_W; e += ZT_THREADS) {
      const int r = e / ZT_W, t = e - r * ZT_W;
      fl[e] = t < w ? Fl[r * fs + t] : (unsigned char)0;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if (tid < w) {
    const int t = tid;
    const bool any = f0 < n;
    const T a = -tb.off[2];
    const T* inv = tabs;
    const T* cpt = tabs + n;
    const T* g0 = tabs + 2 * n;
    const T* zv = tabs + 3 * n;
    const T* invR = tabs + 4 * n;
    const T* cpR = tabs + 5 * n;
    const int r0 = any ? f0 : 0;
    auto rot = [&](int q) { const int r = r0 + q; return r >= n ? r - n : r; };
    const T x0 = any ? tile[r0 * ZT_W + t] : (T)0;
    // ---- forward
    T prev = (T)0, acc = (T)0;
    int m = 0;
    if (any && (n & 7) == 0) {
      // rows in batches of 8: the batch's rows and flags first, then the
      // segment positions and pivots (they depend on the flags alone), then
      // the recurrence.  A row keeps m + 1 for its c' = cpR[m] (0: a forcing
      // row or the last row, c' = 0); m + 1 <= n - 1 since row q = 0 is a
      // forcing row
      for (int q0 = 0; q0 < n; q0 += 8) {
        T e[8], iv[8], am[8];
        int rr[8];
        unsigned char fb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          rr[u] = rot(q0 + u);
          e[u] = tile[rr[u] * ZT_W + t];
          fb[u] = fl[rr[u] * ZT_W + t];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int q = q0 + u;
          const bool frc = (fb[u] >> c) & 1;
          iv[u] = frc ? (T)1 : invR[m];
          am[u] = frc ? (T)0 : a;
          fb[u] = frc || q == n - 1 ? (unsigned char)0 : (unsigned char)(m + 1);
          m = frc ? 0 : m + 1;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          T dq = e[u];
          if (q0 + u == n - 1 && am[u] != (T)0) dq -= a * x0;
          prev = (dq - am[u] * prev) * iv[u];
          e[u] = prev;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          tile[rr[u] * ZT_W + t] = e[u];
          fl[rr[u] * ZT_W + t] = fb[u];
        }
      }
    } else if (any) {
      for (int q = 0; q < n; ++q) {
        const int r = rot(q);
        const bool frc = (fl[r * ZT_W + t] >> c) & 1;
        T iv = (T)1, am = (T)0;
        if (!frc) {
          iv = invR[m];
          am = a;
        }
        T dq = tile[r * ZT_W + t];
        if (q == n - 1 && am != (T)0) dq -= a * x0;
        prev = (dq - am * prev) * iv;
        tile[r * ZT_W + t] = prev;
        fl[r * ZT_W + t] = frc || q == n - 1 ? (unsigned char)0 : (unsigned char)(m + 1);
        m = frc ? 0 : m + 1;
      }
    } else if ((n & 7) == 0) {
      // rows in batches of 8 through registers, every shared-memory load of
      // a batch issued before its recurrence
      for (int q0 = 0; q0 < n; q0 += 8) {
        T e[8], gg[8], vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { e[u] = tile[(q0 + u) * ZT_W + t]; gg[u] = g0[q0 + u]; vv[u] = inv[q0 + u]; }
#pragma unroll
        for (int u = 0; u < 8; ++u) { acc += gg[u] * e[u]; prev = (e[u] - a * prev) * vv[u]; e[u] = prev; }
#pragma unroll
        for (int u = 0; u < 8; ++u) tile[(q0 + u) * ZT_W + t] = e[u];
      }
    } else {
      for (int q = 0; q < n; ++q) {
        const T dq = tile[q * ZT_W + t];
        acc += g0[q] * dq;
        prev = (dq - a * prev) * inv[q];
        tile[q * ZT_W + t] = prev;
      }
    }
    const T fact = any ? (T)0 : (acc + (a / tb.gam[1]) * prev) / tb.smden[1];
    // ---- backward
    T x = (T)0;
    if (any && (n & 7) == 0) {
      for (int q1 = n - 8; q1 >= 0; q1 -= 8) {
        T e[8], cv[8];
        int rr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          rr[u] = rot(q1 + u);
          e[u] = tile[rr[u] * ZT_W + t];
          const int mq = fl[rr[u] * ZT_W + t];
          cv[u] = mq ? cpR[mq - 1] : (T)0;
        }
#pragma unroll
        for (int u = 7; u >= 0; --u) {
          x = e[u] - cv[u] * x;
          e[u] = x;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) tile[rr[u] * ZT_W + t] = e[u];
      }
    } else if (any) {
      for (int q = n - 1; q >= 0; --q) {
        const int r = rot(q);
        const int mq = fl[r * ZT_W + t];
        const T cv = mq ? cpR[mq - 1] : (T)0;
        x = tile[r * ZT_W + t] - cv * x;
        tile[r * ZT_W + t] = x;
      }
    } else if ((n & 7) == 0) {
      for (int q1 = n - 8; q1 >= 0; q1 -= 8) {
        T e[8], cc[8], zz[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { e[u] = tile[(q1 + u) * ZT_W + t]; cc[u] = cpt[q1 + u]; zz[u] = zv[q1 + u]; }
#pragma unroll
        for (int u = 7; u >= 0; --u) { x = e[u] - cc[u] * x; e[u] = x - fact * zz[u]; }
#pragma unroll
        for (int u = 0; u < 8; ++u) tile[(q1 + u) * ZT_W + t] = e[u];
      }
    } else {
      for (int q = n - 1; q >= 0; --q) {
        x = tile[q * ZT_W + t] - cpt[q] * x;
        tile[q * ZT_W + t] = x - fact * zv[q];
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < n * ZT_W; e += ZT_THREADS) {
    const int r = e / ZT_W, t = e - r * ZT_W;
    if (t < w) Rl[r * sn + t] = tile[e];
  }
}
template <typename T>
struct SweepZTile {
  static constexpr int kThreads = ZT_THREADS;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_z_tile<T>(bk, g, f, flags32, tb, lfirst); }
};

// y-sweep on a non-uniform wall-normal grid, one thread per line: the rows'
// coefficients are those of the y part of the Laplacian of the right-hand
// side, from the spacing table, and a forcing node's row is the identity;
// the line is factorised as it is swept (c' to the scratch array) and du is
// added to the state on the way back (as a (hi, lo) pair in the mixed path).
// The same line in FP32 from the FP32 copies of the row tables (mixed path):
// a line without forcing rows in one wall segment, a line with forcing rows
// restarting at [start row][row] after each identity row (c' to the scratch
// array).  Rows move in batches of SYS_B through registers, every load of a
// batch issued before its recurrence runs.
constexpr int SYS_B = 8;

__device__ __forceinline__ void sweep_y_stretched_f32(const Geo& g, const Fields<float>& f,
                                                      const unsigned* __restrict__ flags32, bool any, int c, int i,
                                                      int k, int n, int jj0, int sn, float* __restrict__ Rl,
                                                      float* __restrict__ Sl, float* __restrict__ Ul,
                                                      float* __restrict__ Ll) {
  const float* __restrict__ ta = g.yt.yswf + (c == 1 ? 3ll * g.ny : 0);
  const float* __restrict__ tv = ta + n;
  const float* __restrict__ tc = tv + n;
  const float* __restrict__ iv2 = g.yt.ysw2f + (c == 1 ? 2ll * g.ny * g.ny : 0);
  const float* __restrict__ cp2 = iv2 + (long long)n * n;
  const unsigned char* __restrict__ Fl = reinterpret_cast<const unsigned char*>(flags32) + cidx(g, i, jj0, k);
  // ---- forward
  float p = 0.0f;
  long long s0 = 0;
  for (int m0 = 0; m0 < n; m0 += SYS_B) {
    float r[SYS_B];
    unsigned char fl[SYS_B];
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m0 + u;
      r[u] = 0.0f;
      fl[u] = 0;
      if (m < n) {
        r[u] = Rl[m * sn];
        if (any) fl[u] = Fl[(long long)m * sn];
      }
    }
    float cq[SYS_B];
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m0 + u;
      cq[u] = 0.0f;
      if (m >= n) continue;
      if (!any) {
        p = fmaf(-__ldg(ta + m), p, r[u]) * __ldg(tv + m);
      } else if ((fl[u] >> c) & 1) {
        p = r[u];
        s0 = m + 1;
      } else {
        const long long id = s0 * n + m;
        p = fmaf(-__ldg(ta + m), p, r[u]) * __ldg(iv2 + id);
        cq[u] = __ldg(cp2 + id);
      }
      r[u] = p;
    }
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m0 + u;
      if (m < n) {
        Rl[m * sn] = r[u];
        if (any) Sl[m * sn] = cq[u];
      }
    }
  }
  // ---- backward: x_m = p_m - c'_m x_{m+1}; uhat = u^s + x
  float x = 0.0f;
  for (int m1 = n - 1; m1 >= 0; m1 -= SYS_B) {
    float pv[SYS_B], cv[SYS_B], uh[SYS_B], ul[SYS_B];
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m1 - u;
      pv[u] = cv[u] = uh[u] = ul[u] = 0.0f;
      if (m >= 0) {
        pv[u] = Rl[m * sn];
        cv[u] = any ? Sl[m * sn] : __ldg(tc + m);
        uh[u] = Ul[m * sn];
        if (Ll) ul[u] = Ll[m * sn];
      }
    }
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m1 - u;
      if (m < 0) break;
      x = fmaf(-cv[u], x, pv[u]);
      if (Ll) {
        ff_add(uh[u], ul[u], x);
      } else {
        uh[u] += x;
      }
    }
#pragma unroll
    for (int u = 0; u < SYS_B; ++u) {
      const int m = m1 - u;
      if (m >= 0) {
        Ul[m * sn] = uh[u];
        if (Ll) Ll[m * sn] = ul[u];
      }
    }
  }
}

// A line without forcing rows (most lines) takes its rows' a, 1/pivot and
// c' from the table built with the grid, with no division and no scratch.
template <typename T>
__device__ __forceinline__ void sweep_y_stretched(const Blk& bk, const Geo& g, const Fields<T>& f,
                                                  const unsigned* __restrict__ flags32,
                                                  const int* __restrict__ lfirst, double beta) {
  const int c = bk.y;
  const long long t = (long long)bk.x * blockDim.x + threadIdx.x;
  if (t >= (long long)g.nx * g.nz) return;
  const int i = (int)(t % g.nx), k = (int)(t / g.nx);
  const int jj0 = c == 1 ? 1 : 0;
  const int n = c == 1 ? g.ny - 1 : g.ny;
  const int sn = g.nx;
  const long long base = fidx(g, c, i, jj0, k);
  T* __restrict__ Rl = f.R[c] + base;
  T* __restrict__ Sl = f.scr + comp_off(g, c) + base;
  T* __restrict__ Ul = comp_ptr(f, c) + base;
  T* __restrict__ Ll = f.lo[c] ? f.lo[c] + base : nullptr;
  if constexpr (sizeof(T) == 4) {
    // mixed path: FP32 rows and recurrences, as the uniform grid's sweeps
    if (g.yt.yswf && (lfirst[line_y(g, c, i, k)] >= g.ny || g.yt.ysw2f)) {
      sweep_y_stretched_f32(g, f, flags32, lfirst[line_y(g, c, i, k)] < g.ny, c, i, k, n, jj0, sn, Rl, Sl, Ul, Ll);
      return;
    }
  }
  if (lfirst[line_y(g, c, i, k)] >= g.ny) {
    const double* __restrict__ ta = g.yt.ysw + (c == 1 ? 3ll * g.ny : 0);
    const double* __restrict__ tv = ta + n;
    const double* __restrict__ tc = tv + n;
    double p = 0.0;
    for (int m = 0; m < n; ++m) {
      p = ((double)Rl[m * sn] - __ldg(ta + m) * p) * __ldg(tv + m);
      Rl[m * sn] = (T)p;
    }
    double x = 0.0;
    for (int m = n - 1; m >= 0; --m) {
      x = (double)Rl[m * sn] - __ldg(tc + m) * x;
      if (Ll) {
        float hi = (float)Ul[m * sn], lo = (float)Ll[m * sn];
        ff_add(hi, lo, (float)x);
        Ul[m * sn] = (T)hi;
        Ll[m * sn] = (T)lo;
      } else {
        Ul[m * sn] = (T)((double)Ul[m * sn] + x);
      }
    }
    return;
  }
  if (g.yt.ysw2) {
    // forcing rows are identity rows; the segment after one restarts the
    // elimination, its pivots read at [start row][row]
    const double* __restrict__ ta = g.yt.ysw + (c == 1 ? 3ll * g.ny : 0);
    const double* __restrict__ iv2 = g.yt.ysw2 + (c == 1 ? 2ll * g.ny * g.ny : 0);
    const double* __restrict__ cp2 = iv2 + (long long)n * n;
    long long s0 = 0;
    double p = 0.0;
    for (int m = 0; m < n; ++m) {
      double cq = 0.0;
      if (is_forcing(flags32, cidx(g, i, jj0 + m, k), c)) {
        p = (double)Rl[m * sn];
        s0 = m + 1;
      } else {
        const long long id = s0 * n + m;
        p = ((double)Rl[m * sn] - __ldg(ta + m) * p) * __ldg(iv2 + id);
        cq = __ldg(cp2 + id);
      }
      Rl[m * sn] = (T)p;
      Sl[m * sn] = (T)cq;
    }
  } else {
    const double gs = g.ybc == 0 ? -1.0 : 1.0;
    double prev = 0.0, cprev = 0.0;
    for (int m = 0; m < n; ++m) {
      const int j = jj0 + m;
      double sb, sn2;
      if (c != 1) {
        sb = beta * g.yt.ihc[j] * g.yt.ihf[j];
        sn2 = beta * g.yt.ihc[j] * g.yt.ihf[j + 1];
      } else {
        sb = beta * g.yt.ihf[j] * g.yt.ihc[j - 1];
        sn2 = beta * g.yt.ihf[j] * g.yt.ihc[j];
      }
      double a = -sb, b = 1.0 + sb + sn2, cc = -sn2;
      if (m == 0) {
        if (c != 1) b -= gs * sb;   // wall ghost du_{-1} = gs du_0
        a = 0.0;
      }
      if (m == n - 1) {
        if (c != 1) b -= gs * sn2;
        cc = 0.0;
      }
      if (is_forcing(flags32, cidx(g, i, j, k), c)) {
        a = 0.0;
        b = 1.0;
        cc = 0.0;
      }
      const double den = b - a * cprev;
      cprev = cc / den;
      prev = ((double)Rl[m * sn] - a * prev) / den;
      Rl[m * sn] = (T)prev;
      Sl[m * sn] = (T)cprev;
    }
  }
  double x = 0.0;
  for (int m = n - 1; m >= 0; --m) {
    x = (double)Rl[m * sn] - (double)Sl[m * sn] * x;
    if (Ll) {
      // velocity state as a (hi, lo) pair: add du without rounding it away
      float hi = (float)Ul[m * sn], lo = (float)Ll[m * sn];
      ff_add(hi, lo, (float)x);
      Ul[m * sn] = (T)hi;
      Ll[m * sn] = (T)lo;
    } else {
      Ul[m * sn] = (T)((double)Ul[m * sn] + x);
    }
  }
}
template <typename T>
struct SweepYStretched {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const int* lfirst;
  double beta;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    sweep_y_stretched<T>(bk, g, f, flags32, lfirst, beta);
  }
};

template <typename T>
struct SweepYStream {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_y_stream<T>(bk, g, f, flags32, tb, lfirst); }
};

// y-sweep with each tile staged by TMA: one CTA (one warp) per 32
// consecutive lines of one (k, component).  R, u^s and, in the mixed path,
// the low parts of the tile are one tensor copy each (a 32 x rows box of the
// [k][j][i] array) into shared memory, completing on one mbarrier; the warp
// then runs the recurrences of the streamed sweep from shared memory (R
// overwritten in place, c' from the tables or, on lines crossing a body,
// the scratch array) and writes uhat to global memory.  So R and u^s are
// read once and u written once, and several CTAs per SM overlap one tile's
// copies with another's recurrences.
constexpr int SYT_W = 32;                              // lines per tile (128 B of FP32 per row)
constexpr long long SYT_WAIT_CYCLES = 4000000000ll;   // about 2 s at the top SM clock

// One box of a 3-D tensor map (coordinates x fastest) into shared memory.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <typename T>
struct SweepYTma;

template <typename T>
__device__ __forceinline__ void sweep_y_tma(const Blk& bk, const SweepYTma<T>& op) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar_mem;
  const Geo& g = op.g;
  const Fields<T>& f = op.f;
  const SweepTables<T>& tb = op.tb;
  const int c = (int)bk.z, k = (int)bk.y;
  const int i0 = (int)bk.x * SYT_W;
  const int lane = threadIdx.x;
  const int jj0 = c == 1 ? 1 : 0;
  const int n = c == 1 ? g.ny - 1 : g.ny;
  const int nl = min(SYT_W, g.nx - i0);
  const int sn = g.nx;
  const long long base = fidx(g, c, i0, jj0, k);
  const bool pair = f.lo[c] != nullptr;
  T* Rt = reinterpret_cast<T*>(smem_raw);
  T* Ut = Rt + (size_t)n * SYT_W;
  T* Lt = Ut + (size_t)n * SYT_W;
  T* ivS = pair ? Lt + (size_t)n * SYT_W : Lt;   // 1/pivot and c' of a line without forcing rows
  T* cqS = ivS + n;
  const unsigned bar = smem_addr(&bar_mem);
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const unsigned box = (unsigned)(SYT_W * n * sizeof(T));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(box * (pair ? 3u : 2u))
                 : "memory");
    tma_load_3d(Rt, &op.tm[c][0], i0, jj0, k, bar);
    tma_load_3d(Ut, &op.tm[c][1], i0, jj0, k, bar);
    if (pair) tma_load_3d(Lt, &op.tm[c][2], i0, jj0, k, bar);
  }
  // while the copies are in flight: the rows of a line without forcing rows
  // (one wall segment) to shared memory, so the recurrences read no global
  // memory
  const bool tang = c != 1;
  for (int r = lane; r < n; r += SYT_W) {
    const bool last = r == n - 1;
    ivS[r] = tang ? __ldg((last ? tb.yinvLW : tb.yinvW) + r) : __ldg(tb.vinvR + r);
    cqS[r] = last ? (T)0 : __ldg((tang ? tb.ycpW : tb.vcpR) + r);
  }
  __syncwarp();
  if (!mbar_wait(bar, 0, SYT_WAIT_CYCLES)) {
    // the copies did not complete: report, give them one more bounded wait
    // (they write this block's shared memory) and leave the tile untouched
    if (lane == 0) atomicOr(&op.ds->err, ERR_WAIT);
    mbar_wait(bar, 0, SYT_WAIT_CYCLES);
    return;
  }
  if (lane >= nl) return;
  T* Ug = comp_ptr(f, c) + base;
  T* Lg = pair ? f.lo[c] + base : nullptr;
  const int i = i0 + lane;
  const T a = -tb.off[1];
  const bool any = op.lfirst[line_y(g, c, i, k)] < g.ny;
  if (!any) {
    // one wall segment: p_j = (r_j - a p_{j-1}) iv_j, x_j = p_j - c'_j x_{j+1}
    T p = (T)0;
#pragma unroll 8
    for (int r = 0; r < n; ++r) {
      p = fma(r == 0 ? (T)0 : -a, p, Rt[r * SYT_W + lane]) * ivS[r];
      Rt[r * SYT_W + lane] = p;
    }
    T x = (T)0;
#pragma unroll 8
    for (int r = n - 1; r >= 0; --r) {
      x = fma(-cqS[r], x, Rt[r * SYT_W + lane]);
      if (pair) {
        float hi = (float)Ut[r * SYT_W + lane], lo = (float)Lt[r * SYT_W + lane];
        ff_add(hi, lo, (float)x);
        Ug[(long long)r * sn + lane] = (T)hi;
        Lg[(long long)r * sn + lane] = (T)lo;
      } else {
        Ug[(long long)r * sn + lane] = Ut[r * SYT_W + lane] + x;
      }
    }
    return;
  }
  T* __restrict__ Sl = f.scr + comp_off(g, c) + base + lane;
  const unsigned char* __restrict__ Fl = reinterpret_cast<const unsigned char*>(op.flags32) + cidx(g, i, jj0, k);
  // ---- forward (the streamed sweep's recurrence, segment restarts at forcing rows)
  T prev = (T)0;
  int m = 0;
  bool segW = tang;
  for (int r = 0; r < n; ++r) {
    const bool frc = any && ((Fl[(long long)r * sn] >> c) & 1);
    const bool last = r == n - 1;
    const T* ivt = !tang ? tb.vinvR : (last ? (segW ? tb.yinvLW : tb.yinvLR) : (segW ? tb.yinvW : tb.yinvR));
    const T* cpt = !tang ? tb.vcpR : (segW ? tb.ycpW : tb.ycpR);
    T iv = (T)1, cq = (T)0, am = (T)0;
    if (!frc) {
      iv = __ldg(ivt + m);
      if (!last) cq = __ldg(cpt + m);
      am = a;
    }
    m = frc ? 0 : m + 1;
    segW = segW && !frc;
    prev = fma(-am, prev, Rt[r * SYT_W + lane]) * iv;
    Rt[r * SYT_W + lane] = prev;
    if (any) Sl[(long long)r * sn] = cq;
  }
  // ---- backward: x_j = p_j - c'_j x_{j+1}; uhat = u^s + x
  const T* cpw = tang ? tb.ycpW : tb.vcpR;   // c' of a line without forcing rows (one wall segment)
  T x = (T)0;
  for (int r = n - 1; r >= 0; --r) {
    const T cv = any ? Sl[(long long)r * sn] : (r == n - 1 ? (T)0 : __ldg(cpw + r));
    x = fma(-cv, x, Rt[r * SYT_W + lane]);
    if (pair) {
      float hi = (float)Ut[r * SYT_W + lane], lo = (float)Lt[r * SYT_W + lane];
      ff_add(hi, lo, (float)x);
      Ug[(long long)r * sn + lane] = (T)hi;
      Lg[(long long)r * sn + lane] = (T)lo;
    } else {
      Ug[(long long)r * sn + lane] = Ut[r * SYT_W + lane] + x;
    }
  }
}
template <typename T>
struct SweepYTma {
  static constexpr int kThreads = SYT_W;
  CUtensorMap tm[3][3];   // [component][R, u^s, low parts]
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  SweepTables<T> tb;
  const int* lfirst;
  DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { sweep_y_tma<T>(bk, *this); }
};

// cuTensorMapEncodeTiled from the driver, looked up once (null if absent).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiled encode_tiled() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// The TMA y sweep's maps for this grid, or false where it cannot run: rows of
// 16-byte multiples on 16-byte boundaries, at least one full tile of lines,
// at most 256 rows (one box), and a tile that fits shared memory.
template <typename T>
static bool sweep_y_tma_maps(const Geo& g, const Fields<T>& f, int ny_shape, SweepYTma<T>& op) {
  const EncodeTiled enc = encode_tiled();
  if (!enc || (g.nx * sizeof(T)) % 16 != 0 || g.nx < SYT_W || g.ny > 256) return false;
  if (((size_t)(f.lo[0] ? 3 : 2) * SYT_W + 2) * ny_shape * sizeof(T) > 200u * 1024u) return false;
  for (int c = 0; c < 3; ++c) {
    T* arr[3] = {f.R[c], c == 0 ? f.u : (c == 1 ? f.v : f.w), f.lo[c]};
    const cuuint64_t pl = (cuuint64_t)planes(g, c);
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, pl, (cuuint64_t)g.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)g.nx * sizeof(T), (cuuint64_t)g.nx * pl * sizeof(T)};
    const cuuint32_t box[3] = {(cuuint32_t)SYT_W, (cuuint32_t)(c == 1 ? g.ny - 1 : g.ny), 1u};
    const cuuint32_t es[3] = {1u, 1u, 1u};
    for (int q = 0; q < 3; ++q) {
      if (!arr[q]) {
        memset(&op.tm[c][q], 0, sizeof(CUtensorMap));
        continue;
      }
      if (reinterpret_cast<uintptr_t>(arr[q]) & 15u) return false;
      if (enc(&op.tm[c][q], sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
              arr[q], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  }
  return true;
}

template <typename T>
static size_t sweep_smem(int W, int n, int ld, int tiles = 1) {
  return (size_t)tiles * W * ld * sizeof(T) + (size_t)W * n;
}

// lines per block: the largest of 64, 32, 16 whose tile fits 160 KB
template <typename T>
static int sweep_width(int n, int tiles = 1) {
  for (int W = 64; W > 16; W /= 2)
    if (sweep_smem<T>(W, n, n + 1, tiles) <= 160 * 1024) return W;
  return 16;
}

template <typename T, int K>
static void sweep_x_warp(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb,
                         Exec& ex) {
  const int lines = g.ny * g.nz;   // upper bound over components
  ex.launch(dim3((lines + 7) / 8, 3), dim3(256), 0, SweepXWarp<T, K>{g, f, b.flags32, tb, b.lines.x});
}

// Lanes-per-line sweep for lines of up to n_max rows (the shape's extent):
// 4 lanes x K rows (K = 4..16), 8 lanes x 16 or 32 rows (16 rows per lane
// keep the kernel near 80 registers); false if too long.
template <typename T, int K, int L>
static void lanes_launch(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb, Exec& ex,
                         int dir, int planes_z) {
  constexpr int per_block = 8 * (32 / L);
  ex.launch(dim3((g.nx + per_block - 1) / per_block, 3, planes_z), dim3(256), 0,
            SweepLanes<T, K, L>{g, f, b.flags32, tb, dir == 2 ? b.lines.z : b.lines.y, dir});
}
template <typename T>
static bool sweep_lanes_launch(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb,
                               Exec& ex, int n_max, int dir, int planes_z) {
  if (n_max <= 16) lanes_launch<T, 4, 4>(g, f, b, tb, ex, dir, planes_z);
  else if (n_max <= 32) lanes_launch<T, 8, 4>(g, f, b, tb, ex, dir, planes_z);
  else if (n_max <= 64) lanes_launch<T, 16, 4>(g, f, b, tb, ex, dir, planes_z);
  else if (n_max <= 128) lanes_launch<T, 16, 8>(g, f, b, tb, ex, dir, planes_z);
  else if (n_max <= 256) lanes_launch<T, 32, 8>(g, f, b, tb, ex, dir, planes_z);
  else return false;
  return true;
}

// The TMA y sweep of one simulation (never a batch: its tensor maps travel
// in the kernel's parameters), if its maps can be made; false otherwise.
template <typename T>
static bool sweep_y_tma_ok(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb,
                           DevState* ds, int ny_shape, Exec& ex) {
  SweepYTma<T> op;
  if (!sweep_y_tma_maps<T>(g, f, ny_shape, op)) return false;
  op.g = g;
  op.f = f;
  op.flags32 = b.flags32;
  op.tb = tb;
  op.lfirst = b.lines.y;
  op.ds = ds;
  const size_t smem = ((size_t)(f.lo[0] ? 3 : 2) * SYT_W + 2) * ny_shape * sizeof(T);
  ex.launch(dim3((unsigned)((g.nx + SYT_W - 1) / SYT_W), (unsigned)g.nz, 3), dim3(SYT_W), smem, op);
  return true;
}

// Launch shapes (lines per block, registers per lane) follow ex.shape, so
// every instance of a batch uses the same ones; grids follow the instance.
template <typename T>
void launch_sweeps(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb, DevState* ds,
                   Exec& ex) {
  const Geo& sh = ex.shape;
  ex.mark(ST_SWEEP_X);
  if (sizeof(T) == 4 && sh.nx <= 1024) {
    const int K = (sh.nx + 31) / 32;
    if (K <= 1) sweep_x_warp<T, 1>(g, f, b, tb, ex);
    else if (K <= 2) sweep_x_warp<T, 2>(g, f, b, tb, ex);
    else if (K <= 3) sweep_x_warp<T, 3>(g, f, b, tb, ex);
    else if (K <= 4) sweep_x_warp<T, 4>(g, f, b, tb, ex);
    else if (K <= 8) sweep_x_warp<T, 8>(g, f, b, tb, ex);
    else if (K <= 16) sweep_x_warp<T, 16>(g, f, b, tb, ex);
    else sweep_x_warp<T, 32>(g, f, b, tb, ex);
  } else {
    const int W = sweep_width<T>(sh.nx);
    const int nlines = g.ny * g.nz;     // upper bound over components (v has ny-1 rows of lines)
    ex.launch(dim3((nlines + W - 1) / W, 3), dim3(W), sweep_smem<T>(W, sh.nx, sh.nx + 1),
              SweepX<T>{g, f, b.flags32, tb, b.lines.x});
  }
  // z and y: several lanes per line (FP32, lines up to 256 rows) unless the
  // tuning asks for the shared-memory tile with one thread per line
  const bool lanes = sizeof(T) == 4 && ex.tune.sweep_zy != 1;
  ex.mark(ST_SWEEP_Z);
  if (ex.tune.sweep_y == 4 && sh.nz <= 256) {
    ex.launch(dim3((unsigned)((g.nx + ZT_W - 1) / ZT_W), (unsigned)g.ny, 3), dim3(ZT_THREADS),
              sweep_z_tile_smem<T>(sh.nz), SweepZTile<T>{g, f, b.flags32, tb, b.lines.z});
  } else if (ex.tune.sweep_y >= 1) {
    const long long lines = (long long)g.nx * g.ny;
    ex.launch(dim3((unsigned)((lines + 127) / 128), 3), dim3(128), 0, SweepZStream<T>{g, f, b.flags32, tb, b.lines.z});
  } else if (!(lanes && sweep_lanes_launch(g, f, b, tb, ex, sh.nz, 2, g.ny))) {
    int W = sweep_width<T>(sh.nz);
    if (ex.tune.sweep_w > 0 && ex.tune.sweep_w < W) W = ex.tune.sweep_w;
    ex.launch(dim3((g.nx + W - 1) / W, 3, g.ny), dim3(W), sweep_smem<T>(W, sh.nz, sh.nz),
              SweepZY<T>{g, f, b.flags32, tb, b.lines.z, 2});
  }
  ex.mark(ST_SWEEP_Y);
  if (g.yt.ihc) {
    // non-uniform wall-normal spacing (beta from the x coefficient, beta / dx^2)
    const long long lines = (long long)g.nx * g.nz;
    ex.launch(dim3((unsigned)((lines + 127) / 128), 3), dim3(128), 0,
              SweepYStretched<T>{g, f, b.flags32, b.lines.y, (double)tb.off[0] * g.dx * g.dx});
  } else if (ex.tune.sweep_y == 2 && !ex.rec && sweep_y_tma_ok<T>(g, f, b, tb, ds, sh.ny, ex)) {
    // (launched inside the check: the op carries its tensor maps)
  } else if (ex.tune.sweep_y >= 3 && sizeof(T) == 4 && sh.ny <= 1024 && g.yt.yswf && g.yt.ysw2f) {
    // the tabulated FP32 rows (uniform spacing written as the non-uniform
    // grid's tables; built for every mixed grid of at most 1024 rows)
    const long long lines = (long long)g.nx * g.nz;
    ex.launch(dim3((unsigned)((lines + 127) / 128), 3), dim3(128), 0,
              SweepYStretched<T>{g, f, b.flags32, b.lines.y, (double)tb.off[0] * g.dx * g.dx});
  } else if (ex.tune.sweep_y >= 1) {
    const long long lines = (long long)g.nx * g.nz;
    ex.launch(dim3((unsigned)((lines + 127) / 128), 3), dim3(128), 0, SweepYStream<T>{g, f, b.flags32, tb, b.lines.y});
  } else if (!(lanes && sweep_lanes_launch(g, f, b, tb, ex, sh.ny, 1, g.nz))) {
    const int tiles = f.lo[0] ? 3 : 2;
    int W = sweep_width<T>(sh.ny, tiles);
    if (ex.tune.sweep_w > 0 && ex.tune.sweep_w < W) W = ex.tune.sweep_w;
    ex.launch(dim3((g.nx + W - 1) / W, 3, g.nz), dim3(W), sweep_smem<T>(W, sh.ny, sh.ny, tiles),
              SweepZY<T>{g, f, b.flags32, tb, b.lines.y, 1});
  }
}

template <typename T>
static void sweep_attrs() {
  op_smem_limit<SweepX<T>>(200 * 1024);
  op_smem_limit<SweepZY<T>>(200 * 1024);
  op_smem_limit<SweepYTma<T>>(200 * 1024);
  op_smem_limit<SweepZTile<T>>((int)sweep_z_tile_smem<T>(256));
}

void init_sweep_attributes() {
  sweep_attrs<double>();
  sweep_attrs<float>();
}

// ---------------------------------------------------------------------------
// No-slip error on the forcing points (Section 4.4): the flow is
// interpolated on the wall with the interpolator of Eq. new_IB,
// u_w = (u(x^f) - alpha u(x^e)) / (1 - alpha), eps = u_w - U.
// Fixed-order two-level reduction of sum |eps| per component.
// ---------------------------------------------------------------------------
constexpr int SLIP_BLOCKS = 256, SLIP_THREADS = 256;   // SLIP_BLOCKS: the most partial sums

template <typename T>
__device__ __forceinline__ void slip_partial(const Blk& bk, const Geo& g, const Surf& s, const Fields<T>& f,
                                                               const ForceNode* __restrict__ flist, unsigned cap,
                                                               DevState* ds, double* partial, double* __restrict__ probe) {
  __shared__ double red[3][SLIP_THREADS];
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  const unsigned per = (n + bk.gx - 1) / bk.gx;
  const unsigned e0 = bk.x * per, e1 = min(n, e0 + per);
  double acc[3] = {0.0, 0.0, 0.0};
  for (unsigned e = e0 + threadIdx.x; e < e1; e += SLIP_THREADS) {
    const ForceNode fn = flist[e];
    const int c = (int)(fn.key >> 30);
    double xe[3], alpha, U;
    forcing_probe(g, s, fn, probe + 5ull * e, false, xe, alpha, U);
    const T* fc = comp_ptr(f, c);
    const double ux = (double)fc[fn.key & KEY_MASK] + (f.lo[c] ? (double)f.lo[c][fn.key & KEY_MASK] : 0.0);
    double uw = ux;
    if (alpha != 0.0) {
      double ue;
      if (!trilinear<T>(g, c, fc, xe, &ue)) {
        atomicOr(&ds->err, ERR_PROBE);
        ue = 0.0;
      }
      uw = (ux - alpha * ue) / (1.0 - alpha);
    }
    acc[c] += fabs(uw - U);
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = SLIP_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) partial[bk.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}
template <typename T>
struct SlipPartial {
  static constexpr int kThreads = SLIP_THREADS;
  Geo g;
  Surf s;
  Fields<T> f;
  const ForceNode* flist;
  unsigned cap;
  DevState* ds;
  double* partial;
  double* probe;
  __device__ __forceinline__ void operator()(const Blk& bk) const { slip_partial<T>(bk, g, s, f, flist, cap, ds, partial, probe); }
};

__device__ __forceinline__ void slip_final(const Blk& bk, const double* partial, DevState* ds, int nblk) {
  for (int c = 0; c < 3; ++c) {
    const double s = warp_sum_fixed(partial, nblk, 3, c);
    if (threadIdx.x == 0) {
      ds->slip_sum[c] = s;
      if (!isfinite(s)) atomicOr(&ds->err, ERR_NONFINITE);
    }
  }
}
struct SlipFinal {
  static constexpr int kThreads = 32;
  const double* partial;
  DevState* ds;
  int nblk;
  __device__ __forceinline__ void operator()(const Blk& bk) const { slip_final(bk, partial, ds, nblk); }
};

template <typename T>
void launch_slip(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double* partial,
                 DevState* ds, Exec& ex) {
  ex.mark(ST_SLIP);
  const int nblk = reduce_blocks(g, 8192, SLIP_BLOCKS);
  ex.launch(grid_if(s.nt > 0, dim3(nblk)), dim3(SLIP_THREADS), 0, SlipPartial<T>{g, s, f, b.flist, b.cap, ds, partial, b.probe});
  ex.launch(grid_if(s.nt > 0, dim3(1)), dim3(32), 0, SlipFinal{partial, ds, nblk});
}

#define IBM_INST(T)                                                                                             \
  template void launch_ib_force<T>(const Geo&, const Surf&, const Fields<T>&, const TagBuffers&, DevState*,     \
                                   bool, Exec&);                                                                      \
  template void launch_rhs<T>(const Geo&, const Fields<T>&, const TagBuffers&, const Stage&, double, double,    \
                              bool, bool, DevState*, Exec&);                                                    \
  template void launch_sweeps<T>(const Geo&, const Fields<T>&, const TagBuffers&, const SweepTables<T>&,        \
                                 DevState*, Exec&);                                                             \
  template void launch_slip<T>(const Geo&, const Surf&, const Fields<T>&, const TagBuffers&, double*,           \
                               DevState*, Exec&);
IBM_INST(double)
IBM_INST(float)
#undef IBM_INST

}  // namespace ibm
