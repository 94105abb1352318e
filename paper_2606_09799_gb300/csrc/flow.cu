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
#include "launch.h"

namespace ibm {

template <typename T>
__device__ __forceinline__ T* comp_ptr(const Fields<T>& f, int c) {
  return c == 0 ? f.u : (c == 1 ? f.v : f.w);
}

// Trilinear interpolation of component c at P from the 8 surrounding nodes
// of the same staggered lattice.  x and z wrap; in y the stencil must lie
// in the stored planes (u, w: 0..ny-1; v: 0..ny with the wall planes).
template <typename T>
__device__ bool trilinear(const Geo& g, int c, const T* __restrict__ f, const double P[3], double* out) {
  const double sx = P[0] * g.idx - (c == 0 ? 0.0 : 0.5);
  const double sy = P[1] * g.idy - (c == 1 ? 0.0 : 0.5);
  const double sz = P[2] * g.idz - (c == 2 ? 0.0 : 0.5);
  const double fx = floor(sx), fy = floor(sy), fz = floor(sz);
  const long long i0 = (long long)fx, j0 = (long long)fy, k0 = (long long)fz;
  if (j0 < 0 || j0 + 1 > planes(g, c) - 1) return false;
  const double tx = sx - fx, ty = sy - fy, tz = sz - fz;
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
};

__device__ inline void forcing_geometry(const Geo& g, const Surf& s, unsigned key, unsigned tri, NodeGeom& ng) {
  const int c = (int)(key >> 30);
  const long long node = key & KEY_MASK;
  const int pl = planes(g, c);
  const long long i = node % g.nx, j = (node / g.nx) % pl, k = node / ((long long)g.nx * pl);
  const int va = __ldg(s.t + tri), vb = __ldg(s.t + s.nt + tri), vc = __ldg(s.t + 2 * (long long)s.nt + tri);
  double A[3], B[3], C[3];
  load_vertex(s, va, A);
  load_vertex(s, vb, B);
  load_vertex(s, vc, C);
  double cen[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) cen[d] = (A[d] + B[d] + C[d]) / 3.0;
  node_pos(g, c, i, j, k, ng.x);
  const long long mi = llround((cen[0] - ng.x[0]) / g.lx);
  const long long mk = llround((cen[2] - ng.x[2]) / g.lz);
  if (mi != 0 || mk != 0) node_pos(g, c, i + mi * g.nx, j, k + mk * g.nz, ng.x);
  double wb[3];
  closest_point_exact(ng.x, A, B, C, ng.X, wb);
#pragma unroll
  for (int d = 0; d < 3; ++d) ng.N[d] = dsub(ng.x[d], ng.X[d]);
  ng.n2 = ddot(ng.N, ng.N);
  const long long nv = s.nv;
  ng.U = wb[0] * __ldg(s.u + c * nv + va) + wb[1] * __ldg(s.u + c * nv + vb) + wb[2] * __ldg(s.u + c * nv + vc);
}

// Eq. new_IB for every forcing node, reading u^e from the unmodified state
// (a snapshot: the values are written by a second kernel).
template <typename T>
__global__ void k_ib_force(Geo g, Surf s, Fields<T> f, const ForceNode* __restrict__ flist, unsigned cap,
                           DevState* ds) {
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const ForceNode fn = flist[e];
    const int c = (int)(fn.key >> 30);
    NodeGeom ng;
    forcing_geometry(g, s, fn.key, fn.tri, ng);
    double uf = ng.U;
    if (ng.n2 != 0.0) {
      const double nl = sqrt(ng.n2);
      double xe[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) xe[d] = ng.X[d] + g.h * (ng.N[d] / nl);
      double ue;
      if (!trilinear<T>(g, c, comp_ptr(f, c), xe, &ue)) {
        atomicOr(&ds->err, ERR_PROBE);
        ue = 0.0;
      }
      const double alpha = nl / g.h;
      uf = (1.0 - alpha) * ng.U + alpha * ue;
    }
    f.uf[e] = (T)uf;
  }
}

template <typename T>
__global__ void k_ib_scatter(Fields<T> f, const ForceNode* __restrict__ flist, unsigned cap, const DevState* ds) {
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const ForceNode fn = flist[e];
    comp_ptr(f, (int)(fn.key >> 30))[fn.key & KEY_MASK] = f.uf[e];
  }
}

template <typename T>
void launch_ib_force(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds,
                     cudaStream_t st) {
  const int gb = num_sms() * 4;
  stage_mark(st, ST_FORCE);
  k_ib_force<T><<<gb, 128, 0, st>>>(g, s, f, b.flist, b.cap, ds);
  k_ib_scatter<T><<<gb, 256, 0, st>>>(f, b.flist, b.cap, ds);
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
template <typename T>
__global__ void __launch_bounds__(256) k_rhs(Geo g, Fields<T> f, const unsigned* __restrict__ flags32, Stage sg,
                                             double dt, double re, int use_hp, int write_h, const DevState* ds) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long total = g.ncell;
  const T idx = (T)g.idx, idy = (T)g.idy, idz = (T)g.idz;
  const T idx2 = idx * idx, idy2 = idy * idy, idz2 = idz * idz;
  const T gs = g.ybc == 0 ? (T)-1 : (T)1;
  const T q = (T)0.25;
  const T cg = (T)sg.gam, cr = (T)sg.rho, ca = (T)sg.alp, cv = (T)(sg.alp / re), tdt = (T)dt;
  const T fbx = (T)(sg.alp * ds->fb[0]), fby = (T)(sg.alp * ds->fb[1]), fbz = (T)(sg.alp * ds->fb[2]);
  const long long pv = (long long)(ny + 1) * nx;   // v plane stride (k)
  const long long pu = (long long)ny * nx;         // u, w, p plane stride
  const T* __restrict__ U = f.u;
  const T* __restrict__ V = f.v;
  const T* __restrict__ W = f.w;
  const T* __restrict__ P = f.p;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < total;
       cell += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(cell % nx);
    const int j = (int)((cell / nx) % ny);
    const int k = (int)(cell / pu);
    const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
    const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
    const long long r0 = (long long)k * pu + (long long)j * nx;      // row (j,k) of u, w, p
    const long long rkp = (long long)kp * pu + (long long)j * nx, rkm = (long long)km * pu + (long long)j * nx;
    const long long v0 = (long long)k * pv + (long long)j * nx;      // row (j,k) of v
    const long long v1 = v0 + nx;                                    // row (j+1,k) of v
    const long long vkm0 = (long long)km * pv + (long long)j * nx, vkp0 = (long long)kp * pv + (long long)j * nx;
    const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
    const bool jlo = j == 0, jhi = j + 1 == ny;
    const T pc = P[r0 + i];
    // ---------------- u at (i dx, (j+1/2) dy, (k+1/2) dz) ----------------
    {
      const T uc = U[r0 + i], ue = U[r0 + ip], uw = U[r0 + im];
      const T un = jhi ? gs * uc : U[r0 + nx + i];
      const T us = jlo ? gs * uc : U[r0 - nx + i];
      const T uf = U[rkp + i], ub = U[rkm + i];
      const T adx = ((uc + ue) * (uc + ue) - (uw + uc) * (uw + uc)) * q * idx;
      const T vt = jhi ? (T)0 : (V[v1 + im] + V[v1 + i]) * (uc + un);
      const T vb = jlo ? (T)0 : (V[v0 + im] + V[v0 + i]) * (us + uc);
      const T ady = (vt - vb) * q * idy;
      const T wf = (W[rkp + im] + W[rkp + i]) * (uc + uf);
      const T wb = (W[r0 + im] + W[r0 + i]) * (ub + uc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lap = (ue - (T)2 * uc + uw) * idx2 + (un - (T)2 * uc + us) * idy2 + (uf - (T)2 * uc + ub) * idz2;
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
      const T ady = (vt - vb) * q * idy;
      const T adz = ((wc + wf) * (wc + wf) - (wb + wc) * (wb + wc)) * q * idz;
      const T H = -(adx + ady + adz);
      const T lap = (we - (T)2 * wc + ww) * idx2 + (wn - (T)2 * wc + ws) * idy2 + (wf - (T)2 * wc + wb) * idz2;
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
      const T ady = ((vc + vn) * (vc + vn) - (vs + vc) * (vs + vc)) * q * idy;
      const T wf = (W[rkp - nx + i] + W[rkp + i]) * (vc + vf);
      const T wb = (W[r0 - nx + i] + W[r0 + i]) * (vbk + vc);
      const T adz = (wf - wb) * q * idz;
      const T H = -(adx + ady + adz);
      const T lap = (ve - (T)2 * vc + vw) * idx2 + (vn - (T)2 * vc + vs) * idy2 + (vf - (T)2 * vc + vbk) * idz2;
      const T G = (pc - P[r0 - nx + i]) * idy;
      T r = cg * H - ca * G + cv * lap + fby;
      if (use_hp) r += cr * f.Hp[1][v0 + i];
      if (write_h) f.H[1][v0 + i] = H;
      f.R[1][v0 + i] = (fl & FLAG_V) ? (T)0 : tdt * r;
    } else {
      // wall planes of v carry no unknown
      f.R[1][v0 + i] = (T)0;
      f.R[1][(long long)k * pv + (long long)ny * nx + i] = (T)0;
      if (write_h) {
        f.H[1][v0 + i] = (T)0;
        f.H[1][(long long)k * pv + (long long)ny * nx + i] = (T)0;
      }
    }
  }
}

template <typename T>
void launch_rhs(const Geo& g, const Fields<T>& f, const TagBuffers& b, const Stage& sg, double dt, double re,
                bool use_hp, bool write_h, DevState* ds, cudaStream_t st) {
  const long long blocks = (g.ncell + 255) / 256;
  stage_mark(st, ST_RHS);
  k_rhs<T><<<(unsigned)blocks, 256, 0, st>>>(g, f, b.flags32, sg, dt, re, use_hp ? 1 : 0, write_h ? 1 : 0, ds);
}

// ---------------------------------------------------------------------------
// Approximate factorisation: (1 - beta L_x)(1 - beta L_z)(1 - beta L_y) du = R
// Each factor is a tridiagonal system per grid line; forcing nodes are
// identity rows (the provisional equation is not solved there).  A line
// without forcing nodes has constant coefficients and uses tabulated
// recurrences (no division, no scratch); a line with forcing nodes is
// solved by Thomas with its c' kept in the scratch array.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool is_forcing(const unsigned* flags32, long long cell, int c) {
  return (flags32[cell >> 2] >> (8 * (cell & 3) + c)) & 1u;
}

// periodic direction dir (0 = x, 2 = z) for component blockIdx.y
template <typename T>
__global__ void __launch_bounds__(128) k_sweep_periodic(Geo g, Fields<T> f, const unsigned* __restrict__ flags32,
                                                        SweepTables<T> tb, int dir) {
  const int c = blockIdx.y;
  const int j0 = c == 1 ? 1 : 0, nj = c == 1 ? g.ny - 1 : g.ny;
  const int pl = planes(g, c);
  long long nlines, n, stride, fstride;
  if (dir == 0) { nlines = (long long)nj * g.nz; n = g.nx; stride = 1; fstride = 1; }
  else { nlines = (long long)nj * g.nx; n = g.nz; stride = (long long)pl * g.nx; fstride = (long long)g.ny * g.nx; }
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= nlines) return;
  long long base, fbase;
  if (dir == 0) {
    const long long j = j0 + l % nj, k = l / nj;
    base = fidx(g, c, 0, j, k);
    fbase = cidx(g, 0, j, k);
  } else {
    const long long i = l % g.nx, j = j0 + l / g.nx;
    base = fidx(g, c, i, j, 0);
    fbase = cidx(g, i, j, 0);
  }
  T* __restrict__ R = f.R[c];
  T* __restrict__ S = f.scr + comp_off(g, c);
  const int d = dir == 0 ? 0 : 1;
  const T off = dir == 0 ? tb.off[0] : tb.off[2];
  const T a = -off;
  long long f0 = -1;
  for (long long m = 0; m < n; ++m)
    if (is_forcing(flags32, fbase + m * fstride, c)) { f0 = m; break; }
  if (f0 < 0) {
    // Sherman-Morrison with tabulated recurrences of the modified matrix
    const T* __restrict__ inv = tb.inv[d];
    const T* __restrict__ cp = tb.cp[d];
    const T* __restrict__ zv = tb.zv[d];
    const T* __restrict__ g0 = tb.g0[d];
    T prev = R[base] * inv[0];
    T acc = g0[0] * R[base];
    R[base] = prev;
    for (long long m = 1; m < n; ++m) {
      const T dm = R[base + m * stride];
      acc += g0[m] * dm;
      prev = (dm - a * prev) * inv[m];
      R[base + m * stride] = prev;
    }
    const T fact = (acc + (a / tb.gam[d]) * prev) / tb.smden[d];
    T y = prev;
    R[base + (n - 1) * stride] = y - fact * zv[n - 1];
    for (long long m = n - 2; m >= 0; --m) {
      y = R[base + m * stride] - cp[m] * y;
      R[base + m * stride] = y - fact * zv[m];
    }
    return;
  }
  // rotate the line to start at its first forcing row: the periodic system
  // becomes an ordinary one whose row 0 is the identity
  const T bf = (T)1 + (T)2 * off;
  const long long id0 = base + f0 * stride;
  const T x0 = R[id0];
  S[id0] = (T)0;
  T cprev = (T)0, dprev = x0;
  for (long long m = 1; m < n; ++m) {
    const long long r = (f0 + m) % n;
    const long long id = base + r * stride;
    T dm = R[id];
    T am, bm, cm;
    if (is_forcing(flags32, fbase + r * fstride, c)) { am = (T)0; bm = (T)1; cm = (T)0; }
    else { am = a; bm = bf; cm = a; }
    if (m == n - 1) { dm -= cm * x0; cm = (T)0; }
    const T den = bm - am * cprev;
    cprev = cm / den;
    dprev = (dm - am * dprev) / den;
    S[id] = cprev;
    R[id] = dprev;
  }
  T x = dprev;
  for (long long m = n - 2; m >= 1; --m) {
    const long long id = base + ((f0 + m) % n) * stride;
    x = R[id] - S[id] * x;
    R[id] = x;
  }
}

// wall-normal direction; the result du is added to the state: uhat = u^s + du
template <typename T>
__global__ void __launch_bounds__(128) k_sweep_y(Geo g, Fields<T> f, const unsigned* __restrict__ flags32,
                                                 SweepTables<T> tb) {
  const int c = blockIdx.y;
  const int j0 = c == 1 ? 1 : 0, n = c == 1 ? g.ny - 1 : g.ny;
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)g.nx * g.nz) return;
  const long long i = l % g.nx, k = l / g.nx;
  const long long base = fidx(g, c, i, j0, k), stride = g.nx;
  const long long fbase = cidx(g, i, j0, k);
  T* __restrict__ R = f.R[c];
  T* __restrict__ S = f.scr + comp_off(g, c);
  T* __restrict__ Uc = comp_ptr(f, c);
  const T off = tb.off[1];
  const T a = -off;
  bool any = false;
  for (int m = 0; m < n && !any; ++m) any = is_forcing(flags32, fbase + (long long)m * stride, c);
  if (!any) {
    const int cls = c == 1 ? 1 : 0;
    const T* __restrict__ inv = tb.yinv[cls];
    const T* __restrict__ cp = tb.ycp[cls];
    T prev = R[base] * inv[0];
    R[base] = prev;
    for (int m = 1; m < n; ++m) {
      const long long id = base + (long long)m * stride;
      prev = (R[id] - a * prev) * inv[m];
      R[id] = prev;
    }
    T x = prev;
    Uc[base + (long long)(n - 1) * stride] += x;
    for (int m = n - 2; m >= 0; --m) {
      const long long id = base + (long long)m * stride;
      x = R[id] - cp[m] * x;
      Uc[id] += x;
    }
    return;
  }
  const T gs = g.ybc == 0 ? (T)-1 : (T)1;
  const T bf = (T)1 + (T)2 * off;
  T cprev = (T)0, dprev = (T)0;
  for (int m = 0; m < n; ++m) {
    const long long id = base + (long long)m * stride;
    T am, bm, cm;
    if (is_forcing(flags32, fbase + (long long)m * stride, c)) { am = (T)0; bm = (T)1; cm = (T)0; }
    else {
      am = m == 0 ? (T)0 : a;
      cm = m == n - 1 ? (T)0 : a;
      bm = bf;
      if (c != 1 && (m == 0 || m == n - 1)) bm -= gs * off;
    }
    const T den = bm - am * cprev;
    cprev = cm / den;
    dprev = (R[id] - am * dprev) / den;
    S[id] = cprev;
    R[id] = dprev;
  }
  T x = dprev;
  Uc[base + (long long)(n - 1) * stride] += x;
  for (int m = n - 2; m >= 0; --m) {
    const long long id = base + (long long)m * stride;
    x = R[id] - S[id] * x;
    Uc[id] += x;
  }
}

template <typename T>
void launch_sweeps(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb,
                   cudaStream_t st) {
  const long long lx = (long long)g.ny * g.nz, lz = (long long)g.ny * g.nx, ly = (long long)g.nx * g.nz;
  stage_mark(st, ST_SWEEP_X);
  k_sweep_periodic<T><<<dim3((unsigned)((lx + 127) / 128), 3), 128, 0, st>>>(g, f, b.flags32, tb, 0);
  stage_mark(st, ST_SWEEP_Z);
  k_sweep_periodic<T><<<dim3((unsigned)((lz + 127) / 128), 3), 128, 0, st>>>(g, f, b.flags32, tb, 2);
  stage_mark(st, ST_SWEEP_Y);
  k_sweep_y<T><<<dim3((unsigned)((ly + 127) / 128), 3), 128, 0, st>>>(g, f, b.flags32, tb);
}

// ---------------------------------------------------------------------------
// No-slip error on the forcing points (Section 4.4): the flow is
// interpolated on the wall with the interpolator of Eq. new_IB,
// u_w = (u(x^f) - alpha u(x^e)) / (1 - alpha), eps = u_w - U.
// Fixed-order two-level reduction of sum |eps| per component.
// ---------------------------------------------------------------------------
constexpr int SLIP_BLOCKS = 256, SLIP_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(SLIP_THREADS) k_slip_partial(Geo g, Surf s, Fields<T> f,
                                                               const ForceNode* __restrict__ flist, unsigned cap,
                                                               DevState* ds, double* partial) {
  __shared__ double red[3][SLIP_THREADS];
  const unsigned n = min(ds->nforce_c[0] + ds->nforce_c[1] + ds->nforce_c[2], cap);
  const unsigned per = (n + SLIP_BLOCKS - 1) / SLIP_BLOCKS;
  const unsigned e0 = blockIdx.x * per, e1 = min(n, e0 + per);
  double acc[3] = {0.0, 0.0, 0.0};
  for (unsigned e = e0 + threadIdx.x; e < e1; e += SLIP_THREADS) {
    const ForceNode fn = flist[e];
    const int c = (int)(fn.key >> 30);
    NodeGeom ng;
    forcing_geometry(g, s, fn.key, fn.tri, ng);
    const T* fc = comp_ptr(f, c);
    const double ux = (double)fc[fn.key & KEY_MASK];
    double uw = ux;
    if (ng.n2 != 0.0) {
      const double nl = sqrt(ng.n2);
      double xe[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) xe[d] = ng.X[d] + g.h * (ng.N[d] / nl);
      double ue;
      if (!trilinear<T>(g, c, fc, xe, &ue)) {
        atomicOr(&ds->err, ERR_PROBE);
        ue = 0.0;
      }
      const double alpha = nl / g.h;
      uw = (ux - alpha * ue) / (1.0 - alpha);
    }
    acc[c] += fabs(uw - ng.U);
  }
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int w = SLIP_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) partial[blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_slip_final(const double* partial, DevState* ds) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int b = 0; b < SLIP_BLOCKS; ++b) s += partial[b * 3 + threadIdx.x];
    ds->slip_sum[threadIdx.x] = s;
    if (!isfinite(s)) atomicOr(&ds->err, ERR_NONFINITE);
  }
}

template <typename T>
void launch_slip(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double* partial,
                 DevState* ds, cudaStream_t st) {
  stage_mark(st, ST_SLIP);
  k_slip_partial<T><<<SLIP_BLOCKS, SLIP_THREADS, 0, st>>>(g, s, f, b.flist, b.cap, ds, partial);
  k_slip_final<<<1, 32, 0, st>>>(partial, ds);
}

#define IBM_INST(T)                                                                                             \
  template void launch_ib_force<T>(const Geo&, const Surf&, const Fields<T>&, const TagBuffers&, DevState*,     \
                                   cudaStream_t);                                                               \
  template void launch_rhs<T>(const Geo&, const Fields<T>&, const TagBuffers&, const Stage&, double, double,    \
                              bool, bool, DevState*, cudaStream_t);                                             \
  template void launch_sweeps<T>(const Geo&, const Fields<T>&, const TagBuffers&, const SweepTables<T>&,        \
                                 cudaStream_t);                                                                 \
  template void launch_slip<T>(const Geo&, const Surf&, const Fields<T>&, const TagBuffers&, double*,           \
                               DevState*, cudaStream_t);
IBM_INST(double)
IBM_INST(float)
#undef IBM_INST

}  // namespace ibm
