// poisson.cu -- consistent elliptic step of arXiv 2606.09799:
//   mass correction q (Section 3.2: q_B = D uhat on boundary cells, q_F
//   uniform on the fluid cells, Eq. constraint_q), right-hand side of
//   Eq. elliptic_mod, direct solve of L_c phi = rhs (FFT in the periodic x
//   and z, Thomas per wavenumber in y, homogeneous Neumann walls; Eq.
//   elliptic), projection (Eq. projection) and pressure update (Eq.
//   update_pressure).
//
// The FFTs are hand-written self-sorting (Stockham) transforms in shared
// memory with radix-4, -2 and -3 butterflies, so every size 2^a 3^b up to
// 1024 is supported.  Two real rows are packed into one complex transform.
// The wall-normal Thomas solve always runs in FP64 with pivots tabulated
// once per grid (they depend only on the wavenumber pair).
#include <math.h>

#include "common.cuh"
#include "launch.h"

namespace ibm {

template <typename T>
struct Cplx;
template <>
struct Cplx<double> { using type = double2; };
template <>
struct Cplx<float> { using type = float2; };

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// ---------------------------------------------------------------------------
// FFT plan: radices in order of application (product = n)
// ---------------------------------------------------------------------------
struct FftPlan {
  int n, nst;
  int rad[12];
};

static FftPlan make_plan(int n) {
  FftPlan p;
  p.n = n;
  p.nst = 0;
  int m = n;
  while (m % 4 == 0) { p.rad[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.rad[p.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p.rad[p.nst++] = 3; m /= 3; }
  return p;
}

// One Stockham pass over `lines` transforms of length n stored contiguously
// (line-major) in src, written to dst.  tw[m] = exp(-2 pi i m / n).
template <typename T, bool INV>
__device__ void fft_pass(const typename Cplx<T>::type* src, typename Cplx<T>::type* dst, int lines, int n, int R,
                         int Ns, const typename Cplx<T>::type* __restrict__ tw) {
  using C = typename Cplx<T>::type;
  const int nb = n / R;
  const int scale = n / (Ns * R);
  for (int t = threadIdx.x; t < lines * nb; t += blockDim.x) {
    const int line = t / nb, j = t - line * nb;
    const C* s = src + line * n;
    C* d = dst + line * n;
    const int k = j % Ns;
    C v[4];
    for (int r = 0; r < R; ++r) {
      C x = s[j + r * nb];
      if (r > 0 && k > 0) {
        C w = __ldg(reinterpret_cast<const C*>(tw) + (r * k * scale));
        if (INV) w = cconj(w);
        x = cmul(x, w);
      }
      v[r] = x;
    }
    if (R == 2) {
      const C a = v[0], b = v[1];
      v[0] = cadd(a, b);
      v[1] = csub(a, b);
    } else if (R == 4) {
      const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
      const C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
      C jd13;  // -i d13 (forward) or +i d13 (inverse)
      if (INV) { jd13.x = -d13.y; jd13.y = d13.x; }
      else { jd13.x = d13.y; jd13.y = -d13.x; }
      v[0] = cadd(s02, s13);
      v[2] = csub(s02, s13);
      v[1] = cadd(d02, jd13);
      v[3] = csub(d02, jd13);
    } else {  // R == 3
      const T h = (T)0.86602540378443864676;  // sin(2 pi / 3)
      const C a = v[0], b = v[1], c = v[2];
      const C sbc = cadd(b, c), dbc = csub(b, c);
      C m;
      m.x = a.x - (T)0.5 * sbc.x;
      m.y = a.y - (T)0.5 * sbc.y;
      C rot;  // -i h (b - c) forward, +i h (b - c) inverse
      if (INV) { rot.x = -h * dbc.y; rot.y = h * dbc.x; }
      else { rot.x = h * dbc.y; rot.y = -h * dbc.x; }
      v[0] = cadd(a, sbc);
      v[1] = cadd(m, rot);
      v[2] = csub(m, rot);
    }
    const int base = (j / Ns) * Ns * R + k;
    for (int r = 0; r < R; ++r) d[base + r * Ns] = v[r];
  }
}

// Full transform; returns the buffer that holds the result (0 = a, 1 = b).
template <typename T, bool INV>
__device__ int fft_lines(typename Cplx<T>::type* a, typename Cplx<T>::type* b, int lines, const FftPlan& p,
                         const typename Cplx<T>::type* __restrict__ tw) {
  int Ns = 1, cur = 0;
  for (int s = 0; s < p.nst; ++s) {
    __syncthreads();
    if (cur == 0) fft_pass<T, INV>(a, b, lines, p.n, p.rad[s], Ns, tw);
    else fft_pass<T, INV>(b, a, lines, p.n, p.rad[s], Ns, tw);
    cur ^= 1;
    Ns *= p.rad[s];
  }
  __syncthreads();
  return cur;
}

// ---------------------------------------------------------------------------
// q_F: fixed-order two-level reduction of sum_{C_B} D uhat dV over the
// sorted boundary-cell list; q_F = -A / |C_F| (uniform on fluid cells).
// ---------------------------------------------------------------------------
constexpr int QB_BLOCKS = 128, QB_THREADS = 256;

template <typename T>
__device__ __forceinline__ double div_at(const Geo& g, const T* __restrict__ u, const T* __restrict__ v,
                                         const T* __restrict__ w, long long i, long long j, long long k) {
  const long long ip = i + 1 == g.nx ? 0 : i + 1, kp = k + 1 == g.nz ? 0 : k + 1;
  const double du = ((double)u[fidx(g, 0, ip, j, k)] - (double)u[fidx(g, 0, i, j, k)]) * g.idx;
  const double dv = ((double)v[fidx(g, 1, i, j + 1, k)] - (double)v[fidx(g, 1, i, j, k)]) * g.idy;
  const double dw = ((double)w[fidx(g, 2, i, j, kp)] - (double)w[fidx(g, 2, i, j, k)]) * g.idz;
  return du + dv + dw;
}

template <typename T>
__global__ void __launch_bounds__(QB_THREADS) k_q_partial(Geo g, Fields<T> f, const unsigned* __restrict__ blist,
                                                          unsigned cap, const DevState* ds, double* partial) {
  __shared__ double red[QB_THREADS];
  const unsigned n = min(ds->nbound, cap);
  const unsigned per = (n + QB_BLOCKS - 1) / QB_BLOCKS;
  const unsigned e0 = blockIdx.x * per, e1 = min(n, e0 + per);
  double acc = 0.0;
  for (unsigned e = e0 + threadIdx.x; e < e1; e += QB_THREADS) {
    const long long cell = blist[e];
    const long long i = cell % g.nx, j = (cell / g.nx) % g.ny, k = cell / ((long long)g.nx * g.ny);
    acc += div_at<T>(g, f.u, f.v, f.w, i, j, k);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = QB_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_q_final(Geo g, const double* partial, DevState* ds, int s, int use_q) {
  if (threadIdx.x != 0) return;
  double sum = 0.0;
  for (int b = 0; b < QB_BLOCKS; ++b) sum += partial[b];
  const double dV = g.dx * g.dy * g.dz;
  const double A = sum * dV;
  const double VF = (double)(g.ncell - (long long)ds->nbound) * dV;
  ds->sum_a[s] = A;
  ds->qf[s] = (use_q && VF > 0.0) ? -A / VF : 0.0;
  if (!isfinite(A)) atomicOr(&ds->err, ERR_NONFINITE);
}

// ---------------------------------------------------------------------------
// forward x transform fused with the right-hand side of Eq. elliptic_mod:
// rhs = (D uhat - q) / (alpha dt) on C_F, 0 on C_B (q_B = D uhat), scaled by
// 1/(nx nz) so the inverse transforms need no normalisation.  Two real rows
// form one complex line; the two half-spectra are separated on output.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fft_x_fwd(Geo g, Fields<T> f, const unsigned* __restrict__ flags32, const T* __restrict__ tw,
                            FftPlan plan, int lines_per_block, const DevState* ds, int s, int use_q,
                            double scale) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + lines_per_block * g.nx;
  const int n = g.nx;
  const long long rows = (long long)g.ny * g.nz;
  const long long line0 = (long long)blockIdx.x * lines_per_block;
  const double qf = use_q ? ds->qf[s] : 0.0;
  // load: rows 2 l and 2 l + 1 of line l
  for (int t = threadIdx.x; t < lines_per_block * n; t += blockDim.x) {
    const int l = t / n, i = t - l * n;
    C z;
    z.x = (T)0;
    z.y = (T)0;
    for (int h = 0; h < 2; ++h) {
      const long long row = 2 * (line0 + l) + h;
      if (row >= rows) continue;
      const long long j = row % g.ny, k = row / g.ny;
      const long long cell = cidx(g, i, j, k);
      const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
      double r = 0.0;
      if (!(use_q && (fl & FLAG_B))) r = (div_at<T>(g, f.u, f.v, f.w, i, j, k) - qf) * scale;
      if (h == 0) z.x = (T)r;
      else z.y = (T)r;
    }
    bufa[t] = z;
  }
  const int res = fft_lines<T, false>(bufa, bufb, lines_per_block, plan, reinterpret_cast<const C*>(tw));
  const C* out = res == 0 ? bufa : bufb;
  C* spec = reinterpret_cast<C*>(f.spec);
  const int nkx = g.nkx;
  for (int t = threadIdx.x; t < lines_per_block * nkx; t += blockDim.x) {
    const int l = t / nkx, kx = t - l * nkx;
    const C Z = out[l * n + kx];
    const C Zc = cconj(out[l * n + (kx == 0 ? 0 : n - kx)]);
    C Xa, Xb;
    Xa.x = (T)0.5 * (Z.x + Zc.x);
    Xa.y = (T)0.5 * (Z.y + Zc.y);
    // Xb = (Z - Zc) / (2 i)
    Xb.x = (T)0.5 * (Z.y - Zc.y);
    Xb.y = (T)-0.5 * (Z.x - Zc.x);
    const long long ra = 2 * (line0 + l), rb = ra + 1;
    if (ra < rows) spec[ra * nkx + kx] = Xa;
    if (rb < rows) spec[rb * nkx + kx] = Xb;
  }
}

// inverse x transform: two half-spectra -> one complex line -> two real rows of phi
template <typename T>
__global__ void k_fft_x_inv(Geo g, Fields<T> f, const T* __restrict__ tw, FftPlan plan, int lines_per_block) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + lines_per_block * g.nx;
  const int n = g.nx, nkx = g.nkx;
  const long long rows = (long long)g.ny * g.nz;
  const long long line0 = (long long)blockIdx.x * lines_per_block;
  const C* spec = reinterpret_cast<const C*>(f.spec);
  for (int t = threadIdx.x; t < lines_per_block * n; t += blockDim.x) {
    const int l = t / n, kx = t - l * n;
    const long long ra = 2 * (line0 + l), rb = ra + 1;
    const bool mirror = kx >= nkx;
    const int q = mirror ? n - kx : kx;
    C A, B;
    A.x = A.y = B.x = B.y = (T)0;
    if (ra < rows) A = spec[ra * nkx + q];
    if (rb < rows) B = spec[rb * nkx + q];
    if (q == 0 || 2 * q == n) { A.y = (T)0; B.y = (T)0; }   // real DC / Nyquist bins
    if (mirror) { A = cconj(A); B = cconj(B); }
    C z;  // A + i B
    z.x = A.x - B.y;
    z.y = A.y + B.x;
    bufa[t] = z;
  }
  const int res = fft_lines<T, true>(bufa, bufb, lines_per_block, plan, reinterpret_cast<const C*>(tw));
  const C* out = res == 0 ? bufa : bufb;
  for (int t = threadIdx.x; t < lines_per_block * n; t += blockDim.x) {
    const int l = t / n, i = t - l * n;
    const long long ra = 2 * (line0 + l), rb = ra + 1;
    if (ra < rows) f.phi[ra * n + i] = out[t].x;
    if (rb < rows) f.phi[rb * n + i] = out[t].y;
  }
}

// z transform of the half-spectrum, in place; a block takes `cols` adjacent
// kx columns of one y-plane (coalesced rows of `cols` complex values).
template <typename T, bool INV>
__global__ void k_fft_z(Geo g, Fields<T> f, const T* __restrict__ tw, FftPlan plan, int cols) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + cols * g.nz;
  const int n = g.nz, nkx = g.nkx;
  const int ntile = (nkx + cols - 1) / cols;
  const int j = blockIdx.x / ntile;
  const int kx0 = (blockIdx.x - j * ntile) * cols;
  const int w = min(cols, nkx - kx0);
  C* spec = reinterpret_cast<C*>(f.spec);
  for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
    const int k = t / cols, c = t - k * cols;
    C z;
    z.x = z.y = (T)0;
    if (c < w) z = spec[((long long)k * g.ny + j) * nkx + kx0 + c];
    bufa[c * n + k] = z;
  }
  const int res = fft_lines<T, INV>(bufa, bufb, cols, plan, reinterpret_cast<const C*>(tw));
  const C* out = res == 0 ? bufa : bufb;
  for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
    const int k = t / cols, c = t - k * cols;
    if (c < w) spec[((long long)k * g.ny + j) * nkx + kx0 + c] = out[c * n + k];
  }
}

// ---------------------------------------------------------------------------
// Wall-normal Thomas per wavenumber pair (kx, kz), FP64:
//   (phi_{j+1} - 2 phi_j + phi_{j-1})/dy^2 - (lx + lz) phi_j = r_j,
// Neumann rows at both walls; mode (0,0) pins phi_0 = 0 and removes the
// mean over j afterwards (zero-mean gauge).  Pivots are tabulated.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128) k_tri_y(Geo g, Fields<T> f, const double* __restrict__ cp,
                                               const double* __restrict__ inv, double2* fwd) {
  using C = typename Cplx<T>::type;
  const int nkx = g.nkx;
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)nkx * g.nz) return;
  const long long kx = l % nkx, kz = l / nkx;
  const long long base = kz * (long long)g.ny * nkx + kx, stride = nkx;
  C* spec = reinterpret_cast<C*>(f.spec);
  // forward values stay FP64: in place for the FP64 path, in an FP64 scratch
  // spectrum for the mixed path
  double2* F = fwd ? fwd : reinterpret_cast<double2*>(f.spec);
  const double a = g.idy * g.idy;
  const bool singular = (kx == 0 && kz == 0);
  double pr = 0.0, pi = 0.0;
  for (int j = 0; j < g.ny; ++j) {
    const long long id = base + (long long)j * stride;
    const C zj = spec[id];
    if (j == 0) {
      pr = singular ? 0.0 : (double)zj.x * inv[id];
      pi = singular ? 0.0 : (double)zj.y * inv[id];
    } else {
      pr = ((double)zj.x - a * pr) * inv[id];
      pi = ((double)zj.y - a * pi) * inv[id];
    }
    F[id] = make_double2(pr, pi);
  }
  double xr = pr, xi = pi;
  double sr = xr, si = xi;
  spec[base + (long long)(g.ny - 1) * stride].x = (T)xr;
  spec[base + (long long)(g.ny - 1) * stride].y = (T)xi;
  for (int j = g.ny - 2; j >= 0; --j) {
    const long long id = base + (long long)j * stride;
    const double2 zj = F[id];
    xr = zj.x - cp[id] * xr;
    xi = zj.y - cp[id] * xi;
    if (singular) F[id] = make_double2(xr, xi);
    spec[id].x = (T)xr;
    spec[id].y = (T)xi;
    sr += xr;
    si += xi;
  }
  if (singular) {
    // zero-mean gauge, from the FP64 values
    const double mr = sr / g.ny, mi = si / g.ny;
    for (int j = 0; j < g.ny; ++j) {
      const long long id = base + (long long)j * stride;
      const double2 v = (j == g.ny - 1) ? make_double2(pr, pi) : F[id];
      spec[id].x = (T)(v.x - mr);
      spec[id].y = (T)(v.y - mi);
    }
  }
}

// Tabulate the pivots of every (kx, kz) system once per grid.
__global__ void k_build_tri_tables(Geo g, const double* __restrict__ lamx, const double* __restrict__ lamz,
                                   double* cp, double* inv) {
  const int nkx = g.nkx;
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)nkx * g.nz) return;
  const long long kx = l % nkx, kz = l / nkx;
  const long long base = kz * (long long)g.ny * nkx + kx, stride = nkx;
  const double a = g.idy * g.idy;
  const double lam = lamx[kx] + lamz[kz];
  const bool singular = (kx == 0 && kz == 0);
  double cprev = 0.0;
  for (int j = 0; j < g.ny; ++j) {
    const double am = j > 0 ? a : 0.0;
    double cm = j < g.ny - 1 ? a : 0.0;
    double bm = -am - cm - lam;
    if (singular && j == 0) { bm = 1.0; cm = 0.0; }
    const double sub = (singular && j == 0) ? 0.0 : am;
    const double den = bm - sub * cprev;
    const double iv = 1.0 / den;
    cprev = cm * iv;
    inv[base + (long long)j * stride] = iv;
    cp[base + (long long)j * stride] = cprev;
  }
}

void launch_build_poisson_tables(const Geo& g, const double* lamx, const double* lamz, double* cp, double* inv,
                                 cudaStream_t st) {
  const long long lines = (long long)g.nkx * g.nz;
  k_build_tri_tables<<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(g, lamx, lamz, cp, inv);
}

// ---------------------------------------------------------------------------
// projection (Eq. projection) and pressure update (Eq. update_pressure):
//   u <- uhat - alpha dt G phi   (v on the wall planes untouched)
//   p <- p + phi - alpha dt / (2 Re) L_c phi,  L_c with Neumann walls
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_project(Geo g, Fields<T> f, double adt, double re) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long pu = (long long)ny * nx, pv = (long long)(ny + 1) * nx;
  const T cadt = (T)adt;
  const T beta = (T)(adt / (2.0 * re));
  const T idx = (T)g.idx, idy = (T)g.idy, idz = (T)g.idz;
  const T* __restrict__ ph = f.phi;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < g.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(cell % nx);
    const int j = (int)((cell / nx) % ny);
    const int k = (int)(cell / pu);
    const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
    const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
    const long long r0 = (long long)k * pu + (long long)j * nx;
    const T c0 = ph[r0 + i];
    const T pw = ph[r0 + im], pe = ph[r0 + ip];
    const T pb = ph[(long long)km * pu + (long long)j * nx + i], pf = ph[(long long)kp * pu + (long long)j * nx + i];
    const T up = j + 1 < ny ? ph[r0 + nx + i] - c0 : (T)0;
    const T dn = j > 0 ? c0 - ph[r0 - nx + i] : (T)0;
    f.u[r0 + i] -= cadt * (c0 - pw) * idx;
    f.w[r0 + i] -= cadt * (c0 - pb) * idz;
    if (j > 0) f.v[(long long)k * pv + (long long)j * nx + i] -= cadt * dn * idy;
    const T lap = (pe - (T)2 * c0 + pw) * idx * idx + (up - dn) * idy * idy + (pf - (T)2 * c0 + pb) * idz * idz;
    f.p[r0 + i] += c0 - beta * lap;
  }
}

// ---------------------------------------------------------------------------
// host launcher: the whole elliptic step of one sub-stage
// ---------------------------------------------------------------------------
static int lines_for(int n) {
  int l = 2048 / n;
  return l < 1 ? 1 : l;
}

template <typename T>
void launch_poisson(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SpecTables<T>& tb,
                    const Stage& sg, double dt, double re, int use_q, double* partial, DevState* ds,
                    cudaStream_t st) {
  using C = typename Cplx<T>::type;
  if (use_q) {
    stage_mark(st, ST_QRED);
    k_q_partial<T><<<QB_BLOCKS, QB_THREADS, 0, st>>>(g, f, b.blist, b.cap, ds, partial);
    k_q_final<<<1, 32, 0, st>>>(g, partial, ds, sg.s, use_q);
  }
  const double scale = 1.0 / (sg.alp * dt * (double)g.nx * (double)g.nz);
  const FftPlan px = make_plan(g.nx), pz = make_plan(g.nz);
  // x forward (fused divergence / q / rhs)
  {
    const int lpb = lines_for(g.nx);
    const long long lines = ((long long)g.ny * g.nz + 1) / 2;
    const size_t sm = 2ull * lpb * g.nx * sizeof(C);
    stage_mark(st, ST_FFT_X_FWD);
    k_fft_x_fwd<T><<<(unsigned)((lines + lpb - 1) / lpb), 256, sm, st>>>(g, f, b.flags32, tb.twx, px, lpb, ds, sg.s,
                                                                        use_q, scale);
  }
  const int cols = lines_for(g.nz) < 16 ? lines_for(g.nz) : 16;
  const int ntile = (g.nkx + cols - 1) / cols;
  const size_t smz = 2ull * cols * g.nz * sizeof(C);
  stage_mark(st, ST_FFT_Z_FWD);
  k_fft_z<T, false><<<g.ny * ntile, 256, smz, st>>>(g, f, tb.twz, pz, cols);
  {
    stage_mark(st, ST_TRI_Y);
    const long long lines = (long long)g.nkx * g.nz;
    double2* fwd = sizeof(T) == sizeof(double) ? nullptr : reinterpret_cast<double2*>(f.scr);
    k_tri_y<T><<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(g, f, tb.cp, tb.inv, fwd);
  }
  stage_mark(st, ST_FFT_Z_INV);
  k_fft_z<T, true><<<g.ny * ntile, 256, smz, st>>>(g, f, tb.twz, pz, cols);
  {
    stage_mark(st, ST_FFT_X_INV);
    const int lpb = lines_for(g.nx);
    const long long lines = ((long long)g.ny * g.nz + 1) / 2;
    const size_t sm = 2ull * lpb * g.nx * sizeof(C);
    k_fft_x_inv<T><<<(unsigned)((lines + lpb - 1) / lpb), 256, sm, st>>>(g, f, tb.twx, px, lpb);
  }
  stage_mark(st, ST_PROJECT);
  k_project<T><<<(unsigned)((g.ncell + 255) / 256), 256, 0, st>>>(g, f, sg.alp * dt, re);
}

template <typename T>
void set_fft_smem_limits() {
  using C = typename Cplx<T>::type;
  const int maxsm = 2 * 2048 * (int)sizeof(C) + 1024;
  cudaFuncSetAttribute(k_fft_x_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
  cudaFuncSetAttribute(k_fft_x_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
  cudaFuncSetAttribute(k_fft_z<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
  cudaFuncSetAttribute(k_fft_z<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm);
}

void init_kernel_attributes() {
  set_fft_smem_limits<double>();
  set_fft_smem_limits<float>();
}

template void launch_poisson<double>(const Geo&, const Fields<double>&, const TagBuffers&,
                                     const SpecTables<double>&, const Stage&, double, double, int, double*,
                                     DevState*, cudaStream_t);
template void launch_poisson<float>(const Geo&, const Fields<float>&, const TagBuffers&, const SpecTables<float>&,
                                    const Stage&, double, double, int, double*, DevState*, cudaStream_t);

}  // namespace ibm
