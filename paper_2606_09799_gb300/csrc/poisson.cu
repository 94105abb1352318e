// poisson.cu -- consistent elliptic step of arXiv 2606.09799:
//   mass correction q (Section 3.2: q_B = D uhat on boundary cells, q_F
//   uniform on the fluid cells, Eq. constraint_q), right-hand side of
//   Eq. elliptic_mod, direct solve of L_c phi = rhs (FFT in the periodic x
//   and z, Thomas per wavenumber in y, homogeneous Neumann walls; Eq.
//   elliptic), projection (Eq. projection) and pressure update (Eq.
//   update_pressure).
//
// The FFTs are hand-written self-sorting (Stockham) transforms in shared
// memory with radix-8 (FP32 path), -4, -2, -3 and -5 butterflies, so every
// size 2^a 3^b 5^c up to 1024 is supported.  Two real rows are packed into
// one complex transform.
// The wall-normal Thomas solve always runs in FP64 with pivots tabulated
// once per grid (they depend only on the wavenumber pair).
#include <math.h>

#include <algorithm>
#include <type_traits>

#include <cooperative_groups.h>

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
// FFT plan: radices in order of application (product = n), with the exact
// multipliers that replace the integer divisions of each stage
// ---------------------------------------------------------------------------
struct FftStage {
  int R, Ns, nb, scale;   // radix, span so far, butterflies per line, twiddle stride
  unsigned mNs, mnb;      // ceil(2^32 / Ns), ceil(2^32 / nb)
};
struct FftPlan {
  int n, nst;
  FftStage st[12];
};

static unsigned magic_div(unsigned d) { return (unsigned)((0x100000000ull + d - 1) / d); }

__device__ __forceinline__ unsigned magic_div_dev(unsigned d) {
  return (unsigned)((0x100000000ull + d - 1) / d);
}

// q = x / d with m = ceil(2^32 / d): exact for x < 2^16 and d < 2^16, since
// x * (m d - 2^32) < 2^32.  d = 1 has no 32-bit multiplier (2^32 wraps to
// m = 0) and is taken as the identity.
__device__ __forceinline__ unsigned fdiv(unsigned x, unsigned m) { return m ? __umulhi(x, m) : x; }

static FftPlan make_plan(int n, bool radix8) {
  FftPlan p;
  p.n = n;
  p.nst = 0;
  int m = n, Ns = 1;
  int rad[12], nr = 0;
  while (radix8 && m % 8 == 0) { rad[nr++] = 8; m /= 8; }
  while (m % 4 == 0) { rad[nr++] = 4; m /= 4; }
  while (m % 2 == 0) { rad[nr++] = 2; m /= 2; }
  while (m % 3 == 0) { rad[nr++] = 3; m /= 3; }
  while (m % 5 == 0) { rad[nr++] = 5; m /= 5; }
  for (int s = 0; s < nr; ++s) {
    FftStage& st = p.st[p.nst++];
    st.R = rad[s];
    st.Ns = Ns;
    st.nb = n / st.R;
    st.scale = n / (Ns * st.R);
    st.mNs = magic_div((unsigned)Ns);
    st.mnb = magic_div((unsigned)st.nb);
    Ns *= st.R;
  }
  return p;
}

// Radix-R butterfly on v (inputs already twiddled), in place.
template <typename T, bool INV, int R>
__device__ __forceinline__ void butterfly(typename Cplx<T>::type (&v)[R]) {
  using C = typename Cplx<T>::type;
  if constexpr (R == 2) {
    const C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    const C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    C jd13;  // -i d13 (forward) or +i d13 (inverse)
    if (INV) { jd13.x = -d13.y; jd13.y = d13.x; }
    else { jd13.x = d13.y; jd13.y = -d13.x; }
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, jd13);
    v[3] = csub(d02, jd13);
  } else if constexpr (R == 8) {
    // 4-point transforms of the even and the odd inputs, then
    // X_k = E_k + w^k O_k and X_{k+4} = E_k - w^k O_k, w = exp(-+ 2 pi i / 8)
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    butterfly<T, INV, 4>(e);
    butterfly<T, INV, 4>(o);
    const T h = (T)0.70710678118654752440;   // 1 / sqrt(2)
    C t1, t2, t3;   // w O_1, w^2 O_2, w^3 O_3
    if (INV) {      // w = (1 + i) / sqrt2, w^2 = i, w^3 = (-1 + i) / sqrt2
      t1.x = h * (o[1].x - o[1].y);
      t1.y = h * (o[1].x + o[1].y);
      t2.x = -o[2].y;
      t2.y = o[2].x;
      t3.x = -h * (o[3].x + o[3].y);
      t3.y = h * (o[3].x - o[3].y);
    } else {        // w = (1 - i) / sqrt2, w^2 = -i, w^3 = (-1 - i) / sqrt2
      t1.x = h * (o[1].x + o[1].y);
      t1.y = h * (o[1].y - o[1].x);
      t2.x = o[2].y;
      t2.y = -o[2].x;
      t3.x = h * (o[3].y - o[3].x);
      t3.y = -h * (o[3].x + o[3].y);
    }
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], t1);
    v[5] = csub(e[1], t1);
    v[2] = cadd(e[2], t2);
    v[6] = csub(e[2], t2);
    v[3] = cadd(e[3], t3);
    v[7] = csub(e[3], t3);
  } else if constexpr (R == 5) {
    // X_k = sum_r v_r w^{rk}, w = exp(-+ 2 pi i / 5): pair the inputs
    // symmetric about r = 0 (t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4,
    // t4 = v2 - v3); the cosines and sines of 2 pi / 5 and 4 pi / 5 from
    // sqrt(5): cos = (sqrt5 - 1)/4, -(sqrt5 + 1)/4; sin = sqrt(10 +- 2 sqrt5)/4
    const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;
    const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;
    const C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]), t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C a1, a2, b1, b2;
    a1.x = v[0].x + c1 * t1.x + c2 * t2.x;
    a1.y = v[0].y + c1 * t1.y + c2 * t2.y;
    a2.x = v[0].x + c2 * t1.x + c1 * t2.x;
    a2.y = v[0].y + c2 * t1.y + c1 * t2.y;
    b1.x = s1 * t3.x + s2 * t4.x;
    b1.y = s1 * t3.y + s2 * t4.y;
    b2.x = s2 * t3.x - s1 * t4.x;
    b2.y = s2 * t3.y - s1 * t4.y;
    // forward: X1 = a1 - i b1, X4 = a1 + i b1, X2 = a2 - i b2, X3 = a2 + i b2
    C ib1, ib2;   // -i b (forward) or +i b (inverse)
    if (INV) { ib1.x = -b1.y; ib1.y = b1.x; ib2.x = -b2.y; ib2.y = b2.x; }
    else { ib1.x = b1.y; ib1.y = -b1.x; ib2.x = b2.y; ib2.y = -b2.x; }
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, ib1);
    v[4] = csub(a1, ib1);
    v[2] = cadd(a2, ib2);
    v[3] = csub(a2, ib2);
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
}

// One Stockham pass of radix R over `lines` transforms of length n; element
// e of line l sits at l * ls + e * es (src and dst alike).
// tw[m] = exp(-2 pi i m/n).  Threads take butterflies (line, j) with the
// line index fastest when es > 1 (column tiles: neighbouring lines are
// neighbouring words) or when lfast is set (rows padded to an odd number of
// words' pairs, ls = n + 1: neighbouring lines then fall in neighbouring
// banks, whatever stride the pass writes with), and j fastest otherwise.
// R is a template parameter so the butterfly's values stay in registers.
template <typename T, bool INV, int R>
__device__ __forceinline__ void fft_pass_r(const typename Cplx<T>::type* src, typename Cplx<T>::type* dst,
                                           int lines, const FftStage& S,
                                           const typename Cplx<T>::type* __restrict__ tw, int es, int ls,
                                           unsigned mlines, bool lfast) {
  using C = typename Cplx<T>::type;
  const int Ns = S.Ns, nb = S.nb, scale = S.scale;
  const unsigned mNs = S.mNs, mnb = S.mnb;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const int total = lines * nb;
  for (int t = tid; t < total; t += nth) {
    int line, j;
    if (es > 1 || lfast) {
      j = (int)fdiv((unsigned)t, mlines);
      line = t - j * lines;
    } else {
      line = (int)fdiv((unsigned)t, mnb);
      j = t - line * nb;
    }
    const C* sp = src + line * ls;
    C* dp = dst + line * ls;
    const int jn = (int)fdiv((unsigned)j, mNs);
    const int k = j - jn * Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = sp[(j + r * nb) * es];
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = __ldg(tw + (r * k * scale));
        if (INV) w = cconj(w);
        v[r] = cmul(v[r], w);
      }
    }
    butterfly<T, INV, R>(v);
    const int dbase = jn * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dp[(dbase + r * Ns) * es] = v[r];
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void fft_pass(const typename Cplx<T>::type* src, typename Cplx<T>::type* dst,
                                         int lines, const FftStage& S,
                                         const typename Cplx<T>::type* __restrict__ tw, int es, int ls,
                                         unsigned mlines, bool lfast) {
  switch (S.R) {
    case 8: fft_pass_r<T, INV, 8>(src, dst, lines, S, tw, es, ls, mlines, lfast); break;
    case 4: fft_pass_r<T, INV, 4>(src, dst, lines, S, tw, es, ls, mlines, lfast); break;
    case 2: fft_pass_r<T, INV, 2>(src, dst, lines, S, tw, es, ls, mlines, lfast); break;
    case 3: fft_pass_r<T, INV, 3>(src, dst, lines, S, tw, es, ls, mlines, lfast); break;
    default: fft_pass_r<T, INV, 5>(src, dst, lines, S, tw, es, ls, mlines, lfast); break;
  }
}

// Full transform; returns the buffer that holds the result (0 = a, 1 = b).
template <typename T, bool INV>
__device__ int fft_lines(typename Cplx<T>::type* a, typename Cplx<T>::type* b, int lines, const FftPlan& p,
                         const typename Cplx<T>::type* __restrict__ tw, int es = 1, int ls = -1,
                         unsigned mlines = 0, bool lfast = false) {
  if (ls < 0) ls = p.n;
  int cur = 0;
  for (int s = 0; s < p.nst; ++s) {
    __syncthreads();
    if (cur == 0) fft_pass<T, INV>(a, b, lines, p.st[s], tw, es, ls, mlines, lfast);
    else fft_pass<T, INV>(b, a, lines, p.st[s], tw, es, ls, mlines, lfast);
    cur ^= 1;
  }
  __syncthreads();
  return cur;
}

// ---------------------------------------------------------------------------
// q_F: fixed-order two-level reduction of sum_{C_B} D uhat dV over the
// sorted boundary-cell list; q_F = -A / |C_F| (uniform on fluid cells).
// Each block leaves two partial sums: D uhat and the volume of its boundary
// cells, both per unit dx dz on the non-uniform wall-normal grid (whose cell
// heights differ), the first per unit dV and the second unused otherwise.
// ---------------------------------------------------------------------------
constexpr int QB_BLOCKS = 128, QB_THREADS = 256;   // QB_BLOCKS: the most partial sums

template <typename T>
__device__ __forceinline__ double div_at(const Geo& g, const T* __restrict__ u, const T* __restrict__ v,
                                         const T* __restrict__ w, long long i, long long j, long long k) {
  const long long ip = i + 1 == g.nx ? 0 : i + 1, kp = k + 1 == g.nz ? 0 : k + 1;
  const double du = ((double)u[fidx(g, 0, ip, j, k)] - (double)u[fidx(g, 0, i, j, k)]) * g.idx;
  const double dv = ((double)v[fidx(g, 1, i, j + 1, k)] - (double)v[fidx(g, 1, i, j, k)]) * (g.yt.ihc ? g.yt.ihc[j] : g.idy);
  const double dw = ((double)w[fidx(g, 2, i, j, kp)] - (double)w[fidx(g, 2, i, j, k)]) * g.idz;
  return du + dv + dw;
}

template <typename T>
__device__ __forceinline__ void q_partial(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ blist,
                                                          unsigned cap, const DevState* ds, double* partial) {
  __shared__ double red[QB_THREADS];
  const unsigned n = min(ds->nbound, cap);
  const unsigned per = (n + bk.gx - 1) / bk.gx;
  const unsigned e0 = bk.x * per, e1 = min(n, e0 + per);
  __shared__ double redv[QB_THREADS];
  double acc = 0.0, vol = 0.0;
  for (unsigned e = e0 + threadIdx.x; e < e1; e += QB_THREADS) {
    const long long cell = blist[e];
    long long i, j, k;
    split3(cell, g.nx, g.ny, i, j, k);
    const double du = div_at<T>(g, f.u, f.v, f.w, i, j, k);
    if (g.yt.hc) {
      acc += du * g.yt.hc[j];
      vol += g.yt.hc[j];
    } else {
      acc += du;
    }
  }
  red[threadIdx.x] = acc;
  redv[threadIdx.x] = vol;
  __syncthreads();
  for (int s = QB_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[threadIdx.x] += red[threadIdx.x + s];
      redv[threadIdx.x] += redv[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * bk.x] = red[0];
    partial[2 * bk.x + 1] = redv[0];
  }
}
template <typename T>
struct QPartial {
  static constexpr int kThreads = QB_THREADS;
  Geo g;
  Fields<T> f;
  const unsigned* blist;
  unsigned cap;
  const DevState* ds;
  double* partial;
  __device__ __forceinline__ void operator()(const Blk& bk) const { q_partial<T>(bk, g, f, blist, cap, ds, partial); }
};

__device__ __forceinline__ void q_final(const Blk& bk, const Geo& g, const double* partial, DevState* ds, int s, int use_q,
                                        int nblk) {
  const double sum = warp_sum_fixed(partial, nblk, 2, 0);
  const double vb = warp_sum_fixed(partial, nblk, 2, 1);
  if (threadIdx.x != 0) return;
  double A, VF;
  if (g.yt.hc) {   // heights summed per unit dx dz: the box volume less the boundary cells
    const double dxz = g.dx * g.dz;
    A = sum * dxz;
    VF = g.lx * g.ly * g.lz - vb * dxz;
  } else {
    const double dV = g.dx * g.dy * g.dz;
    A = sum * dV;
    VF = (double)(g.ncell - (long long)ds->nbound) * dV;
  }
  ds->sum_a[s] = A;
  const double qf = (use_q && VF > 0.0) ? -A / VF : 0.0;
  ds->qf[s] = qf;
  ds->sum_qdv[s] = A + qf * VF;
  const float qh = (float)qf;
  ds->qf_hi[s] = qh;
  ds->qf_lo[s] = (float)(qf - (double)qh);
  if (!isfinite(A)) atomicOr(&ds->err, ERR_NONFINITE);
}
struct QFinal {
  static constexpr int kThreads = 32;
  Geo g;
  const double* partial;
  DevState* ds;
  int s;
  int use_q;
  int nblk;
  __device__ __forceinline__ void operator()(const Blk& bk) const { q_final(bk, g, partial, ds, s, use_q, nblk); }
};

// ---------------------------------------------------------------------------
// Energy- and mass-conserving shape of q (App. B):
//   q_F^k = (-A S2 + B S1)/C + (A S1 - B S0)/C (p^k - e^k),  C = S0 S2 - S1^2,
// S_i = sum_F (p - e)^i dV, A = sum_B Du dV, B = sum_B (p - e) Du dV, with
// e = |u|^2/2 of the provisional velocity averaged to the cell centre and p
// the pressure of the sub-stage.  Fixed-order two-level FP64 reduction.
// ---------------------------------------------------------------------------
constexpr int QE_THREADS = 256;

// p - e at a cell from the provisional state (bulk type)
template <typename T>
__device__ __forceinline__ T p_minus_e(const Geo& g, const Fields<T>& f, long long i, long long j, long long k) {
  const long long ip = i + 1 == g.nx ? 0 : i + 1, kp = k + 1 == g.nz ? 0 : k + 1;
  const T uc = (T)0.5 * (f.u[fidx(g, 0, i, j, k)] + f.u[fidx(g, 0, ip, j, k)]);
  const T vc = (T)0.5 * (f.v[fidx(g, 1, i, j, k)] + f.v[fidx(g, 1, i, j + 1, k)]);
  const T wc = (T)0.5 * (f.w[fidx(g, 2, i, j, k)] + f.w[fidx(g, 2, i, j, kp)]);
  return f.p[cidx(g, i, j, k)] - (T)0.5 * (uc * uc + vc * vc + wc * wc);
}

template <typename T>
__device__ __forceinline__ void q_energy_partial(const Blk& bk, const Geo& g, const Fields<T>& f,
                                                 const unsigned* __restrict__ flags32, double* partial) {
  __shared__ double red[5][QE_THREADS];
  const unsigned n = (unsigned)g.ncell;
  const unsigned per = (n + bk.gx - 1) / bk.gx;
  const unsigned c0 = bk.x * per, c1 = min(n, c0 + per);
  // fluid volume, S1, S2, A, B per unit dV (uniform grid) or per unit dx dz
  // (non-uniform wall-normal grid: each cell weighted by its height)
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (unsigned cell = c0 + threadIdx.x; cell < c1; cell += QE_THREADS) {
    const unsigned i = cell % (unsigned)g.nx, r = cell / (unsigned)g.nx;
    const unsigned j = r % (unsigned)g.ny, k = r / (unsigned)g.ny;
    const double pe = (double)p_minus_e<T>(g, f, i, j, k);
    const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
    if (g.yt.hc) {
      const double wv = g.yt.hc[j];
      if (fl & FLAG_B) {
        const double du = div_at<T>(g, f.u, f.v, f.w, i, j, k) * wv;
        acc[3] += du;
        acc[4] += pe * du;
      } else {
        acc[0] += wv;
        acc[1] += pe * wv;
        acc[2] += pe * (pe * wv);
      }
    } else if (fl & FLAG_B) {
      const double du = div_at<T>(g, f.u, f.v, f.w, i, j, k);
      acc[3] += du;
      acc[4] += pe * du;
    } else {
      acc[0] += 1.0;
      acc[1] += pe;
      acc[2] += pe * pe;
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int st = QE_THREADS / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st)
#pragma unroll
      for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[5 * bk.x + threadIdx.x] = red[threadIdx.x][0];
}
template <typename T>
struct QEnergyPartial {
  static constexpr int kThreads = QE_THREADS;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  double* partial;
  __device__ __forceinline__ void operator()(const Blk& bk) const { q_energy_partial<T>(bk, g, f, flags32, partial); }
};

__device__ __forceinline__ void q_energy_final(const Blk&, const Geo& g, const double* partial, DevState* ds, int s,
                                               int nblk) {
  double t[5];
  for (int q = 0; q < 5; ++q) t[q] = warp_sum_fixed(partial, nblk, 5, q);
  if (threadIdx.x != 0) return;
  const double dV = g.yt.hc ? g.dx * g.dz : g.dx * g.dy * g.dz;
  const double S0 = t[0] * dV, S1 = t[1] * dV, S2 = t[2] * dV, A = t[3] * dV, B = t[4] * dV;
  const double C = S0 * S2 - S1 * S1;
  double qa, qb;
  if (S0 > 0.0 && C > 1e-14 * S0 * S2) {
    qa = (-A * S2 + B * S1) / C;
    qb = (A * S1 - B * S0) / C;
  } else {   // p - e uniform on the fluid cells: the mass constraint alone
    qa = S0 > 0.0 ? -A / S0 : 0.0;
    qb = 0.0;
  }
  ds->qa[s] = qa;
  ds->qb[s] = qb;
  ds->qf[s] = qa;
  ds->sum_a[s] = A;
  ds->sum_qdv[s] = A + qa * S0 + qb * S1;
  if (!isfinite(qa) || !isfinite(qb)) atomicOr(&ds->err, ERR_NONFINITE);
}
struct QEnergyFinal {
  static constexpr int kThreads = 32;
  Geo g;
  const double* partial;
  DevState* ds;
  int s;
  int nblk;
  __device__ __forceinline__ void operator()(const Blk& bk) const { q_energy_final(bk, g, partial, ds, s, nblk); }
};

// ---------------------------------------------------------------------------
// forward x transform fused with the right-hand side of Eq. elliptic_mod:
// rhs = (D uhat - q) / (alpha dt) on C_F, 0 on C_B (q_B = D uhat), scaled by
// 1/(nx nz) so the inverse transforms need no normalisation.  Two real rows
// form one complex line; the two half-spectra are separated on output.
// ---------------------------------------------------------------------------
// (H[a] + L[a]) - (H[b] + L[b]) times (ih + il), as a big part and a small
// correction whose sum carries the product to ~FP32^2 relative accuracy
// (a - b) * (ih + il) for pairs a = (ha, la), b = (hb, lb), as a pair
__device__ __forceinline__ void pair_diff_v(float ha, float la, float hb, float lb, float ih, float il, float& big,
                                            float& small) {
  float s, e, p, pe;
  two_sum(ha, -hb, s, e);
  e += la - lb;
  two_prod(s, ih, p, pe);
  big = p;
  small = pe + e * ih + s * il;
}

// Projection coefficients (Eqs. projection, update_pressure).
template <typename T>
struct ProjCoef {
  T cx, cy, cz;          // alpha dt / d
  T bx, by, bz;          // alpha dt / (2 Re d^2)
  T adt, bb;             // alpha dt and alpha dt / (2 Re), for a non-uniform wall-normal spacing
  // the right-hand side's constants in the bulk type, converted once on the
  // host: a conversion from FP64 inside the per-cell arithmetic would run on
  // the narrow FP64 pipe (or be repeated there when the compiler
  // rematerialises it)
  T sc;                  // 1 / (alpha dt nx nz)
  T idx, idy, idz;       // 1 / d
  float scf;             // sc in FP32
  float ih[3][2];        // 1 / d as FP32 (hi, lo) pairs
};

// One face of the projected state held as a (hi, lo) pair: the projection's
// FP32 gradient g subtracted without rounding it away.
__device__ __forceinline__ void proj_face(float& hi, float& lo, float g) { ff_add(hi, lo, -g); }

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Largest |D u' - q| over the fluid cells after the first solve of the mixed
// path (Eq. mod_div), kept as the bits of a non-negative FP32 value (their
// integer order is the numbers' order; NaN sorts above every number).  The
// first solve's forward transform clears the word, the correction solve's
// forward transform folds every cell into it: a block maximum, then one
// atomicMax per block, and only when the word does not already hold as much
// (thousands of blocks would otherwise queue on one address).  Every thread
// of the block calls this (the last warp may be partial).
__device__ __forceinline__ void fold_residual(unsigned* res1, unsigned rmax) {
  __shared__ unsigned wmax[32];
  const unsigned tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const unsigned nt = blockDim.x * blockDim.y * blockDim.z;
  const unsigned lanes = min(32u, nt - (tid & ~31u));
  const unsigned mask = lanes == 32u ? 0xFFFFFFFFu : (1u << lanes) - 1u;
  const unsigned m = __reduce_max_sync(mask, rmax);
  if ((tid & 31u) == 0u) wmax[tid >> 5] = m;
  __syncthreads();
  if (tid < 32u) {
    const unsigned nw = (nt + 31u) >> 5;
    const unsigned b = __reduce_max_sync(nt >= 32u ? 0xFFFFFFFFu : (1u << nt) - 1u, tid < nw ? wmax[tid] : 0u);
    if (tid == 0u && b > *reinterpret_cast<volatile unsigned*>(res1)) atomicMax(res1, b);
  }
}
__device__ __forceinline__ void clear_residual(const Blk& bk, unsigned* res1) {
  if (bk.x == 0 && bk.y == 0 && bk.z == 0 && threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) *res1 = 0u;
}
// The correction solve is needed unless the first solve's residual is
// within the budget (a NaN residual or budget always runs it).
__device__ __forceinline__ bool correction_needed(const DevState* ds, int s) {
  return !(__uint_as_float(ds->res1[s]) <= ds->div_budget);
}

// Right-hand side of Eq. elliptic_mod at cell (i, j, k), scaled by
// 1/(alpha dt nx nz): mode 0 from the provisional state (bulk type), mode 3
// the correction solve's rhs from the projected (hi, lo) state in pair
// arithmetic (the state u' = uhat - G phi is formed at the cell's faces
// here); 0 on boundary cells when q is on (q_B = D uhat).
// Wall-normal coefficients of one row j of cells: the projection's gradient
// coefficients of the faces below and above (cy0, cy1), 1/h of the row as a
// (hi, lo) pair for the pair divergence, and 1/h in the bulk type.  On a
// uniform grid they are the grid's own constants.  The per-plane transform
// forms them once per plane; the per-line transform per cell (measured
// faster there than holding both rows' values across the line).
template <typename T>
struct RowY {
  T cy0, cy1, ih;
  float ihh, ihl;
};
template <typename T>
__device__ __forceinline__ RowY<T> row_y(const Geo& g, const Fields<T>& f, const ProjCoef<T>& cf, int j) {
  RowY<T> r{cf.cy, cf.cy, cf.idy, cf.ih[1][0], cf.ih[1][1]};
  if (g.yt.ihc) {
    r.cy0 = mul_rn(cf.adt, (T)g.yt.ihf[j]);
    r.cy1 = mul_rn(cf.adt, (T)g.yt.ihf[j + 1]);
    const double ih = g.yt.ihc[j];
    r.ih = (T)ih;
    r.ihh = (float)ih;
    r.ihl = (float)(ih - (double)r.ihh);
  }
  return r;
}

template <typename T>
__device__ __forceinline__ T poisson_rhs(const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32,
                                         const DevState* ds, int s, int use_q, double scale, int mode,
                                         const ProjCoef<T>& cf, const RowY<T>& ry, T qf, T qa, T qb, int i, int j,
                                         int k, unsigned& rmax) {
  const int n = g.nx, ny = g.ny;
  const long long pu = (long long)ny * n, pv = (long long)(ny + 1) * n;
  const T sc = cf.sc, idx = cf.idx, idz = cf.idz;
  const int ip = i + 1 == n ? 0 : i + 1;
  const int kp = k + 1 == g.nz ? 0 : k + 1;
  const long long r0 = (long long)k * pu + (long long)j * n;
  const long long cell = r0 + i;
  const unsigned fl = (flags32[cell >> 2] >> (8 * (cell & 3))) & 0xFFu;
  T r = (T)0;
  if (mode == 3) {
    if (!(use_q && (fl & FLAG_B))) {
      const long long v0 = (long long)k * pv + (long long)j * n + i;
      const long long wk = (long long)kp * pu + (long long)j * n + i;
      float bx, sx, by, sy, bz, sz, a1, e1, a2, e2, a3, e3;
      {
        // the faces of the projected state u' = uhat - G phi formed here, with
        // the projection's own arithmetic (FP32 gradient, pair update), so the
        // first projection need not write u'
        const int im = i == 0 ? n - 1 : i - 1;
        const int km = k == 0 ? g.nz - 1 : k - 1;
        const long long rkm = (long long)km * pu + (long long)j * n, rkp = (long long)kp * pu + (long long)j * n;
        const T* __restrict__ ph = f.phi;
        const float p0 = (float)ph[cell];
        float uh0 = (float)f.u[cell], ul0 = (float)f.lo[0][cell];
        float uh1 = (float)f.u[r0 + ip], ul1 = (float)f.lo[0][r0 + ip];
        proj_face(uh0, ul0, (float)mul_rn(cf.cx, (T)p0 - ph[r0 + im]));
        proj_face(uh1, ul1, (float)mul_rn(cf.cx, ph[r0 + ip] - (T)p0));
        float vh0 = (float)f.v[v0], vl0 = (float)f.lo[1][v0];
        float vh1 = (float)f.v[v0 + n], vl1 = (float)f.lo[1][v0 + n];
        // each face's own gradient coefficient, as the projection forms it
        if (j > 0) proj_face(vh0, vl0, (float)mul_rn(ry.cy0, (T)p0 - ph[cell - n]));
        if (j + 1 < ny) proj_face(vh1, vl1, (float)mul_rn(ry.cy1, ph[cell + n] - (T)p0));
        float wh0 = (float)f.w[cell], wl0 = (float)f.lo[2][cell];
        float wh1 = (float)f.w[wk], wl1 = (float)f.lo[2][wk];
        proj_face(wh0, wl0, (float)mul_rn(cf.cz, (T)p0 - ph[rkm + i]));
        proj_face(wh1, wl1, (float)mul_rn(cf.cz, ph[rkp + i] - (T)p0));
        pair_diff_v(uh1, ul1, uh0, ul0, cf.ih[0][0], cf.ih[0][1], bx, sx);
        pair_diff_v(vh1, vl1, vh0, vl0, ry.ihh, ry.ihl, by, sy);
        pair_diff_v(wh1, wl1, wh0, wl0, cf.ih[2][0], cf.ih[2][1], bz, sz);
      }
      two_sum(bx, by, a1, e1);
      two_sum(a1, bz, a2, e2);
      // the target q of the first solve: uniform (an FP32 pair) or the
      // energy-conserving shape stored per cell by mode 0
      const float qh = use_q == 2 ? (float)f.qk[cell] : (use_q ? ds->qf_hi[s] : 0.0f);
      const float ql = use_q == 1 ? ds->qf_lo[s] : 0.0f;
      two_sum(a2, -qh, a3, e3);
      const float d = a3 + (((e1 + e2) + e3) + ((sx + sy) + sz) - ql);   // D u' - q
      rmax = max(rmax, __float_as_uint(d) & 0x7FFFFFFFu);                 // |d| (NaN above every number)
      r = (T)(d * cf.scf);
    }
  } else if (!(use_q && (fl & FLAG_B))) {
    const long long v0 = (long long)k * pv + (long long)j * n + i;
    // explicit rounding (no contraction): the single-simulation and the
    // batched kernels compile this body separately and must round alike
    const T du = mul_rn(f.u[r0 + ip] - f.u[cell], idx);
    const T dv = mul_rn(f.v[v0 + n] - f.v[v0], ry.ih);
    const T dw = mul_rn(f.w[(long long)kp * pu + (long long)j * n + i] - f.w[cell], idz);
    T q = qf;
    if (use_q == 2) {   // App. B shape, kept per cell for the correction solve
      q = qa + qb * p_minus_e<T>(g, f, i, j, k);
      f.qk[cell] = q;
    }
    r = mul_rn(add_rn(add_rn(du, dv), dw) - q, sc);
  }
  return r;
}

// Mode 0 of poisson_rhs for the FP32 cells (i, j, k) and (i + 1, j, k), i even
// (nx is even on every grid, so the pairs are 8-byte aligned; every field has
// fewer than 2^30 entries): each row is read as one float2, with the x-
// neighbour i + 2 of the second cell as a scalar, and each cell takes
// poisson_rhs's operations in the same order.
__device__ __forceinline__ void rhs_pair0(const Geo& g, const Fields<float>& f, const unsigned* __restrict__ flags32,
                                          int use_q, const ProjCoef<float>& cf, const RowY<float>& ry, float qf,
                                          int i, int j, int k, float& ra, float& rb) {
  const int n = g.nx, ny = g.ny;
  const int pu = ny * n, pv = (ny + 1) * n;
  const int kp = k + 1 == g.nz ? 0 : k + 1;
  const int ip2 = i + 2 == n ? 0 : i + 2;
  const int r0 = k * pu + j * n, cell = r0 + i;
  const int v0 = k * pv + j * n + i, wk = kp * pu + j * n + i;
  const float2 uu = *reinterpret_cast<const float2*>(f.u + cell);
  const float u2 = f.u[r0 + ip2];
  const float2 va = *reinterpret_cast<const float2*>(f.v + v0), vb = *reinterpret_cast<const float2*>(f.v + v0 + n);
  const float2 w0 = *reinterpret_cast<const float2*>(f.w + cell), w1 = *reinterpret_cast<const float2*>(f.w + wk);
  const unsigned fw = flags32[cell >> 2];
  const unsigned sh = 8u * (unsigned)(cell & 3);
  const unsigned fla = (fw >> sh) & 0xFFu, flb = (fw >> (sh + 8u)) & 0xFFu;
  const float sc = cf.sc, idx = cf.idx, idz = cf.idz;
  {
    const float du = mul_rn(uu.y - uu.x, idx);
    const float dv = mul_rn(vb.x - va.x, ry.ih);
    const float dw = mul_rn(w1.x - w0.x, idz);
    ra = (use_q && (fla & FLAG_B)) ? 0.0f : mul_rn(add_rn(add_rn(du, dv), dw) - qf, sc);
  }
  {
    const float du = mul_rn(u2 - uu.y, idx);
    const float dv = mul_rn(vb.y - va.y, ry.ih);
    const float dw = mul_rn(w1.y - w0.y, idz);
    rb = (use_q && (flb & FLAG_B)) ? 0.0f : mul_rn(add_rn(add_rn(du, dv), dw) - qf, sc);
  }
}

// Mode 3 of poisson_rhs (the correction's right-hand side from the projected
// (hi, lo) state) for the FP32 cells (i, j, k) and (i + 1, j, k), i even:
// phi, the state's hi and lo words and the rows above, below and beside are
// read as float2 pairs (scalars for the x-neighbours i - 1 and i + 2), and
// each cell takes poisson_rhs's operations in the same order.
__device__ __forceinline__ void rhs_pair3(const Geo& g, const Fields<float>& f, const unsigned* __restrict__ flags32,
                                          const DevState* ds, int s, int use_q, const ProjCoef<float>& cf,
                                          const RowY<float>& ry, int i, int j, int k, float& ra, float& rb,
                                          unsigned& rmax) {
  const int n = g.nx, ny = g.ny;
  const int pu = ny * n, pv = (ny + 1) * n;
  const int kp = k + 1 == g.nz ? 0 : k + 1, km = k == 0 ? g.nz - 1 : k - 1;
  const int im = i == 0 ? n - 1 : i - 1, ip2 = i + 2 == n ? 0 : i + 2;
  const int r0 = k * pu + j * n, cell = r0 + i;
  const int v0 = k * pv + j * n + i, wk = kp * pu + j * n + i;
  const int rkm = km * pu + j * n, rkp = kp * pu + j * n;
  auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
  const float* __restrict__ ph = f.phi;
  const float2 P0 = ld2(ph + cell);
  const float Pm = ph[r0 + im], Pp = ph[r0 + ip2];
  const float2 Ps = j > 0 ? ld2(ph + cell - n) : make_float2(0.0f, 0.0f);
  const float2 Pn = j + 1 < ny ? ld2(ph + cell + n) : make_float2(0.0f, 0.0f);
  const float2 Pkm = ld2(ph + rkm + i), Pkp = ld2(ph + rkp + i);
  const float2 Uh = ld2(f.u + cell), Ul = ld2(f.lo[0] + cell);
  const float Uhp = f.u[r0 + ip2], Ulp = f.lo[0][r0 + ip2];
  const float2 V0h = ld2(f.v + v0), V0l = ld2(f.lo[1] + v0), V1h = ld2(f.v + v0 + n), V1l = ld2(f.lo[1] + v0 + n);
  const float2 W0h = ld2(f.w + cell), W0l = ld2(f.lo[2] + cell), W1h = ld2(f.w + wk), W1l = ld2(f.lo[2] + wk);
  const unsigned fw = flags32[cell >> 2];
  const unsigned sh = 8u * (unsigned)(cell & 3);
  const unsigned fla = (fw >> sh) & 0xFFu, flb = (fw >> (sh + 8u)) & 0xFFu;
  const float2 Qk = use_q == 2 ? ld2(f.qk + cell) : make_float2(0.0f, 0.0f);
  const float qh1 = use_q ? ds->qf_hi[s] : 0.0f, ql = use_q == 1 ? ds->qf_lo[s] : 0.0f;
  auto one = [&](unsigned fl, float p0, float pw, float pe, float pso, float pno, float pkm, float pkp, float uh0,
                 float ul0, float uh1, float ul1, float vh0, float vl0, float vh1, float vl1, float wh0, float wl0,
                 float wh1, float wl1, float qk) {
    if (use_q && (fl & FLAG_B)) return 0.0f;
    float bx, sx, by, sy, bz, sz, a1, e1, a2, e2, a3, e3;
    proj_face(uh0, ul0, mul_rn(cf.cx, p0 - pw));
    proj_face(uh1, ul1, mul_rn(cf.cx, pe - p0));
    if (j > 0) proj_face(vh0, vl0, mul_rn(ry.cy0, p0 - pso));
    if (j + 1 < ny) proj_face(vh1, vl1, mul_rn(ry.cy1, pno - p0));
    proj_face(wh0, wl0, mul_rn(cf.cz, p0 - pkm));
    proj_face(wh1, wl1, mul_rn(cf.cz, pkp - p0));
    pair_diff_v(uh1, ul1, uh0, ul0, cf.ih[0][0], cf.ih[0][1], bx, sx);
    pair_diff_v(vh1, vl1, vh0, vl0, ry.ihh, ry.ihl, by, sy);
    pair_diff_v(wh1, wl1, wh0, wl0, cf.ih[2][0], cf.ih[2][1], bz, sz);
    two_sum(bx, by, a1, e1);
    two_sum(a1, bz, a2, e2);
    const float qh = use_q == 2 ? qk : qh1;
    two_sum(a2, -qh, a3, e3);
    const float d = a3 + (((e1 + e2) + e3) + ((sx + sy) + sz) - ql);   // D u' - q
    rmax = max(rmax, __float_as_uint(d) & 0x7FFFFFFF);
    return d * cf.scf;
  };
  ra = one(fla, P0.x, Pm, P0.y, Ps.x, Pn.x, Pkm.x, Pkp.x, Uh.x, Ul.x, Uh.y, Ul.y, V0h.x, V0l.x, V1h.x, V1l.x, W0h.x,
           W0l.x, W1h.x, W1l.x, Qk.x);
  rb = one(flb, P0.y, P0.x, Pp, Ps.y, Pn.y, Pkm.y, Pkp.y, Uh.y, Ul.y, Uhp, Ulp, V0h.y, V0l.y, V1h.y, V1l.y, W0h.y,
           W0l.y, W1h.y, W1l.y, Qk.y);
}

// mode 0: rhs = (D uhat - q)/(alpha dt) from the (hi part of the) state;
// mode 3: rhs of the correction solve, (D u' - q_F)/(alpha dt) on fluid
// cells from the projected state u' = uhat - G phi as (hi, lo) pairs, in
// pair arithmetic
template <typename T>
__device__ __forceinline__ void fft_x_fwd(const Blk& bk, const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32, const T* __restrict__ tw,
                            const FftPlan& plan, int lines_per_block, const DevState* ds, int s, int use_q,
                            double scale, int mode, const ProjCoef<T>& cf, unsigned* res1) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + lines_per_block * (g.nx + 1);   // lines padded to nx + 1 words (see fft_pass_r)
  const int n = g.nx, ny = g.ny, xs = n + 1;
  const int rows = g.ny * g.nz;
  const int line0 = bk.x * lines_per_block;
  const T qf = use_q ? (T)ds->qf[s] : (T)0;
  const T qa = use_q == 2 ? (T)ds->qa[s] : (T)0, qb = use_q == 2 ? (T)ds->qb[s] : (T)0;
  if (mode == 0) clear_residual(bk, res1);
  unsigned rmax = 0u;
  // load: rows 2 l and 2 l + 1 of line l; divergence in the bulk type
  for (int l = threadIdx.y; l < lines_per_block; l += blockDim.y) {
    int jj[2], kk[2];
    bool ok[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int row = 2 * (line0 + l) + hh;
      ok[hh] = row < rows;
      jj[hh] = row % ny;
      kk[hh] = row / ny;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      C z;
      z.x = (T)0;
      z.y = (T)0;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        if (!ok[hh]) continue;
        const T r = poisson_rhs<T>(g, f, flags32, ds, s, use_q, scale, mode, cf, row_y<T>(g, f, cf, jj[hh]), qf, qa,
                                   qb, i, jj[hh], kk[hh], rmax);
        if (hh == 0) z.x = r;
        else z.y = r;
      }
      bufa[l * xs + i] = z;
    }
  }
  if (mode == 3) fold_residual(res1, rmax);
  const int res = fft_lines<T, false>(bufa, bufb, lines_per_block, plan, reinterpret_cast<const C*>(tw), 1, xs,
                                      magic_div_dev((unsigned)lines_per_block), true);
  const C* out = res == 0 ? bufa : bufb;
  C* spec = reinterpret_cast<C*>(f.spec);
  const int nkx = g.nkx;
  for (int l = threadIdx.y; l < lines_per_block; l += blockDim.y)
  for (int kx = threadIdx.x; kx < nkx; kx += blockDim.x) {
    const C Z = out[l * xs + kx];
    const C Zc = cconj(out[l * xs + (kx == 0 ? 0 : n - kx)]);
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
template <typename T>
struct FftXFwd {
  static constexpr int kThreads = 256;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const T* tw;
  FftPlan plan;
  int lines_per_block;
  const DevState* ds;
  int s;
  int use_q;
  double scale;
  int mode;
  ProjCoef<T> cf;
  unsigned* res1;   // the sub-stage's residual word
  __device__ __forceinline__ void operator()(const Blk& bk) const { fft_x_fwd<T>(bk, g, f, flags32, tw, plan, lines_per_block, ds, s, use_q, scale, mode, cf, res1); }
};

// inverse x transform: two half-spectra -> one complex line -> two real rows of phi
template <typename T>
__device__ __forceinline__ void fft_x_inv(const Blk& bk, const Geo& g, const Fields<T>& f, const T* __restrict__ tw, const FftPlan& plan, int lines_per_block,
                            T* __restrict__ out_phi) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + lines_per_block * (g.nx + 1);   // lines padded to nx + 1 words (see fft_pass_r)
  const int n = g.nx, nkx = g.nkx, xs = n + 1;
  const long long rows = (long long)g.ny * g.nz;
  const long long line0 = (long long)bk.x * lines_per_block;
  const C* spec = reinterpret_cast<const C*>(f.spec);
  for (int l = threadIdx.y; l < lines_per_block; l += blockDim.y)
  for (int kx = threadIdx.x; kx < n; kx += blockDim.x) {
    const int t = l * xs + kx;
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
  const int res = fft_lines<T, true>(bufa, bufb, lines_per_block, plan, reinterpret_cast<const C*>(tw), 1, xs,
                                     magic_div_dev((unsigned)lines_per_block), true);
  const C* out = res == 0 ? bufa : bufb;
  for (int l = threadIdx.y; l < lines_per_block; l += blockDim.y)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int t = l * xs + i;
    const long long ra = 2 * (line0 + l), rb = ra + 1;
    if (ra < rows) out_phi[ra * n + i] = out[t].x;
    if (rb < rows) out_phi[rb * n + i] = out[t].y;
  }
}
template <typename T>
struct FftXInv {
  static constexpr int kThreads = 256;
  Geo g;
  Fields<T> f;
  const T* tw;
  FftPlan plan;
  int lines_per_block;
  T* out_phi;
  __device__ __forceinline__ void operator()(const Blk& bk) const { fft_x_inv<T>(bk, g, f, tw, plan, lines_per_block, out_phi); }
};

// ---------------------------------------------------------------------------
// Fused per-plane transforms: one block per y-plane j keeps the plane's x
// half-spectra [k][kx] in shared memory between the x and the z passes, so
// the forward spectrum leaves the block once and the inverse one arrives
// once (no global round trip between the two directions).  Used when the
// plane (nz * nkx complex values) and two work buffers fit.  Rows k and
// k + 1 of the plane form one complex line of the x transform.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void fft_plane_fwd(const Blk& bk, const Geo& g, const Fields<T>& f,
                                              const unsigned* __restrict__ flags32, const T* __restrict__ twx,
                                              const T* __restrict__ twz, const FftPlan& px, const FftPlan& pz, int wbuf,
                                              int cz, const DevState* ds, int s, int use_q, double scale, int mode,
                                              const ProjCoef<T>& cf, unsigned* res1) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  const int nx = g.nx, nz = g.nz, nkx = g.nkx, ny = g.ny;
  C* S = reinterpret_cast<C*>(smem_raw);   // [k][kx]
  C* bufa = S + (size_t)nz * nkx;
  C* bufb = bufa + wbuf;
  const int j = bk.x;
  const int xs = nx + 1;   // padded line stride of the x transforms (see fft_pass_r)
  const int lc = max(1, wbuf / xs);
  const T qf = use_q ? (T)ds->qf[s] : (T)0;
  const T qa = use_q == 2 ? (T)ds->qa[s] : (T)0, qb = use_q == 2 ? (T)ds->qb[s] : (T)0;
  const int nlines = nz / 2;
  const RowY<T> ry = row_y<T>(g, f, cf, j);
  if (mode == 0) clear_residual(bk, res1);
  unsigned rmax = 0u;
  // x: lc complex lines (row pairs) at a time into S
  for (int l0 = 0; l0 < nlines; l0 += lc) {
    const int nl = min(lc, nlines - l0);
    __syncthreads();
    bool paired = false;
    if constexpr (sizeof(T) == 4) {
      // FP32: two cells per thread along x, paired row loads (the first
      // solve's right-hand side, or the correction's from the (hi, lo) state)
      if ((mode == 0 && use_q != 2) || (mode == 3 && f.lo[0])) {
        paired = true;
        const int hx = nx / 2;
#pragma unroll 2
        for (int t = threadIdx.x; t < nl * hx; t += blockDim.x) {
          const int l = t / hx, i = 2 * (t - l * hx);
          const int k0 = 2 * (l0 + l);
          float a0, b0, a1, b1;
          if (mode == 0) {
            rhs_pair0(g, f, flags32, use_q, cf, ry, qf, i, j, k0, a0, b0);
            rhs_pair0(g, f, flags32, use_q, cf, ry, qf, i, j, k0 + 1, a1, b1);
          } else {
            rhs_pair3(g, f, flags32, ds, s, use_q, cf, ry, i, j, k0, a0, b0, rmax);
            rhs_pair3(g, f, flags32, ds, s, use_q, cf, ry, i, j, k0 + 1, a1, b1, rmax);
          }
          C za, zb;
          za.x = a0;
          za.y = a1;
          zb.x = b0;
          zb.y = b1;
          bufa[l * xs + i] = za;
          bufa[l * xs + i + 1] = zb;
        }
      }
    }
    if (!paired) {
#pragma unroll 4
      for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
        const int l = t / nx, i = t - l * nx;
        const int k0 = 2 * (l0 + l);
        C z;
        z.x = poisson_rhs<T>(g, f, flags32, ds, s, use_q, scale, mode, cf, ry, qf, qa, qb, i, j, k0, rmax);
        z.y = poisson_rhs<T>(g, f, flags32, ds, s, use_q, scale, mode, cf, ry, qf, qa, qb, i, j, k0 + 1, rmax);
        bufa[l * xs + i] = z;
      }
    }
    const int res = fft_lines<T, false>(bufa, bufb, nl, px, reinterpret_cast<const C*>(twx), 1, xs,
                                        magic_div_dev((unsigned)nl), true);
    const C* out = res == 0 ? bufa : bufb;
    for (int t = threadIdx.x; t < nl * nkx; t += blockDim.x) {
      const int l = t / nkx, kx = t - l * nkx;
      const C Z = out[l * xs + kx];
      const C Zc = cconj(out[l * xs + (kx == 0 ? 0 : nx - kx)]);
      C Xa, Xb;
      Xa.x = (T)0.5 * (Z.x + Zc.x);
      Xa.y = (T)0.5 * (Z.y + Zc.y);
      Xb.x = (T)0.5 * (Z.y - Zc.y);   // Xb = (Z - Zc) / (2 i)
      Xb.y = (T)-0.5 * (Z.x - Zc.x);
      const int k0 = 2 * (l0 + l);
      S[k0 * nkx + kx] = Xa;
      S[(k0 + 1) * nkx + kx] = Xb;
    }
  }
  if (mode == 3) fold_residual(res1, rmax);
  // z: cz columns at a time (any cz: the host balances the chunks), strided
  // lines in the work buffers, to global
  C* spec = reinterpret_cast<C*>(f.spec);
  const unsigned mcz = magic_div_dev(cz);
  for (int kx0 = 0; kx0 < nkx; kx0 += cz) {
    const int w = min(cz, nkx - kx0);
    __syncthreads();
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      C z;
      z.x = z.y = (T)0;
      if (c < w) z = S[k * nkx + kx0 + c];
      bufa[t] = z;
    }
    const int res = fft_lines<T, false>(bufa, bufb, cz, pz, reinterpret_cast<const C*>(twz), cz, 1, mcz);
    const C* out = res == 0 ? bufa : bufb;
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      if (c < w) spec[((long long)k * ny + j) * nkx + kx0 + c] = out[t];
    }
  }
}
template <typename T>
struct FftPlaneFwd {
  static constexpr int kThreads = 1024;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const T* twx;
  const T* twz;
  FftPlan px, pz;
  int wbuf, cz;
  const DevState* ds;
  int s, use_q;
  double scale;
  int mode;
  ProjCoef<T> cf;
  unsigned* res1;   // the sub-stage's residual word
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    fft_plane_fwd<T>(bk, g, f, flags32, twx, twz, px, pz, wbuf, cz, ds, s, use_q, scale, mode, cf, res1);
  }
};

template <typename T>
__device__ __forceinline__ void fft_plane_inv(const Blk& bk, const Geo& g, const Fields<T>& f, const T* __restrict__ twx,
                                              const T* __restrict__ twz, const FftPlan& px, const FftPlan& pz, int wbuf,
                                              int cz, T* __restrict__ out_phi) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  const int nx = g.nx, nz = g.nz, nkx = g.nkx, ny = g.ny;
  C* S = reinterpret_cast<C*>(smem_raw);   // [k][kx]
  C* bufa = S + (size_t)nz * nkx;
  C* bufb = bufa + wbuf;
  const int j = bk.x;
  const C* spec = reinterpret_cast<const C*>(f.spec);
  // z inverse: cz columns at a time from global into S
  const unsigned mcz = magic_div_dev(cz);
  for (int kx0 = 0; kx0 < nkx; kx0 += cz) {
    const int w = min(cz, nkx - kx0);
    __syncthreads();
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      C z;
      z.x = z.y = (T)0;
      if (c < w) z = spec[((long long)k * ny + j) * nkx + kx0 + c];
      bufa[t] = z;
    }
    const int res = fft_lines<T, true>(bufa, bufb, cz, pz, reinterpret_cast<const C*>(twz), cz, 1, mcz);
    const C* out = res == 0 ? bufa : bufb;
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      if (c < w) S[k * nkx + kx0 + c] = out[t];
    }
  }
  // x inverse: two half-spectra (rows k, k + 1) -> one complex line -> two real rows
  const int xs = nx + 1;   // padded line stride of the x transforms (see fft_pass_r)
  const int lc = max(1, wbuf / xs);
  const int nlines = nz / 2;
  for (int l0 = 0; l0 < nlines; l0 += lc) {
    const int nl = min(lc, nlines - l0);
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
      const int l = t / nx, kx = t - l * nx;
      const int k0 = 2 * (l0 + l);
      const bool mirror = kx >= nkx;
      const int q = mirror ? nx - kx : kx;
      C A = S[k0 * nkx + q], B = S[(k0 + 1) * nkx + q];
      if (q == 0 || 2 * q == nx) { A.y = (T)0; B.y = (T)0; }   // real DC / Nyquist bins
      if (mirror) { A = cconj(A); B = cconj(B); }
      C z;  // A + i B
      z.x = A.x - B.y;
      z.y = A.y + B.x;
      bufa[l * xs + kx] = z;
    }
    const int res = fft_lines<T, true>(bufa, bufb, nl, px, reinterpret_cast<const C*>(twx), 1, xs,
                                       magic_div_dev((unsigned)nl), true);
    const C* out = res == 0 ? bufa : bufb;
#pragma unroll 4
    for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
      const int l = t / nx, i = t - l * nx;
      const int k0 = 2 * (l0 + l);
      out_phi[((long long)k0 * ny + j) * nx + i] = out[l * xs + i].x;
      out_phi[((long long)(k0 + 1) * ny + j) * nx + i] = out[l * xs + i].y;
    }
  }
}
template <typename T>
struct FftPlaneInv {
  static constexpr int kThreads = 1024;
  Geo g;
  Fields<T> f;
  const T* twx;
  const T* twz;
  FftPlan px, pz;
  int wbuf, cz;
  T* out_phi;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    fft_plane_inv<T>(bk, g, f, twx, twz, px, pz, wbuf, cz, out_phi);
  }
};

// ---------------------------------------------------------------------------
// The per-plane transforms split over a cluster of CL blocks (distributed
// shared memory).  Block r of a plane's cluster holds rows k of
// [r nzc, (r + 1) nzc), nzc = nz / CL, of the plane's half-spectrum in its own
// shared memory.  Forward: each block forms and x-transforms its own rows,
// then, after a cluster barrier, z-transforms its share of the kx columns,
// reading every column's rows from the blocks that hold them.  Inverse: the
// z transforms write their columns' rows into the holders' shared memory,
// and after the barrier each block x-transforms its own rows.  A 128^3 plane
// then runs as 4 blocks of 256 threads with 52 KB each, several clusters
// per SM, so one block's global loads overlap another's transforms, on
// every SM.
// ---------------------------------------------------------------------------
template <typename T, int CL>
__device__ __forceinline__ void fft_plane_fwd_cl(const Blk& bk, const Geo& g, const Fields<T>& f,
                                                 const unsigned* __restrict__ flags32, const T* __restrict__ twx,
                                                 const T* __restrict__ twz, const FftPlan& px, const FftPlan& pz,
                                                 int wbuf, int cz, const DevState* ds, int s, int use_q,
                                                 double scale, int mode, const ProjCoef<T>& cf, unsigned* res1) {
  using C = typename Cplx<T>::type;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ unsigned char smem_raw[];
  const int nx = g.nx, nz = g.nz, nkx = g.nkx, ny = g.ny;
  const int r = (int)cl.block_rank();
  const int j = (int)(bk.x / CL);
  const int nzc = nz / CL;
  C* S = reinterpret_cast<C*>(smem_raw);   // [k - r nzc][kx]
  C* bufa = S + (size_t)nzc * nkx;
  C* bufb = bufa + wbuf;
  const int xs = nx + 1;   // padded line stride of the x transforms (see fft_pass_r)
  const int lc = max(1, wbuf / xs);
  const T qf = use_q ? (T)ds->qf[s] : (T)0;
  const T qa = use_q == 2 ? (T)ds->qa[s] : (T)0, qb = use_q == 2 ? (T)ds->qb[s] : (T)0;
  const int nlines = nzc / 2;
  const RowY<T> ry = row_y<T>(g, f, cf, j);
  if (mode == 0) clear_residual(bk, res1);
  unsigned rmax = 0u;
  // x: this block's rows, lc complex lines (row pairs) at a time
  for (int l0 = 0; l0 < nlines; l0 += lc) {
    const int nl = min(lc, nlines - l0);
    __syncthreads();
#pragma unroll 4
    for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
      const int l = t / nx, i = t - l * nx;
      const int k0 = r * nzc + 2 * (l0 + l);
      C z;
      z.x = poisson_rhs<T>(g, f, flags32, ds, s, use_q, scale, mode, cf, ry, qf, qa, qb, i, j, k0, rmax);
      z.y = poisson_rhs<T>(g, f, flags32, ds, s, use_q, scale, mode, cf, ry, qf, qa, qb, i, j, k0 + 1, rmax);
      bufa[l * xs + i] = z;
    }
    const int res = fft_lines<T, false>(bufa, bufb, nl, px, reinterpret_cast<const C*>(twx), 1, xs,
                                        magic_div_dev((unsigned)nl), true);
    const C* out = res == 0 ? bufa : bufb;
    for (int t = threadIdx.x; t < nl * nkx; t += blockDim.x) {
      const int l = t / nkx, kx = t - l * nkx;
      const C Z = out[l * xs + kx];
      const C Zc = cconj(out[l * xs + (kx == 0 ? 0 : nx - kx)]);
      C Xa, Xb;
      Xa.x = (T)0.5 * (Z.x + Zc.x);
      Xa.y = (T)0.5 * (Z.y + Zc.y);
      Xb.x = (T)0.5 * (Z.y - Zc.y);   // Xb = (Z - Zc) / (2 i)
      Xb.y = (T)-0.5 * (Z.x - Zc.x);
      const int kl = 2 * (l0 + l);
      S[kl * nkx + kx] = Xa;
      S[(kl + 1) * nkx + kx] = Xb;
    }
  }
  if (mode == 3) fold_residual(res1, rmax);
  cl.sync();   // every block's rows are in its shared memory
  // z: this block's columns [c0, c1), cz at a time, gathered from the holders
  const int cw = (nkx + CL - 1) / CL;
  const int c0 = r * cw, c1 = min(nkx, c0 + cw);
  const unsigned mcz = magic_div_dev(cz);
  C* spec = reinterpret_cast<C*>(f.spec);
  for (int kx0 = c0; kx0 < c1; kx0 += cz) {
    const int w = min(cz, c1 - kx0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < CL; ++q) {
      const C* Sq = cl.map_shared_rank(S, q);
      C* dst = bufa + (size_t)q * nzc * cz;
      for (int t = threadIdx.x; t < nzc * cz; t += blockDim.x) {
        const int kl = (int)fdiv((unsigned)t, mcz), c = t - kl * cz;
        C z;
        z.x = z.y = (T)0;
        if (c < w) z = Sq[kl * nkx + kx0 + c];
        dst[t] = z;
      }
    }
    const int res = fft_lines<T, false>(bufa, bufb, cz, pz, reinterpret_cast<const C*>(twz), cz, 1, mcz);
    const C* out = res == 0 ? bufa : bufb;
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      if (c < w) spec[((long long)k * ny + j) * nkx + kx0 + c] = out[t];
    }
  }
  cl.sync();   // no block leaves while a peer may still read its rows
}
template <typename T, int CL>
struct FftPlaneFwdCl {
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const T* twx;
  const T* twz;
  FftPlan px, pz;
  int wbuf, cz;
  const DevState* ds;
  int s, use_q;
  double scale;
  int mode;
  ProjCoef<T> cf;
  unsigned* res1;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    fft_plane_fwd_cl<T, CL>(bk, g, f, flags32, twx, twz, px, pz, wbuf, cz, ds, s, use_q, scale, mode, cf, res1);
  }
};

template <typename T, int CL>
__device__ __forceinline__ void fft_plane_inv_cl(const Blk& bk, const Geo& g, const Fields<T>& f,
                                                 const T* __restrict__ twx, const T* __restrict__ twz,
                                                 const FftPlan& px, const FftPlan& pz, int wbuf, int cz,
                                                 T* __restrict__ out_phi) {
  using C = typename Cplx<T>::type;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ unsigned char smem_raw[];
  const int nx = g.nx, nz = g.nz, nkx = g.nkx, ny = g.ny;
  const int r = (int)cl.block_rank();
  const int j = (int)(bk.x / CL);
  const int nzc = nz / CL;
  C* S = reinterpret_cast<C*>(smem_raw);   // [k - r nzc][kx]
  C* bufa = S + (size_t)nzc * nkx;
  C* bufb = bufa + wbuf;
  const C* spec = reinterpret_cast<const C*>(f.spec);
  // z inverse: this block's columns from global, into the holders' rows
  const int cw = (nkx + CL - 1) / CL;
  const int c0 = r * cw, c1 = min(nkx, c0 + cw);
  const unsigned mcz = magic_div_dev(cz);
  for (int kx0 = c0; kx0 < c1; kx0 += cz) {
    const int w = min(cz, c1 - kx0);
    __syncthreads();
#pragma unroll 4
    for (int t = threadIdx.x; t < nz * cz; t += blockDim.x) {
      const int k = (int)fdiv((unsigned)t, mcz), c = t - k * cz;
      C z;
      z.x = z.y = (T)0;
      if (c < w) z = spec[((long long)k * ny + j) * nkx + kx0 + c];
      bufa[t] = z;
    }
    const int res = fft_lines<T, true>(bufa, bufb, cz, pz, reinterpret_cast<const C*>(twz), cz, 1, mcz);
    const C* out = res == 0 ? bufa : bufb;
#pragma unroll
    for (int q = 0; q < CL; ++q) {
      C* Sq = cl.map_shared_rank(S, q);
      const C* src = out + (size_t)q * nzc * cz;
      for (int t = threadIdx.x; t < nzc * cz; t += blockDim.x) {
        const int kl = (int)fdiv((unsigned)t, mcz), c = t - kl * cz;
        if (c < w) Sq[kl * nkx + kx0 + c] = src[t];
      }
    }
  }
  cl.sync();   // every block's rows are complete (written by the whole cluster)
  // x inverse: two half-spectra (rows k, k + 1) -> one complex line -> two real rows
  const int xs = nx + 1;   // padded line stride of the x transforms (see fft_pass_r)
  const int lc = max(1, wbuf / xs);
  const int nlines = nzc / 2;
  for (int l0 = 0; l0 < nlines; l0 += lc) {
    const int nl = min(lc, nlines - l0);
    __syncthreads();
    for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
      const int l = t / nx, kx = t - l * nx;
      const int kl = 2 * (l0 + l);
      const bool mirror = kx >= nkx;
      const int q = mirror ? nx - kx : kx;
      C A = S[kl * nkx + q], B = S[(kl + 1) * nkx + q];
      if (q == 0 || 2 * q == nx) { A.y = (T)0; B.y = (T)0; }   // real DC / Nyquist bins
      if (mirror) { A = cconj(A); B = cconj(B); }
      C z;  // A + i B
      z.x = A.x - B.y;
      z.y = A.y + B.x;
      bufa[l * xs + kx] = z;
    }
    const int res = fft_lines<T, true>(bufa, bufb, nl, px, reinterpret_cast<const C*>(twx), 1, xs,
                                       magic_div_dev((unsigned)nl), true);
    const C* out = res == 0 ? bufa : bufb;
#pragma unroll 4
    for (int t = threadIdx.x; t < nl * nx; t += blockDim.x) {
      const int l = t / nx, i = t - l * nx;
      const int k0 = r * nzc + 2 * (l0 + l);
      out_phi[((long long)k0 * ny + j) * nx + i] = out[l * xs + i].x;
      out_phi[((long long)(k0 + 1) * ny + j) * nx + i] = out[l * xs + i].y;
    }
  }
}
template <typename T, int CL>
struct FftPlaneInvCl {
  static constexpr int kThreads = 256;
  static constexpr int kMinBlocks = 4;
  Geo g;
  Fields<T> f;
  const T* twx;
  const T* twz;
  FftPlan px, pz;
  int wbuf, cz;
  T* out_phi;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    fft_plane_inv_cl<T, CL>(bk, g, f, twx, twz, px, pz, wbuf, cz, out_phi);
  }
};

// z transform of the half-spectrum, in place; a block takes `cols` adjacent
// kx columns of one y-plane (coalesced rows of `cols` complex values), kept
// in shared memory in load order [k][column] and transformed as strided
// lines (no bank conflicts on load, store or butterflies).  cols is a power
// of two.
template <typename T, bool INV>
__device__ __forceinline__ void fft_z(const Blk& bk, const Geo& g, const Fields<T>& f, const T* __restrict__ tw, const FftPlan& plan, int cols) {
  using C = typename Cplx<T>::type;
  extern __shared__ unsigned char smem_raw[];
  C* bufa = reinterpret_cast<C*>(smem_raw);
  C* bufb = bufa + cols * g.nz;
  const int n = g.nz, nkx = g.nkx;
  const int ntile = (nkx + cols - 1) / cols;
  const int j = bk.x / ntile;
  const int kx0 = (bk.x - j * ntile) * cols;
  const int w = min(cols, nkx - kx0);
  const int lc = __ffs(cols) - 1;
  C* spec = reinterpret_cast<C*>(f.spec);
  for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
    const int k = t >> lc, c = t & (cols - 1);
    C z;
    z.x = z.y = (T)0;
    if (c < w) z = spec[((long long)k * g.ny + j) * nkx + kx0 + c];
    bufa[t] = z;
  }
  const int res = fft_lines<T, INV>(bufa, bufb, cols, plan, reinterpret_cast<const C*>(tw), cols, 1,
                                    magic_div_dev(cols));
  const C* out = res == 0 ? bufa : bufb;
  for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
    const int k = t >> lc, c = t & (cols - 1);
    if (c < w) spec[((long long)k * g.ny + j) * nkx + kx0 + c] = out[t];
  }
}
template <typename T, bool INV>
struct FftZ {
  static constexpr int kThreads = 256;
  Geo g;
  Fields<T> f;
  const T* tw;
  FftPlan plan;
  int cols;
  __device__ __forceinline__ void operator()(const Blk& bk) const { fft_z<T, INV>(bk, g, f, tw, plan, cols); }
};

// ---------------------------------------------------------------------------
// Wall-normal Thomas per wavenumber pair (kx, kz), FP64:
//   (phi_{j+1} - 2 phi_j + phi_{j-1})/dy^2 - (lx + lz) phi_j = r_j,
// Neumann rows at both walls; mode (0,0) pins phi_0 = 0 and removes the
// mean over j afterwards (zero-mean gauge).  Pivots are tabulated.
// ---------------------------------------------------------------------------
// FP32 spectrum value -> FP64 on the integer pipes (FP64 spectrum: as is);
// `special` collects the inputs the integer path leaves to the hardware.
__device__ __forceinline__ double widen(float v, bool& special) { return f2d_int(v, special); }
__device__ __forceinline__ double widen(double v, bool&) { return v; }
__device__ __forceinline__ float narrow_to(float*, double v, bool& special) { return d2f_int(v, special); }
__device__ __forceinline__ double narrow_to(double*, double v, bool&) { return v; }

template <typename T>
__device__ __forceinline__ void tri_y(const Blk& bk, const Geo& g, const Fields<T>& f, const double* __restrict__ cp,
                                               const double* __restrict__ inv, double* fwd) {
  // one thread per real or imaginary part of a (kx, kz) system: the two
  // share the pivots and are independent.  Only the recurrences use the FP64
  // pipe (one FMA and one multiply forward, one FMA backward per row): the
  // FP32 spectrum is widened and narrowed on the integer pipes, and every
  // load of the next batch of rows is issued before the current batch's
  // recurrence, so a warp that holds its SM sub-partition alone still
  // overlaps its loads with its arithmetic.
  const int nkx = g.nkx, ny = g.ny;
  const unsigned FULL = 0xFFFFFFFFu;
  const long long l = bk.x * (long long)blockDim.x + threadIdx.x;
  const bool live = l < 2ll * nkx * g.nz;       // whole warps stay in the loops (warp votes)
  const int part = (int)(l & 1);
  const long long mode = live ? l >> 1 : 0;
  const long long kx = mode % nkx, kz = mode / nkx;
  const long long base = kz * (long long)ny * nkx + kx, stride = nkx;
  T* __restrict__ sp = reinterpret_cast<T*>(f.spec);
  // forward values stay FP64: in place for the FP64 path, in an FP64 scratch
  // spectrum for the mixed path
  double* __restrict__ F = fwd ? fwd : reinterpret_cast<double*>(f.spec);
  const double a = g.idy * g.idy;
  const bool singular = live && kx == 0 && kz == 0;
  constexpr int B = 8;   // rows per batch
  auto at = [&](int j) { return 2 * (base + (long long)j * stride) + part; };
  // ---- forward: p_j = (r_j - a p_{j-1}) / piv_j
  double zc[B], ic[B];
  bool special = false;
#pragma unroll
  for (int u = 0; u < B; ++u)
    if (live && u < ny) {
      zc[u] = widen(sp[at(u)], special);
      ic[u] = __ldg(inv + base + (long long)u * stride);
    }
  double pr = 0.0;
  for (int j0 = 0; j0 < ny; j0 += B) {
    double zn[B], in[B];
    bool sn = false;
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (live && j0 + B + u < ny) {
        zn[u] = widen(sp[at(j0 + B + u)], sn);
        in[u] = __ldg(inv + base + (long long)(j0 + B + u) * stride);
      }
    if (sizeof(T) == 4 && __any_sync(FULL, special)) {   // subnormal, infinite or NaN inputs: hardware widening
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (live && j0 + u < ny) zc[u] = (double)sp[at(j0 + u)];
    }
    if (j0 == 0 && singular) zc[0] = 0.0;   // pinned phi_0 of the (0,0) mode
    // (row 0 takes the same formula: p_{-1} = 0 leaves r_0 / piv_0)
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (live && j0 + u < ny) {
        pr = (zc[u] - a * pr) * ic[u];
        F[at(j0 + u)] = pr;
      }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      zc[u] = zn[u];
      ic[u] = in[u];
    }
    special = sn;
  }
  // ---- backward: x_j = p_j - c'_j x_{j+1}
  double xr = pr, sr = pr;
  if (live) {
    bool s0 = false;
    const T o = narrow_to((T*)nullptr, xr, s0);
    sp[at(ny - 1)] = s0 ? (T)xr : o;
  }
  double fc[B], cc[B];
#pragma unroll
  for (int u = 0; u < B; ++u)
    if (live && ny - 2 - u >= 0) {
      fc[u] = F[at(ny - 2 - u)];
      cc[u] = __ldg(cp + base + (long long)(ny - 2 - u) * stride);
    }
  for (int j1 = ny - 2; j1 >= 0; j1 -= B) {
    double fn[B], cn[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (live && j1 - B - u >= 0) {
        fn[u] = F[at(j1 - B - u)];
        cn[u] = __ldg(cp + base + (long long)(j1 - B - u) * stride);
      }
    double xs[B];
    bool so = false;
    T ob[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (live && j1 - u >= 0) {
        xr = fc[u] - cc[u] * xr;
        xs[u] = xr;
        ob[u] = narrow_to((T*)nullptr, xr, so);
        if (singular) sr += xr;
      }
    if (sizeof(T) == 4 && __any_sync(FULL, so)) {   // results outside the normal FP32 range: hardware narrowing
#pragma unroll
      for (int u = 0; u < B; ++u)
        if (live && j1 - u >= 0) ob[u] = (T)xs[u];
    }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (live && j1 - u >= 0) {
        sp[at(j1 - u)] = ob[u];
        if (singular) F[at(j1 - u)] = xs[u];
      }
#pragma unroll
    for (int u = 0; u < B; ++u) {
      fc[u] = fn[u];
      cc[u] = cn[u];
    }
  }
  if (singular) {
    // zero-mean gauge, from the FP64 values
    const double mr = sr / ny;
    for (int j = 0; j < ny; ++j) {
      const double v = (j == ny - 1) ? pr : F[at(j)];
      sp[at(j)] = (T)(v - mr);
    }
  }
}
// Per-wavenumber Thomas on a non-uniform wall-normal grid (FP64 path, one
// thread per real or imaginary part).  Row j of Eq. elliptic is scaled by
// the cell height, which makes the matrix symmetric: sub = 1/hf_j,
// super = 1/hf_{j+1}, diagonal -(sub + super) - lambda hc_j.  Tables: ivh_j =
// hc_j / pivot_j (the scaled right-hand side folded in), al_j = -sub_j /
// pivot_j, c'_j.  Mode (0,0) pins phi_0 = 0 (its row 0 has zero entries),
// then removes the volume-weighted mean over j.
template <typename T>
__device__ __forceinline__ void tri_y_nu(const Blk& bk, const Geo& g, const Fields<T>& f, const double* __restrict__ cp,
                                         const double* __restrict__ ivh, const double* __restrict__ al) {
  const long long l = (long long)bk.x * blockDim.x + threadIdx.x;
  const int nkx = g.nkx;
  if (l >= 2ll * nkx * g.nz) return;
  const int part = (int)(l & 1);
  const long long mode = l >> 1;
  const long long kx = mode % nkx, kz = mode / nkx;
  const long long base = kz * (long long)g.ny * nkx + kx, stride = nkx;
  T* __restrict__ sp = reinterpret_cast<T*>(f.spec);
  const bool singular = kx == 0 && kz == 0;
  double pr = 0.0;
  for (int j = 0; j < g.ny; ++j) {
    const long long id = base + (long long)j * stride;
    pr = fma(__ldg(al + id), pr, (double)sp[2 * id + part] * __ldg(ivh + id));
    sp[2 * id + part] = (T)pr;
  }
  double x = pr, sw = pr * g.yt.hc[g.ny - 1];
  for (int j = g.ny - 2; j >= 0; --j) {
    const long long id = base + (long long)j * stride;
    x = (double)sp[2 * id + part] - __ldg(cp + id) * x;
    sp[2 * id + part] = (T)x;
    sw += x * g.yt.hc[j];
  }
  if (singular) {
    const double mean = sw / g.ly;
    for (int j = 0; j < g.ny; ++j) {
      const long long id = base + (long long)j * stride;
      sp[2 * id + part] = (T)((double)sp[2 * id + part] - mean);
    }
  }
}
template <typename T>
struct TriYNU {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const double* cp;
  const double* ivh;
  const double* al;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_y_nu<T>(bk, g, f, cp, ivh, al); }
};

// The same systems warp-cooperatively (non-uniform wall-normal spacing): L
// lanes per (kx, kz) system, TRI_SEG rows per lane.  Forward p_j = al_j
// p_{j-1} + r_j / pivot_j and backward x_j = p_j - c'_j x_{j+1} are affine
// maps: each lane composes its rows' maps (the products formed here from the
// rows' multipliers), a shuffle scan over the lanes composes the prefixes,
// and each lane then replays its rows from its incoming value.  The (0,0)
// system takes the volume-weighted zero-mean gauge, as the sequential form.
template <typename T, int L>
__device__ __forceinline__ void tri_y_warp_nu(const Blk& bk, const Geo& g, const Fields<T>& f,
                                              const double* __restrict__ cp, const double* __restrict__ ivh,
                                              const double* __restrict__ al) {
  using C = typename Cplx<T>::type;
  constexpr int Rr = TRI_SEG;
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31;
  const int sl = lane % L;
  const int nkx = g.nkx, ny = g.ny;
  const int groups_x = (nkx + G - 1) / G;
  const long long wid = ((long long)bk.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)groups_x * g.nz) return;     // whole warps only
  const int kz = (int)(wid / groups_x);
  const int kx = (int)(wid % groups_x) * G + lane / L;
  const bool live = kx < nkx;
  const long long base = (long long)kz * ny * nkx + (live ? kx : 0);
  const long long stride = nkx;
  C* spec = reinterpret_cast<C*>(f.spec);
  const bool singular = live && kx == 0 && kz == 0;
  const bool gauge = kz == 0 && (int)(wid % groups_x) == 0;   // warp of the (0,0) system
  const int j0 = sl * Rr;
  const unsigned FULL = 0xFFFFFFFFu;
  double br[Rr], bi[Rr], am[Rr], cq[Rr];
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    br[u] = bi[u] = cq[u] = 0.0;
    am[u] = 1.0;
    if (live && j < ny) {
      const long long id = base + (long long)j * stride;
      const C z = spec[id];
      const double iv = __ldg(ivh + id);
      am[u] = __ldg(al + id);
      cq[u] = __ldg(cp + id);
      br[u] = (double)z.x * iv;
      bi[u] = (double)z.y * iv;
    }
  }
  // ---- forward: the lane's composite map p -> A p + B
  double A = 1.0, Br = 0.0, Bi = 0.0;
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    Br = fma(am[u], Br, br[u]);
    Bi = fma(am[u], Bi, bi[u]);
    A = A * am[u];
  }
  for (int o = 1; o < L; o <<= 1) {
    const double pa = __shfl_up_sync(FULL, A, o, L), pr = __shfl_up_sync(FULL, Br, o, L),
                 pi = __shfl_up_sync(FULL, Bi, o, L);
    if (sl >= o) {
      Br = fma(A, pr, Br);
      Bi = fma(A, pi, Bi);
      A = A * pa;
    }
  }
  double pr = __shfl_up_sync(FULL, Br, 1, L), pi = __shfl_up_sync(FULL, Bi, 1, L);
  if (sl == 0) { pr = 0.0; pi = 0.0; }
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    pr = fma(am[u], pr, br[u]);
    pi = fma(am[u], pi, bi[u]);
    br[u] = pr;
    bi[u] = pi;
  }
  // ---- backward: the lane's composite map from the row above its top row
  A = 1.0;
  Br = 0.0;
  Bi = 0.0;
#pragma unroll
  for (int u = Rr - 1; u >= 0; --u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == ny - 1) {   // the top row: x = p
      A = 0.0;
      Br = br[u];
      Bi = bi[u];
    } else {
      Br = fma(-cq[u], Br, br[u]);
      Bi = fma(-cq[u], Bi, bi[u]);
      A = A * -cq[u];
    }
  }
  for (int o = 1; o < L; o <<= 1) {
    const double na = __shfl_down_sync(FULL, A, o, L), nr = __shfl_down_sync(FULL, Br, o, L),
                 ni = __shfl_down_sync(FULL, Bi, o, L);
    if (sl + o < L) {
      Br = fma(A, nr, Br);
      Bi = fma(A, ni, Bi);
      A = A * na;
    }
  }
  double xr = __shfl_down_sync(FULL, Br, 1, L), xi = __shfl_down_sync(FULL, Bi, 1, L);
  if (sl == L - 1) { xr = 0.0; xi = 0.0; }
  double sr = 0.0, si = 0.0;
#pragma unroll
  for (int u = Rr - 1; u >= 0; --u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == ny - 1) {
      xr = br[u];
      xi = bi[u];
    } else {
      xr = fma(-cq[u], xr, br[u]);
      xi = fma(-cq[u], xi, bi[u]);
    }
    br[u] = xr;
    bi[u] = xi;
    if (gauge) {
      sr = fma(xr, g.yt.hc[j], sr);
      si = fma(xi, g.yt.hc[j], si);
    }
  }
  if (gauge) {
    // volume-weighted zero mean of the (0,0) system (first group of kz = 0)
    for (int o = 1; o < L; o <<= 1) {
      sr += __shfl_xor_sync(FULL, sr, o, L);
      si += __shfl_xor_sync(FULL, si, o, L);
    }
    if (singular) {
      const double mr = sr / g.ly, mi = si / g.ly;
#pragma unroll
      for (int u = 0; u < Rr; ++u) {
        br[u] -= mr;
        bi[u] -= mi;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    C o;
    o.x = (T)br[u];
    o.y = (T)bi[u];
    if (live && j < ny) spec[base + (long long)j * stride] = o;
  }
}
template <typename T, int L>
struct TriYWarpNU {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const double* cp;
  const double* ivh;
  const double* al;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_y_warp_nu<T, L>(bk, g, f, cp, ivh, al); }
};

template <typename T>
struct TriY {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const double* cp;
  const double* inv;
  double* fwd;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_y<T>(bk, g, f, cp, inv, fwd); }
};

// Warp-cooperative variant: a warp holds G = 32/L consecutive kx of one kz,
// L lanes per system, each lane TRI_SEG consecutive rows of j in registers
// (so a warp load touches whole 32-byte sectors of G adjacent wavenumbers).
// Both Thomas passes are affine recurrences with real multipliers,
//   forward  p_j = -c'_j p_{j-1} + r_j / piv_j   (c'_j = a / piv_j, a = 1/dy^2)
//   backward x_j = -c'_j x_{j+1} + p_j,
// composed per lane, then across the L lanes of a system by a segmented
// shuffle scan, in FP64.  The multiplier products of each lane's rows depend
// on the wavenumber only and are tabulated (segf, segb), so a row costs one
// FMA per part and pass in the compositions and one in each recurrence.  A
// lane issues the loads of all its rows before the first use; no forward
// values leave the registers.
template <typename T, int L>
__device__ __forceinline__ void tri_y_warp(const Blk& bk, const Geo& g, const Fields<T>& f, const double* __restrict__ cp,
                                           const double* __restrict__ inv, const double* __restrict__ segf,
                                           const double* __restrict__ segb, const int* __restrict__ jcv) {
  using C = typename Cplx<T>::type;
  constexpr int Rr = TRI_SEG;
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31;
  const int sl = lane % L;                      // lane inside its system
  const int nkx = g.nkx, ny = g.ny;
  const int nseg = (ny + Rr - 1) / Rr;
  const int groups_x = (nkx + G - 1) / G;
  const long long wid = ((long long)bk.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)groups_x * g.nz) return;     // whole warps only
  const int kz = (int)(wid / groups_x);
  const int kx = (int)(wid % groups_x) * G + lane / L;
  const bool live = kx < nkx;
  const long long base = (long long)kz * ny * nkx + (live ? kx : 0);
  const long long stride = nkx;
  C* spec = reinterpret_cast<C*>(f.spec);
  const bool singular = live && kx == 0 && kz == 0;
  const bool gauge = kz == 0 && (int)(wid % groups_x) == 0;   // warp of the (0,0) system
  const int j0 = sl * Rr;
  const bool rows = live && j0 < ny;            // the lane holds at least one row
  const unsigned FULL = 0xFFFFFFFFu;
  // rows jc .. ny-2 share one (1/pivot, c') pair, read once
  const int jc = live ? __ldg(jcv + (long long)kz * nkx + kx) : ny;
  double ivc = 0.0, cpc = 0.0;
  if (live && jc < ny - 1 && j0 + Rr > jc) {
    const long long idc = base + (long long)jc * stride;
    ivc = __ldg(inv + idc);
    cpc = __ldg(cp + idc);
  }
  // ---- every load of the lane's rows, issued together; br = r / piv
  double br[Rr], bi[Rr], cq[Rr];
  bool special = false;   // an FP32 input the integer conversion leaves to the hardware
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    br[u] = bi[u] = cq[u] = 0.0;
    if (live && j < ny) {
      const long long id = base + (long long)j * stride;
      const C z = spec[id];
      const bool tab = j < jc || j == ny - 1;
      const double iv = tab ? __ldg(inv + id) : ivc;
      cq[u] = tab ? __ldg(cp + id) : cpc;
      if constexpr (sizeof(T) == 4) {
        br[u] = f2d_int(z.x, special) * iv;
        bi[u] = f2d_int(z.y, special) * iv;
      } else {
        br[u] = (double)z.x * iv;
        bi[u] = (double)z.y * iv;
      }
    }
  }
  if (sizeof(T) == 4 && __any_sync(FULL, special)) {
#pragma unroll
    for (int u = 0; u < Rr; ++u) {
      const int j = j0 + u;
      if (live && j < ny) {
        const long long id = base + (long long)j * stride;
        const C z = spec[id];
        const double iv = (j < jc || j == ny - 1) ? __ldg(inv + id) : ivc;
        br[u] = (double)z.x * iv;
        bi[u] = (double)z.y * iv;
      }
    }
  }
  if (singular && j0 == 0) br[0] = bi[0] = 0.0;   // pinned phi_0 of the (0,0) mode
  const long long sid = ((long long)kz * nseg + sl) * nkx + (live ? kx : 0);
  // ---- forward: compose the lane's maps
  double A = rows ? __ldg(segf + sid) : 1.0, Br = 0.0, Bi = 0.0;
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == 0) {
      Br = br[u];
      Bi = bi[u];
    } else {
      Br = fma(-cq[u], Br, br[u]);
      Bi = fma(-cq[u], Bi, bi[u]);
    }
  }
  for (int o = 1; o < L; o <<= 1) {
    const double pa = __shfl_up_sync(FULL, A, o, L), pr = __shfl_up_sync(FULL, Br, o, L),
                 pi = __shfl_up_sync(FULL, Bi, o, L);
    if (sl >= o) {
      Br = fma(A, pr, Br);
      Bi = fma(A, pi, Bi);
      A = A * pa;
    }
  }
  double pr = __shfl_up_sync(FULL, Br, 1, L), pi = __shfl_up_sync(FULL, Bi, 1, L);
  if (sl == 0) { pr = 0.0; pi = 0.0; }
  // forward values p_j, in place of br
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == 0) {
      pr = br[u];
      pi = bi[u];
    } else {
      pr = fma(-cq[u], pr, br[u]);
      pi = fma(-cq[u], pi, bi[u]);
    }
    br[u] = pr;
    bi[u] = pi;
  }
  // ---- backward: compose from the top row of the lane down
  A = rows ? __ldg(segb + sid) : 1.0;
  Br = 0.0;
  Bi = 0.0;
#pragma unroll
  for (int u = Rr - 1; u >= 0; --u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == ny - 1) {
      Br = br[u];
      Bi = bi[u];
    } else {
      Br = fma(-cq[u], Br, br[u]);
      Bi = fma(-cq[u], Bi, bi[u]);
    }
  }
  for (int o = 1; o < L; o <<= 1) {
    const double na = __shfl_down_sync(FULL, A, o, L), nr = __shfl_down_sync(FULL, Br, o, L),
                 ni = __shfl_down_sync(FULL, Bi, o, L);
    if (sl + o < L) {
      Br = fma(A, nr, Br);
      Bi = fma(A, ni, Bi);
      A = A * na;
    }
  }
  double xr = __shfl_down_sync(FULL, Br, 1, L), xi = __shfl_down_sync(FULL, Bi, 1, L);
  if (sl == L - 1) { xr = 0.0; xi = 0.0; }
  double sr = 0.0, si = 0.0;
#pragma unroll
  for (int u = Rr - 1; u >= 0; --u) {
    const int j = j0 + u;
    if (!live || j >= ny) continue;
    if (j == ny - 1) {
      xr = br[u];
      xi = bi[u];
    } else {
      xr = fma(-cq[u], xr, br[u]);
      xi = fma(-cq[u], xi, bi[u]);
    }
    br[u] = xr;
    bi[u] = xi;
    if (gauge) {
      sr += xr;
      si += xi;
    }
  }
  if (gauge) {
    // the (0,0) system lives in the first group of kz = 0: zero-mean gauge
    for (int o = 1; o < L; o <<= 1) {
      sr += __shfl_xor_sync(FULL, sr, o, L);
      si += __shfl_xor_sync(FULL, si, o, L);
    }
    if (singular) {
      const double mr = sr / ny, mi = si / ny;
#pragma unroll
      for (int u = 0; u < Rr; ++u) {
        br[u] -= mr;
        bi[u] -= mi;
      }
    }
  }
  special = false;
#pragma unroll
  for (int u = 0; u < Rr; ++u) {
    const int j = j0 + u;
    C o;
    if constexpr (sizeof(T) == 4) {
      o.x = d2f_int(br[u], special);
      o.y = d2f_int(bi[u], special);
    } else {
      o.x = (T)br[u];
      o.y = (T)bi[u];
    }
    if (live && j < ny) spec[base + (long long)j * stride] = o;
  }
  if (sizeof(T) == 4 && __any_sync(FULL, special)) {
    // a value outside the normal binary32 range: store the hardware results
#pragma unroll
    for (int u = 0; u < Rr; ++u) {
      const int j = j0 + u;
      C o;
      o.x = (T)br[u];
      o.y = (T)bi[u];
      if (live && j < ny) spec[base + (long long)j * stride] = o;
    }
  }
}
template <typename T, int L, int MB = 1>
struct TriYWarp {
  static constexpr int kThreads = 128;
  static constexpr int kMinBlocks = MB;   // 7: registers capped so 7 blocks fit an SM
  Geo g;
  Fields<T> f;
  const double* cp;
  const double* inv;
  const double* segf;
  const double* segb;
  const int* jc;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_y_warp<T, L>(bk, g, f, cp, inv, segf, segb, jc); }
};

// Sequential Thomas per (kx, kz, part) with the forward values in shared
// memory: the fewest FP64 operations per row (forward: one FMA and one
// multiply; backward: one FMA), no scratch traffic, loads issued 16 rows at
// a time.  Block: `blockDim.x` systems (consecutive kx, real and imaginary
// parts interleaved, so loads of the spectrum are coalesced); shared memory
// [row][thread] FP64.
template <typename T>
__device__ __forceinline__ void tri_y_smem(const Blk& bk, const Geo& g, const Fields<T>& f, const double* __restrict__ cp,
                                           const double* __restrict__ inv) {
  extern __shared__ unsigned char smem_raw[];
  double* fw = reinterpret_cast<double*>(smem_raw);
  const int nkx = g.nkx, ny = g.ny, nt = blockDim.x, tid = threadIdx.x;
  const long long l = (long long)bk.x * blockDim.x + threadIdx.x;
  if (l >= 2ll * nkx * g.nz) return;   // no barrier below: early exit is safe
  const int part = (int)(l & 1);
  const long long mode = l >> 1;
  const long long kx = mode % nkx, kz = mode / nkx;
  const long long base = kz * (long long)ny * nkx + kx, stride = nkx;
  T* __restrict__ sp = reinterpret_cast<T*>(f.spec);
  const double a = g.idy * g.idy;
  const bool singular = (kx == 0 && kz == 0);
  constexpr int B = 16;
  double pr = 0.0;
  for (int j0 = 0; j0 < ny; j0 += B) {
    double zb[B], ib[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j0 + u < ny) {
        const long long id = base + (long long)(j0 + u) * stride;
        zb[u] = (double)sp[2 * id + part];
        ib[u] = __ldg(inv + id);
      }
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j0 + u < ny) {
        const int j = j0 + u;
        pr = (j == 0) ? (singular ? 0.0 : zb[u] * ib[u]) : (zb[u] - a * pr) * ib[u];
        fw[j * nt + tid] = pr;
      }
  }
  double x = pr, sr = pr;
  if (!singular) sp[2 * (base + (long long)(ny - 1) * stride) + part] = (T)x;
  for (int j1 = ny - 2; j1 >= 0; j1 -= B) {
    double cb[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j1 - u >= 0) cb[u] = __ldg(cp + base + (long long)(j1 - u) * stride);
#pragma unroll
    for (int u = 0; u < B; ++u)
      if (j1 - u >= 0) {
        const int j = j1 - u;
        x = fw[j * nt + tid] - cb[u] * x;
        if (singular) {
          fw[j * nt + tid] = x;
          sr += x;
        } else {
          sp[2 * (base + (long long)j * stride) + part] = (T)x;
        }
      }
  }
  if (singular) {
    // zero-mean gauge of the (0, 0) system, from the FP64 values
    fw[(ny - 1) * nt + tid] = pr;
    const double mr = sr / ny;
    for (int j = 0; j < ny; ++j) sp[2 * (base + (long long)j * stride) + part] = (T)(fw[j * nt + tid] - mr);
  }
}
template <typename T>
struct TriYSmem {
  static constexpr int kThreads = 64;
  Geo g;
  Fields<T> f;
  const double* cp;
  const double* inv;
  __device__ __forceinline__ void operator()(const Blk& bk) const { tri_y_smem<T>(bk, g, f, cp, inv); }
};

// Tabulate the pivots of every (kx, kz) system once per grid.
__global__ void k_build_tri_tables(Geo g, const double* __restrict__ lamx, const double* __restrict__ lamz,
                                   double* cp, double* inv, double* segf, double* segb, int* jc) {
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
    // the last row has no super-diagonal; its entry holds a / pivot, the
    // multiplier of its forward step (no backward step reads it)
    cp[base + (long long)j * stride] = j == g.ny - 1 ? a * iv : cprev;
  }
  // With lam > 0 the pivots of the constant-coefficient rows converge
  // geometrically in j and reach a fixed point in FP64 well before the last
  // row for all but the smallest wavenumbers.  The run of rows that repeat
  // row ny - 2's pair exactly, bit for bit, is found here; the solve holds
  // that pair in registers instead of reading it per row.
  int j1 = g.ny - 1;
  if (g.ny >= 3) {
    const long long e = base + (long long)(g.ny - 2) * stride;
    const long long ive = __double_as_longlong(inv[e]), cpe = __double_as_longlong(cp[e]);
    j1 = g.ny - 2;
    while (j1 > 1 && __double_as_longlong(inv[base + (long long)(j1 - 1) * stride]) == ive &&
           __double_as_longlong(cp[base + (long long)(j1 - 1) * stride]) == cpe)
      --j1;
  }
  jc[l] = j1;
  // products of the forward (-c'_j, j > 0) and backward (-c'_j, j < ny - 1)
  // multipliers over each segment of TRI_SEG rows, in the order in which the
  // warp-cooperative solve composes them
  const int nseg = (g.ny + TRI_SEG - 1) / TRI_SEG;
  for (int sg = 0; sg < nseg; ++sg) {
    double af = 1.0, ab = 1.0;
    for (int u = 0; u < TRI_SEG; ++u) {
      const int j = sg * TRI_SEG + u;
      if (j >= g.ny) break;
      const double al = j == 0 ? 0.0 : -cp[base + (long long)j * stride];
      af = al * af;
    }
    for (int u = TRI_SEG - 1; u >= 0; --u) {
      const int j = sg * TRI_SEG + u;
      if (j >= g.ny) continue;
      const double al = j == g.ny - 1 ? 0.0 : -cp[base + (long long)j * stride];
      ab = al * ab;
    }
    const long long sid = ((long long)kz * nseg + sg) * nkx + kx;
    segf[sid] = af;
    segb[sid] = ab;
  }
}

// Pivots of the height-scaled rows of a non-uniform wall-normal grid (see
// tri_y_nu), per (kx, kz) system.
__global__ void k_build_tri_tables_nu(Geo g, const double* __restrict__ lamx, const double* __restrict__ lamz,
                                      double* cp, double* ivh, double* al) {
  const int nkx = g.nkx;
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= (long long)nkx * g.nz) return;
  const long long kx = l % nkx, kz = l / nkx;
  const long long base = kz * (long long)g.ny * nkx + kx, stride = nkx;
  const double lam = lamx[kx] + lamz[kz];
  const bool singular = (kx == 0 && kz == 0);
  double cprev = 0.0;
  for (int j = 0; j < g.ny; ++j) {
    double sub = j > 0 ? g.yt.ihf[j] : 0.0;
    double sup = j < g.ny - 1 ? g.yt.ihf[j + 1] : 0.0;
    double diag = -sub - sup - lam * g.yt.hc[j];
    double scale = g.yt.hc[j];
    if (singular && j == 0) { diag = 1.0; sup = 0.0; sub = 0.0; scale = 0.0; }
    const double iv = 1.0 / (diag - sub * cprev);
    cprev = sup * iv;
    const long long id = base + (long long)j * stride;
    cp[id] = cprev;
    al[id] = -sub * iv;
    ivh[id] = scale * iv;
  }
}

void launch_build_poisson_tables_nu(const Geo& g, const double* lamx, const double* lamz, double* cp, double* ivh,
                                    double* al, cudaStream_t st) {
  const long long lines = (long long)g.nkx * g.nz;
  k_build_tri_tables_nu<<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(g, lamx, lamz, cp, ivh, al);
}

void launch_build_poisson_tables(const Geo& g, const double* lamx, const double* lamz, double* cp, double* inv,
                                 double* segf, double* segb, int* jc, cudaStream_t st) {
  const long long lines = (long long)g.nkx * g.nz;
  k_build_tri_tables<<<(unsigned)((lines + 127) / 128), 128, 0, st>>>(g, lamx, lamz, cp, inv, segf, segb, jc);
}

// ---------------------------------------------------------------------------
// Residual check of the mixed path's first solve on its own (launch shape
// corr_check = 2): max |D u' - q| over the fluid cells of the projected (hi,
// lo) state u' = uhat - G phi, with the arithmetic of the correction's
// right-hand side (poisson_rhs, mode 3), folded into the sub-stage's
// residual word; the correction's forward transform then runs gated, like
// its Thomas and inverse transforms.  Where the first solve usually meets
// the budget, this pass (no transform, no spectrum written) replaces the
// correction's forward transform.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void residual_check(const Blk& bk, const Geo& g, const Fields<T>& f,
                                               const unsigned* __restrict__ flags32, const DevState* ds, int s,
                                               int use_q, const ProjCoef<T>& cf, unsigned* res1) {
  const int i = bk.x * blockDim.x + threadIdx.x;
  const int j = bk.y * blockDim.y + threadIdx.y;
  const int k = bk.z;
  unsigned rmax = 0u;
  if (i < g.nx && j < g.ny) {
    const RowY<T> ry = row_y<T>(g, f, cf, j);
    const T qz = (T)0;
    (void)poisson_rhs<T>(g, f, flags32, ds, s, use_q, 0.0, 3, cf, ry, qz, qz, qz, i, j, k, rmax);
  }
  fold_residual(res1, rmax);
}
template <typename T>
struct ResidualCheck {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const DevState* ds;
  int s, use_q;
  ProjCoef<T> cf;
  unsigned* res1;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    residual_check<T>(bk, g, f, flags32, ds, s, use_q, cf, res1);
  }
};

// ---------------------------------------------------------------------------
// projection (Eq. projection) and pressure update (Eq. update_pressure):
//   u <- uhat - alpha dt G phi   (v on the wall planes untouched)
//   p <- p + phi - alpha dt / (2 Re) L_c phi,  L_c with Neumann walls
// ---------------------------------------------------------------------------

// mode 0: u <- uhat - alpha dt G phi and p <- p + phi - beta L_c phi;
// mode 3 (mixed path): the (hi, lo) state takes the FP32 gradient of phi,
//         then that of the correction phi2, each subtracted as a pair update;
//         the pressure takes phi + phi2
template <typename T>
__device__ __forceinline__ void project(const Blk& bk, const Geo& g, const Fields<T>& f, const ProjCoef<T>& cf, int mode,
                                       DevState* ds, int s) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long pu = (long long)ny * nx, pv = (long long)(ny + 1) * nx;
  const int i = bk.x * blockDim.x + threadIdx.x;
  const int j = bk.y * blockDim.y + threadIdx.y;
  const int k = bk.z;
  if (i >= nx || j >= ny) return;
  const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int kp = k + 1 == nz ? 0 : k + 1, km = k == 0 ? nz - 1 : k - 1;
  const long long r0 = (long long)k * pu + (long long)j * nx;
  const long long rkm = (long long)km * pu + (long long)j * nx, rkp = (long long)kp * pu + (long long)j * nx;
  // every pseudo-pressure value of the stencil first: the field stores below
  // could alias them for the compiler, which would reload them
  const T* __restrict__ ph = f.phi;
  const T a0 = ph[r0 + i], aw = ph[r0 + im], ae = ph[r0 + ip], ab = ph[rkm + i], af = ph[rkp + i];
  const T as = j > 0 ? ph[r0 - nx + i] : a0, an = j + 1 < ny ? ph[r0 + nx + i] : a0;
  T b0 = (T)0, bw = (T)0, be = (T)0, bb = (T)0, bf = (T)0, bs = (T)0, bn = (T)0;
  // phi2 = 0 when the correction solve was skipped (the pair updates by -0
  // below then leave the state as the first projection made it)
  const bool corr = mode == 3 && correction_needed(ds, s);
  if (mode == 3 && corr && bk.x == 0 && bk.y == 0 && bk.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
    ds->ncorr += 1;
  if (corr) {
    const T* __restrict__ p2 = f.phi2;
    b0 = p2[r0 + i];
    bw = p2[r0 + im];
    be = p2[r0 + ip];
    bb = p2[rkm + i];
    bf = p2[rkp + i];
    bs = j > 0 ? p2[r0 - nx + i] : b0;
    bn = j + 1 < ny ? p2[r0 + nx + i] : b0;
  }
  // every gradient rounded on its own (no contraction into the update that
  // follows: the pair updates must stay error-free, and the single and the
  // batched kernels must round alike)
  const bool nun = g.yt.ihc != nullptr;   // non-uniform wall-normal spacing
  const T gx = mul_rn(cf.cx, a0 - aw);
  const T gz = mul_rn(cf.cz, a0 - ab);
  const T cyj = nun ? mul_rn(cf.adt, (T)g.yt.ihf[j]) : cf.cy;
  const T gy = j > 0 ? mul_rn(cyj, a0 - as) : (T)0;
  const long long vi = (long long)k * pv + (long long)j * nx + i;
  if (mode == 3) {
    // both projections of the mixed path in turn on the (hi, lo) state held
    // since the provisional step: G phi of the first solve, then G phi2 of
    // the correction, each subtracted as a pair update
    const T hx = mul_rn(cf.cx, b0 - bw);
    const T hz = mul_rn(cf.cz, b0 - bb);
    const T hy = j > 0 ? mul_rn(cf.cy, b0 - bs) : (T)0;
    float hi = (float)f.u[r0 + i], lo = (float)f.lo[0][r0 + i];
    ff_add(hi, lo, -(float)gx);
    ff_add(hi, lo, -(float)hx);
    f.u[r0 + i] = (T)hi;
    f.lo[0][r0 + i] = (T)lo;
    hi = (float)f.w[r0 + i];
    lo = (float)f.lo[2][r0 + i];
    ff_add(hi, lo, -(float)gz);
    ff_add(hi, lo, -(float)hz);
    f.w[r0 + i] = (T)hi;
    f.lo[2][r0 + i] = (T)lo;
    if (j > 0) {
      hi = (float)f.v[vi];
      lo = (float)f.lo[1][vi];
      ff_add(hi, lo, -(float)gy);
      ff_add(hi, lo, -(float)hy);
      f.v[vi] = (T)hi;
      f.lo[1][vi] = (T)lo;
    }
  } else {
    f.u[r0 + i] = add_rn(f.u[r0 + i], -gx);
    f.w[r0 + i] = add_rn(f.w[r0 + i], -gz);
    if (j > 0) f.v[vi] = add_rn(f.v[vi], -gy);
  }
  // pressure update with the whole pseudo-pressure
  const bool two = mode == 3;
  const T q0 = two ? a0 + b0 : a0;
  const T pw = two ? aw + bw : aw, pe = two ? ae + be : ae, pb = two ? ab + bb : ab, pf = two ? af + bf : af;
  const T up = j + 1 < ny ? (two ? an + bn : an) - q0 : (T)0;
  const T dn = j > 0 ? q0 - (two ? as + bs : as) : (T)0;
  // explicit fma / rounding: the single-simulation and the batched kernels
  // compile this body separately and must round alike
  const T lx = add_rn(fma((T)-2, q0, pe), pw);
  const T lz = add_rn(fma((T)-2, q0, pf), pb);
  T lap;
  if (nun) {
    const T ly = mul_rn(mul_rn(cf.bb, (T)g.yt.ihc[j]),
                        add_rn(mul_rn(up, (T)g.yt.ihf[j + 1]), -mul_rn(dn, (T)g.yt.ihf[j])));
    lap = fma(cf.bx, lx, add_rn(ly, mul_rn(cf.bz, lz)));
  } else {
    lap = fma(cf.bx, lx, fma(cf.by, add_rn(up, -dn), mul_rn(cf.bz, lz)));
  }
  f.p[r0 + i] = add_rn(f.p[r0 + i], add_rn(q0, -lap));
}
template <typename T>
struct Project {
  static constexpr int kThreads = 128;
  Geo g;
  Fields<T> f;
  ProjCoef<T> cf;
  int mode;
  DevState* ds;   // mode 3: the correction-solve decision of sub-stage s
  int s;
  __device__ __forceinline__ void operator()(const Blk& bk) const { project<T>(bk, g, f, cf, mode, ds, s); }
};

// A kernel of the correction solve: does its work only when the first
// solve's residual exceeds the budget (every block reads the decision the
// correction's forward transform completed before this launch).
template <class Op, bool = HasMinBlocks<Op>::value>
struct MinBlocksOf {};
template <class Op>
struct MinBlocksOf<Op, true> {
  static constexpr int kMinBlocks = Op::kMinBlocks;
};
template <class Op>
struct Gated : MinBlocksOf<Op> {
  static constexpr int kThreads = Op::kThreads;
  Op op;
  const DevState* ds;
  int s;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    if (!correction_needed(ds, s)) return;
    op(bk);
  }
};
// ---------------------------------------------------------------------------
// State diagnostics of a step, after its last projection:
//   div_max = max over C_F of |D u - q| (Eq. mod_div: the projected field
//             has D u = q on the fluid cells; every cell when q is off),
//   ke      = 1/2 sum over the velocity nodes of u^2 dV (dV = dx h dz: the
//             cell height for u and w, the distance of the centres for v),
//   cfl     = dt max over the cells of |u_c|/dx + |v_c|/h + |w_c|/dz, u_c the
//             mean of the cell's two faces of each component.
// A cell counts the nodes of its three lower faces for the energy (the top
// wall plane of v holds no unknown).  The mixed path forms D u in pair
// arithmetic from the (hi, lo) state, q as the FP32 pair of q_F, and the
// energy and CFL number from the hi parts.  Fixed-order two-level reduction:
// each thread walks a fixed set of cells, sums go through a fixed butterfly.
// ---------------------------------------------------------------------------
constexpr int DG_BLOCKS = 4096, DG_THREADS = 256;   // DG_BLOCKS: the most partial triples

// FP32 constants of the mixed path's diagnostics, formed on the host (a
// conversion from FP64 occupies this GPU's narrow FP64 pipe): 1/dx, 1/dz,
// the reciprocal spacings as (hi, lo) pairs, dy.
struct DiagF32 {
  float idx, idz, ixh, ixl, izh, izl, uyh, uyl, dy;
};

template <typename T>
__device__ __forceinline__ void state_diag(const Blk& bk, const Geo& g, const Fields<T>& f,
                                           const unsigned* __restrict__ flags32, const DevState* ds, int s,
                                           int use_q, const DiagF32& fc, double* partial) {
  __shared__ double red[DG_THREADS / 32][3];
  // a warp walks whole x-rows (j, k) -- the row's constants once, cells along
  // the lanes -- rows in a fixed order per warp
  const int nx = g.nx, ny = g.ny;
  const long long pu = (long long)ny * nx, pv = (long long)(ny + 1) * nx;
  const bool nun = g.yt.ihc != nullptr;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long nrows = (long long)ny * g.nz;
  const long long wstride = (long long)bk.gx * (DG_THREADS / 32);
  double dmax = 0.0, ke = 0.0, cmax = 0.0;
  if (f.lo[0]) {
    const float idx = fc.idx, idz = fc.idz;
    const float ixh = fc.ixh, ixl = fc.ixl, izh = fc.izh, izl = fc.izl;
    const float qh1 = use_q == 1 ? ds->qf_hi[s] : 0.0f, ql1 = use_q == 1 ? ds->qf_lo[s] : 0.0f;
    float fdmax = 0.0f, fke = 0.0f, fcmax = 0.0f;
    for (long long r = (long long)bk.x * (DG_THREADS / 32) + wid; r < nrows; r += wstride) {
      const int j = (int)(r % ny), k = (int)(r / ny);
      // row constants: FP32 pair of 1/h and the node volumes' heights
      float ihh = fc.uyh, ihl = fc.uyl, hc = fc.dy, hf = fc.dy;
      if (nun) {
        bool sp = false;
        const double ih = g.yt.ihc[j];
        ihh = d2f_int(ih, sp);
        ihl = d2f_int(ih - f2d_int(ihh, sp), sp);
        hc = d2f_int(g.yt.hc[j], sp);
        hf = d2f_int(g.yt.hf[j], sp);
      }
      const long long e0 = (long long)k * pu + (long long)j * nx;
      const long long kp0 = (k + 1 == g.nz ? 0 : (long long)(k + 1) * pu) + (long long)j * nx;
      const long long v00 = (long long)k * pv + (long long)j * nx;
      for (int i = lane; i < nx; i += 32) {
        const long long e = e0 + i, ip = e0 + (i + 1 == nx ? 0 : i + 1), kp = kp0 + i, v0 = v00 + i;
        const float uh0 = (float)f.u[e], uh1 = (float)f.u[ip], vh0 = (float)f.v[v0], vh1 = (float)f.v[v0 + nx];
        const float wh0 = (float)f.w[e], wh1 = (float)f.w[kp];
        fke += (uh0 * uh0 + wh0 * wh0) * hc + vh0 * vh0 * hf;
        fcmax = fmaxf(fcmax, fabsf(uh0 + uh1) * idx + fabsf(vh0 + vh1) * ihh + fabsf(wh0 + wh1) * idz);
        const unsigned fl = (flags32[e >> 2] >> (8 * (e & 3))) & 0xFFu;
        if (!(use_q && (fl & FLAG_B))) {
          float bx, sx, by, sy, bz, sz, a1, er1, a2, er2, a3, er3;
          pair_diff_v(uh1, (float)f.lo[0][ip], uh0, (float)f.lo[0][e], ixh, ixl, bx, sx);
          pair_diff_v(vh1, (float)f.lo[1][v0 + nx], vh0, (float)f.lo[1][v0], ihh, ihl, by, sy);
          pair_diff_v(wh1, (float)f.lo[2][kp], wh0, (float)f.lo[2][e], izh, izl, bz, sz);
          two_sum(bx, by, a1, er1);
          two_sum(a1, bz, a2, er2);
          const float qh = use_q == 2 ? (float)f.qk[e] : qh1;
          two_sum(a2, -qh, a3, er3);
          const float rr = a3 + ((((er1 + er2) + er3) + ((sx + sy) + sz)) - ql1);
          fdmax = fmaxf(fdmax, fabsf(rr));
        }
      }
    }
    // warp reduction in FP32 (an FP64 shuffle reduction per thread would
    // keep this GPU's narrow FP64 pipe busy longer than the loads take)
    for (int o = 16; o > 0; o >>= 1) {
      fdmax = fmaxf(fdmax, __shfl_xor_sync(0xFFFFFFFFu, fdmax, o));
      fke += __shfl_xor_sync(0xFFFFFFFFu, fke, o);
      fcmax = fmaxf(fcmax, __shfl_xor_sync(0xFFFFFFFFu, fcmax, o));
    }
    if (lane == 0) {   // (one conversion per warp)
      dmax = (double)fdmax;
      ke = (double)fke;
      cmax = (double)fcmax;
    }
  } else {
    for (long long r = (long long)bk.x * (DG_THREADS / 32) + wid; r < nrows; r += wstride) {
      const int j = (int)(r % ny), k = (int)(r / ny);
      const double ih = nun ? g.yt.ihc[j] : g.idy;
      const double hc = nun ? g.yt.hc[j] : g.dy, hf = nun ? g.yt.hf[j] : g.dy;
      const long long e0 = (long long)k * pu + (long long)j * nx;
      const long long kp0 = (k + 1 == g.nz ? 0 : (long long)(k + 1) * pu) + (long long)j * nx;
      const long long v00 = (long long)k * pv + (long long)j * nx;
      for (int i = lane; i < nx; i += 32) {
        const long long e = e0 + i, ip = e0 + (i + 1 == nx ? 0 : i + 1), kp = kp0 + i, v0 = v00 + i;
        const double u0 = (double)f.u[e], u1 = (double)f.u[ip], vv0 = (double)f.v[v0], vv1 = (double)f.v[v0 + nx];
        const double w0 = (double)f.w[e], w1 = (double)f.w[kp];
        ke += (u0 * u0 + w0 * w0) * hc + vv0 * vv0 * hf;
        cmax = fmax(cmax, fabs(u0 + u1) * g.idx + fabs(vv0 + vv1) * ih + fabs(w0 + w1) * g.idz);
        const unsigned fl = (flags32[e >> 2] >> (8 * (e & 3))) & 0xFFu;
        if (!(use_q && (fl & FLAG_B))) {
          const double d = ((u1 - u0) * g.idx + (vv1 - vv0) * ih) + (w1 - w0) * g.idz;
          const double q = use_q == 2 ? (double)f.qk[e] : (use_q ? ds->qf[s] : 0.0);
          dmax = fmax(dmax, fabs(d - q));
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      dmax = fmax(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, o));
      ke += __shfl_xor_sync(0xFFFFFFFFu, ke, o);
      cmax = fmax(cmax, __shfl_xor_sync(0xFFFFFFFFu, cmax, o));
    }
  }
  if (lane == 0) {
    red[wid][0] = dmax;
    red[wid][1] = ke;
    red[wid][2] = cmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < DG_THREADS / 32; ++w) {
      a = fmax(a, red[w][0]);
      b += red[w][1];
      c = fmax(c, red[w][2]);
    }
    partial[3 * bk.x] = a;
    partial[3 * bk.x + 1] = b;
    partial[3 * bk.x + 2] = c;
  }
}
template <typename T>
struct StateDiag {
  static constexpr int kThreads = DG_THREADS;
  Geo g;
  Fields<T> f;
  const unsigned* flags32;
  const DevState* ds;
  int s;
  int use_q;
  DiagF32 fc;
  double* partial;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    state_diag<T>(bk, g, f, flags32, ds, s, use_q, fc, partial);
  }
};

// 256 threads: thread t adds the partials t, t + 256, ... in turn, then a
// fixed tree over the threads (reproducible: the order depends only on the
// number of partials)
constexpr int DGF_THREADS = 256;
__device__ __forceinline__ void state_diag_final(const Geo& g, const double* partial, DevState* ds, double dt,
                                                 int nblk) {
  __shared__ double red[3][DGF_THREADS];
  const int t = threadIdx.x;
  double a = 0.0, k = 0.0, c = 0.0;
  for (int b = t; b < nblk; b += DGF_THREADS) {
    a = fmax(a, partial[3 * b]);
    k += partial[3 * b + 1];
    c = fmax(c, partial[3 * b + 2]);
  }
  red[0][t] = a;
  red[1][t] = k;
  red[2][t] = c;
  __syncthreads();
  for (int w = DGF_THREADS / 2; w > 0; w >>= 1) {
    if (t < w) {
      red[0][t] = fmax(red[0][t], red[0][t + w]);
      red[1][t] += red[1][t + w];
      red[2][t] = fmax(red[2][t], red[2][t + w]);
    }
    __syncthreads();
  }
  if (t == 0) {
    const double dm = red[0][0], ke = red[1][0], cm = red[2][0];
    ds->div_max = dm;
    ds->ke = 0.5 * g.dx * g.dz * ke;
    ds->cfl = 0.5 * dt * cm;
    if (!isfinite(ke) || !isfinite(cm) || !isfinite(dm)) atomicOr(&ds->err, ERR_NONFINITE);
  }
}
struct StateDiagFinal {
  static constexpr int kThreads = DGF_THREADS;
  Geo g;
  const double* partial;
  DevState* ds;
  double dt;
  int nblk;
  __device__ __forceinline__ void operator()(const Blk&) const { state_diag_final(g, partial, ds, dt, nblk); }
};

template <typename T>
void launch_state_diag(const Geo& g, const Fields<T>& f, const TagBuffers& b, int s, int use_q, double dt,
                       double* partial, DevState* ds, Exec& ex) {
  ex.mark(ST_DIAG);
  // about two rows of cells per warp
  const int nblk = (int)std::min<long long>(DG_BLOCKS, std::max<long long>(
      8, ((long long)g.ny * g.nz + 2 * (DG_THREADS / 32) - 1) / (2 * (DG_THREADS / 32))));
  const DiagF32 fc{(float)g.idx, (float)g.idz, (float)f.idh[0][0], (float)f.idh[0][1], (float)f.idh[2][0],
                   (float)f.idh[2][1], (float)f.idh[1][0], (float)f.idh[1][1], (float)g.dy};
  ex.launch(dim3(nblk), dim3(DG_THREADS), 0, StateDiag<T>{g, f, b.flags32, ds, s, use_q, fc, partial});
  ex.launch(dim3(1), dim3(DGF_THREADS), 0, StateDiagFinal{g, partial, ds, dt, nblk});
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
                    const Stage& sg, double dt, double re, int use_q, double* partial, DevState* ds, Exec& ex) {
  using C = typename Cplx<T>::type;
  const Geo& sh = ex.shape;
  const Tune& tu = ex.tune;
  if (use_q == 1) {
    ex.mark(ST_QRED);
    const int nq = reduce_blocks(g, 16384, QB_BLOCKS);
    ex.launch(dim3(nq), dim3(QB_THREADS), 0, QPartial<T>{g, f, b.blist, b.cap, ds, partial});
    ex.launch(dim3(1), dim3(32), 0, QFinal{g, partial, ds, sg.s, use_q, nq});
  } else if (use_q == 2) {
    ex.mark(ST_QRED);
    const int nq = reduce_blocks(g, 16384, QB_BLOCKS);
    ex.launch(dim3(nq), dim3(QE_THREADS), 0, QEnergyPartial<T>{g, f, b.flags32, partial});
    ex.launch(dim3(1), dim3(32), 0, QEnergyFinal{g, partial, ds, sg.s, nq});
  }
  const double scale = 1.0 / (sg.alp * dt * (double)g.nx * (double)g.nz);
  // radix-8 passes in the FP32 path (the FP64 path keeps radix 4 and 2: eight
  // FP64 complex values per thread would crowd the capped registers)
  const FftPlan px = make_plan(g.nx, sizeof(T) == 4), pz = make_plan(g.nz, sizeof(T) == 4);
  // launch shapes from the batch shape (tiles sized for its largest extents)
  int cols = 16;
  while (cols > 1 && cols * sh.nz > 2048) cols >>= 1;
  if (tu.fft_cols > 0)
    while (cols > tu.fft_cols) cols >>= 1;
  const int ntile = (g.nkx + cols - 1) / cols;
  const size_t smz = 2ull * cols * sh.nz * sizeof(C);
  int lpb = lines_for(sh.nx);
  if (tu.fft_lpb > 0 && tu.fft_lpb < lpb) lpb = tu.fft_lpb;
  const long long xlines = ((long long)g.ny * g.nz + 1) / 2;
  const size_t smx = 2ull * lpb * (sh.nx + 1) * sizeof(C);   // lines padded to nx + 1 words
  const int tx = sh.nx < 128 ? sh.nx : 128;
  const dim3 xblk(tx, 256 / tx);
  const dim3 xgrid((unsigned)((xlines + lpb - 1) / lpb));
  const long long tlines = (long long)g.nkx * g.nz;
  double* fwd = sizeof(T) == sizeof(double) ? nullptr : reinterpret_cast<double*>(f.scr);
  // wall-normal Thomas for every (kx, kz): warp-cooperative when the rows fit
  // the registers (16 per lane), else one thread per real/imaginary part
  // threads per block of the shared-memory variant: its FP64 forward values
  // (8 B per row and system) must fit 160 KB
  const int tsm = 64ll * 8 * sh.ny <= 160 * 1024 ? 64 : (32ll * 8 * sh.ny <= 160 * 1024 ? 32 : 0);
  int tri = tu.tri_y == 2 || sh.ny > 32 * TRI_SEG ? 2 : 1;
  if (tu.tri_y == 3 && tsm > 0) tri = 3;
  // the kernels of the correction solve after its forward transform run
  // gated: they return at once when the first solve met the budget
  // gate: 0 none, 1 the correction solve's gate (Gated)
  int gate = 0;
  auto glaunch = [&](dim3 gr, dim3 bl, size_t sm, const auto& op) {
    using Op = std::decay_t<decltype(op)>;
    if constexpr (sizeof(T) == 4) {
      if (gate == 1) {
        ex.launch(gr, bl, sm, Gated<Op>{{}, op, ds, sg.s});
        return;
      }
    }
    ex.launch(gr, bl, sm, op);
  };
  auto tri_solve = [&]() {
    if (tb.pal) {   // non-uniform wall-normal spacing
      if (tu.tri_y == 2 || sh.ny > 32 * TRI_SEG) {
        glaunch(dim3((unsigned)((2 * tlines + 127) / 128)), dim3(128), 0, TriYNU<T>{g, f, tb.cp, tb.inv, tb.pal});
      } else if (sh.ny <= 8 * TRI_SEG) {
        const long long warps = (long long)((g.nkx + 3) / 4) * g.nz;
        glaunch(dim3((unsigned)((warps * 32 + 127) / 128)), dim3(128), 0,
                  TriYWarpNU<T, 8>{g, f, tb.cp, tb.inv, tb.pal});
      } else if (sh.ny <= 16 * TRI_SEG) {
        const long long warps = (long long)((g.nkx + 1) / 2) * g.nz;
        glaunch(dim3((unsigned)((warps * 32 + 127) / 128)), dim3(128), 0,
                  TriYWarpNU<T, 16>{g, f, tb.cp, tb.inv, tb.pal});
      } else {
        const long long warps = (long long)g.nkx * g.nz;
        glaunch(dim3((unsigned)((warps * 32 + 127) / 128)), dim3(128), 0,
                  TriYWarpNU<T, 32>{g, f, tb.cp, tb.inv, tb.pal});
      }
      return;
    }
    if (tri == 3) {
      glaunch(dim3((unsigned)((2 * tlines + tsm - 1) / tsm)), dim3(tsm), (size_t)tsm * 8 * sh.ny,
                TriYSmem<T>{g, f, tb.cp, tb.inv});
    } else if (tri == 1) {
      // L lanes per system: G = 32 / L systems per warp.  Unless the tuning
      // asks for the uncapped form (1), registers are capped so that 7
      // blocks fit an SM (a 128^2-wavenumber grid then runs in one wave)
      const bool cap = tu.tri_y != 1;
      const int L = sh.ny <= 8 * TRI_SEG ? 8 : (sh.ny <= 16 * TRI_SEG ? 16 : 32);
      const long long warps = (long long)((g.nkx + 32 / L - 1) / (32 / L)) * g.nz;
      const dim3 gr((unsigned)((warps * 32 + 127) / 128)), bl(128);
      auto warp_op = [&](auto lanes, auto mb) {
        glaunch(gr, bl, 0, TriYWarp<T, decltype(lanes)::value, decltype(mb)::value>{g, f, tb.cp, tb.inv, tb.segf,
                                                                                    tb.segb, tb.jc});
      };
      using I1 = std::integral_constant<int, 1>;
      using I7 = std::integral_constant<int, 7>;
      if (L == 8) cap ? warp_op(std::integral_constant<int, 8>{}, I7{}) : warp_op(std::integral_constant<int, 8>{}, I1{});
      else if (L == 16) cap ? warp_op(std::integral_constant<int, 16>{}, I7{}) : warp_op(std::integral_constant<int, 16>{}, I1{});
      else cap ? warp_op(std::integral_constant<int, 32>{}, I7{}) : warp_op(std::integral_constant<int, 32>{}, I1{});
    } else {
      // blocks of two warps: the systems of a 128^3 grid then spread over
      // every SM, about one warp per SM sub-partition
      glaunch(dim3((unsigned)((2 * tlines + 63) / 64)), dim3(64), 0, TriY<T>{g, f, tb.cp, tb.inv, fwd});
    }
  };
  // fused per-plane transforms when the plane's half-spectrum and two work
  // buffers fit 200 KB of shared memory; the buffers take what is left, so
  // a small plane goes through each direction in one or two chunks
  const long long plane_b = (long long)sh.nz * sh.nkx * (long long)sizeof(C);
  const long long wmax = (200ll * 1024 - plane_b) / (2 * (long long)sizeof(C));
  int lcp = (int)std::min<long long>(sh.nz / 2, wmax / (sh.nx + 1));   // x lines padded to nx + 1
  // z columns per chunk: the fewest chunks that fit the work buffers, of
  // equal width (65 columns of a 128^3 grid go in one chunk, not 64 + 1)
  int czp = 1;
  {
    const long long cmax = std::max<long long>(1, std::min<long long>(sh.nkx, wmax / sh.nz));
    const long long nch = (sh.nkx + cmax - 1) / cmax;
    czp = (int)((sh.nkx + nch - 1) / nch);
  }
  const int wbuf = std::max(lcp * (sh.nx + 1), czp * sh.nz);
  const size_t smp = (size_t)plane_b + 2ull * wbuf * sizeof(C);
  // the built-in choice for one simulation: one block per plane where the
  // plane fits, else a cluster of blocks per plane (below), else the
  // separate kernels; a batch keeps the separate kernels unless asked
  const bool plane_fits = lcp >= 1 && (long long)czp * sh.nz <= wmax && smp <= 200 * 1024;
  const bool plane = (tu.fft_plane == 2 || (tu.fft_plane == 0 && !ex.rec)) && plane_fits;
  // the per-plane transforms split over a cluster of CLN blocks (one
  // simulation, nz a multiple of 2 CLN): each block's rows and work buffers
  // within 100 KB of shared memory, so at least two blocks share an SM
  constexpr int CLN = 4;
  bool cluster = false;
  int wbc = 0, czc = 0;
  size_t smc = 0;
  if (!ex.rec && !plane && (tu.fft_plane == 3 || tu.fft_plane == 0) && sh.nz % (2 * CLN) == 0 && sh.nkx >= CLN) {
    const int nzc = sh.nz / CLN, cw = (sh.nkx + CLN - 1) / CLN;
    const long long sb = (long long)nzc * sh.nkx * (long long)sizeof(C);
    const long long wm = (100ll * 1024 - sb) / (2 * (long long)sizeof(C));
    const long long lcc = std::min<long long>(nzc / 2, wm / (sh.nx + 1));
    const long long cmax = std::min<long long>(cw, wm / sh.nz);
    if (lcc >= 1 && cmax >= 1) {
      const long long nch = (cw + cmax - 1) / cmax;
      czc = (int)((cw + nch - 1) / nch);
      wbc = (int)std::max<long long>(lcc * (sh.nx + 1), (long long)czc * sh.nz);
      smc = (size_t)sb + 2ull * wbc * sizeof(C);
      cluster = true;
    }
  }
  auto glaunch_cl = [&](dim3 gr, dim3 bl, size_t sm, const auto& op) {
    using Op = std::decay_t<decltype(op)>;
    if constexpr (sizeof(T) == 4) {
      if (gate == 1) {
        ex.launch_cluster(gr, bl, sm, Gated<Op>{{}, op, ds, sg.s}, CLN);
        return;
      }
    }
    ex.launch_cluster(gr, bl, sm, op, CLN);
  };
  // the rest of one solve: z transform, wall-normal Thomas, inverse z and x
  // (the first solve marks each kernel group; the correction solve keeps its
  // forward transforms in one group and marks its Thomas and inverse
  // transforms separately)
  auto solve_rest = [&](T* out, bool first) {
    if (!plane && !cluster) {
      if (first) ex.mark(ST_FFT_Z_FWD);
      glaunch(dim3(g.ny * ntile), dim3(256), smz, FftZ<T, false>{g, f, tb.twz, pz, cols});
    }
    ex.mark(first ? ST_TRI_Y : ST_CORR_TRI);
    tri_solve();
    if (cluster) {
      ex.mark(first ? ST_FFT_X_INV : ST_CORR_INV);
      glaunch_cl(dim3(g.ny * CLN), dim3(256), smc, FftPlaneInvCl<T, CLN>{g, f, tb.twx, tb.twz, px, pz, wbc, czc, out});
      return;
    }
    if (plane) {
      ex.mark(first ? ST_FFT_X_INV : ST_CORR_INV);
      glaunch(dim3(g.ny), dim3(1024), smp, FftPlaneInv<T>{g, f, tb.twx, tb.twz, px, pz, wbuf, czp, out});
      return;
    }
    ex.mark(first ? ST_FFT_Z_INV : ST_CORR_INV);
    glaunch(dim3(g.ny * ntile), dim3(256), smz, FftZ<T, true>{g, f, tb.twz, pz, cols});
    if (first) ex.mark(ST_FFT_X_INV);
    glaunch(xgrid, xblk, smx, FftXInv<T>{g, f, tb.twx, px, lpb, out});
  };
  // forward x (and z, fused per plane) with the right-hand side of Eq. elliptic_mod
  const double adt = sg.alp * dt, bb = adt / (2.0 * re);
  ProjCoef<T> cf;
  cf.cx = (T)(adt * g.idx); cf.cy = (T)(adt * g.idy); cf.cz = (T)(adt * g.idz);
  cf.bx = (T)(bb * g.idx * g.idx); cf.by = (T)(bb * g.idy * g.idy); cf.bz = (T)(bb * g.idz * g.idz);
  cf.adt = (T)adt; cf.bb = (T)bb;
  cf.sc = (T)scale;
  cf.idx = (T)g.idx; cf.idy = (T)g.idy; cf.idz = (T)g.idz;
  cf.scf = (float)scale;
  for (int d = 0; d < 3; ++d) {
    cf.ih[d][0] = (float)f.idh[d][0];
    cf.ih[d][1] = (float)f.idh[d][1];
  }
  auto forward = [&](int mode) {   // (gated while `gate` is set)
    if (cluster)
      glaunch_cl(dim3(g.ny * CLN), dim3(256), smc,
                 FftPlaneFwdCl<T, CLN>{g, f, b.flags32, tb.twx, tb.twz, px, pz, wbc, czc, ds, sg.s, use_q, scale,
                                       mode, cf, ds->res1 + sg.s});
    else if (plane)
      glaunch(dim3(g.ny), dim3(1024), smp,
              FftPlaneFwd<T>{g, f, b.flags32, tb.twx, tb.twz, px, pz, wbuf, czp, ds, sg.s, use_q, scale, mode, cf,
                             ds->res1 + sg.s});
    else
      glaunch(xgrid, xblk, smx,
              FftXFwd<T>{g, f, b.flags32, tb.twx, px, lpb, ds, sg.s, use_q, scale, mode, cf, ds->res1 + sg.s});
  };
  const dim3 pgrid((g.nx + 31) / 32, (g.ny + 3) / 4, g.nz), pblk(32, 4);
  ex.mark(ST_FFT_X_FWD);
  forward(0);
  solve_rest(f.phi, true);
  if (!f.lo[0]) {
    ex.mark(ST_PROJECT);
    ex.launch(pgrid, pblk, 0, Project<T>{g, f, cf, 0, ds, sg.s});
    return;
  }
  // mixed path: solve again for the residual divergence of the projected
  // (hi, lo) state u' = uhat - G phi (formed face by face inside the
  // right-hand side, mode 3), then apply both projections and the pressure
  // update in one pass
  ex.mark(ST_CORRECT);
  if (tu.corr_check == 2) {   // the residual alone, then the whole correction solve gated
    ex.launch(pgrid, pblk, 0, ResidualCheck<T>{g, f, b.flags32, ds, sg.s, use_q, cf, ds->res1 + sg.s});
    gate = 1;
    forward(3);
  } else {                    // the correction's forward transform forms the residual (built-in)
    forward(3);
    gate = 1;
  }
  solve_rest(f.phi2, false);
  gate = 0;
  ex.mark(ST_PROJECT);
  ex.launch(pgrid, pblk, 0, Project<T>{g, f, cf, 3, ds, sg.s});
}

template <typename T>
void set_fft_smem_limits() {
  using C = typename Cplx<T>::type;
  const int maxsm = 2 * 4096 * (int)sizeof(C);   // x lines padded to nx + 1 words
  op_smem_limit<FftXFwd<T>>(maxsm);
  op_smem_limit<FftXInv<T>>(maxsm);
  op_smem_limit<FftZ<T, false>>(maxsm);
  op_smem_limit<FftZ<T, true>>(maxsm);
  op_smem_limit<TriYSmem<T>>(160 * 1024);
  op_smem_limit<FftPlaneFwd<T>>(200 * 1024);
  op_smem_limit<FftPlaneInv<T>>(200 * 1024);
  op_smem_limit<FftPlaneFwdCl<T, 4>>(100 * 1024);
  op_smem_limit<FftPlaneInvCl<T, 4>>(100 * 1024);
  if constexpr (sizeof(T) == 4) {   // the correction solve's kernels (mixed path)
    op_smem_limit<Gated<FftPlaneInvCl<T, 4>>>(100 * 1024);
    op_smem_limit<Gated<FftPlaneFwdCl<T, 4>>>(100 * 1024);
    op_smem_limit<Gated<FftPlaneFwd<T>>>(200 * 1024);
    op_smem_limit<Gated<FftXFwd<T>>>(maxsm);
    op_smem_limit<Gated<FftXInv<T>>>(maxsm);
    op_smem_limit<Gated<FftZ<T, false>>>(maxsm);
    op_smem_limit<Gated<FftZ<T, true>>>(maxsm);
    op_smem_limit<Gated<TriYSmem<T>>>(160 * 1024);
    op_smem_limit<Gated<FftPlaneInv<T>>>(200 * 1024);
  }
}

void init_kernel_attributes() {
  set_fft_smem_limits<double>();
  set_fft_smem_limits<float>();
}

template void launch_state_diag<double>(const Geo&, const Fields<double>&, const TagBuffers&, int, int, double,
                                        double*, DevState*, Exec&);
template void launch_state_diag<float>(const Geo&, const Fields<float>&, const TagBuffers&, int, int, double,
                                       double*, DevState*, Exec&);
template void launch_poisson<double>(const Geo&, const Fields<double>&, const TagBuffers&,
                                     const SpecTables<double>&, const Stage&, double, double, int, double*,
                                     DevState*, Exec&);
template void launch_poisson<float>(const Geo&, const Fields<float>&, const TagBuffers&, const SpecTables<float>&,
                                    const Stage&, double, double, int, double*, DevState*, Exec&);

}  // namespace ibm
