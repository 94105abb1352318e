// loads.cu -- hydrodynamic loads on the surface (Section 3.3 of arXiv
// 2606.09799) and the pressure of the boundary cells (Section 3.2), both
// post-processing of a finished step.
//
// Loads: the markers are the triangle centroids X^l with the oriented unit
// normal n^l and area A^l.  A probe x^e = X^l + h n^l (h the IB probe
// length, twice the cell diagonal) samples the flow; p and the velocity
// gradient there come from second-order moving-least-squares fits and are
// carried back to the wall by the Taylor series of Section 3.3:
//   p^l = p^e - h dp/dn + h^2/2 d2p/dn2,  grad u^l = grad u^e - h d(grad u)/dn
// (a quadratic fit has no third derivatives, so the h^2 term of grad u is
// zero), t^l = -p^l n + (grad u^l + grad u^l^T) n / Re.  The fit of each
// quantity takes the 4 x 4 x 4 nearest nodes of its own lattice (x and z
// wrap, y clamped to the stored planes) with weights exp(-(r/diag)^2) and
// the basis {1, xi, xi^2, cross terms}, xi = (x - x^e)/diag, leaving out
// nodes behind the marker's plane and, for p, the boundary cells; with
// fewer than ten such nodes (or a singular system) the fit is linear.
// sides = 2 adds the opposite face (normal -n) for zero-thickness surfaces.
//
// Boundary-cell pressure: the solution does not define p on C_B (Eq.
// mod_div replaces continuity there); each boundary cell takes the value
// at the probe point of its centre, x^e = X + h N/|N| with X the closest
// point on the triangle owning the cell's lower u face (zero normal
// gradient at the wall), interpolated trilinearly from the cell centres.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "exec.cuh"
#include "geometry.cuh"
#include "launch.h"

namespace ibm {

// Cholesky solve of the m x m SPD system A x = b, A row-major, in place;
// false if A is not positive definite.
template <int MM>
__device__ bool chol(int m, double* A, double* b) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = A[i * MM + j];
      for (int k = 0; k < j; ++k) s -= A[i * MM + k] * A[j * MM + k];
      if (i == j) {
        if (!(s > 0.0)) return false;
        A[i * MM + i] = sqrt(s);
      } else {
        A[i * MM + j] = s / A[j * MM + j];
      }
    }
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= A[i * MM + k] * b[k];
    b[i] = s / A[i * MM + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < m; ++k) s -= A[k * MM + i] * b[k];
    b[i] = s / A[i * MM + i];
  }
  return true;
}

// value of lattice `lat` (0..2 velocity components, 3 cell centres) at a
// stored node; the velocity in the mixed path is its (hi, lo) pair
template <typename T>
__device__ __forceinline__ double lattice_value(const Fields<T>& f, int lat, long long id) {
  if (lat == 3) return (double)f.p[id];
  const T* hi = lat == 0 ? f.u : (lat == 1 ? f.v : f.w);
  const T* lo = f.lo[lat];
  return (double)hi[id] + (lo ? (double)lo[id] : 0.0);
}

// Quadratic MLS fit of lattice `lat` around xe: value, gradient, Hessian.
template <typename T>
__device__ void mls_fit(const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32, int lat,
                        const double xe[3], const double X[3], const double n[3], double& val, double grad[3],
                        double H[9]) {
  const double del[3] = {g.dx, g.dy, g.dz};
  const double diag = sqrt(g.diag2);
  double off[3] = {0.5, 0.5, 0.5};
  if (lat < 3) off[lat] = 0.0;
  const long long pl = lat == 1 ? g.ny + 1 : g.ny;
  long long i0[3];
  for (int d = 0; d < 3; ++d) i0[d] = (long long)floor(xe[d] / del[d] - off[d]) - 1;
  if (i0[1] < 0) i0[1] = 0;
  if (i0[1] > pl - 4) i0[1] = pl - 4;
  double M[100], b[10];
  for (int r = 0; r < 100; ++r) M[r] = 0.0;
  for (int r = 0; r < 10; ++r) b[r] = 0.0;
  int used = 0;
  for (int a = 0; a < 4; ++a)
    for (int bb = 0; bb < 4; ++bb)
      for (int c = 0; c < 4; ++c) {
        const long long ii = i0[0] + a, jj = i0[1] + bb, kk = i0[2] + c;
        const double x[3] = {((double)ii + off[0]) * g.dx, ((double)jj + off[1]) * g.dy, ((double)kk + off[2]) * g.dz};
        const double side = (x[0] - X[0]) * n[0] + (x[1] - X[1]) * n[1] + (x[2] - X[2]) * n[2];
        if (!(side > 0.0)) continue;
        const long long iw = wrapi(ii, g.nx), kw = wrapi(kk, g.nz);
        const long long id = (kw * pl + jj) * g.nx + iw;
        if (lat == 3 && ((flags32[id >> 2] >> (8 * (id & 3))) & FLAG_B)) continue;
        double xi[3], r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          xi[d] = (x[d] - xe[d]) / diag;
          r2 += xi[d] * xi[d];
        }
        const double w = exp(-r2);
        const double P[10] = {1.0, xi[0], xi[1], xi[2], xi[0] * xi[0], xi[1] * xi[1], xi[2] * xi[2],
                              xi[0] * xi[1], xi[0] * xi[2], xi[1] * xi[2]};
        const double q = lattice_value<T>(f, lat, id);
        for (int r = 0; r < 10; ++r) {
          b[r] += w * P[r] * q;
          for (int s = 0; s < 10; ++s) M[r * 10 + s] += w * P[r] * P[s];
        }
        ++used;
      }
  double cf[10];
  for (int r = 0; r < 10; ++r) cf[r] = 0.0;
  bool ok = false;
  if (used >= 10) {
    double Mc[100], bc[10];
    for (int r = 0; r < 100; ++r) Mc[r] = M[r];
    for (int r = 0; r < 10; ++r) bc[r] = b[r];
    if (chol<10>(10, Mc, bc)) {
      for (int r = 0; r < 10; ++r) cf[r] = bc[r];
      ok = true;
    }
  }
  if (!ok) {
    double Ml[16], bl[4];
    for (int r = 0; r < 4; ++r) {
      bl[r] = b[r];
      for (int s = 0; s < 4; ++s) Ml[r * 4 + s] = M[r * 10 + s];
    }
    if (chol<4>(4, Ml, bl))
      for (int r = 0; r < 4; ++r) cf[r] = bl[r];
  }
  val = cf[0];
  for (int d = 0; d < 3; ++d) grad[d] = cf[1 + d] / diag;
  const double id2 = 1.0 / (diag * diag);
  H[0] = 2.0 * cf[4] * id2;
  H[4] = 2.0 * cf[5] * id2;
  H[8] = 2.0 * cf[6] * id2;
  H[1] = H[3] = cf[7] * id2;
  H[2] = H[6] = cf[8] * id2;
  H[5] = H[7] = cf[9] * id2;
}

// traction and wall pressure of one marker side
template <typename T>
__device__ void marker_traction(const Geo& g, const Fields<T>& f, const unsigned* __restrict__ flags32, double re,
                                const double X[3], const double n[3], double t[3], double& pwall) {
  const double h = g.h;
  double xe[3];
  for (int d = 0; d < 3; ++d) xe[d] = X[d] + h * n[d];
  double pe, gp[3], Hp[9];
  mls_fit<T>(g, f, flags32, 3, xe, X, n, pe, gp, Hp);
  const double dpn = gp[0] * n[0] + gp[1] * n[1] + gp[2] * n[2];
  double d2pn = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) d2pn += n[a] * Hp[a * 3 + b] * n[b];
  const double pl = pe - h * dpn + 0.5 * h * h * d2pn;
  double G[9];   // G[i 3 + j] = d u_i / d x_j at the wall
  for (int i = 0; i < 3; ++i) {
    double val, gr[3], H[9];
    mls_fit<T>(g, f, flags32, i, xe, X, n, val, gr, H);
    for (int j = 0; j < 3; ++j) G[i * 3 + j] = gr[j] - h * (H[j * 3 + 0] * n[0] + H[j * 3 + 1] * n[1] + H[j * 3 + 2] * n[2]);
  }
  for (int i = 0; i < 3; ++i) {
    double s = 0.0;
    for (int j = 0; j < 3; ++j) s += (G[i * 3 + j] + G[j * 3 + i]) * n[j];
    t[i] = -pl * n[i] + s / re;
  }
  pwall = pl;
}

// one thread per triangle: tr[6 t] = force t A and torque (X - pole) x t A
// summed over the sides; pw[t] the wall pressure on the normal's side
template <typename T>
__device__ __forceinline__ void loads_body(const Blk& bk, const Geo& g, const Surf& s, const Fields<T>& f,
                                           const unsigned* __restrict__ flags32, double re, int sides, double px,
                                           double py, double pz, double* tr, double* pw) {
  const long long t = (long long)bk.x * blockDim.x + threadIdx.x;
  if (t >= s.nt) return;
  double A[3], B[3], C[3];
  load_triangle(s, (int)t, A, B, C);
  double X[3], e1[3], e2[3], nn[3];
  for (int d = 0; d < 3; ++d) {
    X[d] = (A[d] + B[d] + C[d]) / 3.0;
    e1[d] = B[d] - A[d];
    e2[d] = C[d] - A[d];
  }
  nn[0] = e1[1] * e2[2] - e1[2] * e2[1];
  nn[1] = e1[2] * e2[0] - e1[0] * e2[2];
  nn[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
  const double area = 0.5 * len;
  double ft[3] = {0.0, 0.0, 0.0};
  for (int sd = 0; sd < sides; ++sd) {
    double n[3], tt[3], p;
    for (int d = 0; d < 3; ++d) n[d] = (sd == 0 ? 1.0 : -1.0) * nn[d] / len;
    marker_traction<T>(g, f, flags32, re, X, n, tt, p);
    if (sd == 0) pw[t] = p;
    for (int d = 0; d < 3; ++d) ft[d] += tt[d] * area;
  }
  const double r[3] = {X[0] - px, X[1] - py, X[2] - pz};
  tr[6 * t + 0] = ft[0];
  tr[6 * t + 1] = ft[1];
  tr[6 * t + 2] = ft[2];
  tr[6 * t + 3] = r[1] * ft[2] - r[2] * ft[1];
  tr[6 * t + 4] = r[2] * ft[0] - r[0] * ft[2];
  tr[6 * t + 5] = r[0] * ft[1] - r[1] * ft[0];
}
template <typename T>
struct Loads {
  static constexpr int kThreads = 64;
  Geo g;
  Surf s;
  Fields<T> f;
  const unsigned* flags32;
  double re;
  int sides;
  double px, py, pz;
  double* tr;
  double* pw;
  __device__ __forceinline__ void operator()(const Blk& bk) const {
    loads_body<T>(bk, g, s, f, flags32, re, sides, px, py, pz, tr, pw);
  }
};

// trilinear value of the cell-centre field at P (false: stencil leaves the
// stored planes in y)
template <typename T>
__device__ bool trilinear_centres(const Geo& g, const T* __restrict__ p, const double P[3], double& out) {
  const double sx = P[0] * g.idx - 0.5, sy = P[1] * g.idy - 0.5, sz = P[2] * g.idz - 0.5;
  const double fx = floor(sx), fy = floor(sy), fz = floor(sz);
  const long long i0 = (long long)fx, j0 = (long long)fy, k0 = (long long)fz;
  if (j0 < 0 || j0 + 1 > g.ny - 1) return false;
  const double tx = sx - fx, ty = sy - fy, tz = sz - fz;
  double acc = 0.0;
  for (int dk = 0; dk <= 1; ++dk)
    for (int dj = 0; dj <= 1; ++dj)
      for (int di = 0; di <= 1; ++di) {
        const double w = (di ? tx : 1.0 - tx) * (dj ? ty : 1.0 - ty) * (dk ? tz : 1.0 - tz);
        acc += w * (double)p[cidx(g, wrapi(i0 + di, g.nx), j0 + dj, wrapi(k0 + dk, g.nz))];
      }
  out = acc;
  return true;
}

// one thread per listed boundary cell: q[cell] = p at the cell's probe point
template <typename T>
__device__ __forceinline__ void precon_body(const Blk& bk, const Geo& g, const Surf& s, const T* __restrict__ p,
                                            const unsigned* __restrict__ blist, const unsigned* __restrict__ owner,
                                            const DevState* ds, unsigned cap, double* q) {
  const unsigned nb = min(ds->nbound, cap);
  const unsigned e = bk.x * blockDim.x + threadIdx.x;
  if (e >= nb) return;
  const long long cell = blist[e];
  const unsigned t = owner[cell];   // the u grid shares the cells' [k][j][i] layout
  if (t == 0xFFFFFFFFu) return;
  const long long i = cell % g.nx, j = (cell / g.nx) % g.ny, k = cell / ((long long)g.nx * g.ny);
  double A[3], B[3], C[3];
  load_triangle(s, (int)t, A, B, C);
  double x[3] = {((double)i + 0.5) * g.dx, ((double)j + 0.5) * g.dy, ((double)k + 0.5) * g.dz};
  const double cx = (A[0] + B[0] + C[0]) / 3.0, cz = (A[2] + B[2] + C[2]) / 3.0;
  x[0] += g.lx * round((cx - x[0]) / g.lx);
  x[2] += g.lz * round((cz - x[2]) / g.lz);
  TriConst TC;
  tri_const(A, B, C, TC);
  double X[3], wb[3], N[3];
  closest_point_exact(x, TC, X, wb);
  double nl = 0.0;
  for (int d = 0; d < 3; ++d) {
    N[d] = x[d] - X[d];
    nl += N[d] * N[d];
  }
  nl = sqrt(nl);
  if (nl == 0.0) {
    N[0] = TC.ab[1] * TC.ac[2] - TC.ab[2] * TC.ac[1];
    N[1] = TC.ab[2] * TC.ac[0] - TC.ab[0] * TC.ac[2];
    N[2] = TC.ab[0] * TC.ac[1] - TC.ab[1] * TC.ac[0];
    nl = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
  }
  double xe[3], pe;
  for (int d = 0; d < 3; ++d) xe[d] = X[d] + g.h * N[d] / nl;
  if (trilinear_centres<T>(g, p, xe, pe)) q[cell] = pe;
}
template <typename T>
struct PressureRecon {
  static constexpr int kThreads = 128;
  Geo g;
  Surf s;
  const T* p;
  const unsigned* blist;
  const unsigned* owner;
  const DevState* ds;
  unsigned cap;
  double* q;
  __device__ __forceinline__ void operator()(const Blk& bk) const { precon_body<T>(bk, g, s, p, blist, owner, ds, cap, q); }
};

template <typename T>
void launch_loads(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double re, int sides,
                  const double pole[3], double* tr, double* pw, cudaStream_t st) {
  if (s.nt <= 0) return;
  Exec ex;
  ex.st = st;
  ex.shape = g;
  ex.launch(dim3((unsigned)((s.nt + 63) / 64)), dim3(64), 0,
            Loads<T>{g, s, f, b.flags32, re, sides, pole[0], pole[1], pole[2], tr, pw});
}

template <typename T>
void launch_pressure_recon(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds,
                           double* q, cudaStream_t st) {
  if (s.nt <= 0) return;
  Exec ex;
  ex.st = st;
  ex.shape = g;
  // grid for the most boundary cells possible; threads past the device-side
  // count return
  const long long most = std::min<long long>(b.cap, g.ncell);
  ex.launch(dim3((unsigned)((most + 127) / 128)), dim3(128), 0,
            PressureRecon<T>{g, s, f.p, b.blist, b.owner, ds, b.cap, q});
}

template void launch_loads<double>(const Geo&, const Surf&, const Fields<double>&, const TagBuffers&, double, int,
                                   const double*, double*, double*, cudaStream_t);
template void launch_loads<float>(const Geo&, const Surf&, const Fields<float>&, const TagBuffers&, double, int,
                                  const double*, double*, double*, cudaStream_t);
template void launch_pressure_recon<double>(const Geo&, const Surf&, const Fields<double>&, const TagBuffers&,
                                            DevState*, double*, cudaStream_t);
template void launch_pressure_recon<float>(const Geo&, const Surf&, const Fields<float>&, const TagBuffers&,
                                           DevState*, double*, cudaStream_t);

}  // namespace ibm
