// runtime.cu -- C ABI of the GB300 sharp-interface IBM fractional step
// (declared in include/ibm.h).  Owns the device buffers of a simulation,
// builds the coefficient tables on the host, uploads surfaces, and captures
// one whole time step (tagging, every sub-stage, diagnostics) into a CUDA
// graph that ibm_step replays on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ibm.h"
#include "common.cuh"
#include "exec.cuh"
#include "geometry.cuh"
#include "launch.h"

namespace ibm {

void init_kernel_attributes();
void init_sweep_attributes();

static int g_sms[64];

// ---- stage timing -----------------------------------------------------------
struct StageTimer {
  static constexpr int MAXM = 512;
  cudaEvent_t ev[MAXM];
  int id[MAXM];
  int n;
};
static thread_local StageTimer* t_timer = nullptr;

void stage_mark(cudaStream_t st, int id) {
  StageTimer* t = t_timer;
  if (!t || t->n >= StageTimer::MAXM) return;
  // inside stream capture only an external record becomes a graph node
  cudaEventRecordWithFlags(t->ev[t->n], st, cudaEventRecordExternal);
  t->id[t->n] = id;
  t->n++;
}

static const char* kStageNames[ST_COUNT] = {
    "tagging", "ib_force", "rhs", "sweep_x", "sweep_z", "sweep_y", "q_reduce", "fft_x_fwd", "fft_z_fwd",
    "tri_y", "fft_z_inv", "fft_x_inv", "project", "slip", "correction", "diagnostics", "correction_tri",
    "correction_inv", "other"};

int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (g_sms[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sms[dev] = n > 0 ? n : 152;
  }
  return g_sms[dev];
}

// ---- allocator hook ---------------------------------------------------------
static std::mutex g_alloc_mu;
static ibm_alloc_fn g_alloc = nullptr;
static ibm_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;

struct Allocator {
  ibm_alloc_fn alloc;
  ibm_free_fn free_fn;
  void* ctx;
  void* get(size_t bytes) const {
    if (bytes == 0) bytes = 256;
    if (alloc) return alloc(bytes, ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p) const {
    if (!p) return;
    if (free_fn) free_fn(p, ctx);
    else cudaFree(p);
  }
};

// ---- small helper kernels ----------------------------------------------------
__global__ void k_set_force(DevState* ds, double fx, double fy, double fz) {
  ds->fb[0] = fx;
  ds->fb[1] = fy;
  ds->fb[2] = fz;
  ds->fbf[0] = (float)fx;
  ds->fbf[1] = (float)fy;
  ds->fbf[2] = (float)fz;
}

__global__ void k_set_budget(DevState* ds, float budget) { ds->div_budget = budget; }

__device__ __forceinline__ void step_done(const Blk&, DevState* ds) { ds->steps += 1; }
struct StepDone {
  static constexpr int kThreads = 32;
  DevState* ds;
  __device__ __forceinline__ void operator()(const Blk& bk) const { step_done(bk, ds); }
};

__global__ void k_aos_to_soa(const double* __restrict__ aos, double* soa, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    soa[i] = aos[3 * (long long)i];
    soa[n + i] = aos[3 * (long long)i + 1];
    soa[2 * (long long)n + i] = aos[3 * (long long)i + 2];
  }
}

__global__ void k_tri_to_soa(const int* __restrict__ aos, int* soa, int n, int nv, unsigned* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    for (int m = 0; m < 3; ++m) {
      int v = aos[3 * (long long)i + m];
      if (v < 0 || v >= nv) {   // never let a kernel index outside the surface arrays
        atomicOr(bad, 1u);
        v = 0;
      }
      soa[(long long)m * n + i] = v;
    }
  }
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ src, B* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (B)src[i];
}

// FP64 value -> (hi, lo) FP32 pair and back
__global__ void k_split(const double* __restrict__ src, float* hi, float* lo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = src[i];
    const float h = (float)x;
    hi[i] = h;
    lo[i] = (float)(x - (double)h);
  }
}

__global__ void k_join(const float* __restrict__ hi, const float* __restrict__ lo, double* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)hi[i] + (double)lo[i];
}

__global__ void k_owner_out(const unsigned* __restrict__ own, int32_t* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (int32_t)own[i];
}

}  // namespace ibm

using namespace ibm;

struct ibm_grid {
  ibm_grid_desc desc;
  Geo g;
  Allocator al;
  int device;
  cudaStream_t user;      // caller's stream
  cudaStream_t cap;       // private stream used only for graph capture
  std::vector<void*> owned;
  char err[512];
  // device buffers
  void* fields_mem[16];
  DevState* ds;
  double* partial;
  TagBuffers tb;
  size_t esize;           // bytes of the bulk type
  void* u; void* v; void* w; void* p;
  void* H[3]; void* R[3]; void* scr; void* uf; void* phi; void* spec;
  void* lo[3]; void* phi2;   // mixed path: low parts of the velocity pairs, correction pseudo-pressure
  void* qk;                  // q_F per cell (energy-conserving shape)
  // tables
  void* sweep_mem[24];
  double* pcp; double* pinv; double* psegf; double* psegb; int* pjc; double* lamx; double* lamz;
  double* pal;     // non-uniform wall-normal grid: forward multipliers of the Poisson rows, else null
  double* ytab;    // non-uniform wall-normal grid: 1/heights (ny), 1/centre distances (ny+1), heights (ny),
                   // centre distances (ny+1), centre rows (ny+2), face rows (ny+3)
  double ysp_min;  // non-uniform wall-normal grid: smallest cell height or centre distance, else 0
  void* twx; void* twz;
  double tbl_off[3];
  double tbl_gam[2];
  double tbl_smden[2];
  // surface
  double* sx; double* su; int* st; double* stage_x; int* stage_t; unsigned* bad;
  TriRec* trirec;         // per-triangle constants, rewritten every step
  int nv, nt, nv_cap, nt_cap;
  bool has_topology;
  std::vector<int32_t> host_tri;   // host copy (AoS) of the connectivity when the caller gave one, else empty
  // graph
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graph_ok;
  bool need_full_reset;
  long long steps;
  long long kernels_per_step;
  long long epoch;        // bumped whenever a captured step of this handle goes stale
  Tune tune;              // launch-shape choices (autotuner)
};

// The captured step no longer matches the handle (buffers reallocated,
// surface sizes or tuning changed): recapture before the next step, and
// tell every batch holding the handle.
static void invalidate(ibm_handle h) {
  h->graph_ok = false;
  h->epoch += 1;
}

static void set_err(ibm_handle h, const char* fmt, const char* extra = "") {
  if (h) snprintf(h->err, sizeof(h->err), fmt, extra);
}

static ibm_status cuda_fail(ibm_handle h, cudaError_t e, const char* what) {
  if (h) snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA;
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);    \
  } while (0)

// Report (and clear) any error a launch left in the runtime's last-error
// slot, so it never leaks into the caller's framework.
static ibm_status launch_status(ibm_handle h, const char* what) {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? IBM_OK : cuda_fail(h, e, what);
}

static void* dalloc(ibm_handle h, size_t bytes) {
  void* p = h->al.get(bytes);
  if (p) h->owned.push_back(p);
  return p;
}

static void dfree(ibm_handle h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->owned.size(); ++i)
    if (h->owned[i] == p) {
      h->owned.erase(h->owned.begin() + (long)i);
      break;
    }
  h->al.put(p);
}

static bool good_fft_size(int n) {
  if (n < 4 || n > 1024 || (n % 2) != 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  while (n % 5 == 0) n /= 5;
  return n == 1;
}

// ---- host-side coefficient tables -------------------------------------------
// Thomas recurrences of a tridiagonal matrix with constant off-diagonals a
// (both sides) and diagonal b[m]: inv[m] = 1/pivot, cp[m] = a/pivot.
static void thomas_tables(int n, double a, const std::vector<double>& b, std::vector<double>& inv,
                          std::vector<double>& cp) {
  inv.assign(n, 0.0);
  cp.assign(n, 0.0);
  double prev = 0.0;
  for (int m = 0; m < n; ++m) {
    const double den = b[m] - (m > 0 ? a * prev : 0.0);
    inv[m] = 1.0 / den;
    cp[m] = (m < n - 1 ? a : 0.0) * inv[m];
    prev = cp[m];
  }
}

static void thomas_apply(int n, double a, const std::vector<double>& inv, const std::vector<double>& cp,
                         std::vector<double>& x) {
  double prev = 0.0;
  for (int m = 0; m < n; ++m) {
    prev = (x[m] - (m > 0 ? a * prev : 0.0)) * inv[m];
    x[m] = prev;
  }
  for (int m = n - 2; m >= 0; --m) x[m] = x[m] - cp[m] * x[m + 1];
}

template <typename T>
static void* upload_vec(ibm_handle h, const std::vector<double>& v) {
  std::vector<T> tmp(v.size());
  for (size_t i = 0; i < v.size(); ++i) tmp[i] = (T)v[i];
  void* d = dalloc(h, tmp.size() * sizeof(T) + 16);
  if (!d) return nullptr;
  if (cudaMemcpy(d, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  return d;
}

// Thomas recurrences of a segment of fluid rows with constant off-diagonal a
// and diagonal b, whose first row has diagonal b0 (row after an identity
// row: b0 = b; row at a wall: b0 = the wall diagonal)
static void segment_tables(int n, double a, double b0, double b, std::vector<double>& inv, std::vector<double>& cp) {
  std::vector<double> bb(n, b);
  if (n > 0) bb[0] = b0;
  thomas_tables(n, a, bb, inv, cp);
}

// periodic line of length n: Sherman-Morrison form of (1 - beta L) with
// off = beta/d^2 (modified matrix, correction vector z, first row g0 of its
// inverse) for lines without forcing nodes, and the segment recurrences for
// lines with forcing nodes
template <typename T>
static bool build_periodic(ibm_handle h, int n, double off, int slot) {
  const double a = -off, b = 1.0 + 2.0 * off, gam = -b;
  std::vector<double> bb(n, b);
  bb[0] = b - gam;
  bb[n - 1] = b - a * a / gam;
  std::vector<double> inv, cp;
  thomas_tables(n, a, bb, inv, cp);
  std::vector<double> z(n, 0.0), g0(n, 0.0);
  z[0] = gam;
  z[n - 1] = a;
  thomas_apply(n, a, inv, cp, z);
  g0[0] = 1.0;
  thomas_apply(n, a, inv, cp, g0);
  std::vector<double> invR, cpR;
  segment_tables(n, a, b, b, invR, cpR);
  h->tbl_gam[slot] = gam;
  h->tbl_smden[slot] = 1.0 + z[0] + a * z[n - 1] / gam;
  const std::vector<double>* v[6] = {&inv, &cp, &z, &g0, &invR, &cpR};
  for (int q = 0; q < 6; ++q) {
    h->sweep_mem[6 * slot + q] = upload_vec<T>(h, *v[q]);
    if (!h->sweep_mem[6 * slot + q]) return false;
  }
  return true;
}

// wall-normal lines: tangential components (ny rows, wall diagonal in the
// first and last rows) and v (ny-1 interior rows, Dirichlet walls)
template <typename T>
static bool build_wall(ibm_handle h, double off) {
  const int ny = h->g.ny;
  const double a = -off, b = 1.0 + 2.0 * off;
  const double gs = h->g.ybc == 0 ? -1.0 : 1.0;
  const double bw = b - gs * off;
  std::vector<double> invW, cpW, invR, cpR, invLW(ny), invLR(ny), vinv, vcp;
  segment_tables(ny, a, bw, b, invW, cpW);
  segment_tables(ny, a, b, b, invR, cpR);
  for (int m = 0; m < ny; ++m) {
    invLW[m] = m == 0 ? 1.0 / bw : 1.0 / (bw - a * cpW[m - 1]);
    invLR[m] = m == 0 ? 1.0 / bw : 1.0 / (bw - a * cpR[m - 1]);
  }
  segment_tables(ny - 1, a, b, b, vinv, vcp);
  const std::vector<double>* v[8] = {&invW, &cpW, &invR, &cpR, &invLW, &invLR, &vinv, &vcp};
  for (int q = 0; q < 8; ++q) {
    h->sweep_mem[12 + q] = upload_vec<T>(h, *v[q]);
    if (!h->sweep_mem[12 + q]) return false;
  }
  return true;
}

// Rows of the wall-normal sweep, for lines without forcing nodes and for
// segments that restart after a forcing row.  Row j of the tangential
// components (ny rows, wall ghost in the first and last) and of v (ny - 1
// interior rows) couples to its neighbours with beta / (h_c h_f) from the
// inverse spacings ihc (ny) and ihf (ny + 1).  out1 (6 ny - 3): a, 1/pivot,
// c' of one wall segment, tangential then v; out2 (if not null): 1/pivot and
// c' at [start row][row], tangential (two ny x ny) then v (two (ny-1)^2).
static void y_sweep_rows(int ny, double beta, double gs, const double* ihc, const double* ihf, double* out1,
                         std::vector<double>* out2) {
  if (out2) out2->assign(2ull * ny * ny + 2ull * (ny - 1) * (ny - 1), 0.0);
  for (int kind = 0; kind < 2; ++kind) {
    const bool tang = kind == 0;
    const int n = tang ? ny : ny - 1, jj0 = tang ? 0 : 1;
    double* ta = out1 + (tang ? 0 : 3 * ny);
    double* tv = ta + n;
    double* tcp = tv + n;
    double* iv2 = out2 ? out2->data() + (tang ? 0 : 2ull * ny * ny) : nullptr;
    double* cp2 = iv2 ? iv2 + (size_t)n * n : nullptr;
    for (int s0 = 0; s0 < (out2 ? n : 1); ++s0) {
      double cprev = 0.0;
      for (int m = s0; m < n; ++m) {
        const int j = jj0 + m;
        volatile double sb, sn;
        if (tang) {
          sb = beta * ihc[j] * ihf[j];
          sn = beta * ihc[j] * ihf[j + 1];
        } else {
          sb = beta * ihf[j] * ihc[j - 1];
          sn = beta * ihf[j] * ihc[j];
        }
        volatile double a = -sb, b = 1.0 + sb + sn, cc = -sn;
        if (m == 0) {
          if (tang) b = b - gs * sb;
          a = 0.0;
        }
        if (m == n - 1) {
          if (tang) b = b - gs * sn;
          cc = 0.0;
        }
        volatile double den = b - a * cprev;
        cprev = cc / den;
        if (s0 == 0) {
          ta[m] = a;
          tv[m] = 1.0 / den;
          tcp[m] = cprev;
        }
        if (iv2) {
          iv2[(size_t)s0 * n + m] = 1.0 / den;
          cp2[(size_t)s0 * n + m] = cprev;
        }
      }
    }
  }
}

template <typename T>
static SweepTables<T> sweep_tables(ibm_handle h) {
  SweepTables<T> t;
  for (int d = 0; d < 2; ++d) {
    t.inv[d] = (const T*)h->sweep_mem[6 * d + 0];
    t.cp[d] = (const T*)h->sweep_mem[6 * d + 1];
    t.zv[d] = (const T*)h->sweep_mem[6 * d + 2];
    t.g0[d] = (const T*)h->sweep_mem[6 * d + 3];
    t.invR[d] = (const T*)h->sweep_mem[6 * d + 4];
    t.cpR[d] = (const T*)h->sweep_mem[6 * d + 5];
    t.smden[d] = (T)h->tbl_smden[d];
    t.gam[d] = (T)h->tbl_gam[d];
  }
  t.yinvW = (const T*)h->sweep_mem[12];
  t.ycpW = (const T*)h->sweep_mem[13];
  t.yinvR = (const T*)h->sweep_mem[14];
  t.ycpR = (const T*)h->sweep_mem[15];
  t.yinvLW = (const T*)h->sweep_mem[16];
  t.yinvLR = (const T*)h->sweep_mem[17];
  t.vinvR = (const T*)h->sweep_mem[18];
  t.vcpR = (const T*)h->sweep_mem[19];
  for (int d = 0; d < 3; ++d) t.off[d] = (T)h->tbl_off[d];
  return t;
}

template <typename T>
static Fields<T> fields(ibm_handle h) {
  Fields<T> f;
  f.u = (T*)h->u;
  f.v = (T*)h->v;
  f.w = (T*)h->w;
  f.p = (T*)h->p;
  for (int c = 0; c < 3; ++c) {
    f.H[c] = (T*)h->H[c];
    f.Hp[c] = (T*)h->H[c];
    f.R[c] = (T*)h->R[c];
  }
  f.scr = (T*)h->scr;
  f.uf = (T*)h->uf;
  f.phi = (T*)h->phi;
  f.spec = h->spec;
  for (int c = 0; c < 3; ++c) f.lo[c] = (T*)h->lo[c];
  f.phi2 = (T*)h->phi2;
  f.qk = (T*)h->qk;
  const double id[3] = {h->g.idx, h->g.idy, h->g.idz};
  for (int d = 0; d < 3; ++d) {
    const float hi = (float)id[d];
    f.idh[d][0] = hi;
    f.idh[d][1] = (float)(id[d] - (double)hi);
  }
  return f;
}

template <typename T>
static SpecTables<T> spec_tables(ibm_handle h) {
  SpecTables<T> s;
  s.twx = (const T*)h->twx;
  s.twz = (const T*)h->twz;
  s.cp = h->pcp;
  s.inv = h->pinv;
  s.segf = h->psegf;
  s.segb = h->psegb;
  s.jc = h->pjc;
  s.pal = h->pal;
  return s;
}

static Surf surface(ibm_handle h) {
  Surf s;
  s.x = h->sx;
  s.u = h->su;
  s.t = h->st;
  s.rec = h->trirec;
  s.nv = h->nv;
  s.nt = h->nt;
  return s;
}

// scheme coefficients (gamma, rho, alpha) per sub-stage, Section 2
static int stages(const ibm_grid_desc& d, Stage out[2]) {
  if (d.scheme == IBM_AB_CN) {
    out[0] = Stage{1.5, -0.5, 1.0, 0};
    return 1;
  }
  out[0] = Stage{0.5, 0.0, 0.5, 0};
  out[1] = Stage{1.0, -0.5, 0.5, 1};
  return 2;
}

// enqueue one full time step on stream st
template <typename T>
static void enqueue_step(ibm_handle h, Exec& ex) {
  const Geo& g = h->g;
  const Surf s = surface(h);
  const Fields<T> f = fields<T>(h);
  const SweepTables<T> sw = sweep_tables<T>(h);
  const SpecTables<T> sp = spec_tables<T>(h);
  Stage sg[2];
  const int ns = stages(h->desc, sg);
  launch_tagging(g, s, h->tb, h->ds, ex);
  for (int k = 0; k < ns; ++k) {
    launch_ib_force<T>(g, s, f, h->tb, h->ds, k == 0, ex);
    const bool use_hp = sg[k].rho != 0.0;
    const bool write_h = (h->desc.scheme == IBM_AB_CN) || (k + 1 < ns);
    launch_rhs<T>(g, f, h->tb, sg[k], h->desc.dt, h->desc.re, use_hp, write_h, h->ds, ex);
    launch_sweeps<T>(g, f, h->tb, sw, h->ds, ex);
    launch_poisson<T>(g, f, h->tb, sp, sg[k], h->desc.dt, h->desc.re, h->desc.use_q, h->partial, h->ds, ex);
  }
  launch_state_diag<T>(g, f, h->tb, sg[ns - 1].s, h->desc.use_q, h->desc.dt, h->partial, h->ds, ex);
  launch_slip<T>(g, s, f, h->tb, h->partial, h->ds, ex);
  ex.launch(dim3(1), dim3(1), 0, StepDone{h->ds});
}

// The launch context of one handle stepping alone on stream st.
static Exec solo_exec(ibm_handle h, cudaStream_t st) {
  Exec ex;
  ex.st = st;
  ex.shape = h->g;
  ex.tune = h->tune;
  return ex;
}

static void release_all(ibm_handle h) {
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  for (void* p : h->owned) h->al.put(p);
  h->owned.clear();
  if (h->cap) cudaStreamDestroy(h->cap);
  h->cap = nullptr;
}

static size_t round16(size_t b) { return (b + 15) & ~(size_t)15; }

static ibm_status alloc_lists(ibm_handle h, unsigned cap) {
  dfree(h, h->tb.cand);
  dfree(h, h->tb.flist);
  dfree(h, h->tb.probe);
  dfree(h, h->tb.blist);
  dfree(h, h->tb.ublist);
  dfree(h, h->tb.surv);
  dfree(h, h->uf);
  h->tb.cand = (Cand*)dalloc(h, (size_t)cap * sizeof(Cand));
  h->tb.flist = (ForceNode*)dalloc(h, (size_t)cap * sizeof(ForceNode));
  h->tb.probe = (double*)dalloc(h, (size_t)cap * 5 * sizeof(double));
  h->tb.blist = (unsigned*)dalloc(h, (size_t)cap * sizeof(unsigned));
  h->tb.ublist = (unsigned*)dalloc(h, (size_t)cap * sizeof(unsigned));
  h->tb.surv = (unsigned long long*)dalloc(h, (size_t)cap * sizeof(unsigned long long));
  h->uf = dalloc(h, (size_t)cap * h->esize);
  if (!h->tb.cand || !h->tb.flist || !h->tb.probe || !h->tb.blist || !h->tb.ublist || !h->tb.surv || !h->uf) {
    set_err(h, "device allocation of the work lists failed");
    return IBM_ERR_OOM;
  }
  h->tb.cap = cap;
  invalidate(h);
  h->need_full_reset = true;
  return IBM_OK;
}

static ibm_status full_reset(ibm_handle h, cudaStream_t st) {
  const Geo& g = h->g;
  const long long nall = 2 * g.ncell + g.nvf;
  CK(cudaMemsetAsync(h->tb.d2min, 0xFF, (size_t)nall * 8, st));
  CK(cudaMemsetAsync(h->tb.owner, 0xFF, (size_t)nall * 4, st));
  CK(cudaMemsetAsync(h->tb.ub, 0xFF, (size_t)nall * 4, st));
  CK(cudaMemsetAsync(&h->ds->nub, 0, sizeof(unsigned), st));
  CK(cudaMemsetAsync(h->tb.flags32, 0, round16((size_t)(g.ncell + 3) / 4 * 4), st));
  CK(cudaMemsetAsync(h->tb.lines.x, 0x7F, h->tb.lines.bytes, st));
  CK(cudaMemsetAsync(&h->ds->ncand, 0, sizeof(unsigned), st));
  h->need_full_reset = false;
  return launch_status(h, "reset");
}

static long long count_kernel_nodes(cudaGraph_t gr) {
  size_t n = 0;
  if (cudaGraphGetNodes(gr, nullptr, &n) != cudaSuccess) return -1;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(gr, nodes.data(), &n) != cudaSuccess) return -1;
  long long k = 0;
  for (size_t i = 0; i < n; ++i) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
  }
  return k;
}

template <typename T>
static ibm_status capture(ibm_handle h) {
  if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
  if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
  {
    const ibm_status ls = launch_status(h, "before capture");
    if (ls != IBM_OK) return ls;
  }
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
  Exec ex = solo_exec(h, h->cap);
  enqueue_step<T>(h, ex);
  const cudaError_t le = cudaGetLastError();
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->cap, &gr);
  if (le != cudaSuccess || ex.first_err != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    if (ex.first_err != cudaSuccess) {
      snprintf(h->err, sizeof(h->err), "kernel launch during capture: %s in %.300s",
               cudaGetErrorString(ex.first_err), ex.first_op);
      return IBM_ERR_CUDA;
    }
    return cuda_fail(h, le, "kernel launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "graph capture");
  h->graph = gr;
  CK(cudaGraphInstantiate(&h->exec, gr, 0));
  h->graph_ok = true;
  h->kernels_per_step = count_kernel_nodes(gr);
  return IBM_OK;
}

// Stage timing: one step captured with an (external) event record before
// every kernel group, replayed nsteps times; ms[stage] accumulates the time
// between consecutive records, kernels[stage] the number of groups.
template <class Enqueue>
static ibm_status profile_graph(Enqueue enqueue, cudaStream_t cap, cudaStream_t run, int nsteps, double* ms,
                                int64_t* kernels, char* err, size_t errlen) {
  auto fail = [&](cudaError_t e, const char* what) {
    snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA;
  };
  StageTimer* tm = new (std::nothrow) StageTimer();
  if (!tm) return IBM_ERR_OOM;
  for (int m = 0; m < StageTimer::MAXM; ++m) {
    cudaError_t e = cudaEventCreate(&tm->ev[m]);
    if (e != cudaSuccess) {
      for (int q = 0; q < m; ++q) cudaEventDestroy(tm->ev[q]);
      delete tm;
      return fail(e, "cudaEventCreate");
    }
  }
  double acc[ST_COUNT] = {0};
  int64_t cnt[ST_COUNT] = {0};
  ibm_status rc = IBM_OK;
  cudaGraph_t gr = nullptr;
  cudaGraphExec_t ex = nullptr;
  tm->n = 0;
  t_timer = tm;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    enqueue(cap);
    stage_mark(cap, ST_OTHER);
    e = cudaStreamEndCapture(cap, &gr);
  }
  t_timer = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, gr, 0);
  if (e != cudaSuccess) rc = fail(e, "profiling graph");
  for (int step = 0; step < nsteps && rc == IBM_OK; ++step) {
    e = cudaGraphLaunch(ex, run);
    if (e == cudaSuccess) e = cudaStreamSynchronize(run);
    if (e != cudaSuccess) { rc = fail(e, "profiling step"); break; }
    for (int m = 0; m + 1 < tm->n && rc == IBM_OK; ++m) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, tm->ev[m], tm->ev[m + 1]);
      if (e != cudaSuccess) rc = fail(e, "cudaEventElapsedTime");
      acc[tm->id[m]] += t;
    }
  }
  if (rc == IBM_OK)
    for (int m = 0; m + 1 < tm->n; ++m) cnt[tm->id[m]] += 1;
  if (ex) cudaGraphExecDestroy(ex);
  if (gr) cudaGraphDestroy(gr);
  for (int m = 0; m < StageTimer::MAXM; ++m) cudaEventDestroy(tm->ev[m]);
  delete tm;
  if (rc != IBM_OK) return rc;
  for (int q = 0; q < ST_COUNT; ++q) {
    if (ms) ms[q] = acc[q];
    if (kernels) kernels[q] = cnt[q];
  }
  return IBM_OK;
}

// ---- batches of independent simulations -----------------------------------
// The step of every instance is recorded launch by launch (Exec::rec) with
// one launch shape for all (the largest extent of each axis); position p of
// all instances becomes one grouped launch (k_run_group) whose blocks are
// the concatenation of the instances' grids.  The ops and block offsets of
// every position live in one device buffer written once per build; one
// graph per step replays all positions in order.
struct ibm_batch {
  std::vector<ibm_handle> hs;
  std::vector<long long> epochs;   // handle epochs the graph was built for
  int device;
  cudaStream_t user;               // stream the step graph runs on
  cudaStream_t cap;                // private capture stream
  cudaEvent_t ev;
  Allocator al;
  void* dev;                       // ops + group entries of every position
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool built;
  Tune tune;
  Geo shape;
  long long positions;             // grouped launches per step
  long long kernels_solo;          // kernel launches per step if stepped one by one
  char err[512];
};

static ibm_status bfail(ibm_batch* b, cudaError_t e, const char* what) {
  snprintf(b->err, sizeof(b->err), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? IBM_ERR_OOM : IBM_ERR_CUDA;
}

#define BCK(call)                                             \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return bfail(b, e_, #call);        \
  } while (0)

static void batch_release(ibm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  if (b->dev) b->al.put(b->dev);
  b->dev = nullptr;
  b->built = false;
}

// Launch every recorded position of the batch on stream st (used inside a
// capture).  recs[i] is instance i's launch sequence; layout gives each
// position's device offsets of its ops and group entries.
struct BatchLayout {
  std::vector<size_t> op_off, ge_off;
  std::vector<unsigned> blocks;
  std::vector<size_t> smem;
};

static void batch_enqueue(ibm_batch* b, const std::vector<std::vector<LaunchRec>>& recs, const BatchLayout& L,
                          cudaStream_t st) {
  const int n = (int)recs.size();
  unsigned char* base = static_cast<unsigned char*>(b->dev);
  for (size_t p = 0; p < recs[0].size(); ++p) {
    const LaunchRec& r = recs[0][p];
    if (r.mark >= 0) stage_mark(st, r.mark);
    if (L.blocks[p] == 0) continue;
    r.group(base + L.op_off[p], reinterpret_cast<const GroupEntry*>(base + L.ge_off[p]), n, L.blocks[p], r.block,
            L.smem[p], st);
  }
}

template <typename T>
static ibm_status batch_record(ibm_batch* b, std::vector<std::vector<LaunchRec>>& recs, BatchLayout& L) {
  const int n = (int)b->hs.size();
  recs.assign(n, {});
  for (int i = 0; i < n; ++i) {
    Exec ex;
    ex.st = b->cap;
    ex.rec = &recs[i];
    ex.shape = b->shape;
    ex.tune = b->tune;
    enqueue_step<T>(b->hs[i], ex);
  }
  const size_t P = recs[0].size();
  for (int i = 1; i < n; ++i) {
    if (recs[i].size() != P) {
      snprintf(b->err, sizeof(b->err), "instance %d records %zu launches per step, instance 0 %zu", i,
               recs[i].size(), P);
      return IBM_ERR_STATE;
    }
    for (size_t p = 0; p < P; ++p) {
      const LaunchRec &a = recs[0][p], &c = recs[i][p];
      if (a.kind != c.kind || a.block.x != c.block.x || a.block.y != c.block.y || a.block.z != c.block.z ||
          a.mark != c.mark) {
        snprintf(b->err, sizeof(b->err), "instance %d differs from instance 0 at launch %zu of the step", i, p);
        return IBM_ERR_STATE;
      }
    }
  }
  // device layout: per position the n ops (256-byte aligned) then n entries
  L.op_off.assign(P, 0);
  L.ge_off.assign(P, 0);
  L.blocks.assign(P, 0);
  L.smem.assign(P, 0);
  size_t off = 0;
  for (size_t p = 0; p < P; ++p) {
    off = (off + 255) & ~(size_t)255;
    L.op_off[p] = off;
    off += (size_t)n * recs[0][p].op.size();
    off = (off + 15) & ~(size_t)15;
    L.ge_off[p] = off;
    off += (size_t)n * sizeof(GroupEntry);
  }
  std::vector<unsigned char> img(off > 0 ? off : 16, 0);
  for (size_t p = 0; p < P; ++p) {
    const size_t osz = recs[0][p].op.size();
    unsigned long long start = 0;
    for (int i = 0; i < n; ++i) {
      const LaunchRec& r = recs[i][p];
      memcpy(img.data() + L.op_off[p] + (size_t)i * osz, r.op.data(), osz);
      GroupEntry ge;
      ge.start = (unsigned)start;
      ge.gx = r.grid.x;
      ge.gy = r.grid.y;
      ge.gz = r.grid.z;
      memcpy(img.data() + L.ge_off[p] + (size_t)i * sizeof(GroupEntry), &ge, sizeof(ge));
      start += (unsigned long long)r.grid.x * r.grid.y * r.grid.z;
      if (r.smem > L.smem[p]) L.smem[p] = r.smem;
    }
    if (start > 0x7FFFFFFFull) {
      snprintf(b->err, sizeof(b->err), "launch %zu of the batch needs %llu blocks (limit 2^31-1)", p, start);
      return IBM_ERR_ARG;
    }
    L.blocks[p] = (unsigned)start;
    if (L.smem[p] > 48 * 1024) BCK(recs[0][p].set_smem((int)L.smem[p]));
  }
  if (b->dev) b->al.put(b->dev);
  b->dev = b->al.get(img.size());
  if (!b->dev) {
    snprintf(b->err, sizeof(b->err), "device allocation of the batch launch table failed");
    return IBM_ERR_OOM;
  }
  BCK(cudaMemcpy(b->dev, img.data(), img.size(), cudaMemcpyHostToDevice));
  return IBM_OK;
}

template <typename T>
static ibm_status batch_build(ibm_batch* b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  b->built = false;
  std::vector<std::vector<LaunchRec>> recs;
  BatchLayout L;
  ibm_status s = batch_record<T>(b, recs, L);
  if (s != IBM_OK) return s;
  BCK(cudaGetLastError());
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  batch_enqueue(b, recs, L, b->cap);
  const cudaError_t le = cudaGetLastError();
  cudaGraph_t gr = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &gr);
  if (le != cudaSuccess) {
    if (gr) cudaGraphDestroy(gr);
    return bfail(b, le, "kernel launch during batch capture");
  }
  if (e != cudaSuccess) return bfail(b, e, "batch graph capture");
  b->graph = gr;
  BCK(cudaGraphInstantiate(&b->exec, gr, 0));
  b->positions = count_kernel_nodes(gr);
  long long solo = 0;
  for (const auto& r : recs)
    for (const auto& x : r)
      if ((unsigned long long)x.grid.x * x.grid.y * x.grid.z > 0) ++solo;
  b->kernels_solo = solo;
  for (size_t i = 0; i < b->hs.size(); ++i) b->epochs[i] = b->hs[i]->epoch;
  b->built = true;
  return IBM_OK;
}

static ibm_status batch_prepare(ibm_batch* b) {
  for (ibm_handle h : b->hs)
    if (h->need_full_reset) {
      const ibm_status s = full_reset(h, h->user);
      if (s != IBM_OK) {
        snprintf(b->err, sizeof(b->err), "reset of an instance: %.400s", h->err);
        return s;
      }
    }
  bool stale = !b->built;
  for (size_t i = 0; i < b->hs.size() && !stale; ++i) stale = b->epochs[i] != b->hs[i]->epoch;
  if (!stale) return IBM_OK;
  return b->hs[0]->esize == 8 ? batch_build<double>(b) : batch_build<float>(b);
}

// the batch stream waits for every instance's stream (and vice versa after)
static ibm_status batch_join_in(ibm_batch* b) {
  for (ibm_handle h : b->hs) {
    BCK(cudaEventRecord(b->ev, h->user));
    BCK(cudaStreamWaitEvent(b->user, b->ev, 0));
  }
  return IBM_OK;
}
static ibm_status batch_join_out(ibm_batch* b) {
  BCK(cudaEventRecord(b->ev, b->user));
  for (ibm_handle h : b->hs) BCK(cudaStreamWaitEvent(h->user, b->ev, 0));
  return IBM_OK;
}

// handle lists stepped with ibm_step_batch, with their batch
static std::mutex g_batch_mu;
static std::vector<ibm_batch*> g_batch_cache;

// ---- autotuning ---------------------------------------------------------------
// Coordinate search over the launch-shape choices: every candidate value of
// one knob is timed (whole steps, CUDA events) with the others at their best
// so far.  The simulation state is saved before and restored after, and the
// tagging state is rebuilt at the next step.
struct Knob {
  int Tune::*field;
  std::vector<int> values;
};

static std::vector<Knob> tune_knobs() {
  return {{&Tune::fft_plane, {3, 2, 1}}, {&Tune::sweep_zy, {2, 1}}, {&Tune::sweep_y, {1, 2, 3, 4}}, {&Tune::tri_y, {1, 4, 2, 3}}, {&Tune::rhs, {3, 1, 2}},
          {&Tune::sweep_w, {64, 32, 16}},
          {&Tune::fft_lpb, {0, 8, 4, 2}},
          {&Tune::fft_cols, {16, 8, 4}}};
}

// state a trial step changes that the caller can observe
struct Snapshot {
  std::vector<std::pair<void*, size_t>> bufs;
  void* mem = nullptr;
};

static ibm_status snapshot_take(ibm_handle h, Snapshot& sn, cudaStream_t st) {
  const Geo& g = h->g;
  const size_t es = h->esize;
  sn.bufs.clear();
  sn.bufs.push_back({h->u, g.ncell * es});
  sn.bufs.push_back({h->v, g.nvf * es});
  sn.bufs.push_back({h->w, g.ncell * es});
  sn.bufs.push_back({h->p, g.ncell * es});
  for (int c = 0; c < 3; ++c) {
    const size_t n = (c == 1 ? g.nvf : g.ncell) * es;
    sn.bufs.push_back({h->H[c], n});
    if (h->lo[c]) sn.bufs.push_back({h->lo[c], n});
  }
  sn.bufs.push_back({h->ds, sizeof(DevState)});
  size_t tot = 0;
  for (auto& b : sn.bufs) tot += round16(b.second);
  sn.mem = h->al.get(tot);
  if (!sn.mem) {
    set_err(h, "%s", "device allocation of the autotuning snapshot failed");
    return IBM_ERR_OOM;
  }
  size_t off = 0;
  for (auto& b : sn.bufs) {
    CK(cudaMemcpyAsync((char*)sn.mem + off, b.first, b.second, cudaMemcpyDeviceToDevice, st));
    off += round16(b.second);
  }
  return IBM_OK;
}

static ibm_status snapshot_restore(ibm_handle h, Snapshot& sn, cudaStream_t st) {
  size_t off = 0;
  for (auto& b : sn.bufs) {
    CK(cudaMemcpyAsync(b.first, (char*)sn.mem + off, b.second, cudaMemcpyDeviceToDevice, st));
    off += round16(b.second);
  }
  CK(cudaStreamSynchronize(st));
  h->al.put(sn.mem);
  sn.mem = nullptr;
  h->need_full_reset = true;   // the sparse tagging reset follows the last trial's candidates
  return IBM_OK;
}

static void tune_out(const Tune& t, double ms, ibm_tune* out) {
  if (!out) return;
  out->tri_y = t.tri_y;
  out->sweep_w = t.sweep_w;
  out->fft_lpb = t.fft_lpb;
  out->fft_cols = t.fft_cols;
  out->sweep_zy = t.sweep_zy;
  out->fft_plane = t.fft_plane;
  out->sweep_y = t.sweep_y;
  out->rhs = t.rhs;
  out->corr_check = t.corr_check;
  out->ms_per_step = ms;
}

// Time `steps` replays of graph-making function `run_trial` for every
// candidate; returns the best configuration in `best`.
static void tune_log(const Tune& t, double ms) {
  static const bool on = getenv("IBM_AUTOTUNE_LOG") != nullptr;
  if (on)
    fprintf(stderr,
            "ibm autotune: tri_y %d sweep_w %d fft_lpb %d fft_cols %d sweep_zy %d fft_plane %d sweep_y %d rhs %d"
            " corr_check %d -> %.4f ms/step\n",
            t.tri_y, t.sweep_w, t.fft_lpb, t.fft_cols, t.sweep_zy, t.fft_plane, t.sweep_y, t.rhs, t.corr_check, ms);
}

template <class Trial>
static ibm_status autotune_loop(Tune& best, int steps, Trial trial, double* best_ms) {
  double bms = 0.0;
  ibm_status s = trial(best, steps, &bms);
  if (s != IBM_OK) return s;
  tune_log(best, bms);
  for (const Knob& k : tune_knobs()) {
    for (int v : k.values) {
      if (best.*(k.field) == v) continue;
      Tune cand = best;
      cand.*(k.field) = v;
      double ms = 0.0;
      s = trial(cand, steps, &ms);
      if (s != IBM_OK) return s;
      tune_log(cand, ms);
      if (ms < bms * 0.995) {
        bms = ms;
        best = cand;
      }
    }
  }
  if (best_ms) *best_ms = bms;
  return IBM_OK;
}

// ms per step of `steps` launches of graph exec `ge` on stream st (one
// untimed launch first)
static cudaError_t time_graph(cudaGraphExec_t ge, cudaStream_t st, int steps, double* ms) {
  cudaEvent_t a = nullptr, z = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  for (int i = 0; i < steps && e == cudaSuccess; ++i) e = cudaGraphLaunch(ge, st);
  if (e == cudaSuccess) e = cudaEventRecord(z, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(z);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, z);
  *ms = steps > 0 ? t / steps : 0.0;
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  return e;
}

extern "C" {

ibm_status ibm_set_allocator(ibm_alloc_fn alloc, ibm_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return IBM_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = free_fn;
  g_alloc_ctx = ctx;
  return IBM_OK;
}

const char* ibm_version(void) { return "ibm-gb300 0.1 (sm_103a)"; }

const char* ibm_last_error(ibm_handle h) { return h ? h->err : "null handle"; }

ibm_status ibm_create_grid(const ibm_grid_desc* desc, void* stream, ibm_handle* out) {
  if (!desc || !out) return IBM_ERR_ARG;
  *out = nullptr;
  const ibm_grid_desc d = *desc;
  if (!good_fft_size(d.nx) || !good_fft_size(d.nz) || d.ny < 4 || d.ny > 4096) return IBM_ERR_ARG;
  if (!(d.lx > 0 && d.ly > 0 && d.lz > 0 && d.re > 0 && d.dt > 0)) return IBM_ERR_ARG;
  if (d.scheme != IBM_RK2_CN && d.scheme != IBM_AB_CN) return IBM_ERR_ARG;
  if (d.ybc != IBM_NOSLIP && d.ybc != IBM_FREESLIP) return IBM_ERR_ARG;
  if (d.precision != IBM_FP64 && d.precision != IBM_MIXED && d.precision != IBM_MIXED_FAST) return IBM_ERR_ARG;
  if (d.use_q < 0 || d.use_q > 2) return IBM_ERR_ARG;
  const long long nvf = (long long)d.nx * (d.ny + 1) * d.nz;
  if (nvf >= (1ll << 30)) return IBM_ERR_ARG;   // node indices are packed into 30 bits
  ibm_handle h = new (std::nothrow) ibm_grid();   // value-initialised: every scalar and pointer is zero
  if (!h) return IBM_ERR_OOM;
  h->desc = d;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->al = Allocator{g_alloc, g_free, g_alloc_ctx};
  }
  h->user = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  Geo& g = h->g;
  g.nx = d.nx; g.ny = d.ny; g.nz = d.nz; g.nkx = d.nx / 2 + 1;
  g.ybc = d.ybc;
  g.lx = d.lx; g.ly = d.ly; g.lz = d.lz;
  g.dx = d.lx / (double)d.nx;
  g.dy = d.ly / (double)d.ny;
  g.dz = d.lz / (double)d.nz;
  g.idx = 1.0 / g.dx; g.idy = 1.0 / g.dy; g.idz = 1.0 / g.dz;
  {
    // squared cell diagonal, rounded term by term without contraction
    volatile double sx = g.dx * g.dx, sy = g.dy * g.dy, sz = g.dz * g.dz;
    volatile double sxy = sx + sy;
    g.diag2 = sxy + sz;
  }
  g.h = 2.0 * sqrt(g.diag2);
  g.ncell = (long long)d.nx * d.ny * d.nz;
  g.nvf = nvf;
  h->esize = d.precision == IBM_FP64 ? sizeof(double) : sizeof(float);
  ibm_status rc = IBM_OK;
  cudaError_t ce = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (ce != cudaSuccess) {
    release_all(h);
    delete h;
    return IBM_ERR_CUDA;
  }
  init_kernel_attributes();
  init_sweep_attributes();
  const size_t es = h->esize;
  const long long ncell = g.ncell, nall = 2 * ncell + nvf;
  h->u = dalloc(h, ncell * es);
  h->v = dalloc(h, nvf * es);
  h->w = dalloc(h, ncell * es);
  h->p = dalloc(h, ncell * es);
  for (int c = 0; c < 3; ++c) {
    h->H[c] = dalloc(h, (c == 1 ? nvf : ncell) * es);
    h->R[c] = dalloc(h, (c == 1 ? nvf : ncell) * es);
  }
  h->scr = dalloc(h, nall * es);
  h->phi = dalloc(h, ncell * es);
  h->spec = dalloc(h, (size_t)g.nz * g.ny * g.nkx * 2 * es);
  if (d.precision == IBM_MIXED) {
    for (int c = 0; c < 3; ++c) {
      h->lo[c] = dalloc(h, (c == 1 ? nvf : ncell) * es);
      if (!h->lo[c]) { release_all(h); delete h; return IBM_ERR_OOM; }
    }
    h->phi2 = dalloc(h, ncell * es);
    if (!h->phi2) { release_all(h); delete h; return IBM_ERR_OOM; }
  }
  if (d.use_q == 2) {
    h->qk = dalloc(h, ncell * es);
    if (!h->qk) { release_all(h); delete h; return IBM_ERR_OOM; }
  }
  h->ds = (DevState*)dalloc(h, sizeof(DevState));
  h->partial = (double*)dalloc(h, 16384 * sizeof(double));
  h->tb.d2min = (unsigned long long*)dalloc(h, nall * 8);
  h->tb.owner = (unsigned*)dalloc(h, nall * 4);
  h->tb.ub = (unsigned*)dalloc(h, nall * 4);
  h->tb.flags32 = (unsigned*)dalloc(h, round16((size_t)(ncell + 3) / 4 * 4));
  h->tb.blk = (unsigned*)dalloc(h, (size_t)compaction_blocks(g) * 4 * sizeof(unsigned));
  h->bad = (unsigned*)dalloc(h, 16);
  {
    const size_t nxl = 3ull * g.nz * (g.ny + 1), nzl = 3ull * (g.ny + 1) * g.nx, nyl = 3ull * g.nz * g.nx;
    h->tb.lines.bytes = (nxl + nzl + nyl) * sizeof(int);
    h->tb.lines.x = (int*)dalloc(h, h->tb.lines.bytes);
    h->tb.lines.z = h->tb.lines.x ? h->tb.lines.x + nxl : nullptr;
    h->tb.lines.y = h->tb.lines.x ? h->tb.lines.z + nzl : nullptr;
  }
  void* need[] = {h->u, h->v, h->w, h->p, h->H[0], h->H[1], h->H[2], h->R[0], h->R[1], h->R[2], h->scr,
                  h->phi, h->spec, h->ds, h->partial, h->tb.d2min, h->tb.owner, h->tb.ub, h->tb.flags32, h->tb.blk,
                  h->bad, h->tb.lines.x};
  for (void* q : need)
    if (!q) {
      release_all(h);
      delete h;
      return IBM_ERR_OOM;
    }
  if (alloc_lists(h, 1u << 16) != IBM_OK) {
    release_all(h);
    delete h;
    return IBM_ERR_OOM;
  }
  // coefficient tables: one beta for every sub-stage of the scheme
  Stage sg[2];
  stages(d, sg);
  const double beta = sg[0].alp * d.dt / (2.0 * d.re);
  h->tbl_off[0] = beta / (g.dx * g.dx);
  h->tbl_off[1] = beta / (g.dy * g.dy);
  h->tbl_off[2] = beta / (g.dz * g.dz);
  bool ok;
  if (d.precision == IBM_FP64)
    ok = build_periodic<double>(h, d.nx, h->tbl_off[0], 0) && build_periodic<double>(h, d.nz, h->tbl_off[2], 1) &&
         build_wall<double>(h, h->tbl_off[1]);
  else
    ok = build_periodic<float>(h, d.nx, h->tbl_off[0], 0) && build_periodic<float>(h, d.nz, h->tbl_off[2], 1) &&
         build_wall<float>(h, h->tbl_off[1]);
  if (ok && d.precision != IBM_FP64 && d.ny <= 1024) {
    // FP32 rows of the tabulated y sweep (launch shape sweep_y = 3), the
    // uniform spacing written as the non-uniform grid's tables
    std::vector<double> ih(d.ny + 1, g.idy), t1(6ull * d.ny - 3), t2;
    y_sweep_rows(d.ny, h->tbl_off[0] * g.dx * g.dx, d.ybc == 0 ? -1.0 : 1.0, ih.data(), ih.data(), t1.data(), &t2);
    h->g.yt.yswf = (const float*)upload_vec<float>(h, t1);
    h->g.yt.ysw2f = (const float*)upload_vec<float>(h, t2);
    ok = h->g.yt.yswf && h->g.yt.ysw2f;
  }
  // Poisson: modified wavenumbers, twiddles, pivots
  const double pi = 3.14159265358979323846;
  std::vector<double> lx(g.nkx), lz(g.nz), twx(2 * g.nx), twz(2 * g.nz);
  for (int k = 0; k < g.nkx; ++k) lx[k] = (2.0 - 2.0 * cos(2.0 * pi * k / g.nx)) / (g.dx * g.dx);
  for (int k = 0; k < g.nz; ++k) lz[k] = (2.0 - 2.0 * cos(2.0 * pi * k / g.nz)) / (g.dz * g.dz);
  for (int m = 0; m < g.nx; ++m) { twx[2 * m] = cos(2.0 * pi * m / g.nx); twx[2 * m + 1] = -sin(2.0 * pi * m / g.nx); }
  for (int m = 0; m < g.nz; ++m) { twz[2 * m] = cos(2.0 * pi * m / g.nz); twz[2 * m + 1] = -sin(2.0 * pi * m / g.nz); }
  h->lamx = (double*)upload_vec<double>(h, lx);
  h->lamz = (double*)upload_vec<double>(h, lz);
  if (d.precision == IBM_FP64) {
    h->twx = upload_vec<double>(h, twx);
    h->twz = upload_vec<double>(h, twz);
  } else {
    h->twx = upload_vec<float>(h, twx);
    h->twz = upload_vec<float>(h, twz);
  }
  const size_t nspec = (size_t)g.nz * g.ny * g.nkx;
  h->pcp = (double*)dalloc(h, nspec * 8);
  h->pinv = (double*)dalloc(h, nspec * 8);
  const size_t nsegs = (size_t)g.nz * ((g.ny + TRI_SEG - 1) / TRI_SEG) * g.nkx;
  h->psegf = (double*)dalloc(h, nsegs * 8);
  h->psegb = (double*)dalloc(h, nsegs * 8);
  h->pjc = (int*)dalloc(h, (size_t)g.nz * g.nkx * sizeof(int));
  if (!ok || !h->lamx || !h->lamz || !h->twx || !h->twz || !h->pcp || !h->pinv || !h->psegf || !h->psegb ||
      !h->pjc) {
    release_all(h);
    delete h;
    return IBM_ERR_OOM;
  }
  cudaStream_t st = h->user;
  launch_build_poisson_tables(g, h->lamx, h->lamz, h->pcp, h->pinv, h->psegf, h->psegb, h->pjc, st);
  // state at rest
  cudaMemsetAsync(h->u, 0, ncell * es, st);
  cudaMemsetAsync(h->v, 0, nvf * es, st);
  cudaMemsetAsync(h->w, 0, ncell * es, st);
  cudaMemsetAsync(h->p, 0, ncell * es, st);
  for (int c = 0; c < 3; ++c) {
    cudaMemsetAsync(h->H[c], 0, (c == 1 ? nvf : ncell) * es, st);
    if (h->lo[c]) cudaMemsetAsync(h->lo[c], 0, (c == 1 ? nvf : ncell) * es, st);
  }
  if (h->phi2) cudaMemsetAsync(h->phi2, 0, ncell * es, st);
  cudaMemsetAsync(h->ds, 0, sizeof(DevState), st);
  cudaMemsetAsync(h->bad, 0, 16, st);   // reused device memory is not zero
  cudaMemsetAsync(h->tb.cand, 0, sizeof(Cand), st);
  if (full_reset(h, st) != IBM_OK) rc = IBM_ERR_CUDA;
  ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess || rc != IBM_OK) {
    release_all(h);
    delete h;
    return IBM_ERR_CUDA;
  }
  *out = h;
  return IBM_OK;
}

ibm_status ibm_create_grid_stretched(const ibm_grid_desc* desc, const double* y_faces, void* stream,
                                      ibm_handle* out) {
  if (!desc || !y_faces || !out) return IBM_ERR_ARG;
  *out = nullptr;
  const int ny = desc->ny;
  if (ny < 4 || ny > 4096) return IBM_ERR_ARG;
  if (y_faces[0] != 0.0 || !(fabs(y_faces[ny] - desc->ly) <= 1e-12 * desc->ly)) return IBM_ERR_ARG;
  for (int j = 0; j < ny; ++j)
    if (!(y_faces[j + 1] > y_faces[j])) return IBM_ERR_ARG;
  ibm_handle h = nullptr;
  ibm_status st = ibm_create_grid(desc, stream, &h);
  if (st != IBM_OK) return st;
  // spacing tables: cell heights, centre distances across faces (mirrored
  // centres at the walls), as the oracle defines them
  std::vector<double> t(6ull * ny + 7 + 6ull * ny - 3);
  double* ihc = t.data();
  double* ihf = ihc + ny;
  double* hc = ihf + ny + 1;
  double* hf = hc + ny;
  double* yc = hf + ny + 1;
  double* yv = yc + ny + 2;
  for (int j = 0; j < ny; ++j) hc[j] = y_faces[j + 1] - y_faces[j];
  for (int j = 0; j < ny; ++j) ihc[j] = 1.0 / hc[j];
  hf[0] = hc[0];
  hf[ny] = hc[ny - 1];
  for (int j = 1; j < ny; ++j) hf[j] = 0.5 * (y_faces[j] + y_faces[j + 1]) - 0.5 * (y_faces[j - 1] + y_faces[j]);
  for (int j = 0; j <= ny; ++j) ihf[j] = 1.0 / hf[j];
  // row coordinates, one mirrored row beyond each wall (y_faces[0] = 0)
  for (int j = 0; j < ny; ++j) yc[j + 1] = 0.5 * (y_faces[j] + y_faces[j + 1]);
  yc[0] = -yc[1];
  yc[ny + 1] = 2.0 * y_faces[ny] - yc[ny];
  for (int j = 0; j <= ny; ++j) yv[j + 1] = y_faces[j];
  yv[0] = -y_faces[1];
  yv[ny + 2] = 2.0 * y_faces[ny] - y_faces[ny - 1];
  // y sweep rows (one wall segment; and [start row][row] segments for ny up
  // to 1024), with beta as the sweep kernel receives it (the x table's
  // coefficient times dx^2, in the path's own type)
  std::vector<double> t2;
  {
    const double ox = desc->precision == IBM_FP64 ? h->tbl_off[0] : (double)(float)h->tbl_off[0];
    y_sweep_rows(ny, ox * h->g.dx * h->g.dx, h->g.ybc == 0 ? -1.0 : 1.0, ihc, ihf, yv + ny + 3,
                 ny <= 1024 ? &t2 : nullptr);
  }
  double smin = hc[0], smax = hc[0];
  for (int j = 0; j < ny; ++j) { smin = std::min(smin, hc[j]); smax = std::max(smax, hc[j]); }
  for (int j = 0; j <= ny; ++j) { smin = std::min(smin, hf[j]); smax = std::max(smax, hf[j]); }
  h->ytab = (double*)upload_vec<double>(h, t);
  double* ysw2 = t2.empty() ? nullptr : (double*)upload_vec<double>(h, t2);
  // FP32 copies of the sweep tables for the mixed paths
  float* yswf = nullptr;
  float* ysw2f = nullptr;
  bool f32_ok = true;
  if (desc->precision != IBM_FP64) {
    yswf = (float*)upload_vec<float>(h, std::vector<double>(t.begin() + (6ll * ny + 7), t.end()));
    if (!t2.empty()) ysw2f = (float*)upload_vec<float>(h, t2);
    f32_ok = yswf && (t2.empty() || ysw2f);
  }
  // rows of the tagging pre-screen: FP32 position, wall-normal side of the
  // node's local cell, distances to the rows below and above
  float4* rowf = nullptr;
  {
    std::vector<float> rf(8ull * (ny + 1), 0.0f);
    for (int half = 0; half < 2; ++half)
      for (int j = 0; j <= ny; ++j) {
        const double* yr = half ? yc : yv;   // [j + 1] = row j; one mirrored row beyond each wall
        if (half && j == ny) continue;      // (centre rows end at ny - 1)
        const double y = yr[j + 1], ylo = yr[j], yhi = yr[j + 2];
        const double hy = half ? hc[j] : hf[j];
        float* q = rf.data() + 4ull * (half * (ny + 1) + j);
        q[0] = (float)y;
        q[1] = (float)hy;
        q[2] = (float)(y - ylo);
        q[3] = (float)(yhi - y);
      }
    rowf = (float4*)dalloc(h, rf.size() * sizeof(float));
    if (rowf && cudaMemcpy(rowf, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      rowf = nullptr;
  }
  const size_t nspec = (size_t)h->g.nz * h->g.ny * h->g.nkx;
  h->pal = (double*)dalloc(h, nspec * 8);
  if (!h->ytab || !h->pal || (!t2.empty() && !ysw2) || !f32_ok || !rowf) {
    ibm_destroy(h);
    return IBM_ERR_OOM;
  }
  h->g.yt.ihc = h->ytab;
  h->g.yt.ihf = h->ytab + ny;
  h->g.yt.hc = h->ytab + 2 * ny + 1;
  h->g.yt.hf = h->ytab + 3 * ny + 1;
  h->g.yt.yc = h->ytab + 4 * ny + 2;
  h->g.yt.yv = h->ytab + 5 * ny + 4;
  h->g.yt.ysw = h->ytab + 6 * ny + 7;
  h->g.yt.ysw2 = ysw2;
  h->g.yt.yswf = yswf;
  h->g.yt.ysw2f = ysw2f;
  h->g.yt.rowf = rowf;
  h->g.yt.hmax = smax;
  h->ysp_min = smin;
  launch_build_poisson_tables_nu(h->g, h->lamx, h->lamz, h->pcp, h->pinv, h->pal, h->user);
  if (cudaStreamSynchronize(h->user) != cudaSuccess) {
    ibm_destroy(h);
    return IBM_ERR_CUDA;
  }
  invalidate(h);
  *out = h;
  return IBM_OK;
}

ibm_status ibm_destroy(ibm_handle h) {
  if (!h) return IBM_ERR_ARG;
  cudaStreamSynchronize(h->user);
  {
    // batches made by ibm_step_batch that hold this handle go with it
    std::vector<ibm_batch*> drop;
    {
      std::lock_guard<std::mutex> lk(g_batch_mu);
      for (ibm_batch* b : g_batch_cache)
        if (std::find(b->hs.begin(), b->hs.end(), h) != b->hs.end()) drop.push_back(b);
    }
    for (ibm_batch* b : drop) ibm_batch_destroy(b);
  }
  release_all(h);
  delete h;
  return IBM_OK;
}

ibm_status ibm_set_body_force(ibm_handle h, double fx, double fy, double fz) {
  if (!h) return IBM_ERR_ARG;
  k_set_force<<<1, 1, 0, h->user>>>(h->ds, fx, fy, fz);
  return launch_status(h, "ibm_set_body_force");
}

ibm_status ibm_set_div_budget(ibm_handle h, double budget) {
  if (!h || !(budget >= 0.0)) return IBM_ERR_ARG;
  // rounded down to FP32, so a residual the FP32 comparison lets through is
  // within the budget as given
  float b = (float)budget;
  if ((double)b > budget) b = nextafterf(b, 0.0f);
  k_set_budget<<<1, 1, 0, h->user>>>(h->ds, b);
  return launch_status(h, "ibm_set_div_budget");
}

// upper bound of the candidates a surface can produce: nodes inside every
// triangle's Cartesian box (with the one-cell margin of Algorithm 1)
// (non-uniform wall-normal grid: rows at least ysp_min apart, margins of at
// most g.yt.hmax)
static unsigned long long candidate_bound(const Geo& g, double ysp_min, const double* xyz, const int32_t* tri,
                                          int nt) {
  unsigned long long tot = 0;
  const double del[3] = {g.dx, ysp_min > 0.0 ? ysp_min : g.dy, g.dz};
  const double pad = ysp_min > 0.0 ? 2.0 * g.yt.hmax : 0.0;
  for (int t = 0; t < nt; ++t) {
    unsigned long long prod = 1;
    for (int d = 0; d < 3; ++d) {
      double mn = 1e300, mx = -1e300;
      for (int m = 0; m < 3; ++m) {
        const double x = xyz[3 * (long long)tri[3 * t + m] + d];
        mn = x < mn ? x : mn;
        mx = x > mx ? x : mx;
      }
      long long cnt = (long long)ceil((mx - mn + (d == 1 ? pad : 0.0)) / del[d]) + 4;
      if (d == 1 && cnt > g.ny + 1) cnt = g.ny + 1;
      prod *= (unsigned long long)cnt;
    }
    tot += 3 * prod;
  }
  return tot;
}

ibm_status ibm_set_surface(ibm_handle h, int nverts, const double* xyz, const double* vel, int ntris,
                           const int32_t* tri, int on_device) {
  if (!h || nverts < 0 || ntris < 0) return IBM_ERR_ARG;
  if (ntris == 0) {
    if (h->nt != 0) invalidate(h);
    h->nt = 0;
    h->nv = 0;
    return IBM_OK;
  }
  if (nverts < 3 || !xyz || !vel) return IBM_ERR_ARG;
  if (!tri && (!h->has_topology || ntris != h->nt)) {
    set_err(h, "%s", "ibm_set_surface: tri == NULL needs the previous connectivity with the same ntris");
    return IBM_ERR_STATE;
  }
  cudaStream_t st = h->user;
  // (re)allocate surface storage
  if (nverts > h->nv_cap || ntris > h->nt_cap) {
    const int nvc = nverts > h->nv_cap ? nverts : h->nv_cap;
    const int ntc = ntris > h->nt_cap ? ntris : h->nt_cap;
    CK(cudaStreamSynchronize(st));
    int* old_t = h->st;
    double* nsx = (double*)dalloc(h, 3ull * nvc * 8);
    double* nsu = (double*)dalloc(h, 3ull * nvc * 8);
    int* nst = (int*)dalloc(h, 3ull * ntc * 4);
    double* ngx = (double*)dalloc(h, 3ull * nvc * 8);
    int* ngt = (int*)dalloc(h, 3ull * ntc * 4);
    TriRec* nrec = (TriRec*)dalloc(h, (size_t)ntc * sizeof(TriRec));
    if (!nsx || !nsu || !nst || !ngx || !ngt || !nrec) {
      set_err(h, "%s", "device allocation of the surface failed");
      return IBM_ERR_OOM;
    }
    if (old_t && !tri && h->nt > 0) CK(cudaMemcpy(nst, old_t, 3ull * h->nt * 4, cudaMemcpyDeviceToDevice));
    dfree(h, h->sx); dfree(h, h->su); dfree(h, h->st); dfree(h, h->stage_x); dfree(h, h->stage_t);
    dfree(h, h->trirec);
    h->sx = nsx; h->su = nsu; h->st = nst; h->stage_x = ngx; h->stage_t = ngt; h->trirec = nrec;
    h->nv_cap = nvc;
    h->nt_cap = ntc;
    invalidate(h);
  }
  // host-side checks and the candidate-capacity bound
  if (!on_device) {
    if (tri) {
      for (long long m = 0; m < 3ll * ntris; ++m)
        if (tri[m] < 0 || tri[m] >= nverts) {
          set_err(h, "%s", "ibm_set_surface: triangle vertex index out of range");
          return IBM_ERR_ARG;
        }
      h->host_tri.assign(tri, tri + 3ll * ntris);
    } else if (h->host_tri.size() != 3ull * ntris) {
      // connectivity given on the device earlier: one read back, kept
      std::vector<int> soa(3ull * ntris);
      CK(cudaMemcpy(soa.data(), h->st, 3ull * ntris * 4, cudaMemcpyDeviceToHost));
      h->host_tri.resize(3ull * ntris);
      for (int t = 0; t < ntris; ++t)
        for (int m = 0; m < 3; ++m) h->host_tri[3ull * t + m] = soa[(size_t)m * ntris + t];
    }
    const int32_t* tt = tri ? tri : h->host_tri.data();
    unsigned long long need = candidate_bound(h->g, h->ysp_min, xyz, tt, ntris);
    if (need > 0xF0000000ull) need = 0xF0000000ull;
    if (need > h->tb.cap) {
      CK(cudaStreamSynchronize(st));
      unsigned cap = (unsigned)need;
      if (alloc_lists(h, cap) != IBM_OK) return IBM_ERR_OOM;
    }
  } else if (!h->has_topology || ntris != h->nt) {
    // device surface: size the lists once from a host copy of the first one
    std::vector<double> hx(3ull * nverts);
    std::vector<int32_t> ht(3ull * ntris);
    CK(cudaMemcpy(hx.data(), xyz, hx.size() * 8, cudaMemcpyDeviceToHost));
    if (tri) CK(cudaMemcpy(ht.data(), tri, ht.size() * 4, cudaMemcpyDeviceToHost));
    else {
      std::vector<int> soa(3ull * ntris);
      CK(cudaMemcpy(soa.data(), h->st, 3ull * ntris * 4, cudaMemcpyDeviceToHost));
      for (int t = 0; t < ntris; ++t)
        for (int m = 0; m < 3; ++m) ht[3ull * t + m] = soa[(size_t)m * ntris + t];
    }
    for (long long m = 0; m < 3ll * ntris; ++m)
      if (ht[m] < 0 || ht[m] >= nverts) {
        set_err(h, "%s", "ibm_set_surface: triangle vertex index out of range");
        return IBM_ERR_ARG;
      }
    h->host_tri.swap(ht);
    unsigned long long need = candidate_bound(h->g, h->ysp_min, hx.data(), h->host_tri.data(), ntris) * 3 / 2;
    if (need > 0xF0000000ull) need = 0xF0000000ull;
    if (need > h->tb.cap) {
      CK(cudaStreamSynchronize(st));
      if (alloc_lists(h, (unsigned)need) != IBM_OK) return IBM_ERR_OOM;
    }
  }
  if (on_device && tri && h->has_topology && ntris == h->nt) h->host_tri.clear();   // new device connectivity
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const int tb = 256;
  CK(cudaMemcpyAsync(h->stage_x, xyz, 3ull * nverts * 8, kind, st));
  k_aos_to_soa<<<(nverts + tb - 1) / tb, tb, 0, st>>>(h->stage_x, h->sx, nverts);
  CK(cudaMemcpyAsync(h->stage_x, vel, 3ull * nverts * 8, kind, st));
  k_aos_to_soa<<<(nverts + tb - 1) / tb, tb, 0, st>>>(h->stage_x, h->su, nverts);
  if (tri) {
    CK(cudaMemcpyAsync(h->stage_t, tri, 3ull * ntris * 4, kind, st));
    k_tri_to_soa<<<(ntris + tb - 1) / tb, tb, 0, st>>>(h->stage_t, h->st, ntris, nverts, h->bad);
  }
  CK(cudaGetLastError());
  if (nverts != h->nv || ntris != h->nt) invalidate(h);
  h->nv = nverts;
  h->nt = ntris;
  h->has_topology = true;
  return launch_status(h, "ibm_set_surface");
}

ibm_status ibm_set_fields(ibm_handle h, const double* u, const double* v, const double* w, const double* p,
                          int on_device) {
  if (!h) return IBM_ERR_ARG;
  const Geo& g = h->g;
  cudaStream_t st = h->user;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* src[4] = {u, v, w, p};
  void* dst[4] = {h->u, h->v, h->w, h->p};
  const long long n[4] = {g.ncell, g.nvf, g.ncell, g.ncell};
  for (int q = 0; q < 4; ++q) {
    if (!src[q]) continue;
    if (h->esize == 8) {
      CK(cudaMemcpyAsync(dst[q], src[q], n[q] * 8, kind, st));
    } else {
      // stage through the scratch array (large enough for any field in FP64? use R buffers)
      double* stage = (double*)h->scr;   // scr holds 2*ncell+nvf floats = enough bytes for one FP64 field
      CK(cudaMemcpyAsync(stage, src[q], n[q] * 8, kind, st));
      if (q < 3 && h->lo[q])
        k_split<<<num_sms() * 4, 256, 0, st>>>(stage, (float*)dst[q], (float*)h->lo[q], n[q]);
      else
        k_convert<double, float><<<num_sms() * 4, 256, 0, st>>>(stage, (float*)dst[q], n[q]);
    }
  }
  for (int c = 0; c < 3; ++c) CK(cudaMemsetAsync(h->H[c], 0, (c == 1 ? g.nvf : g.ncell) * h->esize, st));
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

static ibm_status check_device(ibm_handle h, const DevState* have = nullptr);

// Copy the non-linear history H of the three grids out of / into the handle
// (FP64 caller arrays; the mixed paths convert, exactly in both directions).
ibm_status ibm_get_history(ibm_handle h, double* hu, double* hv, double* hw, int on_device) {
  if (!h) return IBM_ERR_ARG;
  const Geo& g = h->g;
  cudaStream_t st = h->user;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dst[3] = {hu, hv, hw};
  for (int c = 0; c < 3; ++c) {
    if (!dst[c]) continue;
    const long long n = comp_size(g, c);
    if (h->esize == 8) {
      CK(cudaMemcpyAsync(dst[c], h->H[c], n * 8, kind, st));
    } else {
      double* stage = (double*)h->scr;
      k_convert<float, double><<<num_sms() * 4, 256, 0, st>>>((const float*)h->H[c], stage, n);
      CK(cudaMemcpyAsync(dst[c], stage, n * 8, kind, st));
    }
    CK(cudaStreamSynchronize(st));
  }
  return check_device(h);
}

ibm_status ibm_set_history(ibm_handle h, const double* hu, const double* hv, const double* hw, int on_device) {
  if (!h) return IBM_ERR_ARG;
  const Geo& g = h->g;
  cudaStream_t st = h->user;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const double* src[3] = {hu, hv, hw};
  for (int c = 0; c < 3; ++c) {
    if (!src[c]) continue;
    const long long n = comp_size(g, c);
    if (h->esize == 8) {
      CK(cudaMemcpyAsync(h->H[c], src[c], n * 8, kind, st));
    } else {
      double* stage = (double*)h->scr;
      CK(cudaMemcpyAsync(stage, src[c], n * 8, kind, st));
      k_convert<double, float><<<num_sms() * 4, 256, 0, st>>>(stage, (float*)h->H[c], n);
    }
  }
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(st));
  return IBM_OK;
}

// Turn the device error word (and the surface-index flag) into a status.
// `have` (optional) is a device-state copy taken after the stream finished.
static ibm_status check_device(ibm_handle h, const DevState* have) {
  DevState ds;
  unsigned bad = 0;
  if (have) {
    ds = *have;
  } else {
    CK(cudaMemcpyAsync(&ds, h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, h->user));
  }
  CK(cudaMemcpyAsync(&bad, h->bad, sizeof(unsigned), cudaMemcpyDeviceToHost, h->user));
  CK(cudaStreamSynchronize(h->user));
  if (bad) {
    CK(cudaMemset(h->bad, 0, sizeof(unsigned)));
    set_err(h, "%s", "triangle vertex index out of range (device surface)");
    return IBM_ERR_ARG;
  }
  if (ds.err) {
    CK(cudaMemset(&h->ds->err, 0, sizeof(unsigned)));
    if (ds.err & (ERR_CAND_OVERFLOW | ERR_LIST_OVERFLOW)) {
      set_err(h, "%s", "a tagging work list overflowed; capacity doubled, redo the step");
      unsigned cap = h->tb.cap;
      unsigned nc = cap > 0x78000000u ? 0xF0000000u : cap * 2;
      if (ds.ncand > nc) nc = ds.ncand + ds.ncand / 2;
      if (alloc_lists(h, nc) != IBM_OK) return IBM_ERR_OOM;
      return IBM_ERR_CAPACITY;
    }
    if (ds.err & ERR_PROBE) {
      set_err(h, "%s", "an IB probe left the domain (body too close to a wall)");
      return IBM_ERR_GEOMETRY;
    }
    if (ds.err & ERR_NONFINITE) {
      set_err(h, "%s", "non-finite values in the solution");
      return IBM_ERR_DIVERGED;
    }
    if (ds.err & ERR_WAIT) {
      set_err(h, "%s", "an asynchronous tile copy did not complete within its wait limit");
      return IBM_ERR_CUDA;
    }
    set_err(h, "%s", "device error");
    return IBM_ERR_CUDA;
  }
  return IBM_OK;
}

ibm_status ibm_sync(ibm_handle h) {
  if (!h) return IBM_ERR_ARG;
  CK(cudaStreamSynchronize(h->user));
  return check_device(h);
}

ibm_status ibm_step(ibm_handle h, int nsteps) {
  if (!h || nsteps < 0) return IBM_ERR_ARG;
  if (h->need_full_reset) {
    ibm_status s = full_reset(h, h->user);
    if (s != IBM_OK) return s;
  }
  if (!h->graph_ok) {
    ibm_status s = h->esize == 8 ? capture<double>(h) : capture<float>(h);
    if (s != IBM_OK) return s;
  }
  for (int n = 0; n < nsteps; ++n) CK(cudaGraphLaunch(h->exec, h->user));
  h->steps += nsteps;
  return launch_status(h, "ibm_step");
}

ibm_status ibm_get_fields(ibm_handle h, double* u, double* v, double* w, double* p, int on_device) {
  if (!h) return IBM_ERR_ARG;
  const Geo& g = h->g;
  cudaStream_t st = h->user;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  double* dst[4] = {u, v, w, p};
  void* src[4] = {h->u, h->v, h->w, h->p};
  const long long n[4] = {g.ncell, g.nvf, g.ncell, g.ncell};
  for (int q = 0; q < 4; ++q) {
    if (!dst[q]) continue;
    if (h->esize == 8) {
      CK(cudaMemcpyAsync(dst[q], src[q], n[q] * 8, kind, st));
    } else {
      double* stage = (double*)h->scr;
      if (q < 3 && h->lo[q])
        k_join<<<num_sms() * 4, 256, 0, st>>>((const float*)src[q], (const float*)h->lo[q], stage, n[q]);
      else
        k_convert<float, double><<<num_sms() * 4, 256, 0, st>>>((const float*)src[q], stage, n[q]);
      CK(cudaMemcpyAsync(dst[q], stage, n[q] * 8, kind, st));
      CK(cudaStreamSynchronize(st));
    }
  }
  CK(cudaStreamSynchronize(st));
  return check_device(h);
}

ibm_status ibm_get_tags(ibm_handle h, int comp, int32_t* owner, int on_device) {
  if (!h || comp < 0 || comp > 2 || !owner) return IBM_ERR_ARG;
  const Geo& g = h->g;
  const long long n = comp_size(g, comp);
  const unsigned* src = h->tb.owner + comp_off(g, comp);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(owner, src, n * 4, kind, h->user));
  CK(cudaStreamSynchronize(h->user));
  return check_device(h);
}

ibm_status ibm_get_diag(ibm_handle h, ibm_diag* out) {
  if (!h || !out) return IBM_ERR_ARG;
  DevState ds;
  CK(cudaMemcpyAsync(&ds, h->ds, sizeof(DevState), cudaMemcpyDeviceToHost, h->user));
  ibm_status s = check_device(h, &ds);
  memset(out, 0, sizeof(*out));
  out->d2h_bytes = (int64_t)(sizeof(DevState) + sizeof(unsigned));
  double tot = 0.0;
  for (int c = 0; c < 3; ++c) {
    out->nforce[c] = ds.nforce_c[c];
    out->slip_comp[c] = ds.nforce_c[c] ? ds.slip_sum[c] / (double)ds.nforce_c[c] : 0.0;
    tot += out->slip_comp[c];
  }
  out->slip_l1 = tot / 3.0;
  out->nboundary = ds.nbound;
  Stage sg[2];
  const int ns = stages(h->desc, sg);
  out->q_f = ds.qf[ns - 1];
  out->sum_q_dv = ds.sum_qdv[ns - 1];   // formed with the fluid volume of the q reduction
  out->steps = (int64_t)ds.steps;
  out->ncandidates = ds.ncand;
  out->kernels_per_step = h->kernels_per_step;
  out->div_max = ds.div_max;
  out->ke = ds.ke;
  out->cfl = ds.cfl;
  if (h->desc.precision == IBM_MIXED) {
    float r = 0.0f;
    for (int i = 0; i < ns; ++i) {
      float v;
      memcpy(&v, &ds.res1[i], sizeof v);
      r = (v > r || v != v) ? v : r;
    }
    out->div_first = r;
    out->corr_solves = (int64_t)ds.ncorr;
  }
  return s;
}

const char* ibm_stage_name(int stage) { return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : ""; }

ibm_status ibm_profile_stages(ibm_handle h, int nsteps, double* ms, int64_t* kernels) {
  if (!h || nsteps < 0) return IBM_ERR_ARG;
  if (h->need_full_reset) {
    ibm_status s = full_reset(h, h->user);
    if (s != IBM_OK) return s;
  }
  const ibm_status rc = profile_graph(
      [&](cudaStream_t st) {
        Exec ex = solo_exec(h, st);
        if (h->esize == 8) enqueue_step<double>(h, ex);
        else enqueue_step<float>(h, ex);
      },
      h->cap, h->user, nsteps, ms, kernels, h->err, sizeof(h->err));
  if (rc != IBM_OK) return rc;
  h->steps += nsteps;
  {
    const ibm_status ls = launch_status(h, "ibm_profile_stages");
    if (ls != IBM_OK) return ls;
  }
  return check_device(h);
}


// ---- tuning -------------------------------------------------------------------
static bool tune_valid(const ibm_tune* t) {
  if (!t) return false;
  if (t->tri_y < 0 || t->tri_y > 4) return false;
  if (t->sweep_w != 0 && t->sweep_w != 16 && t->sweep_w != 32 && t->sweep_w != 64) return false;
  if (t->fft_lpb < 0 || t->fft_lpb > 2048) return false;
  if (t->fft_cols < 0 || t->fft_cols > 16 || (t->fft_cols & (t->fft_cols - 1))) return false;
  if (t->sweep_zy < 0 || t->sweep_zy > 2) return false;
  if (t->fft_plane < 0 || t->fft_plane > 3) return false;
  if (t->sweep_y < 0 || t->sweep_y > 4) return false;
  if (t->rhs < 0 || t->rhs > 3) return false;
  if (t->corr_check < 0 || t->corr_check > 2) return false;
  return true;
}

ibm_status ibm_set_tune(ibm_handle h, const ibm_tune* t) {
  if (!h || !tune_valid(t)) return IBM_ERR_ARG;
  h->tune = Tune{t->tri_y, t->sweep_w, t->fft_lpb, t->fft_cols, t->sweep_zy, t->fft_plane, t->sweep_y, t->rhs,
                 t->corr_check};
  invalidate(h);
  return IBM_OK;
}

ibm_status ibm_get_tune(ibm_handle h, ibm_tune* t) {
  if (!h || !t) return IBM_ERR_ARG;
  tune_out(h->tune, 0.0, t);
  return IBM_OK;
}

ibm_status ibm_autotune(ibm_handle h, int steps, ibm_tune* chosen) {
  if (!h || steps < 1) return IBM_ERR_ARG;
  if (h->need_full_reset) {
    const ibm_status s = full_reset(h, h->user);
    if (s != IBM_OK) return s;
  }
  Snapshot sn;
  ibm_status s = snapshot_take(h, sn, h->user);
  if (s != IBM_OK) return s;
  Tune best = h->tune;
  double bms = 0.0;
  s = autotune_loop(best, steps, [&](const Tune& t, int n, double* ms) -> ibm_status {
    h->tune = t;
    const ibm_status c = h->esize == 8 ? capture<double>(h) : capture<float>(h);
    if (c != IBM_OK) return c;
    const cudaError_t e = time_graph(h->exec, h->user, n, ms);
    return e == cudaSuccess ? IBM_OK : cuda_fail(h, e, "autotune trial");
  }, &bms);
  const ibm_status r = snapshot_restore(h, sn, h->user);
  if (s != IBM_OK) return s;
  if (r != IBM_OK) return r;
  h->tune = best;
  invalidate(h);
  tune_out(best, bms, chosen);
  return launch_status(h, "ibm_autotune");
}

// ---- batches --------------------------------------------------------------------
ibm_status ibm_batch_create(const ibm_handle* hs, int n, void* stream, ibm_batch_handle* out) {
  if (!hs || n < 1 || !out) return IBM_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!hs[i]) return IBM_ERR_ARG;
    if (hs[i]->g.yt.ihc) return IBM_ERR_ARG;   // a non-uniform wall-normal grid steps alone
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return IBM_ERR_ARG;
    const ibm_grid_desc &a = hs[0]->desc, &c = hs[i]->desc;
    if (a.precision != c.precision || a.scheme != c.scheme || a.use_q != c.use_q ||
        hs[0]->device != hs[i]->device)
      return IBM_ERR_ARG;
  }
  ibm_batch* b = new (std::nothrow) ibm_batch();
  if (!b) return IBM_ERR_OOM;
  b->hs.assign(hs, hs + n);
  b->epochs.assign(n, -1);
  b->device = hs[0]->device;
  b->user = (cudaStream_t)stream;
  b->al = hs[0]->al;
  b->tune = hs[0]->tune;
  Geo sh = hs[0]->g;
  for (int i = 1; i < n; ++i) {
    const Geo& g = hs[i]->g;
    sh.nx = std::max(sh.nx, g.nx);
    sh.ny = std::max(sh.ny, g.ny);
    sh.nz = std::max(sh.nz, g.nz);
    sh.nkx = std::max(sh.nkx, g.nkx);
  }
  b->shape = sh;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    if (b->cap) cudaStreamDestroy(b->cap);
    cudaGetLastError();
    delete b;
    return IBM_ERR_CUDA;
  }
  *out = b;
  return IBM_OK;
}

ibm_status ibm_batch_destroy(ibm_batch_handle b) {
  if (!b) return IBM_ERR_ARG;
  cudaStreamSynchronize(b->user);
  batch_release(b);
  if (b->ev) cudaEventDestroy(b->ev);
  if (b->cap) cudaStreamDestroy(b->cap);
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch_cache.size(); ++i)
      if (g_batch_cache[i] == b) {
        g_batch_cache.erase(g_batch_cache.begin() + (long)i);
        break;
      }
  }
  delete b;
  return IBM_OK;
}

const char* ibm_batch_last_error(ibm_batch_handle b) { return b ? b->err : "null batch"; }

ibm_status ibm_batch_step(ibm_batch_handle b, int nsteps) {
  if (!b || nsteps < 0) return IBM_ERR_ARG;
  ibm_status s = batch_prepare(b);
  if (s != IBM_OK) return s;
  s = batch_join_in(b);
  if (s != IBM_OK) return s;
  for (int k = 0; k < nsteps; ++k) BCK(cudaGraphLaunch(b->exec, b->user));
  s = batch_join_out(b);
  if (s != IBM_OK) return s;
  for (ibm_handle h : b->hs) h->steps += nsteps;
  BCK(cudaGetLastError());
  return IBM_OK;
}

ibm_status ibm_batch_sync(ibm_batch_handle b) {
  if (!b) return IBM_ERR_ARG;
  BCK(cudaStreamSynchronize(b->user));
  ibm_status first = IBM_OK;
  for (size_t i = 0; i < b->hs.size(); ++i) {
    const ibm_status s = ibm_sync(b->hs[i]);
    if (s != IBM_OK && first == IBM_OK) {
      first = s;
      snprintf(b->err, sizeof(b->err), "instance %zu: %.400s", i, b->hs[i]->err);
    }
  }
  return first;
}

ibm_status ibm_batch_get_info(ibm_batch_handle b, ibm_batch_info* out) {
  if (!b || !out) return IBM_ERR_ARG;
  const ibm_status s = batch_prepare(b);
  if (s != IBM_OK) return s;
  memset(out, 0, sizeof(*out));
  out->instances = (int64_t)b->hs.size();
  out->launches_per_step = b->positions;
  out->launches_per_step_solo = b->kernels_solo;
  for (ibm_handle h : b->hs) out->cells += h->g.ncell;
  out->shape[0] = b->shape.nx;
  out->shape[1] = b->shape.ny;
  out->shape[2] = b->shape.nz;
  return IBM_OK;
}

ibm_status ibm_batch_profile_stages(ibm_batch_handle b, int nsteps, double* ms, int64_t* kernels) {
  if (!b || nsteps < 0) return IBM_ERR_ARG;
  ibm_status s = batch_prepare(b);
  if (s != IBM_OK) return s;
  std::vector<std::vector<LaunchRec>> recs;
  BatchLayout L;
  s = b->hs[0]->esize == 8 ? batch_record<double>(b, recs, L) : batch_record<float>(b, recs, L);
  if (s != IBM_OK) return s;
  s = batch_join_in(b);
  if (s != IBM_OK) return s;
  s = profile_graph([&](cudaStream_t st) { batch_enqueue(b, recs, L, st); }, b->cap, b->user, nsteps, ms, kernels,
                    b->err, sizeof(b->err));
  if (s != IBM_OK) return s;
  for (ibm_handle h : b->hs) h->steps += nsteps;
  return batch_join_out(b);
}

ibm_status ibm_batch_set_tune(ibm_batch_handle b, const ibm_tune* t) {
  if (!b || !tune_valid(t)) return IBM_ERR_ARG;
  b->tune = Tune{t->tri_y, t->sweep_w, t->fft_lpb, t->fft_cols, t->sweep_zy, t->fft_plane, t->sweep_y, t->rhs,
                 t->corr_check};
  b->built = false;
  return IBM_OK;
}

ibm_status ibm_batch_autotune(ibm_batch_handle b, int steps, ibm_tune* chosen) {
  if (!b || steps < 1) return IBM_ERR_ARG;
  ibm_status s = batch_prepare(b);
  if (s != IBM_OK) return s;
  s = batch_join_in(b);
  if (s != IBM_OK) return s;
  std::vector<Snapshot> sn(b->hs.size());
  for (size_t i = 0; i < b->hs.size() && s == IBM_OK; ++i) s = snapshot_take(b->hs[i], sn[i], b->user);
  Tune best = b->tune;
  double bms = 0.0;
  if (s == IBM_OK)
    s = autotune_loop(best, steps, [&](const Tune& t, int n, double* ms) -> ibm_status {
      b->tune = t;
      const ibm_status c = b->hs[0]->esize == 8 ? batch_build<double>(b) : batch_build<float>(b);
      if (c != IBM_OK) return c;
      const cudaError_t e = time_graph(b->exec, b->user, n, ms);
      return e == cudaSuccess ? IBM_OK : bfail(b, e, "autotune trial");
    }, &bms);
  ibm_status r = IBM_OK;
  for (size_t i = 0; i < b->hs.size(); ++i)
    if (sn[i].mem) {
      const ibm_status q = snapshot_restore(b->hs[i], sn[i], b->user);
      if (q != IBM_OK && r == IBM_OK) r = q;
    }
  if (s != IBM_OK) return s;
  if (r != IBM_OK) return r;
  b->tune = best;
  b->built = false;
  tune_out(best, bms, chosen);
  return batch_join_out(b);
}

ibm_status ibm_step_batch(const ibm_handle* hs, int n, int nsteps) {
  if (!hs || n < 1 || nsteps < 0) return IBM_ERR_ARG;
  ibm_batch* b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (ibm_batch* c : g_batch_cache)
      if ((int)c->hs.size() == n && std::equal(c->hs.begin(), c->hs.end(), hs)) {
        b = c;
        break;
      }
  }
  if (!b) {
    const ibm_status s = ibm_batch_create(hs, n, hs[0]->user, &b);
    if (s != IBM_OK) return s;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batch_cache.push_back(b);
  }
  const ibm_status s = ibm_batch_step(b, nsteps);
  if (s != IBM_OK) snprintf(hs[0]->err, sizeof(hs[0]->err), "ibm_step_batch: %.400s", b->err);
  return s;
}


// ---- post-processing: loads and boundary-cell pressure ---------------------------
ibm_status ibm_get_loads(ibm_handle h, int sides, const double* pole, double* force, double* torque,
                         double* per_triangle, double* p_wall) {
  if (!h || (sides != 1 && sides != 2) || !force || !torque) return IBM_ERR_ARG;
  const double zero[3] = {0.0, 0.0, 0.0};
  const double* pl = pole ? pole : zero;
  for (int d = 0; d < 3; ++d) force[d] = torque[d] = 0.0;
  if (h->g.yt.ihc) {
    set_err(h, "%s", "ibm_get_loads: the MLS probes are written for a uniform grid");
    return IBM_ERR_STATE;
  }
  if (h->nt == 0) return IBM_OK;
  const int nt = h->nt;
  double* dtr = (double*)dalloc(h, (size_t)nt * 7 * sizeof(double));
  if (!dtr) {
    set_err(h, "%s", "device allocation for the loads failed");
    return IBM_ERR_OOM;
  }
  double* dpw = dtr + 6ll * nt;
  if (h->esize == 8)
    launch_loads<double>(h->g, surface(h), fields<double>(h), h->tb, h->desc.re, sides, pl, dtr, dpw, h->user);
  else
    launch_loads<float>(h->g, surface(h), fields<float>(h), h->tb, h->desc.re, sides, pl, dtr, dpw, h->user);
  std::vector<double> host((size_t)nt * 7);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host.data(), dtr, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->user);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->user);
  dfree(h, dtr);
  if (e != cudaSuccess) return cuda_fail(h, e, "ibm_get_loads");
  // fixed order: triangle by triangle
  for (int t = 0; t < nt; ++t)
    for (int d = 0; d < 3; ++d) {
      force[d] += host[6ll * t + d];
      torque[d] += host[6ll * t + 3 + d];
    }
  if (per_triangle) memcpy(per_triangle, host.data(), (size_t)nt * 6 * sizeof(double));
  if (p_wall) memcpy(p_wall, host.data() + 6ll * nt, (size_t)nt * sizeof(double));
  return check_device(h);
}

ibm_status ibm_get_pressure_recon(ibm_handle h, double* p, int on_device) {
  if (!h || !p) return IBM_ERR_ARG;
  if (h->g.yt.ihc) {
    set_err(h, "%s", "ibm_get_pressure_recon: the probes are written for a uniform grid");
    return IBM_ERR_STATE;
  }
  const Geo& g = h->g;
  cudaStream_t st = h->user;
  double* stage = (double*)h->scr;   // holds at least ncell doubles in both precisions
  if (h->esize == 8) {
    CK(cudaMemcpyAsync(stage, h->p, g.ncell * 8, cudaMemcpyDeviceToDevice, st));
    launch_pressure_recon<double>(g, surface(h), fields<double>(h), h->tb, h->ds, stage, st);
  } else {
    k_convert<float, double><<<num_sms() * 4, 256, 0, st>>>((const float*)h->p, stage, g.ncell);
    launch_pressure_recon<float>(g, surface(h), fields<float>(h), h->tb, h->ds, stage, st);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(p, stage, g.ncell * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return check_device(h);
}

}  // extern "C"
