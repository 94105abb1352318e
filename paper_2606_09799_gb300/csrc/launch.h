// launch.h -- host-side launchers of the kernels (one per stage), shared
// between the kernel translation units and the runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "exec.cuh"

namespace ibm {

int num_sms();

// Blocks of a grid-stride kernel whose work grows with the instance: one per
// `cells` cells of the grid, within [lo, hi] (hi: enough to fill the GPU).
// Small instances of a batch then launch few blocks instead of a full GPU's
// worth each.
inline int scaled_blocks(const Geo& g, long long cells, int lo, int hi) {
  const long long b = g.ncell / cells;
  return (int)(b < lo ? lo : (b > hi ? hi : b));
}
// Blocks of the fixed-order two-level reductions (q_F, no-slip error):
// depends on the instance alone, so an instance reduces in the same order
// stepped alone or in a batch.
inline int reduce_blocks(const Geo& g, long long cells, int hi) { return scaled_blocks(g, cells, 8, hi); }

// ---- stage timing -------------------------------------------------------------
// Kernel groups of one time step; ibm_profile_stages reports the device time
// of each.  The order matches the stage names in runtime.cu.
enum StageId {
  ST_TAG = 0, ST_FORCE, ST_RHS, ST_SWEEP_X, ST_SWEEP_Z, ST_SWEEP_Y, ST_QRED, ST_FFT_X_FWD, ST_FFT_Z_FWD,
  ST_TRI_Y, ST_FFT_Z_INV, ST_FFT_X_INV, ST_PROJECT, ST_SLIP, ST_CORRECT, ST_DIAG, ST_CORR_TRI, ST_CORR_INV,
  ST_OTHER, ST_COUNT
};
// Record the start of stage `id` on stream st when stage timing is active
// on this thread (no-op otherwise).  Launchers call Exec::mark.
void stage_mark(cudaStream_t st, int id);

// ---- per-line records of forcing nodes (filled by tagging, read by sweeps) -
// x-lines are indexed (c, k, j), z-lines (c, j, i), y-lines (c, k, i); each
// holds the smallest forcing index along the line, or a large value.
struct LineInfo {
  int* x;          // 3 * nz * (ny+1)
  int* z;          // 3 * (ny+1) * nx
  int* y;          // 3 * nz * nx
  size_t bytes;    // of the three arrays together (x is their start)
};
__host__ __device__ inline long long line_x(const Geo& g, int c, long long j, long long k) {
  return ((long long)c * g.nz + k) * (g.ny + 1) + j;
}
__host__ __device__ inline long long line_z(const Geo& g, int c, long long i, long long j) {
  return ((long long)c * (g.ny + 1) + j) * g.nx + i;
}
__host__ __device__ inline long long line_y(const Geo& g, int c, long long i, long long k) {
  return ((long long)c * g.nz + k) * g.nx + i;
}

// ---- tagging (tagging.cu) --------------------------------------------------
struct TagBuffers {
  Cand* cand;                  // candidate list, capacity cap
  unsigned cap;                // capacity of cand, flist and blist
  unsigned long long* d2min;   // per node of the three grids (comp_off layout)
  unsigned* owner;             // per node of the three grids; 0xFFFFFFFF = fluid
  unsigned* flags32;           // per-cell flag bytes packed four to a word
  unsigned* ub;                // per node of the three grids: FP32 upper bound of the owner's |N|^2 (bits)
  unsigned* ublist;            // nodes whose ub this step set first (capacity cap)
  unsigned long long* surv;    // (triangle << 32 | pair) sent to the exact test (capacity cap)
  unsigned* blk;               // 4 counters per compaction block
  ForceNode* flist;            // forcing nodes, grouped by component, sorted by cell
  double* probe;               // per forcing node, this step: probe point x^e (3), alpha, wall velocity U
  unsigned* blist;             // boundary cells, sorted
  LineInfo lines;
};
void launch_tagging(const Geo& g, const Surf& s, const TagBuffers& b, DevState* ds, Exec& ex);
int compaction_blocks(const Geo& g);

// ---- tridiagonal coefficient tables (built on the host) -------------------
// The factorised sweeps solve (1 - beta L_d) x = r per grid line.  Fluid rows
// have constant coefficients, forcing nodes are identity rows, so every
// pivot is a function of the row's distance m from the start of its segment
// (the line start, or the row after an identity row): the Thomas recurrences
// are tabulated once per (direction, beta) and no line divides.
template <typename T>
struct SweepTables {
  // periodic x (0) and z (1), lines without forcing nodes: Sherman-Morrison
  // form (modified tridiagonal matrix + one correction vector)
  const T* inv[2];    // 1 / pivot of the modified matrix, per row
  const T* cp[2];     // c' of the modified matrix, per row
  const T* zv[2];     // correction vector
  const T* g0[2];     // first row of the modified inverse (y_0 as a dot product)
  T smden[2];         // 1 + v.z
  T gam[2];           // Sherman-Morrison gamma
  // periodic x (0) and z (1), lines with forcing nodes: segment recurrences
  const T* invR[2];
  const T* cpR[2];
  // wall-normal, tangential components: segments from the wall (W) or after
  // an identity row (R); LW / LR: pivot of a last (wall) row at position m
  const T* yinvW;
  const T* ycpW;
  const T* yinvR;
  const T* ycpR;
  const T* yinvLW;
  const T* yinvLR;
  // wall-normal, v (Dirichlet walls): every segment is an R segment
  const T* vinvR;
  const T* vcpR;
  T off[3];           // beta / d^2 per direction x, y, z
};

// ---- flow kernels (flow.cu) ------------------------------------------------
template <typename T>
struct Fields {
  T* u;
  T* v;
  T* w;
  T* p;
  T* H[3];      // non-linear term of the current sub-stage
  T* Hp[3];     // non-linear term of the previous sub-stage (may alias nothing)
  T* R[3];      // right-hand side, then the sweep results
  T* scr;       // scratch for c' of lines crossing bodies (sum of the three grids)
  T* uf;        // IB values of the forcing nodes
  T* phi;       // pseudo-pressure
  void* spec;   // complex half-spectrum nz*ny*nkx
  T* lo[3];     // low parts of the velocity state (mixed path), else null
  T* phi2;      // pseudo-pressure of the correction solve (mixed path)
  T* qk;        // q_F per fluid cell (energy-conserving shape), else null
  double idh[3][2];  // reciprocal spacings as (hi, lo) pairs, for the pair divergence
};

template <typename T>
void launch_ib_force(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds, bool geom,
                     Exec& ex);
template <typename T>
void launch_rhs(const Geo& g, const Fields<T>& f, const TagBuffers& b, const Stage& sg, double dt, double re,
                bool use_hp, bool write_h, DevState* ds, Exec& ex);
template <typename T>
void launch_sweeps(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb, DevState* ds,
                   Exec& ex);
template <typename T>
void launch_slip(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double* partial,
                 DevState* ds, Exec& ex);

// ---- Poisson and projection (poisson.cu) -----------------------------------
constexpr int TRI_SEG = 8;   // rows of j per lane of the warp-cooperative wall-normal Thomas
template <typename T>
struct SpecTables {
  const T* twx;          // exp(-2 pi i m / nx), m < nx, complex interleaved
  const T* twz;          // exp(-2 pi i m / nz)
  const double* cp;      // Thomas c' per (kz, j, kx)
  const double* inv;     // Thomas 1/pivot per (kz, j, kx)
  const double* segf;    // products of the forward multipliers per (kz, segment of TRI_SEG rows, kx)
  const double* segb;    // ... and of the backward multipliers
  const int* jc;         // per (kz, kx): first row of the stationary run of the factorisation (rows
                         // jc .. ny-2 hold the same 1/pivot and c' bit for bit); ny - 1 if none
  const double* pal;     // non-uniform wall-normal grid: forward multipliers (inv then holds
                         // height / pivot and cp the c' of the height-scaled rows); null if uniform
};
template <typename T>
void launch_poisson(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SpecTables<T>& tb,
                    const Stage& sg, double dt, double re, int use_q, double* partial, DevState* ds, Exec& ex);
// State diagnostics of the step after its last projection: max |D u - q| over
// C_F, kinetic energy and CFL number into the device state (poisson.cu).
template <typename T>
void launch_state_diag(const Geo& g, const Fields<T>& f, const TagBuffers& b, int s, int use_q, double dt,
                       double* partial, DevState* ds, Exec& ex);
// ---- post-processing (loads.cu) ----------------------------------------------
template <typename T>
void launch_loads(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double re, int sides,
                  const double pole[3], double* tr, double* pw, cudaStream_t st);
template <typename T>
void launch_pressure_recon(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds,
                           double* q, cudaStream_t st);

void launch_build_poisson_tables_nu(const Geo& g, const double* lamx, const double* lamz, double* cp, double* ivh,
                                    double* al, cudaStream_t st);
void launch_build_poisson_tables(const Geo& g, const double* lamx, const double* lamz, double* cp, double* inv,
                                 double* segf, double* segb, int* jc,
                                 cudaStream_t st);

}  // namespace ibm
