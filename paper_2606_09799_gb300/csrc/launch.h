// launch.h -- host-side launchers of the kernels (one per stage), shared
// between the kernel translation units and the runtime.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ibm {

int num_sms();

// ---- stage timing -------------------------------------------------------------
// Kernel groups of one time step; ibm_profile_stages reports the device time
// of each.  The order matches the stage names in runtime.cu.
enum StageId {
  ST_TAG = 0, ST_FORCE, ST_RHS, ST_SWEEP_X, ST_SWEEP_Z, ST_SWEEP_Y, ST_QRED, ST_FFT_X_FWD, ST_FFT_Z_FWD,
  ST_TRI_Y, ST_FFT_Z_INV, ST_FFT_X_INV, ST_PROJECT, ST_SLIP, ST_OTHER, ST_COUNT
};
// Record the start of stage `id` on stream st when stage timing is active
// on this thread (no-op otherwise, e.g. during graph capture).
void stage_mark(cudaStream_t st, int id);

// ---- tagging (tagging.cu) --------------------------------------------------
struct TagBuffers {
  Cand* cand;                  // candidate list, capacity cap
  unsigned cap;                // capacity of cand, flist and blist
  unsigned long long* d2min;   // per node of the three grids (comp_off layout)
  unsigned* owner;             // per node of the three grids; 0xFFFFFFFF = fluid
  unsigned* flags32;           // per-cell flag bytes packed four to a word
  unsigned* blk;               // 4 counters per compaction block
  ForceNode* flist;            // forcing nodes, grouped by component, sorted by cell
  unsigned* blist;             // boundary cells, sorted
};
void launch_tagging(const Geo& g, const Surf& s, const TagBuffers& b, DevState* ds, cudaStream_t st);
int compaction_blocks(const Geo& g);

// ---- tridiagonal coefficient tables (built on the host) -------------------
// Fast path of the approximate-factorisation sweeps for lines without
// forcing nodes: constant coefficients, so the Thomas recurrences are
// tabulated once per (direction, beta).  Periodic lines use the
// Sherman-Morrison form.
template <typename T>
struct SweepTables {
  // periodic directions x (0) and z (1)
  const T* inv[2];   // 1 / pivot of the modified matrix, per row
  const T* cp[2];    // c' of the modified matrix, per row
  const T* zv[2];    // Sherman-Morrison correction vector
  const T* g0[2];    // first row of the modified inverse
  T smden[2];        // 1 + v.z
  T gam[2];          // Sherman-Morrison gamma
  // wall-normal direction y: tangential components (0) and v (1)
  const T* yinv[2];
  const T* ycp[2];
  T off[3];          // beta / d^2 per direction x, y, z
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
};

template <typename T>
void launch_ib_force(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, DevState* ds,
                     cudaStream_t st);
template <typename T>
void launch_rhs(const Geo& g, const Fields<T>& f, const TagBuffers& b, const Stage& sg, double dt, double re,
                bool use_hp, bool write_h, DevState* ds, cudaStream_t st);
template <typename T>
void launch_sweeps(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SweepTables<T>& tb,
                   cudaStream_t st);
template <typename T>
void launch_slip(const Geo& g, const Surf& s, const Fields<T>& f, const TagBuffers& b, double* partial,
                 DevState* ds, cudaStream_t st);

// ---- Poisson and projection (poisson.cu) -----------------------------------
template <typename T>
struct SpecTables {
  const T* twx;          // exp(-2 pi i m / nx), m < nx, complex interleaved
  const T* twz;          // exp(-2 pi i m / nz)
  const double* cp;      // Thomas c' per (kz, j, kx)
  const double* inv;     // Thomas 1/pivot per (kz, j, kx)
};
template <typename T>
void launch_poisson(const Geo& g, const Fields<T>& f, const TagBuffers& b, const SpecTables<T>& tb,
                    const Stage& sg, double dt, double re, int use_q, double* partial, DevState* ds,
                    cudaStream_t st);
void launch_build_poisson_tables(const Geo& g, const double* lamx, const double* lamz, double* cp, double* inv,
                                 cudaStream_t st);

}  // namespace ibm
