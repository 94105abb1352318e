/*
 * ibm.h -- C ABI of the GB300 sharp-interface immersed-boundary fractional
 * step (Vagnoli, Scarpolini, Verzicco, Viola, arXiv 2606.09799).
 *
 * The library advances the incompressible Navier-Stokes equations (Eq. ns,
 * Section 2) on a staggered Cartesian grid that is periodic in x and z and
 * bounded by walls at y = 0 and y = ly, with moving triangulated bodies of
 * any thickness (including zero) immersed in it.  One call of ibm_step runs,
 * entirely on the GPU:
 *
 *   Algorithm 1 tagging of the forcing nodes of the three velocity grids;
 *   per sub-stage s (RK2+CN: two, AB+CN: one, Section 2):
 *     the IB step on the forcing nodes, Eqs. IB_step, probe and new_IB;
 *     the provisional velocity on the fluid nodes, Eq. NS_prov, with the
 *       approximate factorisation of the CN operator (x, then z, then y);
 *     the consistent mass correction q of Section 3.2 (Eqs. q_boundary and
 *       the uniform q_F) in the right-hand side of Eq. elliptic_mod;
 *     the direct Poisson solve of Eq. elliptic_mod (FFT in x and z, Thomas
 *       per wavenumber in y, homogeneous Neumann walls);
 *     the projection, Eq. projection, and pressure update, Eq.
 *       update_pressure;
 *   the no-slip error of Section 4.4 on the forcing points.
 *
 * Conventions
 *   - Lengths are non-dimensional; U_ref = L_ref = 1.
 *   - Cells nx*ny*nz on [0,lx]x[0,ly]x[0,lz], uniform in each direction.
 *   - u lives on x-faces at (i dx, (j+1/2) dy, (k+1/2) dz),
 *     v on y-faces at ((i+1/2) dx, j dy, (k+1/2) dz), j = 0..ny (the planes
 *       j = 0 and j = ny are the walls and hold 0),
 *     w on z-faces at ((i+1/2) dx, (j+1/2) dy, k dz), p at cell centres.
 *   - Field arrays are C order [k][j][i] (i fastest): u, w, p hold
 *     nz*ny*nx values, v holds nz*(ny+1)*nx.  All field arguments are
 *     FP64 in every precision mode (the mixed mode converts).
 *   - Surface arrays are C order: xyz[3*nv] = (x,y,z) per vertex, vel[3*nv]
 *     the vertex velocities, tri[3*nt] vertex indices per triangle (int32).
 *     Several bodies are passed concatenated; the owner of a forcing node is
 *     the global triangle index.
 *
 * Ownership: the library copies every input into its own device buffers
 *   during the call (stream-ordered); outputs go into caller buffers.  A
 *   handle is not thread-safe; all its GPU work is ordered on the stream
 *   given to ibm_create_grid.
 * Errors: every entry point returns an ibm_status and never aborts.  Device
 *   kernels never trap: they record problems in a device error word that
 *   the next synchronising call (ibm_sync, ibm_get_fields, ibm_get_tags,
 *   ibm_get_diag) turns into a status.  ibm_last_error() describes the last
 *   failure of a handle.
 */
#ifndef IBM_GB300_H
#define IBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_grid* ibm_handle;

typedef enum {
  IBM_OK = 0,
  IBM_ERR_ARG = 1,       /* invalid argument (sizes, pointers, indices) */
  IBM_ERR_CUDA = 2,      /* a CUDA runtime call failed */
  IBM_ERR_OOM = 3,       /* device allocation failed */
  IBM_ERR_GEOMETRY = 4,  /* an IB probe left the domain, or a degenerate triangle */
  IBM_ERR_DIVERGED = 5,  /* non-finite values in the solution */
  IBM_ERR_TIMEOUT = 6,   /* a bounded device wait gave up */
  IBM_ERR_STATE = 7,     /* call not valid in the handle's current state */
  IBM_ERR_CAPACITY = 8   /* a capacity was exceeded.  From ibm_step's synchronising calls: a
                            device work list overflowed; its capacity has been grown, and the step
                            must be redone.  From ibm_tag_noalloc: the grid needs more than the
                            library's fixed array holds (IBM_NOALLOC_MAX_NODES); retrying cannot
                            succeed */
} ibm_status;

enum { IBM_RK2_CN = 0, IBM_AB_CN = 1 };   /* time schemes, Section 2 */
enum { IBM_NOSLIP = 0, IBM_FREESLIP = 1 }; /* condition on the y walls */
/* precision of the bulk arithmetic:
 *   IBM_FP64        everything in FP64;
 *   IBM_MIXED       stencils, forcing interpolation and FFTs in FP32; FP64
 *                   tagging geometry and per-wavenumber Thomas solves; the
 *                   velocity state kept as an unevaluated FP32 pair (hi + lo)
 *                   and a final correction solve on the residual divergence
 *                   computed in that pair arithmetic, so D u = q holds to
 *                   ~1e-12 of U/dx (the correction runs in the sub-stages
 *                   whose first-solve residual exceeds the divergence
 *                   budget, ibm_set_div_budget);
 *   IBM_MIXED_FAST  as IBM_MIXED with an FP32 velocity state and a single
 *                   solve (divergence at the FP32 solve error, ~1e-6 U/dx). */
enum { IBM_FP64 = 0, IBM_MIXED = 1, IBM_MIXED_FAST = 2 };

typedef struct {
  int nx, ny, nz;      /* cells; nx and nz even, factoring into 2s, 3s and 5s, 4 <= n <= 1024; 4 <= ny <= 4096 */
  double lx, ly, lz;   /* box lengths */
  double re;           /* Reynolds number */
  double dt;           /* time step */
  int scheme;          /* IBM_RK2_CN (default) or IBM_AB_CN */
  int ybc;             /* IBM_NOSLIP (default) or IBM_FREESLIP */
  int precision;       /* IBM_FP64, IBM_MIXED or IBM_MIXED_FAST (see above) */
  int use_q;           /* 1: Eq. elliptic_mod with the uniform q_F (the paper's method, mass
                          conserving); 2: the same with the energy- and mass-conserving shape of
                          App. B, q_F^k = a + b (p^k - e^k); 0: Eq. elliptic (no q) */
} ibm_grid_desc;

typedef struct {
  double slip_l1;         /* ||eps||_1 = sum_i ||eps_i||_1 / 3 of the last step (Section 4.4) */
  double slip_comp[3];    /* ||eps_i||_1, the mean |eps_i| over component i's forcing points */
  int64_t nforce[3];      /* forcing nodes per velocity component (last step) */
  int64_t nboundary;      /* boundary cells C_B (last step) */
  double q_f;             /* q_F of the last sub-stage */
  double sum_q_dv;        /* sum over all cells of q dV of the last sub-stage (0 up to rounding) */
  int64_t steps;          /* steps taken by this handle */
  int64_t ncandidates;    /* (node, triangle) pairs that passed Algorithm 1 in the last step */
  int64_t kernels_per_step; /* GPU kernels one ibm_step launches (nodes of its CUDA graph) */
  int64_t d2h_bytes;      /* bytes this ibm_get_diag call copied from the device */
  double div_max;         /* max over the fluid cells C_F of |D u - q| after the step's last projection
                             (Eq. mod_div: the projected field satisfies D u = q; every cell when use_q = 0);
                             the mixed paths form D u in (hi, lo) pair arithmetic */
  double ke;              /* kinetic energy 1/2 sum u^2 dV over the velocity nodes of the three grids
                             (dV = dx h dz, h the cell height for u and w, the centre distance for v) */
  double cfl;             /* dt max over the cells of |u_c|/dx + |v_c|/h + |w_c|/dz, u_c the mean of the
                             cell's two faces of each component (the step's result) */
  double div_first;       /* IBM_MIXED: max over C_F of |D u' - q| after the first Poisson solve of the
                             step's sub-stages (u' the once-projected pair state, FP32), the residual
                             that decides the correction solve; 0 in the other modes */
  int64_t corr_solves;    /* IBM_MIXED: correction solves taken since the handle was created */
} ibm_diag;

/* Create a simulation on the current CUDA device.  stream is a cudaStream_t
 * (NULL = the legacy default stream); all later GPU work of the handle is
 * ordered on it.  Fields start at rest (u = v = w = p = 0), with no surface.
 * Returns IBM_ERR_ARG for unsupported sizes, IBM_ERR_OOM if the device
 * buffers (about 200 B per cell in FP64) do not fit. */
ibm_status ibm_create_grid(const ibm_grid_desc* desc, void* stream, ibm_handle* out);

/* Create a simulation on a non-uniform wall-normal grid (Section 2: the
 * cells keep uniform spacings in the periodic x and z directions and take
 * variable heights in the wall-normal direction).  y_faces: host array of
 * ny + 1 strictly increasing face positions, y_faces[0] = 0 and
 * y_faces[ny] = desc->ly (to 1e-12 relative); it is copied.  Cell j spans
 * [y_faces[j], y_faces[j+1]]; u, w and p sit at the cell centres, v on the
 * faces.  Every wall-normal operator (the explicit terms, the factorised
 * implicit sweep, the divergence, the per-wavenumber tridiagonal of the
 * Poisson solve with a volume-weighted zero-mean gauge, the projection and
 * the pressure update) takes its row's spacings.  Immersed surfaces use the
 * local Eulerian cell (Algorithm 1, Section 3.1): a node's box margin in y and
 * its diagonal come from its own row (cell height for u and w, distance of
 * the centres for v), the probe length is twice that diagonal, and the probe
 * is interpolated between the rows that bracket it; the q term weights every
 * cell by its volume.  Both precisions are supported (the mixed path forms
 * the correction solve's faces and divergence with each row's spacings, in
 * pair arithmetic).  A batch refuses the handle (IBM_ERR_ARG);
 * ibm_get_loads and ibm_get_pressure_recon return IBM_ERR_STATE (their
 * probes assume a uniform grid); invalid face positions return IBM_ERR_ARG. */
ibm_status ibm_create_grid_stretched(const ibm_grid_desc* desc, const double* y_faces, void* stream,
                                     ibm_handle* out);

/* Release every device buffer of h (waits for its stream). */
ibm_status ibm_destroy(ibm_handle h);

/* Set the immersed surface X^n with its vertex velocities U^n (the wall
 * velocity of Eq. new_IB, interpolated barycentrically at X^f).  xyz and
 * vel: 3*nverts FP64; tri: 3*ntris int32, or NULL to keep the previous
 * connectivity (ntris must then match).  on_device = 1 if the pointers are
 * device pointers.  Host pointers must stay valid until the call returns.
 * ntris = 0 removes the surface.  IBM_ERR_ARG for out-of-range indices. */
ibm_status ibm_set_surface(ibm_handle h, int nverts, const double* xyz, const double* vel, int ntris,
                           const int32_t* tri, int on_device);

/* Uniform volume force f of Eq. ns1 (e.g. a mean pressure gradient),
 * applied on the fluid nodes with the weight alpha of each sub-stage. */
ibm_status ibm_set_body_force(ibm_handle h, double fx, double fy, double fz);

/* IBM_MIXED: divergence budget of the correction solve (Eq. mod_div).  After
 * the first Poisson solve of a sub-stage the device takes the largest
 * |D u' - q| over the fluid cells C_F of the once-projected (hi, lo) state;
 * the correction solve runs only when it exceeds `budget` (in the units of
 * D u, velocity / length), otherwise its kernels return at once and the
 * step keeps u'.  Default 0: the correction runs unless the residual is
 * exactly zero.  A mixed run that must meet max |D u - q| <= b passes a
 * budget below b (the first-solve residual is an FP32 value).  Other modes
 * accept and ignore it.  IBM_ERR_ARG for a negative or NaN budget. */
ibm_status ibm_set_div_budget(ibm_handle h, double budget);

/* Overwrite the state u, v, w, p (layouts above; v's wall planes are taken
 * as given).  The non-linear history H^{n-1} of AB+CN is reset to zero (a
 * restart from rest); ibm_set_history afterwards restores a saved one. */
ibm_status ibm_set_fields(ibm_handle h, const double* u, const double* v, const double* w, const double* p,
                          int on_device);

/* The non-linear history that AB+CN carries from step n to step n+1: the
 * explicit terms H^n of Eq. NS_prov (advection of the step's state, one per
 * velocity component, on that component's grid: hu and hw nz*ny*nx, hv
 * nz*(ny+1)*nx, FP64, layouts as the fields).  With ibm_get_fields and
 * ibm_set_fields it makes the whole state of a simulation: a run saved after
 * step n and restored into a new handle (fields, then history, then the
 * surface of step n+1) continues as the original would, bit for bit in
 * FP64.  RK2+CN carries no history across steps (its first sub-stage has
 * rho = 0); the calls then copy the first sub-stage's terms, which the next
 * step overwrites.  In the mixed paths H is FP32 and converts exactly.
 * ibm_get_history synchronises the stream; any pointer may be NULL. */
ibm_status ibm_get_history(ibm_handle h, double* hu, double* hv, double* hw, int on_device);
ibm_status ibm_set_history(ibm_handle h, const double* hu, const double* hv, const double* hw, int on_device);

/* Advance nsteps time steps with the current surface (asynchronous). */
ibm_status ibm_step(ibm_handle h, int nsteps);

/* Copy the state out (synchronises the stream).  Any pointer may be NULL. */
ibm_status ibm_get_fields(ibm_handle h, double* u, double* v, double* w, double* p, int on_device);

/* Tags of the last step for velocity component comp (0 = u, 1 = v, 2 = w):
 * owner[node] = -1 on fluid nodes, else the owning triangle (Algorithm 1,
 * smallest |N|^2, ties to the smallest index).  Array of that component's
 * field size.  Synchronises. */
ibm_status ibm_get_tags(ibm_handle h, int comp, int32_t* owner, int on_device);

/* Diagnostics of the last step (synchronises). */
ibm_status ibm_get_diag(ibm_handle h, ibm_diag* out);

/* Wait for the handle's stream and report any device-side error. */
ibm_status ibm_sync(ibm_handle h);

/* Human-readable description of the last error of h (never NULL). */
const char* ibm_last_error(ibm_handle h);

/* Optional device allocator for all buffers of handles created afterwards
 * (e.g. a framework's caching allocator).  alloc returns NULL on failure.
 * Passing NULL restores cudaMalloc/cudaFree. */
typedef void* (*ibm_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ibm_free_fn)(void* ptr, void* ctx);
ibm_status ibm_set_allocator(ibm_alloc_fn alloc, ibm_free_fn free_fn, void* ctx);

/* Device time of each kernel group of a time step.  Runs nsteps steps
 * (they advance the simulation like ibm_step), each as a CUDA graph with
 * event records between its kernel groups, and returns per group the total
 * device milliseconds in ms[IBM_NSTAGES] and the number of kernels in
 * kernels[IBM_NSTAGES] (either may be NULL).  Synchronises. */
#define IBM_NSTAGES 19
ibm_status ibm_profile_stages(ibm_handle h, int nsteps, double* ms, int64_t* kernels);

/* Name of kernel group `stage` (0 <= stage < IBM_NSTAGES), else "". */
const char* ibm_stage_name(int stage);

/* Tagging without allocation.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory at the time
 * they need the tags -- an application that reserves all of its GPU memory
 * at start-up and hands out nothing afterwards, code running inside another
 * allocator's callback, or a time-critical loop that may not block on the
 * allocator's implicit synchronisation.  It computes the forcing-node owners
 * of Algorithm 1 for one surface on the three staggered grids, bit for bit
 * the tags that ibm_step followed by ibm_get_tags gives for the same surface
 * on a handle made by ibm_create_grid with the same sizes, box and wall
 * condition (uniform spacing in every direction: this call knows nothing of
 * the non-uniform wall-normal rows of ibm_create_grid_stretched), without a
 * handle.
 *
 * All array arguments are device pointers owned by the caller: xyz (3*nverts
 * FP64 vertex positions), tri (3*ntris int32 vertex indices) and the outputs
 * owner_u (nz*ny*nx), owner_v (nz*(ny+1)*nx), owner_w (nz*ny*nx): -1 on fluid
 * nodes, else the owning triangle.  Only desc's nx, ny, nz, lx, ly, lz and
 * ybc are read.
 *
 * Its working memory is a fixed array inside the library, sized for
 * IBM_NOALLOC_MAX_NODES nodes of the three grids together (8 MiB of device
 * memory, held on every GPU that loads the library until the process
 * exits); larger grids are rejected with IBM_ERR_CAPACITY before any work.
 * Every call resolves the array's device address on the current device (a
 * host-side lookup, so a device reset never leaves a stale address); the
 * first call on a device may load the library's device code there, so make
 * it before any stream capture.  Every call shares the one array: calls that overlap on the GPU
 * (on different streams, or from different threads) race and give wrong
 * tags.  The call clears what it uses, runs on `stream`, and waits for it.
 * Returns IBM_ERR_ARG for bad sizes or pointers, or when a triangle names a
 * vertex outside [0, nverts) (such triangles are skipped, never read). */
#define IBM_NOALLOC_MAX_NODES 1048576
ibm_status ibm_tag_noalloc(const ibm_grid_desc* desc, int nverts, const double* xyz, int ntris,
                           const int32_t* tri, int32_t* owner_u, int32_t* owner_v, int32_t* owner_w,
                           void* stream);

/* ---- launch-shape tuning ------------------------------------------------
 * Choices of how the kernels of a step are laid out on the GPU; they change
 * the speed, never the method (the wall-normal Thomas variants differ in
 * rounding order only).  0 in any field means the built-in heuristic. */
typedef struct {
  int tri_y;          /* per-wavenumber Thomas in y: 1 warp-cooperative scan, 2 one thread per real or
                         imaginary part, 3 the same with its forward values in shared memory, 4 as 1
                         with its registers capped so that 7 blocks of 128 threads fit an SM (the
                         built-in choice) */
  int sweep_w;        /* grid lines per block of the z and y sweeps: 16, 32 or 64 */
  int fft_lpb;        /* complex lines per block of the x transforms (capped by shared memory) */
  int fft_cols;       /* kx columns per block of the z transforms: a power of two up to 16 */
  int sweep_zy;       /* z and y sweeps of the FP32 path: 1 shared-memory tile with one thread per line,
                         2 several lanes per line (affine-map scans) */
  int fft_plane;      /* 1 separate x and z transform kernels, 2 both fused per y-plane (when its
                         half-spectrum fits shared memory), 3 both fused per y-plane over a cluster
                         of 4 blocks that share the plane through distributed shared memory (one
                         simulation with nz a multiple of 8).  Built-in: 2 where it fits, else 3,
                         else 1 (a batch: 1) */
  int sweep_y;        /* z and y sweeps: 0 as sweep_zy, 1 one thread per line with its rows streamed
                         through registers (any line length), 2 as 1 for z, and for y tiles of 32
                         lines staged in shared memory by bulk asynchronous copies (where every row
                         starts on a 16-byte boundary and the tile fits; else as 1), 3 as 1 for z,
                         and for y the mixed path's tabulated FP32 rows in register batches (grids of
                         at most 1024 rows; else as 1), 4 z from tiles of 32 lines with all their rows
                         staged in shared memory (nz <= 256; else as 1), y as 3 */
  int rhs;            /* explicit right-hand side: 1 one thread per cell reading its neighbours from
                         global memory (the built-in choice of the FP64 path), 2 tiles of 32 x 4 cells
                         marching in z with the three planes of u, v, w (and two of p) and their halos
                         staged in shared memory, 3 two cells per thread along x with paired (float2)
                         row loads (the built-in choice of the FP32 path; the FP64 path runs 1) */
  int corr_check;     /* mixed path, the first solve's residual against the divergence budget: 1 formed
                         inside the correction's forward transform (the built-in choice), 2 by a pass
                         of its own, the correction's forward transform then skipped with the rest of
                         the correction solve when the budget is met (faster where the budget is met
                         in most sub-stages; the autotuner leaves it alone: how often the correction
                         runs changes along a run) */
  double ms_per_step; /* set by the autotuners: measured time per step of the chosen shapes */
} ibm_tune;

/* Use tuning `t` from the next step on (IBM_ERR_ARG if a field is out of range). */
ibm_status ibm_set_tune(ibm_handle h, const ibm_tune* t);
ibm_status ibm_get_tune(ibm_handle h, ibm_tune* t);

/* Autotuner: times whole steps (CUDA events, `steps` per candidate after one
 * untimed step) for every value of one choice at a time, keeping the others
 * at their best so far, and keeps the fastest.  The simulation state (fields,
 * non-linear terms, device scalars) is saved before and restored after, so
 * the trial steps leave no trace; the tagging state is rebuilt at the next
 * step.  Writes the choice to *chosen (may be NULL).  Synchronises. */
ibm_status ibm_autotune(ibm_handle h, int steps, ibm_tune* chosen);

/* ---- batches of independent simulations ---------------------------------
 * The paper's method advances one simulation; these entry points (no
 * counterpart in the paper) advance many independent ones -- uneven grid
 * sizes, each with its own bodies, Re and dt -- together: every launch of
 * the time step becomes ONE kernel launch over all instances (the blocks of
 * the instances' grids concatenated), and one CUDA graph holds a whole step
 * of the batch.  Each instance computes exactly what ibm_step computes for
 * it alone with the same launch shapes.
 *
 * The instances must share precision, scheme and use_q and live on one
 * device (else IBM_ERR_ARG).  Launch shapes (tiles, FFT lines per block,
 * Thomas variant) follow the largest extent of each axis over the batch.
 * The batch keeps the handle pointers, not copies: destroy a batch before
 * any of its handles.  Surfaces, fields and body forces are set per handle
 * as usual (ibm_set_surface, ...) on the handle's own stream; the batch's
 * stream waits for every handle's stream before a step, and every handle's
 * stream waits for the batch after it, so per-handle calls and batch steps
 * are ordered as issued.  A changed surface size or reallocated work list
 * rebuilds the batch's graph at its next step.  Device errors of an
 * instance are reported by ibm_batch_sync (or the handle's own synchronising
 * calls). */
typedef struct ibm_batch* ibm_batch_handle;

typedef struct {
  int64_t instances;
  int64_t cells;                   /* sum of the instances' cells */
  int64_t launches_per_step;       /* kernel launches of one batched step */
  int64_t launches_per_step_solo;  /* kernel launches if each instance stepped alone */
  int32_t shape[3];                /* nx, ny, nz that choose the launch shapes */
} ibm_batch_info;

ibm_status ibm_batch_create(const ibm_handle* hs, int n, void* stream, ibm_batch_handle* out);
ibm_status ibm_batch_destroy(ibm_batch_handle b);
/* nsteps steps of every instance; asynchronous on the batch's stream. */
ibm_status ibm_batch_step(ibm_batch_handle b, int nsteps);
/* Waits for the batch and checks every instance's device error word; on an
 * error returns the first instance's status (ibm_batch_last_error says which). */
ibm_status ibm_batch_sync(ibm_batch_handle b);
ibm_status ibm_batch_get_info(ibm_batch_handle b, ibm_batch_info* out);
/* ibm_profile_stages for the batched step (summed over the instances). */
ibm_status ibm_batch_profile_stages(ibm_batch_handle b, int nsteps, double* ms, int64_t* kernels);
ibm_status ibm_batch_set_tune(ibm_batch_handle b, const ibm_tune* t);
/* ibm_autotune for the batched step (state of every instance saved and restored). */
ibm_status ibm_batch_autotune(ibm_batch_handle b, int steps, ibm_tune* chosen);
const char* ibm_batch_last_error(ibm_batch_handle b);

/* One-call form: steps the n handles together, keeping one batch per
 * distinct handle list (created on first use on hs[0]'s stream, released
 * with ibm_destroy of any of its handles).  Errors are also described by
 * ibm_last_error(hs[0]). */
ibm_status ibm_step_batch(const ibm_handle* hs, int n, int nsteps);

/* ---- post-processing of a finished step ----------------------------------
 * Hydrodynamic loads (Section 3.3): markers at the triangle centroids, a
 * probe at distance h (twice the cell diagonal) along the oriented normal,
 * second-order moving-least-squares fits of p and of each velocity
 * component there (the 4x4x4 nearest nodes of each lattice, Gaussian
 * weights of width the cell diagonal, nodes behind the marker's plane and
 * boundary cells left out), the Taylor series back to the wall, traction
 * t = -p n + (grad u + grad u^T) n / Re.  sides = 1 uses the normal given by
 * the vertex order (closed bodies: make it outward), sides = 2 adds the
 * opposite face (zero-thickness surfaces).  Writes the total force and the
 * torque about `pole` (NULL: the origin), optionally per triangle the force
 * and torque (6*nt values) and the wall pressure on the normal's side (nt).
 * Uses the current fields and surface; call after ibm_step and before the
 * next ibm_set_surface.  Synchronises. */
ibm_status ibm_get_loads(ibm_handle h, int sides, const double* pole, double* force, double* torque,
                         double* per_triangle, double* p_wall);

/* Pressure with the boundary cells (Section 3.2), where the solution does
 * not define it, replaced by its value at each cell's probe point (zero
 * normal gradient at the wall); p: nz*ny*nx FP64 (host or device, as
 * on_device says).  Synchronises. */
ibm_status ibm_get_pressure_recon(ibm_handle h, double* p, int on_device);

/* Self-check of an implementation detail of the mixed path (no counterpart
 * in the paper): its kernels convert between FP32 and FP64 with integer
 * operations (a hardware conversion costs this GPU's narrow FP64 pipe about
 * two FP64 FMAs).  Runs n cases on the current device -- hashed binary32
 * bit patterns widened, binary64 values narrowed (every rounding case,
 * exact ties included) -- and compares each integer-path result with the
 * hardware conversion bit for bit.  *checked: results the integer path
 * produced (the rest are subnormal, infinite or NaN cases that the kernels
 * leave to the hardware); *mismatches: those that differ (0 expected).
 * Allocates 16 bytes on the device; synchronises the device. */
ibm_status ibm_check_conversions(long long n, long long* mismatches, long long* checked);

/* Self-check of the bounded waits (no counterpart in the paper): kernels
 * whose tiles arrive by asynchronous copies wait on an mbarrier with a
 * cycle limit and report a timeout through the device error word instead of
 * waiting without bound.  Runs one block whose mbarrier can never complete
 * and waits on it with limit_cycles (0 to 4e9 SM cycles).  *timed_out: 1 if
 * the wait gave up (expected); *waited_cycles: the cycles it waited.  The
 * device stays usable afterwards.  Allocates 16 bytes on the device;
 * synchronises the device.  IBM_ERR_ARG for a limit out of range or null
 * outputs. */
ibm_status ibm_check_bounded_wait(long long limit_cycles, int* timed_out, long long* waited_cycles);

/* Arithmetic roofs of the current device (no counterpart in the paper):
 * the FP64 and FP32 fused multiply-add throughput in TFLOP/s (an FMA counts
 * two flops), measured by a kernel whose every thread runs eight
 * independent FMA chains on every SM, timed with CUDA events after an
 * untimed launch (~20 ms per type).  The benchmark reports FP64-bound
 * kernels against *fp64_tflops.  Allocates 16 bytes on the device;
 * synchronises the device. */
ibm_status ibm_measure_alu_peaks(double* fp64_tflops, double* fp32_tflops);

/* Library version string. */
const char* ibm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IBM_GB300_H */
