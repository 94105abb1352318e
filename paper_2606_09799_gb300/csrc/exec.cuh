// exec.cuh -- how the kernels of a time step are launched.
//
// Every kernel body is a device function that takes its block coordinates
// as a Blk instead of reading blockIdx / gridDim, wrapped in a small "op"
// struct that holds the arguments.  An op runs in one of two ways:
//   - one simulation: k_run<Op>, a plain launch with the op as its parameter;
//   - a batch of independent simulations (uneven sizes, own bodies): the
//     launches of every instance are recorded in step order, and position p
//     of all instances becomes ONE launch of k_run_group<Op>, whose blocks
//     are the concatenation of the instances' grids (a block finds its
//     instance by binary search over the block offsets).
// Block shapes, shared-memory sizes and template choices (tiles, FFT lines
// per block, tridiagonal variant) are taken from Exec::shape, which is the
// instance's own grid for one simulation and the largest extent of every
// axis for a batch, so all instances of a group share one launch shape.
#pragma once

#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace ibm {

struct Blk {
  unsigned x, y, z;      // block coordinates inside the instance's grid
  unsigned gx, gy, gz;   // the instance's grid
};

__device__ __forceinline__ Blk blk_builtin() {
  return Blk{blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x, gridDim.y, gridDim.z};
}

// Programmatic dependent launch: every op kernel is launched with the
// programmatic-serialization attribute, so it may be scheduled while its
// predecessor in the stream drains.  It first waits until that predecessor
// has completed and its writes are visible (griddepcontrol.wait), then lets
// its own successor be scheduled.  No op touches memory before the wait.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// An op may ask the compiler to fit kMinBlocks of its blocks on one SM
// (registers capped to suit); its kernels are then the _occ forms.  Ops
// without it keep a plain thread bound (an explicit minimum of 1 would let
// the compiler spend more registers than its own default).
template <class Op, class = void>
struct HasMinBlocks : std::false_type {};
template <class Op>
struct HasMinBlocks<Op, std::void_t<decltype(Op::kMinBlocks)>> : std::true_type {};

template <class Op>
__global__ void __launch_bounds__(Op::kThreads) k_run(const __grid_constant__ Op op) {
  pdl_enter();
  op(blk_builtin());
}
template <class Op>
__global__ void __launch_bounds__(Op::kThreads, Op::kMinBlocks) k_run_occ(const __grid_constant__ Op op) {
  pdl_enter();
  op(blk_builtin());
}

// Block offset and grid of one instance inside a grouped launch.
struct GroupEntry {
  unsigned start;          // first block of the instance
  unsigned gx, gy, gz;
};

template <class Op>
__device__ __forceinline__ void run_group(const Op* __restrict__ ops, const GroupEntry* __restrict__ ge, int n) {
  pdl_enter();
  const unsigned b = blockIdx.x;
  int lo = 0, hi = n - 1;   // last instance whose start <= b (empty instances are skipped)
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&ge[mid].start) <= b) lo = mid;
    else hi = mid - 1;
  }
  const GroupEntry e = ge[lo];
  unsigned r = b - e.start;
  Blk bk;
  bk.gx = e.gx;
  bk.gy = e.gy;
  bk.gz = e.gz;
  bk.x = r % e.gx;
  r /= e.gx;
  bk.y = r % e.gy;
  bk.z = r / e.gy;
  ops[lo](bk);   // the op stays in global memory (a copy would go to local memory)
}
template <class Op>
__global__ void __launch_bounds__(Op::kThreads) k_run_group(const Op* __restrict__ ops,
                                                            const GroupEntry* __restrict__ ge, int n) {
  run_group<Op>(ops, ge, n);
}
template <class Op>
__global__ void __launch_bounds__(Op::kThreads, Op::kMinBlocks) k_run_group_occ(const Op* __restrict__ ops,
                                                                               const GroupEntry* __restrict__ ge,
                                                                               int n) {
  run_group<Op>(ops, ge, n);
}

// The kernels that run an op: alone and in a batch.
template <class Op>
constexpr auto run_kernel() {
  if constexpr (HasMinBlocks<Op>::value) return &k_run_occ<Op>;
  else return &k_run<Op>;
}
template <class Op>
constexpr auto group_kernel() {
  if constexpr (HasMinBlocks<Op>::value) return &k_run_group_occ<Op>;
  else return &k_run_group<Op>;
}

// One recorded launch of one instance.
struct LaunchRec {
  const void* kind;    // identifies the op type (its group launcher)
  void (*group)(const void* ops, const GroupEntry* ge, int n, unsigned blocks, dim3 block, size_t smem,
                cudaStream_t st);
  cudaError_t (*set_smem)(int bytes);
  std::vector<unsigned char> op;   // the op's bytes (ops are plain structs of values and pointers)
  dim3 grid, block;
  size_t smem;
  int mark;            // stage that starts with this launch, or -1
};

// Launch configuration with the programmatic-serialization attribute.
struct PdlConfig {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  PdlConfig(dim3 grid, dim3 block, size_t smem, cudaStream_t st) {
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
};

template <class Op>
void group_launch(const void* ops, const GroupEntry* ge, int n, unsigned blocks, dim3 block, size_t smem,
                  cudaStream_t st) {
  PdlConfig pc(dim3(blocks), block, smem, st);
  cudaLaunchKernelEx(&pc.cfg, group_kernel<Op>(), static_cast<const Op*>(ops), ge, n);
}

// Raise the dynamic shared-memory limit of both launch forms of an op on the
// current device.  The limit only ever grows: a smaller request (a batch
// whose tiles need less) must not undercut what another caller relies on.
template <class Op>
cudaError_t op_smem_limit(int bytes) {
  static std::mutex mu;
  static int high[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (bytes <= high[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(run_kernel<Op>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(group_kernel<Op>(), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  high[dev] = bytes;
  return cudaSuccess;
}

void stage_mark(cudaStream_t st, int id);

// Name of an op type, for error messages.
template <class Op>
const char* op_name() {
  return __PRETTY_FUNCTION__;
}

// Launch-shape choices of the autotuner (0 = the built-in heuristic).  Every
// value is clamped by the launchers to what the shape allows.
struct Tune {
  int tri_y;      // wall-normal Thomas: 1 warp-cooperative scan, 2 one thread per real/imaginary part
                  // (forward values in global scratch), 3 the same with them in shared memory
  int sweep_w;    // lines per block of the z and y sweeps (16, 32 or 64)
  int fft_lpb;    // complex lines per block of the x transforms
  int fft_cols;   // kx columns per block of the z transforms (power of two)
  int sweep_zy;   // z and y sweeps (FP32): 1 shared-memory tile, one thread per line; 2 several lanes per line
  int fft_plane;  // 1 separate x and z transform kernels; 2 fused per y-plane (when the plane fits);
                  // 3 fused per y-plane over a cluster of 4 blocks (one simulation, nz a multiple of 8);
                  // 0: 2 where it fits, else 3, else 1 (a batch: 1)
  int sweep_y;    // z and y sweeps: 0 as sweep_zy; 1 one thread per line, rows streamed through registers;
                  // 2 z as 1, y from tiles staged by bulk asynchronous copies (else as 1);
                  // 3 z as 1, y from the tabulated FP32 rows in register batches (mixed path, else as 1);
                  // 4 z from shared-memory tiles of whole lines (nz <= 256, else as 1), y as 3
  int rhs;        // explicit right-hand side: 1 one thread per cell from global memory; 2 tiles marching
                  // in z with planes and halos staged in shared memory; 3 two cells per thread along x
                  // with float2 row loads (FP32); 0: 3 in FP32, 1 in FP64
  int corr_check; // mixed path: 1 (and 0) the first solve's residual formed inside the correction's forward
                  // transform; 2 a residual pass of its own, the whole correction solve gated (not autotuned)
};

struct Exec {
  cudaStream_t st = nullptr;
  std::vector<LaunchRec>* rec = nullptr;   // batch: record instead of launching
  Geo shape{};                             // sizes that choose launch shapes
  Tune tune{};
  int pending = -1;
  cudaError_t first_err = cudaSuccess;     // first launch error, with the op that caused it
  const char* first_op = nullptr;

  void mark(int stage) {
    if (rec) pending = stage;
    else stage_mark(st, stage);
  }

  // A launch in thread-block clusters of `csize` blocks along x (the op's
  // blocks then share their shared memory within a cluster).  One simulation
  // only: a batch records plain launches, whose block offsets would split
  // the clusters, so its callers choose a plain op instead.
  template <class Op>
  void launch_cluster(dim3 grid, dim3 block, size_t smem, const Op& op, int csize) {
    if (rec) {
      if (first_err == cudaSuccess) {
        first_err = cudaErrorNotSupported;
        first_op = op_name<Op>();
      }
      return;
    }
    if ((unsigned long long)grid.x * grid.y * grid.z == 0) return;
    PdlConfig pc(grid, block, smem, st);
    cudaLaunchAttribute at[2];
    at[0] = pc.attr[0];
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)csize;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    pc.cfg.attrs = at;
    pc.cfg.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&pc.cfg, run_kernel<Op>(), op);
    if (e == cudaSuccess) e = cudaPeekAtLastError();
    if (e != cudaSuccess && first_err == cudaSuccess) {
      first_err = e;
      first_op = op_name<Op>();
    }
  }

  template <class Op>
  void launch(dim3 grid, dim3 block, size_t smem, const Op& op) {
    if (!rec) {
      if ((unsigned long long)grid.x * grid.y * grid.z == 0) return;
      PdlConfig pc(grid, block, smem, st);
      cudaError_t e = cudaLaunchKernelEx(&pc.cfg, run_kernel<Op>(), op);
      if (e == cudaSuccess) e = cudaPeekAtLastError();
      if (e != cudaSuccess && first_err == cudaSuccess) {
        first_err = e;
        first_op = op_name<Op>();
      }
      return;
    }
    LaunchRec r;
    r.kind = reinterpret_cast<const void*>(&group_launch<Op>);
    r.group = &group_launch<Op>;
    r.set_smem = &op_smem_limit<Op>;
    r.op.resize(sizeof(Op));
    memcpy(r.op.data(), &op, sizeof(Op));
    r.grid = grid;
    r.block = block;
    r.smem = smem;
    r.mark = pending;
    pending = -1;
    rec->push_back(r);
  }
};

// A grid that is empty unless `live` (keeps the launch sequences of the
// instances of a batch aligned when one of them has nothing to do).
inline dim3 grid_if(bool live, dim3 g) { return live ? g : dim3(0, 1, 1); }

}  // namespace ibm
