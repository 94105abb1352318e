// selfcheck.cu -- bit-for-bit check of the integer-pipe FP32 <-> FP64
// conversions (common.cuh) against the hardware conversions, a check that
// the bounded mbarrier wait (mbar.cuh) gives up and returns, and the FP64 /
// FP32 fused multiply-add throughput of the device (the arithmetic roofs
// the benchmark reports against).
#include <cuda_runtime.h>

#include "common.cuh"
#include "ibm.h"
#include "mbar.cuh"

namespace ibm {

// 32-bit integer hash "lowbias32" (C. Wellons, hash-prospector): a
// counter-based source of bit patterns for the check.
__device__ __forceinline__ unsigned lowbias32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352dU;
  x ^= x >> 15;
  x *= 0x846ca68bU;
  x ^= x >> 16;
  return x;
}

// Case t: a float with a hashed bit pattern (every class of binary32 value),
// and a double made from a hashed normal float with hashed low 29 mantissa
// bits (every rounding case of the narrowing, exact ties included: one
// pattern in 2^29 is a tie, so some cases force one) or, one case in eight,
// a fully hashed bit pattern (exponents outside the binary32 range).
__global__ void k_check_conversions(long long n, unsigned long long* out) {
  unsigned long long bad = 0, fast = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const unsigned h0 = lowbias32((unsigned)t * 2u + 1u), h1 = lowbias32((unsigned)t * 2u + 2u ^ 0x9e3779b9u);
    // widening
    const float f = __uint_as_float(h0);
    bool sp = false;
    const double w = f2d_int(f, sp);
    if (!sp) {
      ++fast;
      const double ref = (double)f;
      if (__double_as_longlong(w) != __double_as_longlong(ref) && !(f != f)) ++bad;
    }
    // narrowing
    double d;
    if ((h1 & 7u) == 0u) {
      d = __hiloint2double((int)h0, (int)h1);
    } else {
      const unsigned fe = 1u + (h1 >> 8) % 254u;                       // normal binary32 exponent
      const float g = __uint_as_float((h0 & 0x807FFFFFu) | (fe << 23));
      bool s2 = false;
      const double gw = f2d_int(g, s2);
      unsigned low = lowbias32(h1) & 0x1FFFFFFFu;
      if ((h1 & 0xF0u) == 0u) low = 0x10000000u;                       // an exact tie
      d = __hiloint2double(__double2hiint(gw), (int)(((unsigned)__double2loint(gw) & 0xE0000000u) | low));
    }
    bool sp2 = false;
    const float r = d2f_int(d, sp2);
    if (!sp2) {
      ++fast;
      if (__float_as_uint(r) != __float_as_uint((float)d) && !(d != d)) ++bad;
    }
  }
  atomicAdd(out, bad);
  atomicAdd(out + 1, fast);
}

// An mbarrier whose phase cannot complete: one expected arrival, made with
// 16 bytes of transaction count that no copy ever delivers.  Every thread
// waits on it through the bounded wait; out[0] = 1 if thread 0's wait gave
// up, out[1] = the cycles it waited.
__global__ void k_check_bounded_wait(long long limit_cycles, long long* out) {
  __shared__ __align__(8) unsigned long long bar_mem;
  const unsigned bar = smem_addr(&bar_mem);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], 16;\n" ::"r"(bar) : "memory");
  }
  __syncthreads();
  const long long t0 = clock64();
  const bool done = mbar_wait(bar, 0, limit_cycles);
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    out[0] = done ? 0 : 1;
    out[1] = t1 - t0;
  }
}

// Arithmetic throughput probe: every thread runs eight independent chains
// of fused multiply-adds (a <- a m + b), so the pipe of type T, not the
// latency of one chain, bounds the rate.  The result is stored only under a
// condition the data never meets, which keeps the chains alive.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(int iters, T seed, T* out) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = seed + (T)(threadIdx.x + 7 * c);
  const T m = (T)0.9999, b = (T)1e-4;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = fma(a[c], m, b);
  }
  T s = (T)0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  if (s == (T)-1.25) out[0] = s;
}

template <typename T>
static cudaError_t fma_rate(T* out, double* tflops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)(sms * 8)), block(256);
  cudaEvent_t a = nullptr, z = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&z);
  // size the run from a short one so that the timed launch takes ~20 ms
  int iters = 256;
  float ms = 0.f;
  for (int round = 0; round < 3 && e == cudaSuccess; ++round) {
    k_fma_chains<T><<<grid, block>>>(iters, (T)1, out);
    e = cudaEventRecord(a);
    if (e == cudaSuccess) {
      k_fma_chains<T><<<grid, block>>>(iters, (T)1, out);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(z);
    if (e == cudaSuccess) e = cudaEventSynchronize(z);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, z);
    if (e != cudaSuccess || round == 2) break;
    const double scale = ms > 0.f ? 20.0 / ms : 64.0;
    iters = (int)fmin(fmax(iters * scale, 256.0), 1e8);
  }
  if (e == cudaSuccess)
    *tflops = 2.0 * 8.0 * (double)iters * (double)grid.x * block.x / (ms * 1e-3) / 1e12;
  if (a) cudaEventDestroy(a);
  if (z) cudaEventDestroy(z);
  return e;
}

}  // namespace ibm

extern "C" ibm_status ibm_measure_alu_peaks(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return IBM_ERR_ARG;
  double* d = nullptr;
  if (cudaMalloc(&d, 16) != cudaSuccess) return IBM_ERR_OOM;
  ibm_status st = IBM_OK;
  if (ibm::fma_rate<double>(d, fp64_tflops) != cudaSuccess) st = IBM_ERR_CUDA;
  if (st == IBM_OK && ibm::fma_rate<float>(reinterpret_cast<float*>(d), fp32_tflops) != cudaSuccess) st = IBM_ERR_CUDA;
  cudaFree(d);
  return st;
}

extern "C" ibm_status ibm_check_bounded_wait(long long limit_cycles, int* timed_out, long long* waited_cycles) {
  if (limit_cycles < 0 || limit_cycles > 4000000000ll || !timed_out || !waited_cycles) return IBM_ERR_ARG;
  long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(long long)) != cudaSuccess) return IBM_ERR_OOM;
  long long h[2] = {0, 0};
  ibm_status st = IBM_OK;
  ibm::k_check_bounded_wait<<<1, 32>>>(limit_cycles, d);
  if (cudaGetLastError() != cudaSuccess) st = IBM_ERR_CUDA;
  if (st == IBM_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) st = IBM_ERR_CUDA;
  cudaFree(d);
  *timed_out = (int)h[0];
  *waited_cycles = h[1];
  return st;
}

extern "C" ibm_status ibm_check_conversions(long long n, long long* mismatches, long long* checked) {
  if (n < 0 || !mismatches || !checked) return IBM_ERR_ARG;
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return IBM_ERR_OOM;
  unsigned long long h[2] = {0, 0};
  ibm_status st = IBM_OK;
  if (cudaMemset(d, 0, sizeof(h)) != cudaSuccess) st = IBM_ERR_CUDA;
  if (st == IBM_OK && n > 0) {
    ibm::k_check_conversions<<<1024, 256>>>(n, d);
    if (cudaGetLastError() != cudaSuccess) st = IBM_ERR_CUDA;
  }
  if (st == IBM_OK && cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) st = IBM_ERR_CUDA;
  cudaFree(d);
  *mismatches = (long long)h[0];
  *checked = (long long)h[1];
  return st;
}
