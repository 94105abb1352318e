// mbar.cuh -- shared-memory address and the bounded mbarrier wait used by
// kernels whose tiles arrive by asynchronous (TMA) copies.
#pragma once

namespace ibm {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Wait for phase `parity` of the mbarrier at shared address `bar`, giving up
// after `limit_cycles` SM cycles (returns false then).  Never waits without
// bound: the caller reports the timeout through its error word.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit_cycles) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit_cycles) return false;
  }
}

}  // namespace ibm
