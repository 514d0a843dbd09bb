// Bulk asynchronous copies global -> shared memory (the TMA engine's
// untiled cp.async.bulk) completed on shared-memory mbarriers, and a grid
// barrier with a time limit, for the persistent kernels (sm_90 and later
// PTX; written for sm_103a).
//
// Rules the callers keep: a bulk copy's source and destination are 16-byte
// aligned and its size is a multiple of 16 bytes; every wait is bounded
// (kWaitCycles) and reports failure instead of spinning forever.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mg {

// about 1 s at the GB300 SM clock
constexpr long long kWaitCycles = 2000000000LL;

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the async proxy (the copy engine)
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// the calling thread's arrival, announcing `bytes` of transactions to come
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// announces `bytes` of transactions to come, without an arrival
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// the calling thread's arrival (release: its earlier shared-memory writes are
// visible to the threads that see the phase complete)
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// waits for the phase of the given parity to complete; false after the time limit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// bytes from global `src` to shared `dst`, completing `bytes` transactions on bar
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Grid barrier of a cooperative launch.  `count` starts at 0 for the launch
// (the host clears it); every block arrives once per barrier and waits until
// all gridDim.x blocks have arrived, for at most kWaitCycles.  A block that
// times out raises *abort, which releases every other waiting block; the
// return value is false from then on and the callers unwind.  `target` is the
// block's running arrival count (identical in every block).
__device__ __forceinline__ bool grid_barrier(unsigned* count, int* abort, unsigned& target) {
  __shared__ int ok;
  __syncthreads();
  target += gridDim.x;
  if (threadIdx.x == 0) {
    int good = 1;
    __threadfence();
    atomicAdd(count, 1u);
    const long long t0 = clock64();
    while (true) {
      unsigned c;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(c) : "l"(count) : "memory");
      if ((int)(c - target) >= 0) break;
      if (*(volatile int*)abort) {
        good = 0;
        break;
      }
      if (clock64() - t0 > kWaitCycles) {
        atomicExch(abort, 1);
        good = 0;
        break;
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace mg
