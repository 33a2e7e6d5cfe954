// tma.cuh -- bulk asynchronous copies (TMA, cp.async.bulk) global -> shared
// with mbarrier completion, and bounded waits.
//
// Every wait here gives up after a clock budget, sets a device error word
// and returns false; callers then stop issuing work and drain what they
// already issued (again with a bound) before leaving the kernel, so a lost
// completion never hangs the GPU.  The host reads the error word in
// vofl_sync() and reports VOFL_ETIMEDOUT.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace vofl {

// ~0.5 s at 2 GHz: far above any legitimate copy latency (microseconds)
constexpr long long kWaitBudgetCycles = 1LL << 30;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared accesses before later
// async-proxy (TMA) writes to the same shared memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// one contiguous global -> shared copy; dst, src 16-byte aligned, bytes a
// multiple of 16; completion counted on `bar`
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Wait for phase `phase` of `bar` to complete, at most budget cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int* err,
                                                  long long budget = kWaitBudgetCycles) {
  if (mbar_try_wait(bar, phase)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() - t0 > budget) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}

// Grid-wide barrier of a cooperative launch (every CTA resident), bounded.
// bar[0] counts the CTAs that arrived, bar[1] is the generation: each CTA
// reads the generation, then arrives; the last of the grid's CTAs resets
// the count and advances the generation, which releases the others.  (Any
// grid size per launch; launches that use the same counter pair run one
// after another.)  Writes before the barrier are visible to every CTA
// after it (fences around the arrival and the wait).  A wait past the
// budget sets the error word and lets the CTA go on (the launch's results
// are then reported invalid).
__device__ __forceinline__ void grid_barrier_bounded(unsigned long long* bar, int* err,
                                                     long long budget = kWaitBudgetCycles) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long n = (unsigned long long)gridDim.x * gridDim.y * gridDim.z;
    const volatile unsigned long long* vgen = bar + 1;
    const unsigned long long g0 = *vgen;
    __threadfence();
    if (atomicAdd(bar, 1ULL) + 1 == n) {
      atomicExch(bar, 0ULL);
      __threadfence();
      atomicAdd(bar + 1, 1ULL);
    } else {
      const long long t0 = clock64();
      while (*vgen == g0) {
        if (clock64() - t0 > budget) {
          if (err) atomicExch(err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// Hint: bring `bytes` (a multiple of 16) at the 16-byte aligned global
// address p into L2 (no completion to wait for; data may change later).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 2D tiled tensor store (TMA) of a dense shared-memory box to the tensor of
// `tmap` at element coordinates (x inner, y outer); x * element size must
// be a multiple of 16 bytes.  Elements outside the tensor are not written.
__device__ __forceinline__ void tma_store_2d(const void* tmap, int x, int y, const void* smem_src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(tmap), "r"(x),
               "r"(y), "r"(smem_addr(smem_src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the issuing thread's committed bulk stores have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and have completed (their writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// a tensor map read from global memory: order earlier generic writes of it
// before its use by the tensor-copy unit
__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

}  // namespace vofl
