// Asynchronous copies into shared memory (sm_90 and later, written as inline
// PTX): bulk copies by the tensor memory accelerator that complete on an
// mbarrier (contiguous global ranges, 16-byte aligned, sizes a multiple of
// 16 bytes), and per-thread cp.async copies for gathers.  Waits on an
// mbarrier are bounded in time and in polls: a caller that gets `false`
// reports an error instead of spinning forever.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfem {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes initialised mbarriers visible to the asynchronous (bulk copy) proxy
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier shared-memory accesses (and, after a block
// barrier, the block's) before later bulk copies into the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// one arrival that also announces `bytes` of bulk-copy data for this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// bulk copy global -> shared memory of this CTA, completing on `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t kAsyncWaitNs = 2000000000ull;  // 2 s of global time
constexpr uint32_t kAsyncWaitPolls = 1u << 26;

// waits for the phase of `bar` with the given parity to complete; false
// when neither happened within kAsyncWaitNs nor kAsyncWaitPolls polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t k = 1; k < kAsyncWaitPolls; ++k) {
    if (mbar_test(bar, parity)) return true;
    if ((k & 63) == 0 && global_ns() - t0 > kAsyncWaitNs) return false;
  }
  return false;
}

// per-thread asynchronous copy of N (4, 8 or 16) bytes global -> shared
template <int N>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
  static_assert(N == 4 || N == 8 || N == 16, "cp.async copies 4, 8 or 16 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(dst)), "l"(src), "n"(N) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

}  // namespace sfem
