// bcm_bulk.cuh -- bulk asynchronous copies between this GPU's global memory and a block's
// shared memory (cp.async.bulk, no tensor map), their mbarrier completion with bounded
// waits, and the proxy fences that order them against ordinary loads and stores.
//
// Rules the callers keep: both addresses 16-byte aligned and sizes multiples of 16; a
// global write by ordinary stores is read by a bulk copy only after the writing threads
// executed fence_async_global() and a barrier (block or grid) separates them from the
// issuing thread; shared memory written by ordinary stores is read by a bulk store only
// after fence_async_shared() and a block barrier; a buffer filled by a bulk copy is
// reused only after its mbarrier phase completed, and a buffer read by a bulk store only
// after bulk_wait_read().
#pragma once

#include <stdint.h>

#include "bcm_persist.cuh"

namespace bcm {

__device__ __forceinline__ uint32_t s_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(b)), "r"(count) : "memory");
}
// One arrival on b that also raises its expected byte count by `bytes`.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(s_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier to complete, at most limit_ns.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity,
                                          unsigned long long limit_ns) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_test(b, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// Bulk copy of `bytes` from this GPU's global memory into this block's shared memory,
// completing on barrier b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          s_addr(dst)),
      "l"(src), "r"(bytes), "r"(s_addr(b))
      : "memory");
}
// Bulk copy of `bytes` from this block's shared memory to global memory (bulk group of
// the issuing thread; bulk_commit() closes the group).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(s_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// The issuing thread's committed bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// ... and are complete in global memory.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
__device__ __forceinline__ void fence_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace bcm
