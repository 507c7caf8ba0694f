// Inline-PTX helpers shared by the kernels that stage data with the
// asynchronous copy engine (TMA bulk copies) and mbarriers.  Every wait is
// bounded: after 2^24 polls it sets *flag and reports failure, so a caller
// can drain its copies and return instead of hanging.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ofm {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the asynchronous proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Like mbar_test, but the hardware may suspend the thread for a while before
// reporting "not yet" (fewer issue slots spent while waiting).
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
      " selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, int* flag) {
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_test(addr, parity)) return true;
    if (i > 64) __nanosleep(32);
  }
  atomicExch(flag, 1);
  return false;
}

// Arrival of the issuing thread that also announces `bytes` of
// transaction count (the bulk copies issued next complete them).
__device__ __forceinline__ void mbar_arrive_expect(uint32_t addr, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(addr),
      "r"(bytes)
      : "memory");
}

// Plain arrival (count 1, no transactions): completes a phase that has no copy.
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(addr)
               : "memory");
}

// Bulk copy global -> shared of `bytes` (multiple of 16; both addresses
// 16-byte aligned), completing transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// asynchronous-proxy accesses (bulk copies, tensor-core operand reads).
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace ptx
}  // namespace ofm
