// Device helpers shared by the batched block kernels: asynchronous bulk copies (TMA,
// cp.async.bulk) with mbarrier completion, proxy fences, the error-free transformations of
// the compensated residual, and the float sqrt / reciprocal used by the factorizations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace qrkit {
namespace dev {

__device__ __forceinline__ void record(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------------------
// Error-free transformations for the extended-precision residual of the refinement:
// TwoSum (Knuth) and TwoProduct via FMA (Dekker); every operation uses the _rn intrinsics
// so the compiler cannot contract or reassociate them.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// sqrt and reciprocal for float: x * rsqrtf(x) (a few ulp at most, far below the rounding
// the factorization itself accumulates) and the correctly rounded __frcp_rn; IEEE for double.
__device__ __forceinline__ float fsqrt(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double fsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float frcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }

// ---------------------------------------------------------------------------------------
// Asynchronous bulk copies (cp.async.bulk) between global and shared memory.  Both addresses
// 16-byte aligned, size a multiple of 16.  Loads complete on an mbarrier (transaction
// bytes); stores are tracked per thread by bulk async-groups.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// This thread's bulk stores have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// This thread's bulk stores are complete.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}
// Orders this thread's generic-proxy shared-memory accesses with later async-proxy ones.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Per-thread asynchronous 16-byte copies global -> shared (cp.async, tracked per thread by
// commit groups): both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The 16-byte-aligned interior [h, h + ni) of the element range [0, count) starting at g.
template <typename T>
__device__ __forceinline__ void interior(const T* g, int64_t count, int& h, int& ni) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(g);
  const uintptr_t e = a + (uintptr_t)count * sizeof(T);
  const uintptr_t ab = (a + 15) & ~(uintptr_t)15;
  const uintptr_t ae = e & ~(uintptr_t)15;
  if (ae > ab) {
    h = (int)((ab - a) / sizeof(T));
    ni = (int)((ae - ab) / sizeof(T));
  } else {
    h = (int)count;
    ni = 0;
  }
}
// Element offset that makes shared[off + k] share global g[k]'s address modulo 16.
template <typename T>
__device__ __forceinline__ int align_off(const T* g) {
  return (int)((reinterpret_cast<uintptr_t>(g) & 15) / sizeof(T));
}

}  // namespace dev
}  // namespace qrkit
