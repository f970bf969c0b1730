// common.cuh -- sm_103a building blocks shared by the eigensolver kernels:
// shared-memory mbarriers, 1-D bulk copies (cp.async.bulk, the non-tensor
// form of TMA) and bounded waits.  No multicast and no cluster-remote
// accesses: every CTA reads only its own tiles of this GPU's memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace syev3 {

// Device status bits (OR-ed into a per-translation-unit __device__ word).
constexpr unsigned kFlagWaitTimeout = 1u;

// Limit of a wait on an mbarrier, on the GPU's global nanosecond timer: a
// 12 KB bulk copy lands in microseconds, so a wait still open after a second
// is declared lost.  Each poll may suspend the thread for up to
// kSuspendHintNs; kMaxPolls is a backstop should the timer not advance
// (at most kMaxPolls x kSuspendHintNs = 84 s).
constexpr uint64_t kWaitLimitNs = 1000000000ull;
constexpr uint32_t kSuspendHintNs = 20000u;
constexpr uint32_t kMaxPolls = 1u << 22;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make mbarrier initialisation visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Plain arrival (a phase that expects no bulk bytes completes with it).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Returns true once the phase with the given parity has completed, false if
// kWaitLimitNs went by first (timed from the first poll that found the phase
// open; the normal path reads no timer).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t i = 0; i < kMaxPolls; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
    if (i == 0)
      t0 = global_ns();
    else if (global_ns() - t0 > kWaitLimitNs)
      return false;
  }
  return false;
}

// Global -> shared bulk copy completing on `bar`.  dst, src 16-byte aligned;
// bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace syev3
