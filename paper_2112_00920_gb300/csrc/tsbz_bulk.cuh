// Bulk global -> shared copies completed on an mbarrier (sm_90+ async proxy),
// with a bounded wait: a CTA never spins without limit on a barrier.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

__device__ __forceinline__ uint32_t bk_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bk_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  // make the initialised barrier visible to the async proxy
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// The calling thread arrives once and announces bytes of transactions.
__device__ __forceinline__ void bk_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

// bytes (multiple of 16) from 16-byte aligned global src to 16-byte aligned shared dst.
__device__ __forceinline__ void bk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Wait for phase `parity` of the barrier; false if it did not complete within
// max_iter polls (each poll may suspend the thread for a short while).
__device__ __forceinline__ bool bk_mbar_wait(uint32_t bar, uint32_t parity, int max_iter) {
  for (int i = 0; i < max_iter; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

#define BK_WAIT_POLLS (1 << 20)
#define BK_STATUS_TIMEOUT 2   // sub-simulation status bit: a bounded device wait gave up
