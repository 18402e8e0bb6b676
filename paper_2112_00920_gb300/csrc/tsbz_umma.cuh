// Fifth-generation tensor-core building blocks (tcgen05, sm_100 family):
// tensor-memory allocation, single-thread MMA issue with the A operand in
// tensor memory and the B operand in shared memory, completion through an
// mbarrier, and warp-wide tensor-memory loads and stores.
//
// Tensor memory (TMEM) holds 128 lanes x 512 columns of 32-bit cells per SM;
// an address is (lane << 16) | column.  A warp may access only the 32 lanes
// of its quarter: warp w of a CTA uses lanes 32 (w % 4) .. 32 (w % 4) + 31.
// With M = 128 an MMA operand or accumulator row r lives in lane r.
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// a core matrix is 8 rows x 16 bytes (8 x 4 32-bit values) stored as 128
// contiguous bytes; core matrices that follow each other along K are
// `lbo` bytes apart, groups of 8 rows are `sbo` bytes apart.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// ---- tensor memory -----------------------------------------------------------
// The .sync.aligned instructions below need the whole warp converged; each
// helper re-converges it first (__syncwarp), so a divergent branch earlier in
// the caller cannot leave part of the warp behind.
// Allocate ncols columns (power of two, >= 32) for the CTA; executed by one
// whole warp.  The base address is written to shared memory at `slot`.
__device__ __forceinline__ void um_alloc(uint32_t slot, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void um_dealloc(uint32_t taddr, uint32_t ncols) {
  __syncwarp();
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void um_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void um_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// ---- descriptors ---------------------------------------------------------------
// Shared-memory matrix descriptor, K-major, no swizzle (layout type 0);
// bits 46-47 hold the descriptor version of the sm_100 family (1).
__device__ __forceinline__ uint64_t um_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, no negation, dense; N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t um_idesc_tf32(int m, int n) {
  return (1u << 4)                       // D format: F32
         | (2u << 7)                     // A format: TF32
         | (2u << 10)                    // B format: TF32
         | ((uint32_t)(n >> 3) << 17)    // N
         | ((uint32_t)(m >> 4) << 24);   // M
}

// ---- MMA -----------------------------------------------------------------------
// D[tmem] (+)= A[tmem] B[smem]^T: M x N x 8 (TF32), issued by one thread.
__device__ __forceinline__ void um_mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                               bool accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"((uint32_t)accumulate)
      : "memory");
}

// Arrive once on the mbarrier when every MMA issued so far by this thread has
// completed.
__device__ __forceinline__ void um_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
               : "memory");
}

// ---- tensor memory loads and stores (32 lanes x 32 bits per warp) ------------
// Thread i of the warp reads lane (base lane + i), columns c .. c + 15 (c + 31).
// The destination registers of tcgen05.ld are valid only after
// tcgen05.wait::ld, so the load and the wait are one asm statement: the
// compiler cannot move a use of the values ahead of the wait.
__device__ __forceinline__ void um_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void um_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Write then wait: the written cells are complete when this returns.
__device__ __forceinline__ void um_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  __syncwarp();
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// TMEM address of lane quarter q (0..3), column c
__device__ __forceinline__ uint32_t um_addr(uint32_t base, int q, int c) {
  return base + ((uint32_t)(32 * q) << 16) + (uint32_t)c;
}
