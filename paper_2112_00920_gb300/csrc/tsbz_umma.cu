// Self-test of the tcgen05 building blocks used by the projector
// contractions: one CTA computes D = A B^T (M = 128, N = 32, K = 16) with the
// three-product TF32 split (A = A_hi + A_lo, B = B_hi + B_lo, D = A_lo B_hi +
// A_hi B_lo + A_hi B_hi in FP32), A in tensor memory (written by the threads
// with tcgen05.st), B in shared memory in the canonical K-major layout, the
// accumulator in tensor memory, completion through an mbarrier with a
// bounded wait.  The result is compared with a host product by the tests.
#include <cuda_runtime.h>

#include "tsbz.h"
#include "tsbz_bulk.cuh"
#include "tsbz_umma.cuh"

namespace {

constexpr int ST_M = 128, ST_N = 32, ST_K = 16;
constexpr uint32_t ST_COLS = 64;   // A_hi 0..15, A_lo 16..31, D 32..63

__device__ __forceinline__ uint32_t st_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

// B_t[n][k] at the canonical K-major position of (row n, column k).
__device__ __forceinline__ int st_boff(int n, int k, int lbo, int sbo) {
  return (n >> 3) * sbo + (k >> 2) * lbo + (n & 7) * 16 + (k & 3) * 4;
}

__global__ void __launch_bounds__(128) k_selftest_umma(const float* __restrict__ A, const float* __restrict__ B,
                                                       float* __restrict__ D, int swap_lbo_sbo, int polls,
                                                       int* status) {
  __shared__ __align__(1024) unsigned char bsm[2][4096];
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  // K-major core matrices: 128 bytes each, 4 per 8-row group along K (K = 16)
  const int lbo = 128, sbo = 512;
  const int dlbo = swap_lbo_sbo ? sbo : lbo, dsbo = swap_lbo_sbo ? lbo : sbo;
  if (warp == 0) um_alloc((uint32_t)__cvta_generic_to_shared(&tslot), ST_COLS);
  if (tid == 0) bk_mbar_init((uint32_t)__cvta_generic_to_shared(&mbar), 1);
  // B hi / lo in shared memory
  for (int i = tid; i < ST_N * ST_K; i += blockDim.x) {
    const int n = i / ST_K, k = i % ST_K;
    const float x = B[i];
    const uint32_t hi = st_tf32(x), lo = st_tf32(x - __uint_as_float(hi));
    *reinterpret_cast<uint32_t*>(&bsm[0][st_boff(n, k, lbo, sbo)]) = hi;
    *reinterpret_cast<uint32_t*>(&bsm[1][st_boff(n, k, lbo, sbo)]) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  um_fence_before();
  __syncthreads();
  um_fence_after();
  const uint32_t tbase = tslot;
  // row tid of A (lane tid): hi in columns 0..15, lo in 16..31
  uint32_t hi[16], lo[16];
#pragma unroll
  for (int k = 0; k < ST_K; ++k) {
    const float x = A[tid * ST_K + k];
    hi[k] = st_tf32(x);
    lo[k] = st_tf32(x - __uint_as_float(hi[k]));
  }
  um_st16(um_addr(tbase, warp, 0), hi);
  um_st16(um_addr(tbase, warp, 16), lo);
  um_fence_before();
  __syncthreads();
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (tid == 0) {
    um_fence_after();
    constexpr uint32_t idesc = um_idesc_tf32(ST_M, ST_N);
    const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(bsm[0]), b1 = (uint32_t)__cvta_generic_to_shared(bsm[1]);
    const uint32_t dt = tbase + 32;
#pragma unroll
    for (int ks = 0; ks < ST_K / 8; ++ks) {
      // K step ks covers two core matrices along K: 2 ks lbo bytes in
      const uint64_t bh = um_sdesc(b0 + 2 * ks * lbo, dlbo, dsbo), bl = um_sdesc(b1 + 2 * ks * lbo, dlbo, dsbo);
      um_mma_tf32_ts(dt, tbase + 16 + 8 * ks, bh, idesc, ks > 0);   // A_lo B_hi
      um_mma_tf32_ts(dt, tbase + 8 * ks, bl, idesc, true);          // A_hi B_lo
      um_mma_tf32_ts(dt, tbase + 8 * ks, bh, idesc, true);          // A_hi B_hi
    }
    um_commit(bar);
  }
  const bool ok = bk_mbar_wait(bar, 0, polls);
  if (!__syncthreads_and(ok)) {
    // the MMAs did not complete within the limit: wait again (bounded), then
    // release the tensor memory and report
    if (tid == 0) {
      bk_mbar_wait(bar, 0, polls);
      atomicOr(status, BK_STATUS_TIMEOUT);
    }
    __syncthreads();
    if (warp == 0) um_dealloc(tbase, ST_COLS);
    return;
  }
  um_fence_after();
  float d0[32];
  um_ld32(um_addr(tbase, warp, 32), d0);
#pragma unroll
  for (int n = 0; n < 32; ++n) D[tid * ST_N + n] = d0[n];
  um_fence_before();
  __syncthreads();
  if (warp == 0) {
    um_fence_after();
    um_dealloc(tbase, ST_COLS);
  }
}

}  // namespace

extern "C" int tsbz_selftest_umma(int device, int swap_lbo_sbo, const float* a, const float* b, float* d,
                                  int* status_out) {
  if (!a || !b || !d) return TSBZ_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return TSBZ_ECUDA;
  float *da = nullptr, *db = nullptr, *dd = nullptr;
  int* ds = nullptr;
  cudaError_t e = cudaMalloc(&da, sizeof(float) * ST_M * ST_K);
  if (e == cudaSuccess) e = cudaMalloc(&db, sizeof(float) * ST_N * ST_K);
  if (e == cudaSuccess) e = cudaMalloc(&dd, sizeof(float) * ST_M * ST_N);
  if (e == cudaSuccess) e = cudaMalloc(&ds, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(da, a, sizeof(float) * ST_M * ST_K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(db, b, sizeof(float) * ST_N * ST_K, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(ds, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(dd, 0, sizeof(float) * ST_M * ST_N);
  if (e == cudaSuccess) {
    k_selftest_umma<<<1, 128>>>(da, db, dd, swap_lbo_sbo, BK_WAIT_POLLS, ds);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(d, dd, sizeof(float) * ST_M * ST_N, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&st, ds, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(da);
  cudaFree(db);
  cudaFree(dd);
  cudaFree(ds);
  if (e != cudaSuccess) return TSBZ_ECUDA;
  if (status_out) *status_out = st;
  return (st & BK_STATUS_TIMEOUT) ? TSBZ_ETIMEOUT : TSBZ_OK;
}
