// Arithmetic throughput probe: the FP32 and FP64 peaks against which the
// ALU-bound kernels of the library are measured.
//
// Each thread runs NCH independent fused multiply-add chains for `iters`
// unrolled rounds; the grid fills every SM (blocks of 512 threads, 4 per SM),
// so the dependent-latency of one chain is hidden by the others and by the
// other warps.  Flops per launch = threads x NCH x iters x 2 (x 2 for the
// packed FP32x2 form, which does two FMAs per instruction).  The chains'
// final values are folded into one word that is stored only if it equals an
// impossible value, so the compiler keeps every FMA and the kernel writes
// nothing in practice.
#include <cuda_runtime.h>

#include "tsbz.h"

namespace {

constexpr int NCH = 8;
constexpr int PROBE_THREADS = 512;
constexpr int PROBE_BLOCKS_PER_SM = 4;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(int iters, float b, float c, float* sink) {
  float a[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) a[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < NCH; ++i) a[i] = fmaf(a[i], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += a[i];
  if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma2(int iters, float b, float c, float* sink) {
  float2 a[NCH];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
#pragma unroll
  for (int i = 0; i < NCH; ++i) a[i] = make_float2((float)(threadIdx.x + i), (float)(threadIdx.x - i));
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < NCH; ++i) a[i] = __ffma2_rn(a[i], bb, cc);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += a[i].x + a[i].y;
  if (s == -1.2345e30f) sink[blockIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double b, double c, float* sink) {
  double a[NCH];
#pragma unroll
  for (int i = 0; i < NCH; ++i) a[i] = (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int i = 0; i < NCH; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < NCH; ++i) s += a[i];
  if (s == -1.2345e300) sink[blockIdx.x] = (float)s;
}

}  // namespace

extern "C" int tsbz_probe_alu_peak(int device, int kind, int iters, double* flops_per_s, double* ms_out) {
  if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 24) || !flops_per_s) return TSBZ_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return TSBZ_ECUDA;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n_sm < 1)
    return TSBZ_ECUDA;
  const int blocks = n_sm * PROBE_BLOCKS_PER_SM;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return TSBZ_ENOMEM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  // one untimed launch, then the best of three
  for (int rep = 0; err == cudaSuccess && rep < 4; ++rep) {
    err = cudaEventRecord(e0);
    if (err != cudaSuccess) break;
    if (kind == 0)
      k_probe_ffma<<<blocks, PROBE_THREADS>>>(iters, 0.999f, 1e-3f, sink);
    else if (kind == 1)
      k_probe_ffma2<<<blocks, PROBE_THREADS>>>(iters, 0.999f, 1e-3f, sink);
    else
      k_probe_dfma<<<blocks, PROBE_THREADS>>>(iters, 0.999, 1e-3, sink);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e1);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess || best <= 0.f) return TSBZ_ECUDA;
  const double fma_per_launch = (double)blocks * PROBE_THREADS * NCH * 8.0 * (double)iters * (kind == 1 ? 2.0 : 1.0);
  *flops_per_s = 2.0 * fma_per_launch / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return TSBZ_OK;
}
