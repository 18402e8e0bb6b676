// Helpers of the 2.5-D z-march kernels (float orbitals, star stencil of
// half-width 4): the halo-padded periodic plane and packed FP32x2 FMA.
#pragma once
#include <cuda_runtime.h>

#define ZM_ND 4   // stencil half-width of the z-march kernels

// Periodic plane with a halo of ND points on each side in x and y: entry
// (iy + ND) * (n1 + 2 ND) + ix + ND holds t(ix, iy); the halo holds the
// periodic images, so every in-plane neighbour of the star stencil is a
// load at a constant offset from the thread's own entry.
__device__ __forceinline__ void zpad_store(float2* pl, int n1, int n2, int ix, int iy, float2 v) {
  constexpr int ND = ZM_ND;
  const int W = n1 + 2 * ND;
  pl[(iy + ND) * W + ix + ND] = v;
  if (ix < ND) pl[(iy + ND) * W + ix + n1 + ND] = v;
  if (ix >= n1 - ND) pl[(iy + ND) * W + ix - n1 + ND] = v;
  if (iy < ND) pl[(iy + n2 + ND) * W + ix + ND] = v;
  if (iy >= n2 - ND) pl[(iy - n2 + ND) * W + ix + ND] = v;
}

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
