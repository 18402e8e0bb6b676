// Launchers of the tensor-core kernels (single-precision tensor-core mode).
#include "tsbz_internal.h"
#include "tsbz_kernels.cuh"
#include "tsbz_tc.cuh"

static bool tc_attr_set = false;

static void tc_set_attributes() {
  if (tc_attr_set) return;
  cudaFuncSetAttribute(k_bra_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
  cudaFuncSetAttribute(k_stage_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
  tc_attr_set = true;
}

void launch_bra_tc(const LaunchSet& L, const void* psi, void* out, int with_d, void* stream) {
  if (L.n_units == 0 || !L.cell.use_proj) return;
  tc_set_attributes();
  dim3 grid(with_d ? 4 : 1, L.n_units);
  k_bra_tc<<<grid, TC_THREADS, sizeof(TcSmem), (cudaStream_t)stream>>>(L, (const float2*)psi, (float2*)out, with_d);
}

void launch_stage_tc(const LaunchSet& L, const void* tin, void* tout, void* psi, void* P, int m, void* stream) {
  if (L.n_units == 0) return;
  tc_set_attributes();
  k_stage_tc<<<L.n_units, TC_THREADS, sizeof(TcSmem), (cudaStream_t)stream>>>(
      L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)P, (float2*)P, m);
}
