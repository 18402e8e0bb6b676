// Launchers of the tensor-core kernels (single-precision tensor-core mode).
#include "tsbz_internal.h"
#include "tsbz_kernels.cuh"
#include "tsbz_tc.cuh"

static bool tc_attr_set = false;

static void tc_set_attributes() {
  if (tc_attr_set) return;
  cudaFuncSetAttribute(k_bra_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TwSmem));
  cudaFuncSetAttribute(k_ket_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TwSmem));
  tc_attr_set = true;
}

void launch_bra_tc(const LaunchSet& L, const void* psi, void* out, int with_d, void* stream) {
  if (L.n_units == 0 || !L.cell.use_proj) return;
  tc_set_attributes();
  // one CTA per unit (all four current weightings in one pass when with_d)
  k_bra_w<<<L.n_units, 256, sizeof(TwSmem), (cudaStream_t)stream>>>(L, (const float2*)psi, (float2*)out, with_d);
}


void launch_ket_tc(const LaunchSet& L, const void* P, void* V, void* stream) {
  if (L.n_units == 0) return;
  tc_set_attributes();
  const int n_steps = (L.cell.npts + TW_PTS - 1) / TW_PTS;
  dim3 grid((n_steps + 8 * TW_KET_STEPS - 1) / (8 * TW_KET_STEPS), L.n_units);
  k_ket_w<<<grid, 256, sizeof(TwSmem), (cudaStream_t)stream>>>(L, (const float2*)P, (float2*)V);
}

void launch_stage_v(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* V, int m, void* stream) {
  if (L.n_units == 0) return;
  const int n12 = L.cell.n1 * L.cell.n2;
  if (L.cell.n1 == ZB_N && L.cell.n2 == ZB_N && L.cell.n3 == ZB_N && L.variant < 2) {
    // band of t_{m-1} (variant 1: with V and psi) bulk-staged in shared memory, barrier-free z-march
    static bool zb_attr = false;
    if (!zb_attr) {
      cudaFuncSetAttribute(k_stage_zb<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 + 3 * ZB_N * ZB_NP * 8);
      cudaFuncSetAttribute(k_stage_zb<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 + ZB_N * ZB_NP * 8);
      zb_attr = true;
    }
    dim3 grid(L.cell.n_bands, L.n_units);
    if (L.variant == 1)
      k_stage_zb<true><<<grid, ZB_NP, 128 + 3 * ZB_N * ZB_NP * sizeof(float2), (cudaStream_t)stream>>>(
          L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)V, m);
    else
      k_stage_zb<false><<<grid, ZB_NP, 128 + ZB_N * ZB_NP * sizeof(float2), (cudaStream_t)stream>>>(
          L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)V, m);
    return;
  }
  if (n12 <= 256 && L.cell.n3 == 16) {
    // 2.5-D z-march, depth 16 unrolled, packed arithmetic, halo plane per z
    const int threads = ((n12 + 31) / 32) * 32;
    dim3 grid(L.cell.n_bands, L.n_units);
    const size_t pad = (size_t)(L.cell.n1 + 2 * TC_ND) * (L.cell.n2 + 2 * TC_ND) * sizeof(float2);
    k_stage_zf<16><<<grid, threads, pad, (cudaStream_t)stream>>>(
        L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)V, m);
    return;
  }
  if (n12 <= 256) {
    // 2.5-D z-march: one CTA per (band, unit), one thread per (x, y) column
    const int threads = ((n12 + 31) / 32) * 32;
    dim3 grid(L.cell.n_bands, L.n_units);
    k_stage_z<float, TC_ND><<<grid, threads, n12 * sizeof(float2), (cudaStream_t)stream>>>(
        L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)V, m);
    return;
  }
  dim3 grid(L.cell.n_tiles, L.n_units);
  k_stage_v<float, TC_ND><<<grid, TSBZ_PT, 0, (cudaStream_t)stream>>>(L, (const float2*)tin, (float2*)tout,
                                                                      (float2*)psi, (const float2*)V, m);
}

bool launch_observe_zf(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                       void* stream) {
  const int n12 = L.cell.n1 * L.cell.n2;
  if (L.cell.n3 != 16 || L.cell.n1 > 16 || L.cell.n2 > 16 || L.cell.n_bgroups != 1 || L.n_units == 0) return false;
  const int threads = ((n12 + 31) / 32) * 32;
  k_observe_zf<16><<<L.n_units, threads, 0, (cudaStream_t)stream>>>(L, (const float2*)psi, rho_part, jk_part,
                                                                    nrm_part);
  return true;
}
