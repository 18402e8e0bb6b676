// Launchers of the single-precision fused stage and projection kernels.
#include "tsbz_internal.h"
#include "tsbz_sep.cuh"
#include "tsbz_fused.cuh"

// The 16^3 fused kernels run their z contractions per z group when the cell's
// atoms occupy at most 4 distinct z tables with at most two atoms each (NZU = 4),
// else per atom (NZU = 8).
#ifndef FS_ZGROUP
#define FS_ZGROUP 1
#endif
static inline bool fs_grouped(const CellDev& c) {
  if (!FS_ZGROUP || c.n_zg <= 0 || c.n_zg > 4) return false;
  for (int g = 0; g < c.n_zg; ++g)
    if (c.zg_off[g + 1] - c.zg_off[g] > 2) return false;   // the grouped ket adds at most two atoms
  return true;
}

template <typename K> static void fs_attr(K* kernel, size_t bytes) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

static inline bool fs_cube16(const CellDev& c) { return c.n1 == 16 && c.n2 == 16 && c.n3 == 16; }

// Kernel variants of the single-precision path (LaunchSet::variant):
//   16^3 cells with z groups: 0 whole step in one launch with the z
//     contractions on tcgen05, 1 fused stage per launch (mma.sync), 2 z-march
//     stage with CUDA-core projections, 3 whole step with the z contractions
//     on mma.sync;
//   other 16^3 cells and 8^3 cells: 0 fused / bulk-staged stage, 1 z-march stage;
//   other shapes: the z-march stage only.
// Returns 0 (whole step), 1 (fused or bulk-staged stage) or 2 (z-march stage).
static int stage_kind(const LaunchSet& L) {
  const CellDev& c = L.cell;
  if (L.ph_next == nullptr) return 2;
  if (fs_cube16(c) && fs_grouped(c)) return L.variant == 3 ? 0 : L.variant;
  if (fs_cube16(c) || (c.n1 == 8 && c.n2 == 8 && c.n3 == 8)) return L.variant == 0 ? 1 : 2;
  return 2;
}

// The grouped 16^3 whole-step kernel (and the projection pass that matches it)
// runs its z contractions on tcgen05 in variant 0.
static inline bool fs_umma(const LaunchSet& L) { return L.variant == 0; }

int sep_variants(const CellDev& c) {
  if (fs_cube16(c) && fs_grouped(c)) return 4;
  if (fs_cube16(c) || (c.n1 == 8 && c.n2 == 8 && c.n3 == 8)) return 2;
  return 1;
}

bool sep_supported(const CellDev& c) {
  const int n12 = c.n1 * c.n2;
  return c.nd == ZM_ND && n12 <= 256 && (c.n3 == 8 || c.n3 == 16) && c.n_atoms <= SEP_NA;
}

static inline unsigned sep_threads(const CellDev& c) { return (unsigned)(((c.n1 * c.n2 + 31) / 32) * 32); }

void launch_bra_sep(const LaunchSet& L, const void* src, void* out, int with_d, int use_obs, void* stream) {
  if (L.n_units == 0 || !L.cell.use_proj) return;
  const unsigned grid = (unsigned)L.n_units * (unsigned)L.cell.n_bands;
  const CellDev& c = L.cell;
  if (stage_kind(L) <= 1 && !with_d && !use_obs && fs_cube16(c)) {
    // the projections the 16^3 fused stage leaves are formed by the same pass
    static bool attr = false;
    if (!attr) {
      fs_attr(k_bra_fused<4, true>, sizeof(FsSmem));
      fs_attr(k_bra_fused<4, false>, sizeof(FsSmem));
      fs_attr(k_bra_fused<SEP_NA, false>, sizeof(FsSmem));
      attr = true;
    }
    if (fs_grouped(c) && fs_umma(L))
      k_bra_fused<4, true><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src,
                                                                                (float2*)out);
    else if (fs_grouped(c))
      k_bra_fused<4, false><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src,
                                                                                 (float2*)out);
    else
      k_bra_fused<SEP_NA, false><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src,
                                                                                        (float2*)out);
    return;
  }
  if (stage_kind(L) <= 1 && with_d && use_obs && fs_cube16(c)) {
    // the current's projections by the second-order pass of the fused stage 4
    static bool attr_pa = false;
    if (!attr_pa) {
      fs_attr(k_pa_fused<4, true>, sizeof(FsSmem));
      fs_attr(k_pa_fused<4, false>, sizeof(FsSmem));
      fs_attr(k_pa_fused<SEP_NA, false>, sizeof(FsSmem));
      attr_pa = true;
    }
    if (fs_grouped(c) && fs_umma(L))
      k_pa_fused<4, true><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src, (float2*)out);
    else if (fs_grouped(c))
      k_pa_fused<4, false><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src,
                                                                                (float2*)out);
    else
      k_pa_fused<SEP_NA, false><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (const float2*)src,
                                                                                       (float2*)out);
    return;
  }
  const unsigned thr = sep_threads(L.cell);
  cudaStream_t st = (cudaStream_t)stream;
  const float2* s = (const float2*)src;
  float2* o = (float2*)out;
  if (L.cell.n3 == 16) {
    if (with_d)
      k_bra_sep<16, 1><<<grid, thr, 0, st>>>(L, s, o, use_obs);
    else
      k_bra_sep<16, 0><<<grid, thr, 0, st>>>(L, s, o, use_obs);
  } else {
    if (with_d)
      k_bra_sep<8, 1><<<grid, thr, 0, st>>>(L, s, o, use_obs);
    else
      k_bra_sep<8, 0><<<grid, thr, 0, st>>>(L, s, o, use_obs);
  }
}

template <int N>
static void launch_stage_bulk(const LaunchSet& L, const void* tin, void* tout, void* psi, void* P, void* Pa, int m,
                              cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    size_t most = 0;
    for (int k = 1; k <= 4; ++k) most = sep_bulk_smem(N, k) > most ? sep_bulk_smem(N, k) : most;
    cudaFuncSetAttribute(k_stage_bulk<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    attr = true;
  }
  const unsigned grid = (unsigned)L.n_units * (unsigned)L.cell.n_bands;
  const size_t dyn = sep_bulk_smem(N, m);
  k_stage_bulk<N><<<grid, N * N, dyn, st>>>(L, (const float2*)tin, (float2*)tout, (float2*)psi, (float2*)P,
                                            (float2*)Pa, m);
}

bool launch_stage_sep(const LaunchSet& L, const void* tin, void* tout, void* psi, void* P, void* Pa, int m,
                      int same_next, void* stream) {
  if (L.n_units == 0) return false;
  const CellDev& c = L.cell;
  cudaStream_t st = (cudaStream_t)stream;
  const bool next = stage_kind(L) <= 1;
  if (next && fs_cube16(c)) {
    static bool attr = false;
    if (!attr) {
      fs_attr(k_stage_fused<4>, sizeof(FsSmem));
      fs_attr(k_stage_fused<SEP_NA>, sizeof(FsSmem));
      attr = true;
    }
    const unsigned grid = (unsigned)L.n_units * (unsigned)c.n_bands;
    if (fs_grouped(c))
      k_stage_fused<4><<<grid, FS_NP, sizeof(FsSmem), st>>>(L, (const float2*)tin, (float2*)tout, (float2*)psi,
                                                             (float2*)P, (float2*)Pa, m, same_next);
    else
      k_stage_fused<SEP_NA><<<grid, FS_NP, sizeof(FsSmem), st>>>(L, (const float2*)tin, (float2*)tout,
                                                                  (float2*)psi, (float2*)P, (float2*)Pa, m,
                                                                  same_next);
    return true;
  }
  if (next && c.n1 == 8 && c.n2 == 8 && c.n3 == 8) {
    launch_stage_bulk<8>(L, tin, tout, psi, P, Pa, m, st);
    return true;
  }
  const unsigned grid = (unsigned)L.n_units * (unsigned)c.n_bands;
  const unsigned thr = sep_threads(c);
  const size_t pad = (size_t)(c.n1 + 2 * ZM_ND) * (c.n2 + 2 * ZM_ND) * sizeof(float2);
  if (c.n3 == 16)
    k_stage_sep<16><<<grid, thr, pad, st>>>(L, (const float2*)tin, (float2*)tout, (float2*)psi, (float2*)P, m);
  else
    k_stage_sep<8><<<grid, thr, pad, st>>>(L, (const float2*)tin, (float2*)tout, (float2*)psi, (float2*)P, m);
  return false;
}

bool launch_step_fused(const LaunchSet& L, void* psi, void* P, void* Pa, int same_next, void* stream) {
  if (L.n_units == 0 || stage_kind(L) != 0) return false;
  static bool attr = false;
  if (!attr) {
    fs_attr(k_step_fused<4, true>, sizeof(FsSmem));
    fs_attr(k_step_fused<4, false>, sizeof(FsSmem));
    attr = true;
  }
  const unsigned grid = (unsigned)L.n_units * (unsigned)L.cell.n_bands;
  if (fs_umma(L))
    k_step_fused<4, true><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (float2*)psi, (float2*)P,
                                                                                (float2*)Pa, same_next);
  else
    k_step_fused<4, false><<<grid, FS_NP, sizeof(FsSmem), (cudaStream_t)stream>>>(L, (float2*)psi, (float2*)P,
                                                                                 (float2*)Pa, same_next);
  return true;
}

bool launch_observe_fused(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                          void* stream) {
  const CellDev& c = L.cell;
  if (L.n_units == 0 || c.n1 != 16 || c.n2 != 16 || c.n3 != 16 || c.n_bands > FO_MAXB) return false;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_observe_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(FoSmem));
    attr = true;
  }
  k_observe_fused<<<L.n_units, FS_NP, sizeof(FoSmem), (cudaStream_t)stream>>>(L, (const float2*)psi, rho_part,
                                                                              jk_part, nrm_part);
  return true;
}
