// Tensor-core projector contractions (scaled split-FP16, FP32 accumulate) and the
// fused Taylor stage of the single-precision tensor-core mode.
//
// Projector values of one k-point, C_j(r) = conj(beta~_j(r)) = pnorm_j F_x F_y F_z w_j,
// with the per-axis factors F_ax(i) = g_ax(i) exp(+i q_ax d_ax(i)) and
// w_j in {1, d_x, d_y, d_z}, are generated per tile of grid points in
// shared memory as a real matrix Cs[pt][j'] (j' < 32: Re C_j, j' >= 32:
// Im C_j).  Every operand value x is scaled by S = 2^10 and split into an
// FP16 high part and an FP16 low part (S x ~ hi + lo, each round to
// nearest; the scale keeps the low parts in the normal FP16 range).  A
// product A B is evaluated as A_hi B_hi + A_hi B_lo + A_lo B_hi with
// mma.sync m16n8k16 (f16 inputs, FP32 accumulate), about 2^-21 relative
// error per product, and the accumulator is multiplied by 1/S^2 = 2^-20.
//   bra  P_jb = dV sum_r C_j(r) t_b(r):  D[j'][n'] = sum_pt Cs[pt][j'] Ts[n'][pt]
//        (n' < 16: Re t_b, n' >= 16: Im t_b), P_re = D[j][b] - D[32+j][16+b],
//        P_im = D[j][16+b] + D[32+j][b]
//   ket  V_b(r) = sum_j conj(C_j(r)) E_j P_jb:  V[pt][n'] = sum_j' Cs[pt][j'] Wt[n'][j']
//        with Wt built from W = E P so that V[pt][b] = Re V_b, V[pt][16+b] = Im V_b.
// Limits of this mode per cell: bands <= 16, projectors <= 32, grid edges <= 32.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tsbz_bulk.cuh"
#include "tsbz_internal.h"
#include "tsbz_zmarch.cuh"

#define TC_W_PITCH 72      // FP16 values per Wt row
#define TC_D_PITCH 33      // floats per row of the final bra combination
#define TC_ND 4            // stencil half-width of the fused stage
#define TC_NMAX 32         // largest grid edge
#define TC_NA 8            // atoms (projectors / 4)


#define TC_SCALE 1024.0f               // operand scale S
#define TC_UNSCALE (1.0f / 1048576.0f)   // 1 / S^2

// Split a pair (x, y) into packed FP16 high parts and packed FP16 low parts
// of (S x, S y); one packed conversion per part, because conversions issue
// on a narrow pipe.
__device__ __forceinline__ void tc_split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  x *= TC_SCALE;
  y *= TC_SCALE;
  const __half2 h = __floats2half2_rn(x, y);
  const float2 hf = __half22float2(h);
  const __half2 l = __floats2half2_rn(x - hf.x, y - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ uint32_t tc_ld32(const __half* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void tc_st16(__half* p, uint32_t bits) {
  *reinterpret_cast<unsigned short*>(p) = (unsigned short)(bits & 0xFFFFu);
}

__device__ __forceinline__ void tc_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tc_ldsm_x4_trans(uint32_t (&r)[4], const __half* row_ptr) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(row_ptr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// ============================================================================
// Warp-independent forms of the bra and the ket.  Each warp owns 16-point
// slices: it generates its own projector rows and orbital values into a
// private shared-memory tile and runs its products with warp-level
// synchronisation only; CTA barriers occur once, in the final reduction.
// ============================================================================
#define TW_PTS 16          // points per warp step
#define TW_CPITCH 72       // FP16 values per projector row (64 + 8)
#define TW_TPITCH 24       // FP16 values per orbital row (16 + 8)

struct TwTile {
  __half c_hi[TW_PTS * TW_CPITCH];
  __half c_lo[TW_PTS * TW_CPITCH];
  __half t_hi[32 * TW_TPITCH];
  __half t_lo[32 * TW_TPITCH];
};

struct TwSmem {
  TwTile w[8];
  float2 fac[TC_NA * 3 * TC_NMAX];
  float dis[TC_NA * 3 * TC_NMAX];
  float pn[TC_NA * 4];
  __half wk_hi[32 * TC_W_PITCH];
  __half wk_lo[32 * TC_W_PITCH];
};

__device__ __forceinline__ void tw_load_tables(TwSmem& sm, const CellDev& c, const float2* ph) {
  const int nm = c.nmax;
  const int n = c.n_atoms * 3 * nm;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int a = i / (3 * nm), r = i % (3 * nm);
    const int ax = r / nm, ii = r % nm;
    const float g = c.g1f[i];
    const float2 p = ph[i];
    sm.fac[(a * 3 + ax) * TC_NMAX + ii] = make_float2(g * p.x, g * p.y);
    sm.dis[(a * 3 + ax) * TC_NMAX + ii] = c.d1f[i];
  }
  for (int i = threadIdx.x; i < 4 * c.n_atoms; i += blockDim.x) sm.pn[i] = c.pnormf[i];
}

// projector rows of 16 points (p0 .. p0+15) into the warp's tile
__device__ __forceinline__ void tw_gen_c(TwTile& wt, const TwSmem& sm, const CellDev& c, int p0, int alpha,
                                         int lane) {
  // lane -> point pt = lane % 16 and atoms lane / 16 + 2k
  const int pt = lane & (TW_PTS - 1);
  const int p = p0 + pt;
  const bool pv = p < c.npts;
  const int pp = pv ? p : 0;
  const int n12 = c.n1 * c.n2;
  const int iz = pp / n12, rem = pp - iz * n12;
  const int iy = rem / c.n1, ix = rem - iy * c.n1;
#pragma unroll
  for (int k = 0; k < (TW_PTS * TC_NA) / 32; ++k) {
    const int a = (lane >> 4) + 2 * k;
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    if (pv && a < c.n_atoms) {
      const float2* fa = sm.fac + a * 3 * TC_NMAX;
      const float* da = sm.dis + a * 3 * TC_NMAX;
      const float2 fx = fa[ix], fy = fa[TC_NMAX + iy], fz = fa[2 * TC_NMAX + iz];
      const float d[3] = {da[ix], da[TC_NMAX + iy], da[2 * TC_NMAX + iz]};
      const float2 fxy = make_float2(fx.x * fy.x - fx.y * fy.y, fx.x * fy.y + fx.y * fy.x);
      float fr = fxy.x * fz.x - fxy.y * fz.y, fi = fxy.x * fz.y + fxy.y * fz.x;
      if (alpha > 0) {
        fr *= d[alpha - 1];
        fi *= d[alpha - 1];
      }
      const float* pn = sm.pn + 4 * a;
      const float w[4] = {pn[0], pn[1] * d[0], pn[2] * d[1], pn[3] * d[2]};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        cr[t] = fr * w[t];
        ci[t] = fi * w[t];
      }
    }
    uint2 hr, lr, hc, lc;
    tc_split2(cr[0], cr[1], hr.x, lr.x);
    tc_split2(cr[2], cr[3], hr.y, lr.y);
    tc_split2(ci[0], ci[1], hc.x, lc.x);
    tc_split2(ci[2], ci[3], hc.y, lc.y);
    *reinterpret_cast<uint2*>(wt.c_hi + pt * TW_CPITCH + 4 * a) = hr;
    *reinterpret_cast<uint2*>(wt.c_lo + pt * TW_CPITCH + 4 * a) = lr;
    *reinterpret_cast<uint2*>(wt.c_hi + pt * TW_CPITCH + 32 + 4 * a) = hc;
    *reinterpret_cast<uint2*>(wt.c_lo + pt * TW_CPITCH + 32 + 4 * a) = lc;
  }
}

// 8 orbital values per lane of a 16-point step: v[k] = t_b(p0 + pt), i = lane + 32k, pt = i % 16, b = i / 16
__device__ __forceinline__ void tw_fetch(float2 (&v)[8], const float2* src, const CellDev& c, int p0, int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = lane + 32 * k;
    const int pt = i % TW_PTS, b = i / TW_PTS;
    const int p = p0 + pt;
    v[k] = (p < c.npts && b < c.n_bands) ? src[(long long)b * c.npts + p] : make_float2(0.f, 0.f);
  }
}

__device__ __forceinline__ void tw_store_t(TwTile& wt, const float2 (&v)[8], int lane) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = lane + 32 * k;
    const int pt = i % TW_PTS, b = i / TW_PTS;
    uint32_t hi, lo;
    tc_split2(v[k].x, v[k].y, hi, lo);
    tc_st16(wt.t_hi + b * TW_TPITCH + pt, hi);
    tc_st16(wt.t_lo + b * TW_TPITCH + pt, lo);
    tc_st16(wt.t_hi + (16 + b) * TW_TPITCH + pt, hi >> 16);
    tc_st16(wt.t_lo + (16 + b) * TW_TPITCH + pt, lo >> 16);
  }
}

// acc[mt][nt] += C^T T over the 16 points of the warp's tile
__device__ __forceinline__ void tw_bra_step(const TwTile& wt, float (&acc)[4][4][4], int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int q = lane >> 3, r = lane & 7;
  uint32_t bh[4][2], bl[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const __half* ph = wt.t_hi + (8 * nt + g) * TW_TPITCH + 2 * t;
    const __half* pl = wt.t_lo + (8 * nt + g) * TW_TPITCH + 2 * t;
    bh[nt][0] = tc_ld32(ph);
    bh[nt][1] = tc_ld32(ph + 8);
    bl[nt][0] = tc_ld32(pl);
    bl[nt][1] = tc_ld32(pl + 8);
  }
  const int prow = ((q >> 1) << 3) + r;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    const int jcol = 16 * mt + ((q & 1) << 3);
    uint32_t ahi[4], alo[4];
    tc_ldsm_x4_trans(ahi, wt.c_hi + prow * TW_CPITCH + jcol);
    tc_ldsm_x4_trans(alo, wt.c_lo + prow * TW_CPITCH + jcol);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      tc_mma(acc[mt][nt], alo, bh[nt][0], bh[nt][1]);
      tc_mma(acc[mt][nt], ahi, bl[nt][0], bl[nt][1]);
      tc_mma(acc[mt][nt], ahi, bh[nt][0], bh[nt][1]);
    }
  }
}

// ----------------------------------------------------------------------------
// Bra of orbitals on tensor cores, one 8-CTA cluster per unit, warp-independent
// main loop.  with_d = 0: P[u][b][j] (q_half tables), every warp one slice
// sequence; with_d = 1: Pa[u][b][j][alpha] (q_obs tables), warp w takes
// weighting alpha = w % 4 and every other slice.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 2) k_bra_w(LaunchSet L, const float2* __restrict__ src,
                                                  float2* __restrict__ out, int with_d) {
  extern __shared__ __align__(16) unsigned char tw_raw[];
  TwSmem& sm = *reinterpret_cast<TwSmem*>(tw_raw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float2* ph = (const float2*)(with_d ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride;
  tw_load_tables(sm, c, ph);
  __syncthreads();
  const int n_steps_all = (c.npts + TW_PTS - 1) / TW_PTS;
  const int alpha = with_d ? (warp & 3) : 0;
  const int s_first = with_d ? (warp >> 2) : warp;
  const int s_stride = with_d ? 2 : 8;
  TwTile& wt = sm.w[warp];
  const float2* s0 = src + U.psi_off;
  float acc[4][4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;
  float2 v[8];
  if (s_first < n_steps_all) tw_fetch(v, s0, c, s_first * TW_PTS, lane);
  for (int s = s_first; s < n_steps_all; s += s_stride) {
    const int p0 = s * TW_PTS;
    __syncwarp();
    tw_store_t(wt, v, lane);
    if (s + s_stride < n_steps_all) tw_fetch(v, s0, c, (s + s_stride) * TW_PTS, lane);
    tw_gen_c(wt, sm, c, p0, alpha, lane);
    __syncwarp();
    tw_bra_step(wt, acc, lane);
  }
  // reduce the warps in a fixed order into D[slot][64][33] (tile area)
  float* D = reinterpret_cast<float*>(sm.w);
  const int slot = with_d ? (warp & 3) : 0;
  const int order = with_d ? (warp >> 2) : warp;
  const int n_order = with_d ? 2 : 8;
  const int g = lane >> 2, t = lane & 3;
  for (int pass = 0; pass < n_order; ++pass) {
    __syncthreads();
    if (order == pass) {
      float* Ds = D + slot * 64 * TC_D_PITCH;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int row = 16 * mt + g + ((e >> 1) << 3);
            const int col = 8 * nt + 2 * t + (e & 1);
            float* dst = Ds + row * TC_D_PITCH + col;
            *dst = (pass == 0) ? acc[mt][nt][e] : *dst + acc[mt][nt][e];
          }
    }
  }
  __syncthreads();
  const int n_slots = with_d ? 4 : 1;
  const float dv = (float)c.dv * TC_UNSCALE;
  for (int i = threadIdx.x; i < n_slots * 32 * 16; i += blockDim.x) {
    const int sl = i / 512, o = i % 512;
    const int j = o % 32, b = o / 32;
    if (j < c.n_proj && b < c.n_bands) {
      const float* Dl = D + sl * 64 * TC_D_PITCH;
      const float pr = Dl[j * TC_D_PITCH + b] - Dl[(32 + j) * TC_D_PITCH + 16 + b];
      const float pi = Dl[j * TC_D_PITCH + 16 + b] + Dl[(32 + j) * TC_D_PITCH + b];
      const float2 val = make_float2(dv * pr, dv * pi);
      if (with_d)
        out[U.pa_off + (long long)b * 4 * c.n_proj + 4 * j + sl] = val;
      else
        out[U.p_off + (long long)b * c.n_proj + j] = val;
    }
  }
}

// ----------------------------------------------------------------------------
// Ket on tensor cores, warp-independent: V[u][b][r] = sum_j beta~_j(r) E_j P_jb.
// grid (chunks of 8 x TW_KET_STEPS slices, units); warp w takes slices
// w, w + 8, ... of the chunk and writes V from its MMA registers.
// ----------------------------------------------------------------------------
#define TW_KET_STEPS 4
__global__ void __launch_bounds__(256, 2) k_ket_w(LaunchSet L, const float2* __restrict__ P,
                                                  float2* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char tw_raw[];
  TwSmem& sm = *reinterpret_cast<TwSmem*>(tw_raw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  tw_load_tables(sm, c, (const float2*)L.ph_half + (long long)u * L.ph_stride);
  for (int i = threadIdx.x; i < 32 * 16; i += blockDim.x) {
    const int j = i % 32, b = i / 32;
    float wr = 0.f, wi = 0.f;
    if (j < c.n_proj && b < c.n_bands) {
      const float2 p = P[U.p_off + (long long)b * c.n_proj + j];
      const float e = (float)c.ekb[j];
      wr = e * p.x;
      wi = e * p.y;
    }
    uint32_t hi, lo, nhi, nlo;
    tc_split2(wr, wi, hi, lo);
    tc_split2(-wr, wi, nhi, nlo);
    tc_st16(sm.wk_hi + b * TC_W_PITCH + j, hi);
    tc_st16(sm.wk_lo + b * TC_W_PITCH + j, lo);
    tc_st16(sm.wk_hi + (16 + b) * TC_W_PITCH + j, hi >> 16);
    tc_st16(sm.wk_lo + (16 + b) * TC_W_PITCH + j, lo >> 16);
    tc_st16(sm.wk_hi + b * TC_W_PITCH + 32 + j, nhi >> 16);
    tc_st16(sm.wk_lo + b * TC_W_PITCH + 32 + j, nlo >> 16);
    tc_st16(sm.wk_hi + (16 + b) * TC_W_PITCH + 32 + j, nhi);
    tc_st16(sm.wk_lo + (16 + b) * TC_W_PITCH + 32 + j, nlo);
  }
  __syncthreads();
  TwTile& wt = sm.w[warp];
  const int n_steps_all = (c.npts + TW_PTS - 1) / TW_PTS;
  const int s_begin = blockIdx.x * 8 * TW_KET_STEPS;
  const int s_end = min(n_steps_all, s_begin + 8 * TW_KET_STEPS);
  for (int s = s_begin + warp; s < s_end; s += 8) {
    const int p0 = s * TW_PTS;
    __syncwarp();
    tw_gen_c(wt, sm, c, p0, 0, lane);
    __syncwarp();
    float d[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int e = 0; e < 4; ++e) d[nt][e] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int col = 16 * ks + 2 * t4;
      uint32_t ahi[4], alo[4];
      ahi[0] = tc_ld32(wt.c_hi + g * TW_CPITCH + col);
      ahi[1] = tc_ld32(wt.c_hi + (g + 8) * TW_CPITCH + col);
      ahi[2] = tc_ld32(wt.c_hi + g * TW_CPITCH + col + 8);
      ahi[3] = tc_ld32(wt.c_hi + (g + 8) * TW_CPITCH + col + 8);
      alo[0] = tc_ld32(wt.c_lo + g * TW_CPITCH + col);
      alo[1] = tc_ld32(wt.c_lo + (g + 8) * TW_CPITCH + col);
      alo[2] = tc_ld32(wt.c_lo + g * TW_CPITCH + col + 8);
      alo[3] = tc_ld32(wt.c_lo + (g + 8) * TW_CPITCH + col + 8);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = 8 * nt + g;
        const uint32_t bh0 = tc_ld32(sm.wk_hi + n * TC_W_PITCH + col), bh1 = tc_ld32(sm.wk_hi + n * TC_W_PITCH + col + 8);
        const uint32_t bl0 = tc_ld32(sm.wk_lo + n * TC_W_PITCH + col), bl1 = tc_ld32(sm.wk_lo + n * TC_W_PITCH + col + 8);
        tc_mma(d[nt], alo, bh0, bh1);
        tc_mma(d[nt], ahi, bl0, bl1);
        tc_mma(d[nt], ahi, bh0, bh1);
      }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int p = p0 + g + 8 * r;
      if (p >= c.npts) continue;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int b = 2 * t4 + (k & 1) + 8 * (k >> 1);
        if (b < c.n_bands)
          V[U.psi_off + (long long)b * c.npts + p] = make_float2(d[k >> 1][2 * r + (k & 1)] * TC_UNSCALE,
                                                                 d[2 + (k >> 1)][2 * r + (k & 1)] * TC_UNSCALE);
      }
    }
  }
}




// ----------------------------------------------------------------------------
// Taylor stage m, 2.5-D z-march for float orbitals with a compile-time grid
// depth NZ (the z loop is fully unrolled, so the register queue of the 2 ND + 1
// column values rotates by renaming) and packed FP32x2 complex arithmetic.
// One CTA per (band, unit), one thread per (x, y) column (n1 n2 <= 256).
//   t_m = (-i dt/m)[h_loc t + V], psi accumulation as in k_stage.
// ----------------------------------------------------------------------------
template <int NZ>
__global__ void __launch_bounds__(256, 4) k_stage_zf(LaunchSet L, const float2* __restrict__ tin,
                                                     float2* __restrict__ tout, float2* __restrict__ psi,
                                                     const float2* __restrict__ V, int m) {
  constexpr int ND = TC_ND;
  extern __shared__ __align__(16) unsigned char zraw[];
  float2* plane = reinterpret_cast<float2*>(zraw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int n1 = c.n1, n2 = c.n2, n12 = n1 * n2;
  const int col = threadIdx.x;
  const bool act = col < n12;
  const int ix = act ? col % n1 : 0, iy = act ? col / n1 : 0;
  const int W = n1 + 2 * ND;
  const float2* me = plane + (iy + ND) * W + ix + ND;
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const float hdt = (float)(S.dt * L.dt_scale) / (float)m;
  const float* veff = reinterpret_cast<const float*>(S.veff);
  const long long base0 = U.psi_off + (long long)b * c.npts + col;
  const float2* tb = tin + base0;
  const float2 zero = make_float2(0.f, 0.f);
  const float2 neg1 = make_float2(-1.f, -1.f);
  float2 qv[NZ + 2 * ND];   // t(z) for z = -ND .. NZ - 1 + ND (periodic)
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) qv[k] = act ? tb[(long long)((k - ND + NZ) % NZ) * n12] : zero;
  float2 v_cur = act ? V[base0] : zero;
  float2 p_cur = (act && m >= 2) ? psi[base0] : zero;
  float e_cur = act ? veff[col] : 0.f;
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    // t(z + ND) enters the queue (periodic), V, psi, v_eff of plane z + 1 prefetched
    qv[z + 2 * ND] = act ? tb[(long long)((z + ND) % NZ) * n12] : zero;
    float2 v_nxt = zero, p_nxt = zero;
    float e_nxt = 0.f;
    if (act && z + 1 < NZ) {
      const long long idx_n = base0 + (long long)(z + 1) * n12;
      v_nxt = V[idx_n];
      if (m >= 2) p_nxt = psi[idx_n];
      e_nxt = veff[(z + 1) * n12 + col];
    }
    __syncthreads();
    if (act) zpad_store(plane, n1, n2, ix, iy, qv[z + ND]);
    __syncthreads();
    if (act) {
      const float2 ce = qv[z + ND];
      const long long idx = base0 + (long long)z * n12;
      const float dg = dg0 + e_cur;
      float2 h = __fmul2_rn(make_float2(dg, dg), ce);
      float2 gx = zero, gy = zero, gz = zero;
#pragma unroll
      for (int mm = 1; mm <= ND; ++mm) {
        const float2 xu = me[mm], xd = me[-mm];
        const float2 yu = me[mm * W], yd = me[-mm * W];
        const float2 zu = qv[z + ND + mm], zd = qv[z + ND - mm];
        h = f2fma(c.hlap2[0][mm], __fadd2_rn(xu, xd), h);
        h = f2fma(c.hlap2[1][mm], __fadd2_rn(yu, yd), h);
        h = f2fma(c.hlap2[2][mm], __fadd2_rn(zu, zd), h);
        gx = f2fma(c.gradw2[0][mm], f2fma(neg1, xd, xu), gx);
        gy = f2fma(c.gradw2[1][mm], f2fma(neg1, yd, yu), gy);
        gz = f2fma(c.gradw2[2][mm], f2fma(neg1, zd, zu), gz);
      }
      // q.grad t = q0 gx + q1 gy + q2 gz;  h += -i q.grad t + V
      float2 qg = __fmul2_rn(make_float2(q0, q0), gx);
      qg = f2fma(make_float2(q1, q1), gy, qg);
      qg = f2fma(make_float2(q2, q2), gz, qg);
      const float hr = h.x + qg.y + v_cur.x;
      const float hi = h.y - qg.x + v_cur.y;
      const float2 t = make_float2(hdt * hi, -hdt * hr);
      if (m < 4) tout[idx] = t;
      if (m == 2) {
        psi[idx] = __fadd2_rn(p_cur, __fadd2_rn(ce, t));
      } else if (m >= 3) {
        psi[idx] = __fadd2_rn(p_cur, t);
      }
    }
    v_cur = v_nxt;
    p_cur = p_nxt;
    e_cur = e_nxt;
  }
}

// ----------------------------------------------------------------------------
// The same Taylor stage on 16^3 grids with the band of t_{m-1} staged in
// shared memory by bulk copies (issued by one thread at the start of the CTA,
// completed on one mbarrier with a bounded wait), so that the z-march runs
// without a CTA barrier: x and y neighbours are shared-memory loads at
// per-thread addresses plus compile-time plane offsets, z neighbours a
// register queue.  VP = true stages the bands of V = V_NL t_{m-1} and (m >= 2)
// psi in shared memory as well (96 KiB: the CTA's whole input in flight at
// once, 2 CTAs per SM); VP = false reads them per plane from global memory,
// two planes ahead (32 KiB of shared memory, 3 CTAs per SM).  Algorithmic
// bytes per launch: t_{m-1} and V read; t_m written (m < 4); psi read and
// written (m >= 2).  Same arithmetic per point as k_stage_zf.
// ----------------------------------------------------------------------------
#define ZB_N 16
#define ZB_NP 256

template <bool VP>
__global__ void __launch_bounds__(ZB_NP, VP ? 2 : 3) k_stage_zb(LaunchSet L, const float2* __restrict__ tin,
                                                               float2* __restrict__ tout, float2* __restrict__ psi,
                                                               const float2* __restrict__ V, int m) {
  constexpr int ND = TC_ND, N = ZB_N, NP = ZB_NP;
  extern __shared__ __align__(128) unsigned char zbraw[];
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(zbraw);
  float2* st = reinterpret_cast<float2*>(zbraw + 128);
  float2* sv = st + N * NP;
  float2* sp = sv + N * NP;
  const CellDev& c = L.cell;
  const int b = blockIdx.x;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int col = threadIdx.x, ix = col & (N - 1), iy = col / N;
  const long long base = U.psi_off + (long long)b * (N * NP);
  const uint32_t bar = bk_smem(mbar);
  constexpr uint32_t band_bytes = (uint32_t)(N * NP * sizeof(float2));
  if (col == 0) {
    bk_mbar_init(bar, 1);
    bk_mbar_expect_tx(bar, band_bytes * (VP ? (m >= 2 ? 3u : 2u) : 1u));
    bk_copy_g2s(bk_smem(st), tin + base, band_bytes, bar);
    if (VP) {
      bk_copy_g2s(bk_smem(sv), V + base, band_bytes, bar);
      if (m >= 2) bk_copy_g2s(bk_smem(sp), psi + base, band_bytes, bar);
    }
  }
  const float2 zero = make_float2(0.f, 0.f);
  const float2* gv = V + base + col;
  const float2* gp = psi + base + col;
  float2 vq[2], pq[2];   // V and psi of the next two planes (VP = false)
  if (!VP) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      vq[k] = gv[k * NP];
      pq[k] = m >= 2 ? gp[k * NP] : zero;
    }
  }
  const float2* cz = st + col;
  const float2* xp[ND];
  const float2* xm[ND];
  const float2* yp[ND];
  const float2* ym[ND];
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) {
    xp[mm - 1] = st + iy * N + ((ix + mm) & (N - 1));
    xm[mm - 1] = st + iy * N + ((ix - mm) & (N - 1));
    yp[mm - 1] = st + ((iy + mm) & (N - 1)) * N + ix;
    ym[mm - 1] = st + ((iy - mm) & (N - 1)) * N + ix;
  }
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const float hdt = (float)(S.dt * L.dt_scale) / (float)m;
  const float* veff = reinterpret_cast<const float*>(S.veff) + col;
  __syncthreads();   // the barrier is initialised before anyone polls it
  const bool ok = bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
  if (!__syncthreads_and(ok)) {
    if (col == 0) {
      atomicOr(S.status, BK_STATUS_TIMEOUT);
      bk_mbar_wait(bar, 0, BK_WAIT_POLLS);   // let the copies in flight land before the CTA exits
    }
    return;
  }
  const float2 neg1 = make_float2(-1.f, -1.f);
  float2 qv[N + 2 * ND];   // t(z) for z = -ND .. N - 1 + ND (periodic)
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) qv[k] = cz[((k - ND + N) & (N - 1)) * NP];
  float2* to = tout + base + col;
  float2* po = psi + base + col;
#pragma unroll
  for (int z = 0; z < N; ++z) {
    qv[z + 2 * ND] = cz[((z + ND) & (N - 1)) * NP];
    float2 vz, pz;
    if (VP) {
      vz = sv[z * NP + col];
      pz = m >= 2 ? sp[z * NP + col] : zero;
    } else {
      vz = vq[z & 1];
      pz = pq[z & 1];
      if (z + 2 < N) {
        vq[z & 1] = gv[(z + 2) * NP];
        pq[z & 1] = m >= 2 ? gp[(z + 2) * NP] : zero;
      }
    }
    const float2 ce = qv[z + ND];
    const float dg = dg0 + veff[z * NP];
    float2 h = __fmul2_rn(make_float2(dg, dg), ce);
    float2 gx = zero, gy = zero, gz = zero;
#pragma unroll
    for (int mm = 1; mm <= ND; ++mm) {
      const float2 xu = xp[mm - 1][z * NP], xd = xm[mm - 1][z * NP];
      const float2 yu = yp[mm - 1][z * NP], yd = ym[mm - 1][z * NP];
      const float2 zu = qv[z + ND + mm], zd = qv[z + ND - mm];
      h = f2fma(c.hlap2[0][mm], __fadd2_rn(xu, xd), h);
      h = f2fma(c.hlap2[1][mm], __fadd2_rn(yu, yd), h);
      h = f2fma(c.hlap2[2][mm], __fadd2_rn(zu, zd), h);
      gx = f2fma(c.gradw2[0][mm], f2fma(neg1, xd, xu), gx);
      gy = f2fma(c.gradw2[1][mm], f2fma(neg1, yd, yu), gy);
      gz = f2fma(c.gradw2[2][mm], f2fma(neg1, zd, zu), gz);
    }
    float2 qg = __fmul2_rn(make_float2(q0, q0), gx);
    qg = f2fma(make_float2(q1, q1), gy, qg);
    qg = f2fma(make_float2(q2, q2), gz, qg);
    const float hr = h.x + qg.y + vz.x;
    const float hi = h.y - qg.x + vz.y;
    const float2 t = make_float2(hdt * hi, -hdt * hr);
    if (m < 4) to[z * NP] = t;
    if (m == 2) {
      po[z * NP] = __fadd2_rn(pz, __fadd2_rn(ce, t));
    } else if (m >= 3) {
      po[z * NP] = __fadd2_rn(pz, t);
    }
  }
}

// ----------------------------------------------------------------------------
// Observation pass for float orbitals on depth-NZ grids, 2.5-D form: one CTA
// per unit, one thread per (x, y) column; bands outer, z-march inner.  Per
// column and plane it accumulates occ sum_b |u|^2 (rho) over the bands, and
// per thread sum Re(u* (-i grad u)) and per band sum |u|^2 (block-reduced per
// band).  The unit's sums are written to point tile 0 of the partial
// buffers and zeros to the other tiles, which the finalize kernel adds.
// ----------------------------------------------------------------------------
template <int NZ>
__global__ void __launch_bounds__(256) k_observe_zf(LaunchSet L, const float2* __restrict__ psi,
                                                    double* __restrict__ rho_part, double* __restrict__ jk_part,
                                                    double* __restrict__ nrm_part) {
  constexpr int ND = TC_ND;
  __shared__ float2 plane[(16 + 2 * TC_ND) * (16 + 2 * TC_ND)];
  __shared__ float red[8];
  __shared__ double redj[8][3];
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int n1 = c.n1, n2 = c.n2, n12 = n1 * n2;
  const int col = threadIdx.x;
  const bool act = col < n12;
  const int ix = act ? col % n1 : 0, iy = act ? col / n1 : 0;
  const int W = n1 + 2 * ND;
  const float2* me = plane + (iy + ND) * W + ix + ND;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float2 zero = make_float2(0.f, 0.f);
  float rho[NZ];
#pragma unroll
  for (int z = 0; z < NZ; ++z) rho[z] = 0.f;
  double jx = 0.0, jy = 0.0, jz = 0.0;
  for (int b = 0; b < c.n_bands; ++b) {
    const float2* tb = psi + U.psi_off + (long long)b * c.npts + col;
    float2 qv[NZ + 2 * ND];
#pragma unroll
    for (int k = 0; k < 2 * ND; ++k) qv[k] = act ? tb[(long long)((k - ND + NZ) % NZ) * n12] : zero;
    float nb = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      qv[z + 2 * ND] = act ? tb[(long long)((z + ND) % NZ) * n12] : zero;
      __syncthreads();
      if (act) zpad_store(plane, n1, n2, ix, iy, qv[z + ND]);
      __syncthreads();
      if (act) {
        const float2 ce = qv[z + ND];
        float2 gx = zero, gy = zero, gz = zero;
#pragma unroll
        for (int mm = 1; mm <= ND; ++mm) {
          const float2 xu = me[mm], xd = me[-mm];
          const float2 yu = me[mm * W], yd = me[-mm * W];
          const float2 zu = qv[z + ND + mm], zd = qv[z + ND - mm];
          gx.x = fmaf(c.gradwf[0][mm], xu.x - xd.x, gx.x);
          gx.y = fmaf(c.gradwf[0][mm], xu.y - xd.y, gx.y);
          gy.x = fmaf(c.gradwf[1][mm], yu.x - yd.x, gy.x);
          gy.y = fmaf(c.gradwf[1][mm], yu.y - yd.y, gy.y);
          gz.x = fmaf(c.gradwf[2][mm], zu.x - zd.x, gz.x);
          gz.y = fmaf(c.gradwf[2][mm], zu.y - zd.y, gz.y);
        }
        const float n2v = ce.x * ce.x + ce.y * ce.y;
        rho[z] += n2v;
        nb += n2v;
        // Re(conj(u) (-i g)) = u_r g_i - u_i g_r
        bx += ce.x * gx.y - ce.y * gx.x;
        by += ce.x * gy.y - ce.y * gy.x;
        bz += ce.x * gz.y - ce.y * gz.x;
      }
    }
    jx += bx;
    jy += by;
    jz += bz;
    // band norm: warp then block sum (fixed order)
    for (int off = 16; off > 0; off >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, off);
    __syncthreads();
    if (lane == 0) red[warp] = nb;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += (double)red[w];
      nrm_part[U.nrm_off + b] = sum;
    }
  }
  if (act)
#pragma unroll
    for (int z = 0; z < NZ; ++z) rho_part[U.rho_off + (long long)z * n12 + col] = c.occ * (double)rho[z];
  for (int off = 16; off > 0; off >>= 1) {
    jx += __shfl_xor_sync(0xffffffffu, jx, off);
    jy += __shfl_xor_sync(0xffffffffu, jy, off);
    jz += __shfl_xor_sync(0xffffffffu, jz, off);
  }
  if (lane == 0) {
    redj[warp][0] = jx;
    redj[warp][1] = jy;
    redj[warp][2] = jz;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += redj[w][threadIdx.x];
    jk_part[U.jk_off + threadIdx.x] = sum;
  }
  // zeros for the other point tiles of the partial layout
  for (int i = threadIdx.x; i < 3 * (c.n_tiles - 1); i += blockDim.x) jk_part[U.jk_off + 3 + i] = 0.0;
  for (int i = threadIdx.x; i < c.n_bands * (c.n_tiles - 1); i += blockDim.x)
    nrm_part[U.nrm_off + c.n_bands + i] = 0.0;
}
