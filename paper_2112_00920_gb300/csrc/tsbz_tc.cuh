// Tensor-core projector contractions (split-BF16, FP32 accumulate) and the
// fused Taylor stage of the single-precision tensor-core mode.
//
// Projector values of one k-point, C_j(r) = conj(beta~_j(r)) = pnorm_j g(r) w_j(d) exp(+i q.d),
// are generated per tile of TC_PT grid points in shared memory as a real
// matrix Cs[pt][j'] (j' < 32: Re C_j, j' >= 32: Im C_j), each value split into
// a BF16 high part and a BF16 low part (x ~ hi + lo).  A product A B is
// evaluated as A_hi B_hi + A_hi B_lo + A_lo B_hi with mma.sync m16n8k16 and
// FP32 accumulation.
//   bra  P_jb = dV sum_r C_j(r) t_b(r):  D[j'][n'] = sum_pt Cs[pt][j'] Ts[n'][pt]
//        (n' < 16: Re t_b, n' >= 16: Im t_b), P_re = D[j][b] - D[32+j][16+b],
//        P_im = D[j][16+b] + D[32+j][b]
//   ket  V_b(r) = sum_j conj(C_j(r)) E_j P_jb:  V[pt][n'] = sum_j' Cs[pt][j'] Wt[n'][j']
//        with Wt built from W = E P so that V[pt][b] = Re V_b, V[pt][16+b] = Im V_b.
// One CTA handles one unit (k-point, all bands <= 16, projectors <= 32) and
// loops over all point tiles, so every projection is complete inside the CTA.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tsbz_internal.h"

#define TC_PT 128          // grid points per tile
#define TC_THREADS 256     // 8 warps
#define TC_CS_PITCH 72     // bf16 per Cs row (64 + 8 padding)
#define TC_W_PITCH 72      // bf16 per Wt row
#define TC_TS_PITCH 136    // bf16 per Ts row (128 + 8 padding)
#define TC_V_PITCH 33      // floats per Vs row
#define TC_ND 4            // stencil half-width of the fused stage

struct TcSmem {
  __nv_bfloat16 cs_hi[TC_PT * TC_CS_PITCH];
  __nv_bfloat16 cs_lo[TC_PT * TC_CS_PITCH];
  __nv_bfloat16 ts_hi[32 * TC_TS_PITCH];
  __nv_bfloat16 ts_lo[32 * TC_TS_PITCH];
  __nv_bfloat16 w_hi[32 * TC_W_PITCH];
  __nv_bfloat16 w_lo[32 * TC_W_PITCH];
  float vs[TC_PT * TC_V_PITCH];
};

// Split a pair (x, y) into packed BF16 high parts and packed BF16 low parts
// (round to nearest for both); one packed conversion per part, because on
// this GPU conversions issue on a narrow pipe.
__device__ __forceinline__ void tc_split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x - hf.x, y - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ uint32_t tc_ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void tc_st16(__nv_bfloat16* p, uint32_t bits) {
  *reinterpret_cast<unsigned short*>(p) = (unsigned short)(bits & 0xFFFFu);
}

__device__ __forceinline__ void tc_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tc_ldsm_x4_trans(uint32_t (&r)[4], const __nv_bfloat16* row_ptr) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(row_ptr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// Generate Cs for points p0 .. p0+TC_PT-1 of unit u.  alpha = 0: plain
// projector rows; alpha = 1..3: rows multiplied by d_x, d_y, d_z.
__device__ __forceinline__ void tc_gen_c(TcSmem& sm, const CellDev& c, const float2* ph, int p0, int alpha) {
  const int nm = c.nmax;
  for (int i = threadIdx.x; i < TC_PT * 8; i += TC_THREADS) {
    const int pt = i % TC_PT, a = i / TC_PT;
    const int p = p0 + pt;
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    if (p < c.npts && a < c.n_atoms) {
      const int ix = p % c.n1, iy = (p / c.n1) % c.n2, iz = p / (c.n1 * c.n2);
      const float* ga = c.g1f + (long long)a * 3 * nm;
      const float* da = c.d1f + (long long)a * 3 * nm;
      const float g = ga[ix] * ga[nm + iy] * ga[2 * nm + iz];
      const float d[3] = {da[ix], da[nm + iy], da[2 * nm + iz]};
      const float2* pa = ph + (long long)a * 3 * nm;
      const float2 px = pa[ix], py = pa[nm + iy], pz = pa[2 * nm + iz];
      const float2 pxy = make_float2(px.x * py.x - px.y * py.y, px.x * py.y + px.y * py.x);
      float fr = pxy.x * pz.x - pxy.y * pz.y, fi = pxy.x * pz.y + pxy.y * pz.x;
      float sc = g;
      if (alpha > 0) sc *= d[alpha - 1];
      fr *= sc;
      fi *= sc;
      const float* pn = c.pnormf + 4 * a;
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
    *reinterpret_cast<uint2*>(sm.cs_hi + pt * TC_CS_PITCH + 4 * a) = hr;
    *reinterpret_cast<uint2*>(sm.cs_lo + pt * TC_CS_PITCH + 4 * a) = lr;
    *reinterpret_cast<uint2*>(sm.cs_hi + pt * TC_CS_PITCH + 32 + 4 * a) = hc;
    *reinterpret_cast<uint2*>(sm.cs_lo + pt * TC_CS_PITCH + 32 + 4 * a) = lc;
  }
}

// D[j'][n'] += sum over the tile of Cs[pt][j'] Ts[n'][pt]; warp w owns j'-tile
// w/2 and n'-tiles 2(w%2), 2(w%2)+1.
__device__ __forceinline__ void tc_bra_tile(const TcSmem& sm, float (&acc)[2][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp >> 1, nt0 = 2 * (warp & 1);
  const int q = lane >> 3, r = lane & 7;
#pragma unroll 2
  for (int ks = 0; ks < TC_PT / 16; ++ks) {
    const int prow = 16 * ks + ((q >> 1) << 3) + r;
    const int jcol = 16 * mt + ((q & 1) << 3);
    uint32_t ahi[4], alo[4];
    tc_ldsm_x4_trans(ahi, sm.cs_hi + prow * TC_CS_PITCH + jcol);
    tc_ldsm_x4_trans(alo, sm.cs_lo + prow * TC_CS_PITCH + jcol);
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int n = 8 * (nt0 + j) + g;
      const __nv_bfloat16* bh = sm.ts_hi + n * TC_TS_PITCH + 16 * ks + 2 * t;
      const __nv_bfloat16* bl = sm.ts_lo + n * TC_TS_PITCH + 16 * ks + 2 * t;
      const uint32_t bh0 = tc_ld32(bh), bh1 = tc_ld32(bh + 8);
      const uint32_t bl0 = tc_ld32(bl), bl1 = tc_ld32(bl + 8);
      tc_mma(acc[j], alo, bh0, bh1);
      tc_mma(acc[j], ahi, bl0, bl1);
      tc_mma(acc[j], ahi, bh0, bh1);
    }
  }
}

// Write the bra result (dV * complex combination) of one unit: out[b * stride + j * jstep + joff]
__device__ __forceinline__ void tc_bra_store(TcSmem& sm, const float (&acc)[2][4], const CellDev& c, float2* out,
                                             int stride, int jstep, int joff) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int mt = warp >> 1, nt0 = 2 * (warp & 1);
  float* D = sm.vs;  // [64][33]
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int n = 8 * (nt0 + j) + 2 * t;
    const int row = 16 * mt + g;
    D[row * TC_V_PITCH + n] = acc[j][0];
    D[row * TC_V_PITCH + n + 1] = acc[j][1];
    D[(row + 8) * TC_V_PITCH + n] = acc[j][2];
    D[(row + 8) * TC_V_PITCH + n + 1] = acc[j][3];
  }
  __syncthreads();
  const float dv = (float)c.dv;
  for (int i = threadIdx.x; i < 32 * 16; i += TC_THREADS) {
    const int j = i % 32, b = i / 32;
    if (j < c.n_proj && b < c.n_bands) {
      const float pr = D[j * TC_V_PITCH + b] - D[(32 + j) * TC_V_PITCH + 16 + b];
      const float pi = D[j * TC_V_PITCH + 16 + b] + D[(32 + j) * TC_V_PITCH + b];
      out[(long long)b * stride + j * jstep + joff] = make_float2(dv * pr, dv * pi);
    }
  }
}

// Load a tile of orbitals (all bands) into Ts as split BF16.
__device__ __forceinline__ void tc_load_ts(TcSmem& sm, const CellDev& c, const float2* src, int p0) {
  for (int i = threadIdx.x; i < TC_PT * 16; i += TC_THREADS) {
    const int pt = i % TC_PT, b = i / TC_PT;
    const int p = p0 + pt;
    float2 v = make_float2(0.f, 0.f);
    if (p < c.npts && b < c.n_bands) v = src[(long long)b * c.npts + p];
    uint32_t hi, lo;
    tc_split2(v.x, v.y, hi, lo);
    tc_st16(sm.ts_hi + b * TC_TS_PITCH + pt, hi);
    tc_st16(sm.ts_lo + b * TC_TS_PITCH + pt, lo);
    tc_st16(sm.ts_hi + (16 + b) * TC_TS_PITCH + pt, hi >> 16);
    tc_st16(sm.ts_lo + (16 + b) * TC_TS_PITCH + pt, lo >> 16);
  }
}

// ----------------------------------------------------------------------------
// Stand-alone bra of psi on tensor cores.  grid (4 alphas or 1, units).
//   alpha = 0 with with_d = 0: P[u][b][j]            (q_half tables)
//   with_d = 1: Pa[u][b][j][alpha], alpha = blockIdx.x (q_obs tables)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 2) k_bra_tc(LaunchSet L, const float2* __restrict__ psi,
                                                          float2* __restrict__ out, int with_d) {
  extern __shared__ __align__(16) unsigned char tc_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_raw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.y];
  const UnitDev U = L.units[u];
  const int alpha = with_d ? blockIdx.x : 0;
  const float2* ph = (const float2*)(with_d ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int p0 = 0; p0 < c.npts; p0 += TC_PT) {
    __syncthreads();
    tc_gen_c(sm, c, ph, p0, alpha);
    tc_load_ts(sm, c, psi + U.psi_off, p0);
    __syncthreads();
    tc_bra_tile(sm, acc);
  }
  if (with_d)
    tc_bra_store(sm, acc, c, (float2*)out + U.pa_off, 4 * c.n_proj, 4, alpha);
  else
    tc_bra_store(sm, acc, c, (float2*)out + U.p_off, c.n_proj, 1, 0);
}

// ----------------------------------------------------------------------------
// Fused Taylor stage m on tensor cores, one CTA per unit.
//   t_m = (-i dt/m)[ -1/2 lap t - i q.grad t + (|q|^2/2 + v_eff) t + V_NL t ]
//   psi accumulation as in k_stage; for m < 4 also P_m = <beta~|t_m> -> Pout.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 2) k_stage_tc(LaunchSet L, const float2* __restrict__ tin,
                                                            float2* __restrict__ tout, float2* __restrict__ psi,
                                                            const float2* __restrict__ Pin, float2* __restrict__ Pout,
                                                            int m) {
  extern __shared__ __align__(16) unsigned char tc_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(tc_raw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2], q2h = qt[3];
  const float hdt = (float)S.dt / (float)m;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const bool do_bra = m < 4;

  // Wt (ket operand) from W = E_j P_jb:
  //   Wt[b][j] = Wr, Wt[16+b][j] = Wi, Wt[b][32+j] = Wi, Wt[16+b][32+j] = -Wr
  for (int i = threadIdx.x; i < 32 * 16; i += TC_THREADS) {
    const int j = i % 32, b = i / 32;
    float wr = 0.f, wi = 0.f;
    if (j < c.n_proj && b < c.n_bands) {
      const float2 p = Pin[U.p_off + (long long)b * c.n_proj + j];
      const float e = (float)c.ekb[j];
      wr = e * p.x;
      wi = e * p.y;
    }
    uint32_t hi, lo, nhi, nlo;
    tc_split2(wr, wi, hi, lo);        // (Wr, Wi)
    tc_split2(-wr, wi, nhi, nlo);     // (-Wr, Wi)
    tc_st16(sm.w_hi + b * TC_W_PITCH + j, hi);
    tc_st16(sm.w_lo + b * TC_W_PITCH + j, lo);
    tc_st16(sm.w_hi + (16 + b) * TC_W_PITCH + j, hi >> 16);
    tc_st16(sm.w_lo + (16 + b) * TC_W_PITCH + j, lo >> 16);
    tc_st16(sm.w_hi + b * TC_W_PITCH + 32 + j, nhi >> 16);
    tc_st16(sm.w_lo + b * TC_W_PITCH + 32 + j, nlo >> 16);
    tc_st16(sm.w_hi + (16 + b) * TC_W_PITCH + 32 + j, nhi);
    tc_st16(sm.w_lo + (16 + b) * TC_W_PITCH + 32 + j, nlo);
  }
  // per-thread stencil constants (packed float2 pairs)
  float lw[3][TC_ND], gq[3][TC_ND];
  const float qa[3] = {q0, q1, q2};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax)
#pragma unroll
    for (int mm = 1; mm <= TC_ND; ++mm) {
      lw[ax][mm - 1] = (float)(-0.5 * c.lapw[ax][mm]);
      gq[ax][mm - 1] = qa[ax] * (float)c.gradw[ax][mm];
    }
  const float diag0 = (float)(-0.5 * (c.lapw[0][0] + c.lapw[1][0] + c.lapw[2][0])) + q2h;
  const int n12 = c.n1 * c.n2;
  const int pt = threadIdx.x % TC_PT, bh = threadIdx.x / TC_PT;  // point, band half (8 bands)
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};

  for (int p0 = 0; p0 < c.npts; p0 += TC_PT) {
    __syncthreads();
    tc_gen_c(sm, c, ph, p0, 0);
    __syncthreads();
    // ket: warp w -> points 16w..16w+15, all 32 n'
    {
      float d[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[nt][e] = 0.f;
      const int row = 16 * warp + g;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const int col = 16 * ks + 2 * t4;
        uint32_t ahi[4], alo[4];
        ahi[0] = tc_ld32(sm.cs_hi + row * TC_CS_PITCH + col);
        ahi[1] = tc_ld32(sm.cs_hi + (row + 8) * TC_CS_PITCH + col);
        ahi[2] = tc_ld32(sm.cs_hi + row * TC_CS_PITCH + col + 8);
        ahi[3] = tc_ld32(sm.cs_hi + (row + 8) * TC_CS_PITCH + col + 8);
        alo[0] = tc_ld32(sm.cs_lo + row * TC_CS_PITCH + col);
        alo[1] = tc_ld32(sm.cs_lo + (row + 8) * TC_CS_PITCH + col);
        alo[2] = tc_ld32(sm.cs_lo + row * TC_CS_PITCH + col + 8);
        alo[3] = tc_ld32(sm.cs_lo + (row + 8) * TC_CS_PITCH + col + 8);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const int n = 8 * nt + g;
          const uint32_t bh0 = tc_ld32(sm.w_hi + n * TC_W_PITCH + col), bh1 = tc_ld32(sm.w_hi + n * TC_W_PITCH + col + 8);
          const uint32_t bl0 = tc_ld32(sm.w_lo + n * TC_W_PITCH + col), bl1 = tc_ld32(sm.w_lo + n * TC_W_PITCH + col + 8);
          tc_mma(d[nt], alo, bh0, bh1);
          tc_mma(d[nt], ahi, bl0, bl1);
          tc_mma(d[nt], ahi, bh0, bh1);
        }
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int n = 8 * nt + 2 * t4;
        sm.vs[row * TC_V_PITCH + n] = d[nt][0];
        sm.vs[row * TC_V_PITCH + n + 1] = d[nt][1];
        sm.vs[(row + 8) * TC_V_PITCH + n] = d[nt][2];
        sm.vs[(row + 8) * TC_V_PITCH + n + 1] = d[nt][3];
      }
    }
    __syncthreads();
    // stencil + ket + Taylor update for (point pt, bands 8 bh .. 8 bh + 7)
    {
      const int p = p0 + pt;
      const bool valid = p < c.npts;
      const int pp = valid ? p : 0;
      const int ix = pp % c.n1, iy = (pp / c.n1) % c.n2, iz = pp / n12;
      int ox[2 * TC_ND], oy[2 * TC_ND], oz[2 * TC_ND];
#pragma unroll
      for (int mm = 1; mm <= TC_ND; ++mm) {
        ox[2 * mm - 2] = wrap_idx(ix + mm, c.n1) - ix;
        ox[2 * mm - 1] = wrap_idx(ix - mm, c.n1) - ix;
        oy[2 * mm - 2] = (wrap_idx(iy + mm, c.n2) - iy) * c.n1;
        oy[2 * mm - 1] = (wrap_idx(iy - mm, c.n2) - iy) * c.n1;
        oz[2 * mm - 2] = (wrap_idx(iz + mm, c.n3) - iz) * n12;
        oz[2 * mm - 1] = (wrap_idx(iz - mm, c.n3) - iz) * n12;
      }
      const float v = valid ? reinterpret_cast<const float*>(S.veff)[pp] : 0.f;
      const float dg = diag0 + v;
      for (int bl = 0; bl < 8; ++bl) {
        const int b = 8 * bh + bl;
        float tr = 0.f, ti = 0.f;
        if (valid && b < c.n_bands) {
          const long long base = U.psi_off + (long long)b * c.npts + pp;
          const float2* tb = tin + base;
          const float2 ce = tb[0];
          float hx = dg * ce.x, hy = dg * ce.y, gx = 0.f, gy = 0.f;
#pragma unroll
          for (int mm = 1; mm <= TC_ND; ++mm) {
            const float2 xu = tb[ox[2 * mm - 2]], xd = tb[ox[2 * mm - 1]];
            const float2 yu = tb[oy[2 * mm - 2]], yd = tb[oy[2 * mm - 1]];
            const float2 zu = tb[oz[2 * mm - 2]], zd = tb[oz[2 * mm - 1]];
            hx = fmaf(lw[0][mm - 1], xu.x + xd.x, hx);
            hy = fmaf(lw[0][mm - 1], xu.y + xd.y, hy);
            hx = fmaf(lw[1][mm - 1], yu.x + yd.x, hx);
            hy = fmaf(lw[1][mm - 1], yu.y + yd.y, hy);
            hx = fmaf(lw[2][mm - 1], zu.x + zd.x, hx);
            hy = fmaf(lw[2][mm - 1], zu.y + zd.y, hy);
            gx = fmaf(gq[0][mm - 1], xu.x - xd.x, gx);
            gy = fmaf(gq[0][mm - 1], xu.y - xd.y, gy);
            gx = fmaf(gq[1][mm - 1], yu.x - yd.x, gx);
            gy = fmaf(gq[1][mm - 1], yu.y - yd.y, gy);
            gx = fmaf(gq[2][mm - 1], zu.x - zd.x, gx);
            gy = fmaf(gq[2][mm - 1], zu.y - zd.y, gy);
          }
          // -i q.grad t, ket
          const float hr = hx + gy + sm.vs[pt * TC_V_PITCH + b];
          const float hi = hy - gx + sm.vs[pt * TC_V_PITCH + 16 + b];
          tr = hdt * hi;
          ti = -hdt * hr;
          if (m < 4) tout[base] = make_float2(tr, ti);
          if (m == 2) {
            const float2 ps = psi[base];
            psi[base] = make_float2(ps.x + (ce.x + tr), ps.y + (ce.y + ti));
          } else if (m >= 3) {
            const float2 ps = psi[base];
            psi[base] = make_float2(ps.x + tr, ps.y + ti);
          }
        }
        if (do_bra) {
          uint32_t hi, lo;
          tc_split2(tr, ti, hi, lo);
          tc_st16(sm.ts_hi + b * TC_TS_PITCH + pt, hi);
          tc_st16(sm.ts_lo + b * TC_TS_PITCH + pt, lo);
          tc_st16(sm.ts_hi + (16 + b) * TC_TS_PITCH + pt, hi >> 16);
          tc_st16(sm.ts_lo + (16 + b) * TC_TS_PITCH + pt, lo >> 16);
        }
      }
    }
    if (do_bra) {
      __syncthreads();
      tc_bra_tile(sm, acc);
    }
  }
  if (do_bra) tc_bra_store(sm, acc, c, Pout + U.p_off, c.n_proj, 1, 0);
}
