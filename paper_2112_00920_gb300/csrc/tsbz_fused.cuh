// Taylor stage on 16^3 grids with the factorised projector contractions on
// tensor cores (three-product TF32 mma.sync, FP32 accumulate).
//
// Per (unit, band) CTA, with C_{a,t}(r) = pn F^a_x F^a_y F^a_z w_t as in the
// header of the z-march kernels:
//   ket   conj(V_NL t)(col, z) = sum_q A[col][q] Z_q(z): the z dependence is a
//         GEMM over q = (atom, {F_z, d_z F_z}) with the column coefficients
//         A[col][(a,0)] = F_y (G00 + d_y G10), A[col][(a,1)] = F_y G01,
//         G00 = F_x (conj W_s + d_x conj W_px), G10 = F_x conj W_py,
//         G01 = F_x conj W_pz, W = pn E P (x tables first, then y).
//   bra   monomial sums M_a(i,j,k) = sum_r F_x F_y F_z d_x^i d_y^j d_z^k u(r)
//         in three contractions: z as a GEMM S[col][(a,k)] = sum_z u Z_{a,k},
//         then x per (a, k, iy) row, then y per (a, i, j, k) output.
//         P_{a,t} = dV pn M_a(w_t) with w_t = 000, 100, 010, 001 (s, p_x, p_y,
//         p_z); the current needs the second-order sums as well.
// Three-product TF32: x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x -
// x_hi) (round to nearest); A B ~ A_lo B_hi + A_hi B_lo + A_hi B_hi, an
// error of order 2^-21 relative per product, accumulated in FP32.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tsbz_sep.cuh"
#include "tsbz_umma.cuh"

#define FS_N 16
#define FS_NP 256          // columns (threads)
#define FS_NPTS 4096
#define FS_PU 260          // plane pitch of ubuf in float2 (bank-conflict-free fragment stores)
#define FS_BKP 36          // row pitch of the ket B matrix in uint2

__device__ __forceinline__ uint32_t fs_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void fs_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = fs_tf32(x);
  lo = fs_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint2 fs_split2(float x) {
  uint2 r;
  fs_split(x, r.x, r.y);
  return r;
}

__device__ __forceinline__ void fs_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B, A = ah + al, B = (b.x hi, b.y lo) for the two B registers
__device__ __forceinline__ void fs_mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4], uint2 b0,
                                        uint2 b1) {
  fs_mma(d, al, b0.x, b1.x);
  fs_mma(d, ah, b0.y, b1.y);
  fs_mma(d, ah, b0.x, b1.x);
}

struct FsSmem {
  // two plane buffers of pitch FS_PU: the band of t_{m-1}, and V_NL per plane
  // (ket) overwritten by t_m; the projection passes use them as scratch
  float2 xb[FS_N * FS_PU];
  float2 yb[FS_N * FS_PU];
  uint2 bk[32 * FS_BKP];             // ket B matrix (hi, lo); tcgen05 form: and the stage 1-3 bra B_z
  float4 zt[SEP_NA * FS_N];          // (Re F_z, Im F_z, d_z, 0) per atom and plane
  float4 colt[SEP_NA * 2 * FS_N];    // x and y factors (Re F, Im F, d, 0)
  float4 xpk[SEP_NA * FS_N * 3];     // x factors times d^w, w = 0..2, as (Re, Re, Im, Im) pairs
  float2 gt[SEP_NA * 3 * FS_N];      // ket column tables G00, G10, G01 per atom and ix
  float2 wt[SEP_NP];                 // pn E P of the band
  float2 mres[SEP_NA * 10];          // monomial sums of one projection pass
  float vbuf[FS_NPTS];               // v_eff of the sub-simulation (stage kernel)
  int zg[SEP_NA];                    // z group of atom a
  int zrep[4];                       // first atom of group g
  int zmem[4][2];                    // the (at most two) atoms of group g
  int zcnt[4];
  unsigned long long mbar;
  unsigned long long mbar_mma;   // completion of the tcgen05 contractions (one phase per commit)
  uint32_t tslot;                // tensor-memory base address from tcgen05.alloc
};

// z group tables of the cell into shared memory (grouped kernels; read after
// the next barrier)
template <int NZU> __device__ __forceinline__ void fz_load(FsSmem& sm, const CellDev& c) {
  if constexpr (NZU != SEP_NA) {
    const int t = threadIdx.x;
    if (t < SEP_NA) sm.zg[t] = c.zg_of[t];
    if (t < 4) {
      const int lo = c.zg_off[t], n = c.zg_off[t + 1] - lo;
      sm.zrep[t] = c.zg_rep[t];
      sm.zcnt[t] = n;
      sm.zmem[t][0] = n > 0 ? c.zg_mem[lo] : 0;
      sm.zmem[t][1] = n > 1 ? c.zg_mem[lo + 1] : 0;
    }
  }
}

// z factors of one phase table
__device__ __forceinline__ void fs_load_z(float4* zt, const CellDev& c, const float2* ph) {
  const int nm = c.nmax;
  for (int i = threadIdx.x; i < SEP_NA * FS_N; i += blockDim.x) {
    const int a = i / FS_N, z = i - a * FS_N;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < c.n_atoms) {
      const int idx = (a * 3 + 2) * nm + z;
      const float g = c.g1f[idx];
      const float2 p = ph[idx];
      v = make_float4(g * p.x, g * p.y, c.d1f[idx], 0.f);
    }
    zt[i] = v;
  }
}

// Factor tables of one phase table: colt (x and y rows, as the column loader
// of the other kernels) and, for the x contraction of the projection passes,
// d_x^w F_x for w = 0..2 in the (Re, Re, Im, Im) form of the packed products.
__device__ __forceinline__ void fs_load_cols(FsSmem& sm, const CellDev& c, const float2* ph) {
  const int nm = c.nmax;
  for (int i = threadIdx.x; i < SEP_NA * 2 * FS_N; i += blockDim.x) {
    const int a = i / (2 * FS_N), r = i - a * 2 * FS_N, ax = r / FS_N, ii = r - ax * FS_N;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < c.n_atoms && ii < (ax == 0 ? c.n1 : c.n2)) {
      const int idx = (a * 3 + ax) * nm + ii;
      const float g = c.g1f[idx];
      const float2 p = ph[idx];
      v = make_float4(g * p.x, g * p.y, c.d1f[idx], 0.f);
    }
    sm.colt[i] = v;
    if (ax == 0) {
      float fr = v.x, fi = v.y;
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        sm.xpk[(a * FS_N + ii) * 3 + w] = make_float4(fr, fr, fi, fi);
        fr = __fmul_rn(v.z, fr);
        fi = __fmul_rn(v.z, fi);
      }
    }
  }
}

// complex product with explicit round-to-nearest operations (never contracted)
__device__ __forceinline__ float2 fs_cmul_rn(float2 a, float2 b) {
  return make_float2(__fsub_rn(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)),
                     __fadd_rn(__fmul_rn(a.x, b.y), __fmul_rn(a.y, b.x)));
}

// monomial index of d_x^i d_y^j d_z^k (i + j + k <= 2) in the order
// 000, 100, 010, 001, 200, 110, 101, 020, 011, 002
__device__ __forceinline__ int fs_mono(int i, int j, int k) {
  const int deg = i + j + k;
  if (deg == 0) return 0;
  if (deg == 1) return i ? 1 : (j ? 2 : 3);
  if (i == 2) return 4;
  if (i == 1) return j ? 5 : 6;
  if (j == 2) return 7;
  return j ? 8 : 9;
}

// z groups (atoms with identical z factor tables, see CellDev): with NZU =
// SEP_NA every atom is its own group; with NZU < SEP_NA the cell's groups
// (at most NZU of them) are used and every z contraction runs per group.
template <int NZU> __device__ __forceinline__ int fz_grp(const FsSmem& sm, int a) {
  if constexpr (NZU == SEP_NA) return a; else return sm.zg[a];
}
template <int NZU> __device__ __forceinline__ float4 fz_table(const FsSmem& sm, const CellDev& c, int g, int z) {
  if constexpr (NZU == SEP_NA) {
    return sm.zt[g * FS_N + z];
  } else {
    return g < c.n_zg ? sm.zt[sm.zrep[g] * FS_N + z] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ----------------------------------------------------------------------------
// ket: ubuf[z][col] = conj(V_NL t)(col, z) for the warp's 32 columns.  The z
// dependence is a GEMM over q = (z group, {F_z, d_z F_z}): column coefficient
// A[col][q] = sum over the group's atoms of F_y (G00 + d_y G10) or F_y G01.
// ----------------------------------------------------------------------------
template <int NZU>
__device__ __forceinline__ void fs_ket(FsSmem& sm, const CellDev& c, float2* vout, bool build_b) {
  constexpr int Q = 2 * NZU;   // complex columns of the GEMM
  constexpr int KS = Q / 4;    // k steps of 8 over the 2 Q real rows (Re rows, then Im rows)
  constexpr int NI = Q / 4;    // q values per thread: t4 + 4 i
  const int tid = threadIdx.x;
  // column tables G00, G10, G01 (conj W) and the B matrix B[k][n], k < 16: Re rows,
  // k >= 16: Im rows of q = (a, w); n = 2 z + c
  for (int i = tid; i < SEP_NA * FS_N; i += blockDim.x) {
    const int a = i / FS_N, ix = i - a * FS_N;
    const float4 fx = sm.colt[(2 * a) * FS_N + ix];
    const float2 F = make_float2(fx.x, fx.y);
    const float2 ws = sm.wt[4 * a], wx = sm.wt[4 * a + 1], wy = sm.wt[4 * a + 2], wz = sm.wt[4 * a + 3];
    const float2 q0 = make_float2(ws.x + fx.z * wx.x, -(ws.y + fx.z * wx.y));
    sm.gt[(a * 3 + 0) * FS_N + ix] = sep_cmul(F, q0);
    sm.gt[(a * 3 + 1) * FS_N + ix] = sep_cmul(F, make_float2(wy.x, -wy.y));
    sm.gt[(a * 3 + 2) * FS_N + ix] = sep_cmul(F, make_float2(wz.x, -wz.y));
  }
  for (int i = tid; build_b && i < 2 * Q * 2 * FS_N; i += blockDim.x) {
    const int k = i / (2 * FS_N), n = i - k * 2 * FS_N;
    const bool rrow = k < Q;
    const int q = rrow ? k : k - Q, z = n >> 1, cc = n & 1;
    const float4 f = fz_table<NZU>(sm, c, q >> 1, z);
    const float s = (q & 1) ? f.z : 1.f;
    const float zr = s * f.x, zi = s * f.y;
    const float v = rrow ? (cc ? zi : zr) : (cc ? zr : -zi);
    sm.bk[k * FS_BKP + n] = fs_split2(v);
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, g = lane >> 2, t4 = lane & 3;
  // A fragments of both m-tiles: rows = columns 32 warp + 16 mt + g (+8), k = 8 ks + t4 (+4)
  uint32_t ah[2][KS][4], al[2][KS][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int iyc = 2 * warp + mt;
    float re[2][NI], im[2][NI];   // [column A/B][q index i: q = t4 + 4 i]
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int q = t4 + 4 * i, gq = q >> 1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ixc = g + 8 * h;
        float2 v = make_float2(0.f, 0.f);
        auto add_atom = [&](int a) {
          const float4 fy = sm.colt[(2 * a + 1) * FS_N + iyc];
          const float2 F = make_float2(fy.x, fy.y);
          float2 w;
          if (q & 1) {
            w = sep_cmul(F, sm.gt[(a * 3 + 2) * FS_N + ixc]);
          } else {
            const float2 g0 = sm.gt[(a * 3 + 0) * FS_N + ixc], g1 = sm.gt[(a * 3 + 1) * FS_N + ixc];
            w = sep_cmul(F, make_float2(g0.x + fy.z * g1.x, g0.y + fy.z * g1.y));
          }
          v.x += w.x;
          v.y += w.y;
        };
        if constexpr (NZU == SEP_NA) {
          add_atom(gq);
        } else {
          const int cnt = sm.zcnt[gq];
#pragma unroll
          for (int j = 0; j < 2; ++j)
            if (j < cnt) add_atom(sm.zmem[gq][j]);
        }
        re[h][i] = v.x;
        im[h][i] = v.y;
      }
    }
    // the first KS/2 k steps: Re of q = t4 + 8 ks (+4); the others: Im
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const bool rpart = ks < KS / 2;
      const int i0 = 2 * (rpart ? ks : ks - KS / 2);
      const float(&src)[2][NI] = rpart ? re : im;
      fs_split(src[0][i0], ah[mt][ks][0], al[mt][ks][0]);
      fs_split(src[1][i0], ah[mt][ks][1], al[mt][ks][1]);
      fs_split(src[0][i0 + 1], ah[mt][ks][2], al[mt][ks][2]);
      fs_split(src[1][i0 + 1], ah[mt][ks][3], al[mt][ks][3]);
    }
  }
#pragma unroll
  for (int nt = 0; nt < (2 * FS_N) / 8; ++nt) {
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      const uint2 b0 = sm.bk[(8 * ks + t4) * FS_BKP + 8 * nt + g];
      const uint2 b1 = sm.bk[(8 * ks + t4 + 4) * FS_BKP + 8 * nt + g];
      fs_mma3(d[0], ah[0][ks], al[0][ks], b0, b1);
      fs_mma3(d[1], ah[1][ks], al[1][ks], b0, b1);
    }
    const int z = 4 * nt + t4;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int cA = 32 * warp + 16 * mt + g;
      vout[z * FS_PU + cA] = make_float2(d[mt][0], d[mt][1]);
      vout[z * FS_PU + cA + 8] = make_float2(d[mt][2], d[mt][3]);
    }
  }
}

// x and y contractions of a projection pass, from the z sums
// sbuf[q'][iy][ix ^ iy] of the pass's z weights q' = q0 .. q0 + NQ - 1 (read
// after a barrier): leaves mres[(a - a0) * NM + mono] and ends with a barrier.
template <int D, int NQ, int NAP, int NZU>
__device__ __forceinline__ void fs_xy_contract(FsSmem& sm, const CellDev& c, int q0, int a0, const float2* sbuf) {
  constexpr int NM = D == 1 ? 4 : 10;
  const int tid = threadIdx.x;
  // x contraction per row (q', iy): R_i = sum_ix F_x d_x^i S, i <= D - k; then the
  // y contraction M_a(i, j, k) = sum_iy F_y d_y^j R_i over the 16 lanes of the
  // half-warp that holds the rows iy = 0..15 of one q' (fixed-order shuffles).
  constexpr int NR = (D + 1) * NAP * FS_N;
  for (int r0 = 0; r0 < NR; r0 += FS_NP) {
    const int r = r0 + tid;
    const bool live = r < NR;
    const int ql = live ? (r >> 4) : 0, iyr = r & 15;
    const int al_ = ql / (D + 1), kz = ql - al_ * (D + 1), a = a0 + al_;
    const int sq = (D + 1) * fz_grp<NZU>(sm, a) + kz - q0;   // z sums of the atom's group
    // packed FP32x2 products: for w = 0..D - k, A_w accumulates d^w Re F_x (s_re, s_im)
    // and B_w d^w Im F_x (s_re, s_im); R_w = sum d^w F_x s = (A_w.x - B_w.y, A_w.y + B_w.x).
    // Every row runs every w of the pass (no divergence); the D = 1 and D = 2 passes
    // share the operations of w = 0, 1, so their common sums agree bit for bit.
    const float2 zero2 = make_float2(0.f, 0.f);
    float2 A0 = zero2, B0 = zero2, A1 = zero2, B1 = zero2, A2 = zero2, B2 = zero2;
    if (live) {
      const float4* xw = sm.xpk + a * FS_N * 3;
      const float2* sr = sbuf + sq * FS_NP + iyr * FS_N;
#pragma unroll 4
      for (int ixr = 0; ixr < FS_N; ++ixr) {
        const float2 sv = sr[ixr ^ iyr];
        const float4 p0 = xw[ixr * 3 + 0], p1 = xw[ixr * 3 + 1];
        A0 = __ffma2_rn(make_float2(p0.x, p0.y), sv, A0);
        B0 = __ffma2_rn(make_float2(p0.z, p0.w), sv, B0);
        A1 = __ffma2_rn(make_float2(p1.x, p1.y), sv, A1);
        B1 = __ffma2_rn(make_float2(p1.z, p1.w), sv, B1);
        if (D == 2) {
          const float4 p2 = xw[ixr * 3 + 2];
          A2 = __ffma2_rn(make_float2(p2.x, p2.y), sv, A2);
          B2 = __ffma2_rn(make_float2(p2.z, p2.w), sv, B2);
        }
      }
    }
    const float2 R0 = make_float2(__fsub_rn(A0.x, B0.y), __fadd_rn(A0.y, B0.x));
    const float2 R1 = make_float2(__fsub_rn(A1.x, B1.y), __fadd_rn(A1.y, B1.x));
    const float2 R2 = make_float2(__fsub_rn(A2.x, B2.y), __fadd_rn(A2.y, B2.x));
    // y weights of this row: F_y d_y^j
    const float4 fy = sm.colt[(2 * a + 1) * FS_N + iyr];
    const float2 Fy = make_float2(fy.x, fy.y), Fyd = make_float2(__fmul_rn(fy.z, fy.x), __fmul_rn(fy.z, fy.y));
    // contributions, in the order of the monomials this row feeds:
    //   D = 1, k = 0: 000 (F R0), 100 (F R1), 010 (F d R0);  k = 1: 001 (F R0)
    //   D = 2, k = 0: 000, 100, 010, 200 (F R2), 110 (F d R1), 020 (F d^2 R0)
    //          k = 1: 001, 101 (F R1), 011 (F d R0);  k = 2: 002
    constexpr int NC = D == 1 ? 3 : 6;
    float2 v[NC];
    v[0] = fs_cmul_rn(Fy, R0);
    v[1] = fs_cmul_rn(Fy, R1);
    v[2] = fs_cmul_rn(Fyd, R0);
    if (D == 2) {
      v[3 % NC] = fs_cmul_rn(Fy, R2);
      v[4 % NC] = fs_cmul_rn(Fyd, R1);
      v[5 % NC] = fs_cmul_rn(make_float2(__fmul_rn(fy.z, Fyd.x), __fmul_rn(fy.z, Fyd.y)), R0);
    }
#pragma unroll
    for (int off = 1; off < 16; off <<= 1)
#pragma unroll
      for (int e = 0; e < NC; ++e) {
        v[e].x = __fadd_rn(v[e].x, __shfl_xor_sync(0xffffffffu, v[e].x, off));
        v[e].y = __fadd_rn(v[e].y, __shfl_xor_sync(0xffffffffu, v[e].y, off));
      }
    if (live && iyr == 0) {
      float2* M = sm.mres + al_ * NM;
      if (D == 1) {
        if (kz == 0) {
          M[0] = v[0];
          M[1] = v[1];
          M[2] = v[2];
        } else {
          M[3] = v[0];
        }
      } else {
        if (kz == 0) {
          M[0] = v[0];
          M[1] = v[1];
          M[2] = v[2];
          M[4] = v[3 % NC];
          M[5] = v[4 % NC];
          M[7] = v[5 % NC];
        } else if (kz == 1) {
          M[3] = v[0];
          M[6] = v[1];
          M[8] = v[2];
        } else {
          M[9] = v[0];
        }
      }
    }
  }
  __syncthreads();
}


// ----------------------------------------------------------------------------
// Projection pass: monomial sums up to degree D of the atoms a0 .. a0 + NAP - 1,
// from the split A fragments of u (ah/al) and the tables zt / colt of the
// pass.  The z contraction covers the z weights q' = q0 .. q0 + NQ - 1 with
// q' = (D + 1) g + k (g the z group, k the power of d_z); the x and y
// contractions run per atom on the z sums of its group.  Leaves
// mres[(a - a0) * NM + mono] (NM = 4 for D = 1, 10 for D = 2).
// ----------------------------------------------------------------------------
template <int D, int NQ, int NAP, int NZU>
__device__ __forceinline__ void fs_project_pass(FsSmem& sm, const CellDev& c, int q0, int a0,
                                                const uint32_t (&ah)[2][4][4], const uint32_t (&al)[2][4][4],
                                                uint2* bz, float2* sbuf) {
  // bz: B_z (32 x (2 NQ + 4) uint2); sbuf: the z sums [q'][iy][ix ^ iy] (NQ x 256 float2)
  constexpr int NPR = 2 * NQ;          // real n of the pass
  constexpr int BZP = NPR + 4;         // B_z row pitch (uint2)
  constexpr int NM = D == 1 ? 4 : 10;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t4 = lane & 3;
  // B_z[k][n], k = 2 z + c (component of u), n = 2 q' + c' (component of S)
  for (int i = tid; i < 32 * NPR; i += blockDim.x) {
    const int k = i / NPR, n = i - k * NPR;
    const int z = k >> 1, cu = k & 1, qq = q0 + (n >> 1), cs = n & 1;
    const int gz = qq / (D + 1), kz = qq - gz * (D + 1);
    const float4 f = fz_table<NZU>(sm, c, gz, z);
    const float s = kz == 0 ? 1.f : (kz == 1 ? f.z : f.z * f.z);
    const float zr = s * f.x, zi = s * f.y;
    const float v = cs == 0 ? (cu == 0 ? zr : -zi) : (cu == 0 ? zi : zr);
    bz[k * BZP + n] = fs_split2(v);
  }
  __syncthreads();
  // z contraction on tensor cores: S[col][q'] for the warp's columns
#pragma unroll
  for (int nt = 0; nt < NPR / 8; ++nt) {
    float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const uint2 b0 = bz[(8 * ks + t4) * BZP + 8 * nt + g];
      const uint2 b1 = bz[(8 * ks + t4 + 4) * BZP + 8 * nt + g];
      fs_mma3(d[0], ah[0][ks], al[0][ks], b0, b1);
      fs_mma3(d[1], ah[1][ks], al[1][ks], b0, b1);
    }
    const int ql = 4 * nt + t4;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int iyc = 2 * warp + mt;
      sbuf[ql * FS_NP + iyc * FS_N + (g ^ iyc)] = make_float2(d[mt][0], d[mt][1]);
      sbuf[ql * FS_NP + iyc * FS_N + ((g + 8) ^ iyc)] = make_float2(d[mt][2], d[mt][3]);
    }
  }
  __syncthreads();
  fs_xy_contract<D, NQ, NAP, NZU>(sm, c, q0, a0, sbuf);
}

// A fragments (split) of u = ubuf[z][col] for the warp's columns, k = 2 z + c
__device__ __forceinline__ void fs_load_u(const float2* src, uint32_t (&ah)[2][4][4], uint32_t (&al)[2][4][4]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t4 = lane & 3;
  const float* ub = reinterpret_cast<const float*>(src);
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int cA = 32 * warp + 16 * mt + g;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int k0 = 8 * ks + t4, k1 = k0 + 4;
      const int z0 = k0 >> 1, c0 = k0 & 1, z1 = k1 >> 1, c1 = k1 & 1;
      fs_split(ub[2 * (z0 * FS_PU + cA) + c0], ah[mt][ks][0], al[mt][ks][0]);
      fs_split(ub[2 * (z0 * FS_PU + cA + 8) + c0], ah[mt][ks][1], al[mt][ks][1]);
      fs_split(ub[2 * (z1 * FS_PU + cA) + c1], ah[mt][ks][2], al[mt][ks][2]);
      fs_split(ub[2 * (z1 * FS_PU + cA + 8) + c1], ah[mt][ks][3], al[mt][ks][3]);
    }
  }
}

// ----------------------------------------------------------------------------
// The same z contractions on the fifth-generation tensor cores (tcgen05, NZU =
// 4): each thread writes the split row of its column (A operand, TF32 hi and
// lo) into tensor memory with tcgen05.st, the B operand (z factors, hi and
// lo) sits in shared memory in the canonical K-major layout, one thread
// issues the MMAs (M = 128 per half of the 256 columns, K = 8 per
// instruction, three products per K step), their completion arrives on an
// mbarrier (bounded wait), and each thread reads its row of the FP32
// accumulator back with tcgen05.ld.  Same three-product TF32 scheme as the
// mma.sync form; the accumulation order inside the tensor core differs, so
// the two forms agree to FP32 rounding, not bit for bit.
// Tensor-memory columns of a CTA (FU_COLS): ket A (hi, lo per half) and bra
// accumulator in [0, 64), ket accumulator in [64, 128), bra A in [128, 256).
// ----------------------------------------------------------------------------
#define FU_COLS 256u
#define FU_KET_A 0
#define FU_KET_D 64
#define FU_BRA_D 0
#define FU_BRA_A 128
#define FU_BZ_OFF 4096   // byte offset in FsSmem::bk of the stage 1-3 bra B_z (4 KiB after the ket B)

struct FuState {
  uint32_t tbase;   // tensor-memory base of the CTA
  uint32_t bar;     // shared address of FsSmem::mbar_mma
  uint32_t phase;   // parity of the next completion
};

// byte offset of element (row n, k) of a K-major operand with 128-byte core
// matrices: K-direction stride lbo = 128, 8-row groups sbo apart
__device__ __forceinline__ int fu_boff(int n, int k, int sbo) {
  return (n >> 3) * sbo + (k >> 2) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

// Wait for the last commit (bounded); true on every thread when it completed.
__device__ __forceinline__ bool fu_wait(FuState& u) {
  const bool ok = bk_mbar_wait(u.bar, u.phase, BK_WAIT_POLLS);
  u.phase ^= 1u;
  return __syncthreads_and(ok) != 0;
}

// Failure path after fu_wait returned false: record the timeout, give the
// MMAs in flight one more bounded wait, release the tensor memory.
__device__ __forceinline__ void fu_bail(const FuState& u, int* status) {
  if (threadIdx.x == 0) {
    atomicOr(status, BK_STATUS_TIMEOUT);
    bk_mbar_wait(u.bar, u.phase ^ 1u, BK_WAIT_POLLS);
  }
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) um_dealloc(u.tbase, FU_COLS);
}

// Allocation at the start of a kernel (after the CTA knows it has work) and
// release at its end; both are CTA-wide (barriers inside).
__device__ __forceinline__ FuState fu_open(FsSmem& sm) {
  if ((threadIdx.x >> 5) == 0) um_alloc(bk_smem(&sm.tslot), FU_COLS);
  if (threadIdx.x == 0) bk_mbar_init(bk_smem(&sm.mbar_mma), 1);
  um_fence_before();
  __syncthreads();
  um_fence_after();
  FuState u;
  u.tbase = sm.tslot;
  u.bar = bk_smem(&sm.mbar_mma);
  u.phase = 0;
  return u;
}

__device__ __forceinline__ void fu_close(const FuState& u) {
  um_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    um_fence_after();
    um_dealloc(u.tbase, FU_COLS);
  }
}

// ket on tcgen05: vout[z][col] = conj(V_NL t)(col, z) (see fs_ket).  The B
// matrix of z factors (K = 16: Re rows of q, then Im rows; N = 32: n = 2 z + c)
// is built when build_b, in sm.bk (hi at 0, lo at 2 KiB).
template <int NZU>
__device__ __forceinline__ bool fu_ket(FsSmem& sm, const CellDev& c, float2* vout, bool build_b, FuState& u) {
  static_assert(NZU == 4, "the tcgen05 ket covers 4 z groups (K = 16)");
  constexpr int Q = 2 * NZU;
  const int tid = threadIdx.x, warp = tid >> 5, col = tid, ix = col & (FS_N - 1), iy = col / FS_N;
  const int h = warp >> 2, qd = warp & 3;
  unsigned char* bkb = reinterpret_cast<unsigned char*>(sm.bk);
  for (int i = tid; i < SEP_NA * FS_N; i += blockDim.x) {
    const int a = i / FS_N, jx = i - a * FS_N;
    const float4 fx = sm.colt[(2 * a) * FS_N + jx];
    const float2 F = make_float2(fx.x, fx.y);
    const float2 ws = sm.wt[4 * a], wx = sm.wt[4 * a + 1], wy = sm.wt[4 * a + 2], wz = sm.wt[4 * a + 3];
    const float2 q0 = make_float2(ws.x + fx.z * wx.x, -(ws.y + fx.z * wx.y));
    sm.gt[(a * 3 + 0) * FS_N + jx] = sep_cmul(F, q0);
    sm.gt[(a * 3 + 1) * FS_N + jx] = sep_cmul(F, make_float2(wy.x, -wy.y));
    sm.gt[(a * 3 + 2) * FS_N + jx] = sep_cmul(F, make_float2(wz.x, -wz.y));
  }
  for (int i = tid; build_b && i < 2 * Q * 2 * FS_N; i += blockDim.x) {
    const int k = i / (2 * FS_N), n = i - k * 2 * FS_N;
    const bool rrow = k < Q;
    const int q = rrow ? k : k - Q, z = n >> 1, cc = n & 1;
    const float4 f = fz_table<NZU>(sm, c, q >> 1, z);
    const float sc = (q & 1) ? f.z : 1.f;
    const float zr = sc * f.x, zi = sc * f.y;
    const float v = rrow ? (cc ? zi : zr) : (cc ? zr : -zi);
    uint32_t hi, lo;
    fs_split(v, hi, lo);
    *reinterpret_cast<uint32_t*>(bkb + fu_boff(n, k, 512)) = hi;
    *reinterpret_cast<uint32_t*>(bkb + 2048 + fu_boff(n, k, 512)) = lo;
  }
  __syncthreads();
  // A row of this column: k < Q Re, k >= Q Im of A_q = sum over the group's
  // atoms of F_y (G00 + d_y G10) (q even) or F_y G01 (q odd); each atom's
  // tables are read once for both q of its group
  uint32_t ah[16], al[16];
  float2 av[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) av[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int gq = 0; gq < NZU; ++gq) {
    const int cnt = sm.zcnt[gq];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      if (j < cnt) {
        const int a = sm.zmem[gq][j];
        const float4 fy = sm.colt[(2 * a + 1) * FS_N + iy];
        const float2 F = make_float2(fy.x, fy.y);
        const float2 g0 = sm.gt[(a * 3 + 0) * FS_N + ix], g1 = sm.gt[(a * 3 + 1) * FS_N + ix];
        const float2 g2 = sm.gt[(a * 3 + 2) * FS_N + ix];
        const float2 we = sep_cmul(F, make_float2(g0.x + fy.z * g1.x, g0.y + fy.z * g1.y));
        const float2 wo = sep_cmul(F, g2);
        av[2 * gq].x += we.x;
        av[2 * gq].y += we.y;
        av[2 * gq + 1].x += wo.x;
        av[2 * gq + 1].y += wo.y;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    fs_split(av[q].x, ah[q], al[q]);
    fs_split(av[q].y, ah[Q + q], al[Q + q]);
  }
  um_st16(um_addr(u.tbase, qd, FU_KET_A + 32 * h), ah);
  um_st16(um_addr(u.tbase, qd, FU_KET_A + 32 * h + 16), al);
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  um_fence_before();
  __syncthreads();
  if (tid == 0) {
    um_fence_after();
    constexpr uint32_t idesc = um_idesc_tf32(128, 32);
    const uint32_t b0 = bk_smem(bkb), b1 = b0 + 2048;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const uint32_t d = u.tbase + FU_KET_D + 32 * hh;
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint32_t a_hi = u.tbase + FU_KET_A + 32 * hh + 8 * ks, a_lo = a_hi + 16;
        const uint64_t bh = um_sdesc(b0 + 256 * ks, 128, 512), bl = um_sdesc(b1 + 256 * ks, 128, 512);
        um_mma_tf32_ts(d, a_lo, bh, idesc, ks > 0);
        um_mma_tf32_ts(d, a_hi, bl, idesc, true);
        um_mma_tf32_ts(d, a_hi, bh, idesc, true);
      }
    }
    um_commit(u.bar);
  }
  if (!fu_wait(u)) return false;
  um_fence_after();
  float d[32];
  um_ld32(um_addr(u.tbase, qd, FU_KET_D + 32 * h), d);
#pragma unroll
  for (int z = 0; z < 16; ++z) vout[z * FS_PU + col] = make_float2(d[2 * z], d[2 * z + 1]);
  return true;
}

// The A operand of the projection passes: this thread's column of u = src[z][col]
// (k = 2 z + c, K = 32), split into TF32 hi and lo, into tensor memory.
__device__ __forceinline__ void fu_stage_u(const float2* src, const FuState& u) {
  const int col = threadIdx.x, warp = col >> 5, h = warp >> 2, qd = warp & 3;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int zz = 0; zz < 8; ++zz) {
      const float2 v = src[(8 * kk + zz) * FS_PU + col];
      fs_split(v.x, hi[2 * zz], lo[2 * zz]);
      fs_split(v.y, hi[2 * zz + 1], lo[2 * zz + 1]);
    }
    um_st16(um_addr(u.tbase, qd, FU_BRA_A + 64 * h + 16 * kk), hi);
    um_st16(um_addr(u.tbase, qd, FU_BRA_A + 64 * h + 32 + 16 * kk), lo);
  }
}

// Projection pass on tcgen05 (see fs_project_pass); the A operand was staged by
// fu_stage_u.  bz: NPAD/8 KiB of shared memory for B_z (hi, then lo); when
// build_b is false it already holds the B_z of the same z tables and pass.
template <int D, int NQ, int NAP, int NZU>
__device__ __forceinline__ bool fu_project_pass(FsSmem& sm, const CellDev& c, int q0, int a0, FuState& u,
                                                unsigned char* bz, float2* sbuf, bool build_b = true) {
  constexpr int NPR = 2 * NQ;                   // real n of the pass
  constexpr int NPAD = (NPR + 15) / 16 * 16;    // N of the MMA (M = 128 needs a multiple of 16)
  constexpr int LO = NPAD / 8 * 1024;           // byte offset of the lo part
  static_assert(NPAD <= 32, "one pass holds at most 16 complex z weights");
  const int tid = threadIdx.x, warp = tid >> 5, col = tid, ix = col & (FS_N - 1), iy = col / FS_N;
  const int h = warp >> 2, qd = warp & 3;
  // B_z^T[n][k], n = 2 q' + c' (component of S), k = 2 z + c (component of u)
  for (int i = tid; build_b && i < 32 * NPAD; i += blockDim.x) {
    const int n = i / 32, k = i - n * 32;
    float v = 0.f;
    if (n < NPR) {
      const int z = k >> 1, cu = k & 1, qq = q0 + (n >> 1), cs = n & 1;
      const int gz = qq / (D + 1), kz = qq - gz * (D + 1);
      const float4 f = fz_table<NZU>(sm, c, gz, z);
      const float sc = kz == 0 ? 1.f : (kz == 1 ? f.z : f.z * f.z);
      const float zr = sc * f.x, zi = sc * f.y;
      v = cs == 0 ? (cu == 0 ? zr : -zi) : (cu == 0 ? zi : zr);
    }
    uint32_t hi, lo;
    fs_split(v, hi, lo);
    *reinterpret_cast<uint32_t*>(bz + fu_boff(n, k, 1024)) = hi;
    *reinterpret_cast<uint32_t*>(bz + LO + fu_boff(n, k, 1024)) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  um_fence_before();
  __syncthreads();
  if (tid == 0) {
    um_fence_after();
    constexpr uint32_t idesc = um_idesc_tf32(128, NPAD);
    const uint32_t b0 = bk_smem(bz), b1 = b0 + LO;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const uint32_t d = u.tbase + FU_BRA_D + 32 * hh;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t a_hi = u.tbase + FU_BRA_A + 64 * hh + 8 * ks, a_lo = a_hi + 32;
        const uint64_t bh = um_sdesc(b0 + 256 * ks, 128, 1024), bl = um_sdesc(b1 + 256 * ks, 128, 1024);
        um_mma_tf32_ts(d, a_lo, bh, idesc, ks > 0);
        um_mma_tf32_ts(d, a_hi, bl, idesc, true);
        um_mma_tf32_ts(d, a_hi, bh, idesc, true);
      }
    }
    um_commit(u.bar);
  }
  if (!fu_wait(u)) return false;
  um_fence_after();
  if constexpr (NPAD > 16) {
    float d[32];
    um_ld32(um_addr(u.tbase, qd, FU_BRA_D + 32 * h), d);
#pragma unroll
    for (int ql = 0; ql < NQ; ++ql) sbuf[ql * FS_NP + iy * FS_N + (ix ^ iy)] = make_float2(d[2 * ql], d[2 * ql + 1]);
  } else {
    float d[16];
    um_ld16(um_addr(u.tbase, qd, FU_BRA_D + 32 * h), d);
#pragma unroll
    for (int ql = 0; ql < NQ; ++ql) sbuf[ql * FS_NP + iy * FS_N + (ix ^ iy)] = make_float2(d[2 * ql], d[2 * ql + 1]);
  }
  __syncthreads();
  fs_xy_contract<D, NQ, NAP, NZU>(sm, c, q0, a0, sbuf);
  return true;
}

// ----------------------------------------------------------------------------
// Pieces shared by the per-stage and the whole-step kernels.
// ----------------------------------------------------------------------------
// One band (16 planes of 256 complex values) into a buffer of plane pitch FS_PU.
__device__ __forceinline__ void fs_copy_band(float2* dst, const float2* src, uint32_t bar) {
#pragma unroll 1
  for (int z = 0; z < FS_N; ++z)
    bk_copy_g2s(bk_smem(dst + z * FS_PU), src + z * FS_NP, FS_NP * (uint32_t)sizeof(float2), bar);
}

// Factor tables of the unit (q of the step) and W = E P of the band.
__device__ __forceinline__ void fs_unit_tables(FsSmem& sm, const CellDev& c, const float2* ph, const float2* Pu) {
  fs_load_z(sm.zt, c, ph);
  fs_load_cols(sm, c, ph);
  for (int j = threadIdx.x; j < SEP_NP; j += blockDim.x) {
    float2 w = make_float2(0.f, 0.f);
    if (j < c.n_proj) {
      const float2 p = Pu[j];
      const float e = c.wkbf[j];
      w = make_float2(e * p.x, e * p.y);
    }
    sm.wt[j] = w;
  }
}

// z-march of Taylor stage m over the band held in `tin`: t_m = (-i dt/m) h t_{m-1}
// with h t = -1/2 lap t - i q.grad t + (|q|^2/2 + v_eff) t + V_NL t.  `vio`
// holds conj(V_NL t_{m-1}) per plane on entry and receives, column by column,
// t_m (m < 4) or psi(t_{n+1}) (m = 4).
//   STEP = false (one launch per stage): psi in global memory, `acc` holds the
//     psi column (m >= 2), t_m goes to tout (m < 4);
//   STEP = true (the whole step in one launch): psi accumulates in `acc`
//     (acc = t_0 + t_1 at m = 1) and is written once, at m = 4.
template <bool STEP>
__device__ __forceinline__ void fs_march(const FsSmem& sm, const CellDev& c, const float2* tin, float2* vio, int m,
                                         float hdt, float q0, float q1, float q2, float dg0, float2 (&acc)[FS_N],
                                         float2* __restrict__ tout, float2* __restrict__ psi, long long base) {
  constexpr int ND = ZM_ND, N = FS_N, NP = FS_NP;
  const int col = threadIdx.x, ix = col & (N - 1), iy = col / N;
  const float2 zero = make_float2(0.f, 0.f);
  const float2* cz = tin + col;
  const float2* xp[ND];
  const float2* xm[ND];
  const float2* yp[ND];
  const float2* ym[ND];
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) {
    xp[mm - 1] = tin + iy * N + ((ix + mm) & (N - 1));
    xm[mm - 1] = tin + iy * N + ((ix - mm) & (N - 1));
    yp[mm - 1] = tin + ((iy + mm) & (N - 1)) * N + ix;
    ym[mm - 1] = tin + ((iy - mm) & (N - 1)) * N + ix;
  }
  const float2 neg1 = make_float2(-1.f, -1.f);
  float2 qv[N + 2 * ND];
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) qv[k] = cz[((k - ND + N) & (N - 1)) * FS_PU];
#pragma unroll
  for (int z = 0; z < N; ++z) {
    qv[z + 2 * ND] = cz[((z + ND) & (N - 1)) * FS_PU];
    const float2 ce = qv[z + ND];
    const float dg = dg0 + sm.vbuf[z * NP + col];
    float2 h = __fmul2_rn(make_float2(dg, dg), ce);
    float2 gx = zero, gy = zero, gz = zero;
#pragma unroll
    for (int mm = 1; mm <= ND; ++mm) {
      const float2 xu = xp[mm - 1][z * FS_PU], xd = xm[mm - 1][z * FS_PU];
      const float2 yu = yp[mm - 1][z * FS_PU], yd = ym[mm - 1][z * FS_PU];
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
    const float2 vq = vio[z * FS_PU + col];   // conj(V_NL t)
    const float hr = h.x + qg.y + vq.x;
    const float hi = h.y - qg.x - vq.y;
    const float2 t = make_float2(hdt * hi, -hdt * hr);
    const long long idx = base + (long long)z * NP + col;
    float2 uo = t;
    if constexpr (STEP) {
      if (m == 1) {
        acc[z] = __fadd2_rn(ce, t);
      } else if (m < 4) {
        acc[z] = __fadd2_rn(acc[z], t);
      } else {
        uo = __fadd2_rn(acc[z], t);   // psi(t_{n+1})
        psi[idx] = uo;
      }
    } else {
      if (m < 4) tout[idx] = t;
      if (m == 2) {
        psi[idx] = __fadd2_rn(acc[z], __fadd2_rn(ce, t));
      } else if (m == 3) {
        psi[idx] = __fadd2_rn(acc[z], t);
      } else if (m == 4) {
        uo = __fadd2_rn(acc[z], t);   // psi(t_{n+1})
        psi[idx] = uo;
      }
    }
    vio[z * FS_PU + col] = uo;
  }
}

// P_j = dV pn_j M_j of a degree-1 pass (float, as stored in P).
__device__ __forceinline__ float2 fs_proj_value(const FsSmem& sm, const CellDev& c, int j) {
  const float2 M = sm.mres[(j >> 2) * 4 + (j & 3)];
  const double sc = c.dv * (double)c.pnormf[j];
  return make_float2((float)(sc * M.x), (float)(sc * M.y));
}

// Stage 4 after the march: projections of psi(t_{n+1}) (split fragments ah/al)
// for the next step (P, q of the next step) and for the current (Pa, q at
// t_{n+1}).  With a constant field both use the same q, and the first-order
// sums of the current's pass are those of the next step's (same z sums, rows
// and order).  bz / sbuf: scratch (B_z, z sums), both buffers free.
template <int NZU, bool UM>
__device__ __forceinline__ bool fs_stage4_projections(FsSmem& sm, const LaunchSet& L, const CellDev& c, int u,
                                                      const UnitDev& U, int b, float2* __restrict__ Pu,
                                                      float2* __restrict__ Pa, int same_next,
                                                      const uint32_t (&ah)[2][4][4], const uint32_t (&al)[2][4][4],
                                                      FuState& fu, uint2* bz, float2* sbuf) {
  const int tid = threadIdx.x;
  const float2* phn = (const float2*)L.ph_next + (long long)u * L.ph_stride;
  const float2* pho = (const float2*)L.ph_obs + (long long)u * L.ph_stride;
  if (!same_next) {
    fs_load_z(sm.zt, c, phn);
    fs_load_cols(sm, c, phn);
    __syncthreads();
    if constexpr (UM) {
      if (!fu_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, fu, reinterpret_cast<unsigned char*>(bz), sbuf))
        return false;
    } else {
      fs_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, ah, al, bz, sbuf);
    }
    if (tid < c.n_proj) Pu[tid] = fs_proj_value(sm, c, tid);
  }
  fs_load_z(sm.zt, c, pho);
  fs_load_cols(sm, c, pho);
  __syncthreads();
  float2* Pab = Pa + U.pa_off + 4LL * b * c.n_proj;
  // the second-order sums of every atom in one pass when the z groups halve
  // the z weights (12 of them), else in two passes of 4 atoms
  constexpr int NPASS = NZU == SEP_NA ? 2 : 1, NAP = SEP_NA / NPASS;
#pragma unroll 1
  for (int half = 0; half < NPASS; ++half) {
    if constexpr (UM) {
      if (!fu_project_pass<2, 3 * NZU / NPASS, NAP, NZU>(sm, c, half * (3 * NZU / NPASS), half * NAP, fu,
                                                         reinterpret_cast<unsigned char*>(bz), sbuf))
        return false;
    } else {
      fs_project_pass<2, 3 * NZU / NPASS, NAP, NZU>(sm, c, half * (3 * NZU / NPASS), half * NAP, ah, al, bz, sbuf);
    }
    // rows (a, c_x, c_y, c_z) of projector type t: monomials w_t and w_t + e_alpha
    const int o = tid;
    if (o < 4 * 4 * NAP) {
      const int al_ = o >> 4, t = (o >> 2) & 3, s = o & 3;
      const int a = half * NAP + al_;
      const int j = 4 * a + t;
      if (j < c.n_proj) {
        int e[3] = {t == 1 ? 1 : 0, t == 2 ? 1 : 0, t == 3 ? 1 : 0};
        if (s > 0) e[s - 1] += 1;
        const float2 M = sm.mres[al_ * 10 + fs_mono(e[0], e[1], e[2])];
        const double sc = c.dv * (double)c.pnormf[j];
        const float2 v = make_float2((float)(sc * M.x), (float)(sc * M.y));
        Pab[4 * j + s] = v;
        if (same_next && s == 0) Pu[j] = v;
      }
    }
    __syncthreads();
  }
  return true;
}

// ----------------------------------------------------------------------------
// Taylor stage m on a 16^3 grid, one CTA per (unit, band), one thread per
// (x, y) column; same arithmetic contract as k_stage_bulk: t_m, the psi
// accumulation, the projections of t_m (m < 4) or, at m = 4, those of
// psi(t_{n+1}) for the next step (P) and for the current (Pa).  The z
// contractions run on mma.sync.
// ----------------------------------------------------------------------------
template <int NZU>
__global__ void __launch_bounds__(FS_NP, 2) k_stage_fused(LaunchSet L, const float2* __restrict__ tin,
                                                          float2* __restrict__ tout, float2* __restrict__ psi,
                                                          float2* __restrict__ P, float2* __restrict__ Pa, int m,
                                                          int same_next) {
  constexpr int N = FS_N, NP = FS_NP;
  extern __shared__ __align__(128) unsigned char fs_raw[];
  FsSmem& sm = *reinterpret_cast<FsSmem*>(fs_raw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int tid = threadIdx.x, col = tid;
  const bool proj = c.use_proj != 0;
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  float2* Pu = P + U.p_off + (long long)b * c.n_proj;
  const long long base = U.psi_off + (long long)b * FS_NPTS;
  const float2 zero = make_float2(0.f, 0.f);
  const uint32_t bar = bk_smem(&sm.mbar);
  if (tid == 0) bk_mbar_init(bar, 1);
  fz_load<NZU>(sm, c);
  __syncthreads();
  if (tid == 0) {
    // the band of t_{m-1} and the sub-simulation's v_eff, on one barrier
    bk_mbar_expect_tx(bar, FS_NPTS * (uint32_t)(sizeof(float2) + sizeof(float)));
    fs_copy_band(sm.xb, tin + base, bar);
    bk_copy_g2s(bk_smem(sm.vbuf), S.veff, FS_NPTS * sizeof(float), bar);
  }
  // psi of the column in registers (m >= 2), in flight while the ket runs
  float2 pq[N];
#pragma unroll
  for (int z = 0; z < N; ++z) pq[z] = m >= 2 ? psi[base + z * NP + col] : zero;
  if (proj) fs_unit_tables(sm, c, ph, Pu);
  __syncthreads();
  if (proj) {
    fs_ket<NZU>(sm, c, sm.yb, true);
  } else {
#pragma unroll
    for (int z = 0; z < N; ++z) sm.yb[z * FS_PU + col] = zero;
  }
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const bool ok = bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
  if (!__syncthreads_and(ok)) {
    if (tid == 0) {
      atomicOr(S.status, BK_STATUS_TIMEOUT);
      bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
    }
    return;
  }
  fs_march<false>(sm, c, sm.xb, sm.yb, m, (float)(S.dt * L.dt_scale) / (float)m, qt[0], qt[1], qt[2], dg0, pq, tout, psi, base);
  if (!proj) return;
  __syncthreads();
  uint32_t ah[2][4][4], al[2][4][4];
  fs_load_u(sm.yb, ah, al);
  __syncthreads();   // both buffers free for the projection scratch
  uint2* bz = reinterpret_cast<uint2*>(sm.xb);
  if (m < 4) {
    fs_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, ah, al, bz, sm.yb);
    if (tid < c.n_proj) Pu[tid] = fs_proj_value(sm, c, tid);
    return;
  }
  FuState fu{};
  fs_stage4_projections<NZU, false>(sm, L, c, u, U, b, Pu, Pa, same_next, ah, al, fu, bz, sm.yb);
}

// ----------------------------------------------------------------------------
// The whole time step in one launch (cells whose atoms form z groups of at
// most two: NZU = 4), one CTA per (unit, band): the band of psi is brought in
// once, the four Taylor terms live in the two plane buffers (t_{m-1} in one,
// V_NL and then t_m in the other, roles swapping each stage), psi accumulates
// in registers, and each stage's projections go straight to the next stage's
// ket.  Memory traffic per step: psi read and written once, P and Pa.  Same
// arithmetic per stage as k_stage_fused; psi is summed as
// (((t_0 + t_1) + t_2) + t_3) + t_4.  UM: the z contractions on tcgen05, else
// on mma.sync.
// ----------------------------------------------------------------------------
template <int NZU, bool UM>
__global__ void __launch_bounds__(FS_NP, 2) k_step_fused(LaunchSet L, float2* __restrict__ psi,
                                                         float2* __restrict__ P, float2* __restrict__ Pa,
                                                         int same_next) {
  static_assert(NZU == 4, "the projection scratch of a stage fits one plane buffer only with z groups");
  constexpr int N = FS_N;
  extern __shared__ __align__(128) unsigned char fs_raw[];
  FsSmem& sm = *reinterpret_cast<FsSmem*>(fs_raw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int tid = threadIdx.x, col = tid;
  const bool proj = c.use_proj != 0;
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  float2* Pu = P + U.p_off + (long long)b * c.n_proj;
  const long long base = U.psi_off + (long long)b * FS_NPTS;
  const uint32_t bar = bk_smem(&sm.mbar);
  FuState fu{};
  if constexpr (UM) {
    if (proj) fu = fu_open(sm);
  }
  if (tid == 0) bk_mbar_init(bar, 1);
  fz_load<NZU>(sm, c);
  __syncthreads();
  if (tid == 0) {
    bk_mbar_expect_tx(bar, FS_NPTS * (uint32_t)(sizeof(float2) + sizeof(float)));
    fs_copy_band(sm.xb, psi + base, bar);
    bk_copy_g2s(bk_smem(sm.vbuf), S.veff, FS_NPTS * sizeof(float), bar);
  }
  if (proj) fs_unit_tables(sm, c, ph, Pu);
  __syncthreads();
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  float2 acc[N];
  uint32_t ah[2][4][4], al[2][4][4];
  float2* tin = sm.xb;
  float2* vio = sm.yb;
  bool waited = false;
#pragma unroll 1
  for (int m = 1; m <= 4; ++m) {
    bool mma_ok = true;
    if (proj) {
      if constexpr (UM) {
        mma_ok = fu_ket<NZU>(sm, c, vio, m == 1, fu);   // the z-table B matrix once per step
      } else {
        fs_ket<NZU>(sm, c, vio, m == 1);
      }
    } else {
#pragma unroll
      for (int z = 0; z < N; ++z) vio[z * FS_PU + col] = make_float2(0.f, 0.f);
    }
    if (!waited) {
      const bool ok = bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
      if (!__syncthreads_and(ok)) {
        if (tid == 0) {
          atomicOr(S.status, BK_STATUS_TIMEOUT);
          bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
        }
        if constexpr (UM) {
          if (proj) {
            if (mma_ok) fu_close(fu); else fu_bail(fu, S.status);
          }
        }
        return;
      }
      waited = true;
    } else {
      __syncthreads();
    }
    if constexpr (UM) {
      if (!mma_ok) {
        fu_bail(fu, S.status);
        return;
      }
    }
    fs_march<true>(sm, c, tin, vio, m, (float)(S.dt * L.dt_scale) / (float)m, q0, q1, q2, dg0, acc, nullptr, psi, base);
    __syncthreads();
    if (!proj) {
      float2* t = tin;
      tin = vio;
      vio = t;
      continue;
    }
    if constexpr (UM) {
      fu_stage_u(vio, fu);
    } else {
      fs_load_u(vio, ah, al);
    }
    if (m < 4) {
      // projections of t_m for the next stage; scratch in the buffer of t_{m-1}
      if constexpr (UM) {
        // the B_z of stages 1-3 (same z tables) is built once per step, beside the ket B
        if (!fu_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, fu,
                                                      reinterpret_cast<unsigned char*>(sm.bk) + FU_BZ_OFF, tin,
                                                      m == 1)) {
          fu_bail(fu, S.status);
          return;
        }
      } else {
        fs_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, ah, al,
                                                 reinterpret_cast<uint2*>(tin + 2 * NZU * FS_NP), tin);
      }
      if (tid < SEP_NP) {
        float2 w = make_float2(0.f, 0.f);
        if (tid < c.n_proj) {
          const float2 p = fs_proj_value(sm, c, tid);
          const float e = c.wkbf[tid];
          w = make_float2(e * p.x, e * p.y);
        }
        sm.wt[tid] = w;
      }
      __syncthreads();
      float2* t = tin;
      tin = vio;
      vio = t;
    } else {
      __syncthreads();   // both buffers free for the projection scratch
      if (!fs_stage4_projections<NZU, UM>(sm, L, c, u, U, b, Pu, Pa, same_next, ah, al, fu,
                                          reinterpret_cast<uint2*>(tin), vio)) {
        fu_bail(fu, S.status);
        return;
      }
    }
  }
  if constexpr (UM) {
    if (proj) fu_close(fu);
  }
}

// ----------------------------------------------------------------------------
// Projections P[u][b][j] of float orbitals on a 16^3 grid (q_half tables),
// one CTA per (unit, band): the same tensor-core pass as the fused stage, so
// the projections of a restored state equal those the stage leaves, bit for
// bit (UM selects the tcgen05 or the mma.sync form, as the stage kernels do).
// ----------------------------------------------------------------------------
template <int NZU, bool UM>
__global__ void __launch_bounds__(FS_NP, 2) k_bra_fused(LaunchSet L, const float2* __restrict__ src,
                                                        float2* __restrict__ P) {
  static_assert(!UM || NZU == 4, "the tcgen05 contractions cover grouped cells");
  extern __shared__ __align__(128) unsigned char fs_raw[];
  FsSmem& sm = *reinterpret_cast<FsSmem*>(fs_raw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int tid = threadIdx.x;
  FuState fu{};
  if constexpr (UM) fu = fu_open(sm);
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  const float2* sb = src + U.psi_off + (long long)b * FS_NPTS + tid;
  fz_load<NZU>(sm, c);
#pragma unroll
  for (int z = 0; z < FS_N; ++z) sm.yb[z * FS_PU + tid] = sb[z * FS_NP];
  fs_load_z(sm.zt, c, ph);
  fs_load_cols(sm, c, ph);
  __syncthreads();
  if constexpr (UM) {
    fu_stage_u(sm.yb, fu);
    if (!fu_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, fu, reinterpret_cast<unsigned char*>(sm.xb), sm.yb)) {
      fu_bail(fu, L.subs[U.sub].status);
      return;
    }
  } else {
    uint32_t ah[2][4][4], al[2][4][4];
    fs_load_u(sm.yb, ah, al);
    __syncthreads();
    fs_project_pass<1, 2 * NZU, SEP_NA, NZU>(sm, c, 0, 0, ah, al, reinterpret_cast<uint2*>(sm.xb), sm.yb);
  }
  if (tid < c.n_proj) P[U.p_off + (long long)b * c.n_proj + tid] = fs_proj_value(sm, c, tid);
  if constexpr (UM) fu_close(fu);
}

// ----------------------------------------------------------------------------
// Projections of the current, Pa[u][b][j][alpha] = <beta~_j|u>, <d_alpha beta~_j|u>
// on the q_obs tables, one CTA per (unit, band): the second-order pass of the
// whole-step kernel's stage 4 (monomials of degree <= 2), for the evaluations
// of J outside a step (J(0-), J(0+), a restored state).
// ----------------------------------------------------------------------------
template <int NZU, bool UM>
__global__ void __launch_bounds__(FS_NP, 2) k_pa_fused(LaunchSet L, const float2* __restrict__ src,
                                                       float2* __restrict__ Pa) {
  static_assert(!UM || NZU == 4, "the tcgen05 contractions cover grouped cells");
  extern __shared__ __align__(128) unsigned char fs_raw[];
  FsSmem& sm = *reinterpret_cast<FsSmem*>(fs_raw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int tid = threadIdx.x;
  FuState fu{};
  if constexpr (UM) fu = fu_open(sm);
  const float2* ph = (const float2*)L.ph_obs + (long long)u * L.ph_stride;
  const float2* sb = src + U.psi_off + (long long)b * FS_NPTS + tid;
  fz_load<NZU>(sm, c);
#pragma unroll
  for (int z = 0; z < FS_N; ++z) sm.yb[z * FS_PU + tid] = sb[z * FS_NP];
  fs_load_z(sm.zt, c, ph);
  fs_load_cols(sm, c, ph);
  __syncthreads();
  uint32_t ah[2][4][4], al[2][4][4];
  if constexpr (UM) {
    fu_stage_u(sm.yb, fu);
  } else {
    fs_load_u(sm.yb, ah, al);
    __syncthreads();   // yb becomes the z-sum scratch
  }
  float2* Pab = Pa + U.pa_off + 4LL * b * c.n_proj;
  constexpr int NPASS = NZU == SEP_NA ? 2 : 1, NAP = SEP_NA / NPASS;
#pragma unroll 1
  for (int half = 0; half < NPASS; ++half) {
    if constexpr (UM) {
      if (!fu_project_pass<2, 3 * NZU / NPASS, NAP, NZU>(sm, c, half * (3 * NZU / NPASS), half * NAP, fu,
                                                         reinterpret_cast<unsigned char*>(sm.xb), sm.yb)) {
        fu_bail(fu, L.subs[U.sub].status);
        return;
      }
    } else {
      fs_project_pass<2, 3 * NZU / NPASS, NAP, NZU>(sm, c, half * (3 * NZU / NPASS), half * NAP, ah, al,
                                                    reinterpret_cast<uint2*>(sm.xb), sm.yb);
    }
    // rows (a, c_x, c_y, c_z) of projector type t: monomials w_t and w_t + e_alpha
    const int o = tid;
    if (o < 4 * 4 * NAP) {
      const int al_ = o >> 4, t = (o >> 2) & 3, sa = o & 3;
      const int a = half * NAP + al_;
      const int j = 4 * a + t;
      if (j < c.n_proj) {
        int e[3] = {t == 1 ? 1 : 0, t == 2 ? 1 : 0, t == 3 ? 1 : 0};
        if (sa > 0) e[sa - 1] += 1;
        const float2 M = sm.mres[al_ * 10 + fs_mono(e[0], e[1], e[2])];
        const double sc = c.dv * (double)c.pnormf[j];
        Pab[4 * j + sa] = make_float2((float)(sc * M.x), (float)(sc * M.y));
      }
    }
    __syncthreads();
  }
  if constexpr (UM) fu_close(fu);
}

// ----------------------------------------------------------------------------
// Observation pass on 16^3 grids: one CTA per unit, bands in turn through a
// ring of FO_SLOTS band buffers filled by bulk copies.  A slot's "full"
// mbarrier completes when its band has landed, its "empty" mbarrier when all
// warps are done with it; thread 0 refills a slot once it is empty, so warps
// never meet at a CTA barrier between bands.
// Per column and plane it accumulates occ sum_b |u|^2 (rho; over bands as an
// unevaluated float pair s + e updated by the error-free two-sum, which keeps
// the sum to about 2^-44 relative, i.e. FP64-grade, without FP64 arithmetic),
// per thread sum Re(u* (-i grad u)) (FP32 within a band; over bands again as a
// two-sum float pair, so that GB300's narrow FP64 pipe is left alone) and
// per band sum |u|^2 (per-warp partials, added over warps in order at the
// end).  The unit's sums go to point tile 0 of the partial buffers and zeros to
// the other tiles.
// ----------------------------------------------------------------------------
#define FO_SLOTS 3
#define FO_MAXB 128   // bands of the per-warp norm table

struct FoSmem {
  float2 buf[FO_SLOTS][FS_NPTS];
  float nrm[8][FO_MAXB];
  double redj[8][3];
  unsigned long long full[FO_SLOTS];
  unsigned long long empty[FO_SLOTS];
  int fail;
};

// One arrival of the calling thread on a shared-memory mbarrier.
__device__ __forceinline__ void fo_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(FS_NP, 2) k_observe_fused(LaunchSet L, const float2* __restrict__ psi,
                                                            double* __restrict__ rho_part,
                                                            double* __restrict__ jk_part,
                                                            double* __restrict__ nrm_part) {
  constexpr int ND = ZM_ND, N = FS_N, NP = FS_NP;
  extern __shared__ __align__(128) unsigned char fo_raw[];
  FoSmem& sm = *reinterpret_cast<FoSmem*>(fo_raw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int tid = threadIdx.x, col = tid, lane = tid & 31, warp = tid >> 5;
  const int n_warps = (int)(blockDim.x >> 5);
  const int ix = col & (N - 1), iy = col / N;
  const int nb = c.n_bands;
  const float2* src = psi + U.psi_off;
  volatile int* fail = &sm.fail;
  if (tid == 0) {
    for (int k = 0; k < FO_SLOTS; ++k) {
      bk_mbar_init(bk_smem(&sm.full[k]), 1);
      bk_mbar_init(bk_smem(&sm.empty[k]), (uint32_t)n_warps);
    }
    *fail = 0;
  }
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < FO_SLOTS && k < nb; ++k) {
      bk_mbar_expect_tx(bk_smem(&sm.full[k]), FS_NPTS * (uint32_t)sizeof(float2));
      bk_copy_g2s(bk_smem(sm.buf[k]), src + (long long)k * FS_NPTS, FS_NPTS * sizeof(float2), bk_smem(&sm.full[k]));
    }
  float rho[N], rho_e[N];
#pragma unroll
  for (int z = 0; z < N; ++z) rho[z] = rho_e[z] = 0.f;
  float js[3] = {0.f, 0.f, 0.f}, je[3] = {0.f, 0.f, 0.f};   // current over bands: js + je per axis
  int issued = nb < FO_SLOTS ? nb : FO_SLOTS;   // bands whose copy thread 0 has issued
  for (int b = 0; b < nb; ++b) {
    if (*fail) break;
    const int slot = b % FO_SLOTS;
    const uint32_t parity = (uint32_t)((b / FO_SLOTS) & 1);
    if (!bk_mbar_wait(bk_smem(&sm.full[slot]), parity, BK_WAIT_POLLS)) {
      *fail = 1;
      break;
    }
    const float2* tb = sm.buf[slot];
    const float2* cz = tb + col;
    // the current's local part in correlation form: on the periodic grid
    // sum_r Re(u* (-i grad_ax) u) = 2 sum_m w_m Im sum_r u*(r) u(r + m e_ax),
    // which needs the forward neighbours only
    float2 qv[N + ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) qv[k] = cz[k * NP];
    float nbs = 0.f;
    float cx[ND], cy[ND], czs[ND];
#pragma unroll
    for (int mm = 0; mm < ND; ++mm) cx[mm] = cy[mm] = czs[mm] = 0.f;
#pragma unroll
    for (int z = 0; z < N; ++z) {
      qv[z + ND] = cz[((z + ND) & (N - 1)) * NP];
      const float2 ce = qv[z];
#pragma unroll
      for (int mm = 1; mm <= ND; ++mm) {
        const float2 xu = tb[z * NP + iy * N + ((ix + mm) & (N - 1))];
        const float2 yu = tb[z * NP + ((iy + mm) & (N - 1)) * N + ix];
        const float2 zu = qv[z + mm];
        // Im(conj(u) v) = u_r v_i - u_i v_r
        cx[mm - 1] = __fmaf_rn(ce.x, xu.y, __fmaf_rn(-ce.y, xu.x, cx[mm - 1]));
        cy[mm - 1] = __fmaf_rn(ce.x, yu.y, __fmaf_rn(-ce.y, yu.x, cy[mm - 1]));
        czs[mm - 1] = __fmaf_rn(ce.x, zu.y, __fmaf_rn(-ce.y, zu.x, czs[mm - 1]));
      }
      const float n2v = ce.x * ce.x + ce.y * ce.y;
      {
        // two-sum: rho + n2v = t + err exactly
        const float t = rho[z] + n2v, bb = t - rho[z];
        rho_e[z] += (rho[z] - (t - bb)) + (n2v - bb);
        rho[z] = t;
      }
      nbs += n2v;
    }
    float bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int mm = 1; mm <= ND; ++mm) {
      bx = __fmaf_rn(2.f * c.gradwf[0][mm], cx[mm - 1], bx);
      by = __fmaf_rn(2.f * c.gradwf[1][mm], cy[mm - 1], by);
      bz = __fmaf_rn(2.f * c.gradwf[2][mm], czs[mm - 1], bz);
    }
    {
      const float bv[3] = {bx, by, bz};
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const float t = js[ax] + bv[ax], bb = t - js[ax];
        je[ax] += (js[ax] - (t - bb)) + (bv[ax] - bb);
        js[ax] = t;
      }
    }
    for (int off = 16; off > 0; off >>= 1) nbs += __shfl_xor_sync(0xffffffffu, nbs, off);
    if (lane == 0) {
      sm.nrm[warp][b] = nbs;
      fo_arrive(bk_smem(&sm.empty[slot]));   // the warp is done with this slot (reads ordered by the shuffles)
    }
    if (tid == 0 && b + FO_SLOTS < nb) {
      // refill the slot with band b + FO_SLOTS once every warp is done with it
      if (!bk_mbar_wait(bk_smem(&sm.empty[slot]), parity, BK_WAIT_POLLS)) {
        *fail = 1;
        break;
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      bk_mbar_expect_tx(bk_smem(&sm.full[slot]), FS_NPTS * (uint32_t)sizeof(float2));
      bk_copy_g2s(bk_smem(sm.buf[slot]), src + (long long)(b + FO_SLOTS) * FS_NPTS, FS_NPTS * sizeof(float2),
                  bk_smem(&sm.full[slot]));
      issued = b + FO_SLOTS + 1;
    }
  }
  if (__syncthreads_or(*fail)) {
    if (tid == 0) {
      atomicOr(S.status, BK_STATUS_TIMEOUT);
      // let every issued copy land before the CTA's shared memory is released
      for (int k = (issued > FO_SLOTS ? issued - FO_SLOTS : 0); k < issued; ++k)
        bk_mbar_wait(bk_smem(&sm.full[k % FO_SLOTS]), (uint32_t)((k / FO_SLOTS) & 1), BK_WAIT_POLLS);
    }
    return;
  }
#pragma unroll
  for (int z = 0; z < N; ++z) rho_part[U.rho_off + (long long)z * NP + col] = c.occ * ((double)rho[z] + (double)rho_e[z]);
  double jx = (double)js[0] + (double)je[0], jy = (double)js[1] + (double)je[1], jz = (double)js[2] + (double)je[2];
  for (int off = 16; off > 0; off >>= 1) {
    jx += __shfl_xor_sync(0xffffffffu, jx, off);
    jy += __shfl_xor_sync(0xffffffffu, jy, off);
    jz += __shfl_xor_sync(0xffffffffu, jz, off);
  }
  if (lane == 0) {
    sm.redj[warp][0] = jx;
    sm.redj[warp][1] = jy;
    sm.redj[warp][2] = jz;
  }
  __syncthreads();
  if (tid < 3) {
    double sum = 0.0;
    for (int w = 0; w < n_warps; ++w) sum += sm.redj[w][tid];
    jk_part[U.jk_off + tid] = sum;
  }
  for (int b = tid; b < nb; b += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < n_warps; ++w) sum += (double)sm.nrm[w][b];
    nrm_part[U.nrm_off + b] = sum;
  }
  for (int i = tid; i < 3 * (c.n_tiles - 1); i += blockDim.x) jk_part[U.jk_off + 3 + i] = 0.0;
  for (int i = tid; i < c.n_bands * (c.n_tiles - 1); i += blockDim.x) nrm_part[U.nrm_off + c.n_bands + i] = 0.0;
}
