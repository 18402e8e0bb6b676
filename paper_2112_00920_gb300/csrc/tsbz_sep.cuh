// Single-precision Taylor stage with the projector contractions folded in,
// for cells whose projectors are one s and three p Gaussians per atom.
//
// Every projector factorises over the three axes (minimum-image
// displacements and the Gaussian are per-axis, and so is the phase of
// beta~ = beta exp(-i q.d)):
//   C_{a,t}(r) = conj(beta~_{a,t}(r)) = pn_{a,t} F^a_x(ix) F^a_y(iy) F^a_z(iz) w_t(r),
//   F^a_ax(i) = g^a_ax(i) exp(+i q_ax d^a_ax(i)),  w_s = 1,  w_{p_alpha} = d^a_alpha.
// With one thread per (x, y) column marching in z, both contractions become
// per-column sums over z against per-plane factors that all threads share:
//   bra   P_{a,t} = dV pn_{a,t} sum_{ix,iy} F_x F_y w_t^{xy} sum_z F_z w_t^z t(r)
//         (per column S_a = sum_z F_z t, S'_a = sum_z d_z F_z t; one reduction per CTA)
//   ket   V(r) = sum_{a,t} conj(C_{a,t}(r)) E_{a,t} P_{a,t}, i.e.
//         conj(V(r)) = sum_a F_z(iz) K_a + d_z F_z(iz) L_a,
//         K_a = F_x F_y conj(W_s + d_x W_px + d_y W_py),  L_a = F_x F_y conj(W_pz),
//         W_{a,t} = pn_{a,t} E_{a,t} P_{a,t}.
// The stage kernel applies h = h_loc + V_NL to t_{m-1}, writes t_m and the
// psi accumulation, and (m < 4) the projections of t_m for the next stage,
// so the non-local term costs no extra pass over the orbitals.
#pragma once
#include <cuda_runtime.h>

#include "tsbz_bulk.cuh"
#include "tsbz_internal.h"
#include "tsbz_zmarch.cuh"

#define SEP_NA 8                // atoms per cell in this path
#define SEP_NP (4 * SEP_NA)     // projectors
#define SEP_CPITCH 64           // column-table pitch of the runtime-shape kernels (n1, n2 <= 64)
// Dynamic shared memory of k_stage_bulk<N> for stage m: the band of t_{m-1}
// (and of psi for m >= 2); stage 4 reuses it for the next-step and current
// tables (72 N float4) and 20 SEP_NA doubles of reduction results.
__host__ __device__ constexpr size_t sep_bulk_smem(int N, int m) {
  return (m >= 2 ? 2 : 1) * (size_t)N * N * N * 8 > (m == 4 ? (size_t)72 * N * 16 + 20 * SEP_NA * 8 : 0)
             ? (m >= 2 ? 2 : 1) * (size_t)N * N * N * 8
             : (size_t)72 * N * 16 + 20 * SEP_NA * 8;
}
#ifndef SEP_BULK_MINB
#define SEP_BULK_MINB 2         // resident CTAs per SM the 16^3 bulk-staged stage is compiled for
#endif

// A complex factor F is kept as (Re F, Re F, Im F, Im F), so that with b and
// brot = (-Im b, Re b) the product F b is two packed FMAs and needs no moves.
__device__ __forceinline__ float4 sep_bcast(float fr, float fi) { return make_float4(fr, fr, fi, fi); }

__device__ __forceinline__ float2 sep_rot(float2 b) { return make_float2(-b.y, b.x); }

// acc + F b
__device__ __forceinline__ float2 sep_cmac(float4 f, float2 b, float2 brot, float2 acc) {
  acc = __ffma2_rn(make_float2(f.x, f.y), b, acc);
  return __ffma2_rn(make_float2(f.z, f.w), brot, acc);
}

__device__ __forceinline__ float2 sep_cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Per-plane factors of the unit: fzt[(w SEP_NA + a) NZ + z] = d_z^w F^a_z(z) in the (Re, Re, Im, Im) form.
template <int NZ, int NW>
__device__ __forceinline__ void sep_load_z(float4* fzt, const CellDev& c, const float2* ph) {
  const int nm = c.nmax;
  for (int i = threadIdx.x; i < SEP_NA * NZ; i += blockDim.x) {
    const int a = i / NZ, z = i - a * NZ;
    float fr = 0.f, fi = 0.f, d = 0.f;
    if (a < c.n_atoms) {
      const int idx = (a * 3 + 2) * nm + z;
      const float g = c.g1f[idx];
      const float2 p = ph[idx];
      fr = g * p.x;
      fi = g * p.y;
      d = c.d1f[idx];
    }
    fzt[i] = sep_bcast(fr, fi);
    fzt[SEP_NA * NZ + i] = sep_bcast(d * fr, d * fi);
    if (NW > 2) fzt[2 * SEP_NA * NZ + i] = sep_bcast(d * d * fr, d * d * fi);
  }
}

// Column factors of atom a: H = F_x(ix) F_y(iy), d_x(ix), d_y(iy) (zero when inactive).
__device__ __forceinline__ void sep_column(const CellDev& c, const float2* ph, int ix, int iy, bool act, int a,
                                           float2& H, float& dx, float& dy) {
  H = make_float2(0.f, 0.f);
  dx = 0.f;
  dy = 0.f;
  if (act && a < c.n_atoms) {
    const int nm = c.nmax;
    const int ixx = (a * 3) * nm + ix, iyy = (a * 3 + 1) * nm + iy;
    const float gx = c.g1f[ixx], gy = c.g1f[iyy];
    const float2 px = ph[ixx], py = ph[iyy];
    H = sep_cmul(make_float2(gx * px.x, gx * px.y), make_float2(gy * py.x, gy * py.y));
    dx = c.d1f[ixx];
    dy = c.d1f[iyy];
  }
}

// Column tables of the unit in shared memory: colt[(a 2 + ax) PITCH + i] =
// (Re F^a_ax(i), Im F^a_ax(i), d^a_ax(i), 0) for ax = x, y and i < PITCH
// (PITCH >= n1, n2; zero beyond the edge).
template <int PITCH>
__device__ __forceinline__ void sep_load_cols(float4* colt, const CellDev& c, const float2* ph) {
  const int nm = c.nmax;
  for (int i = threadIdx.x; i < SEP_NA * 2 * PITCH; i += blockDim.x) {
    const int a = i / (2 * PITCH), r = i - a * 2 * PITCH, ax = r / PITCH, ii = r - ax * PITCH;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a < c.n_atoms && ii < (ax == 0 ? c.n1 : c.n2)) {
      const int idx = (a * 3 + ax) * nm + ii;
      const float g = c.g1f[idx];
      const float2 p = ph[idx];
      v = make_float4(g * p.x, g * p.y, c.d1f[idx], 0.f);
    }
    colt[i] = v;
  }
}

// Column tables source: global tables (any grid) or the shared copy above.
struct SepColG {
  const CellDev& c;
  const float2* ph;
  __device__ __forceinline__ void operator()(int ix, int iy, bool act, int a, float2& H, float& dx, float& dy) const {
    sep_column(c, ph, ix, iy, act, a, H, dx, dy);
  }
};
template <int PITCH>
struct SepColS {
  const float4* colt;
  __device__ __forceinline__ void operator()(int ix, int iy, bool, int a, float2& H, float& dx, float& dy) const {
    const float4 fx = colt[(2 * a) * PITCH + ix], fy = colt[(2 * a + 1) * PITCH + iy];
    H = sep_cmul(make_float2(fx.x, fx.y), make_float2(fy.x, fy.y));
    dx = fx.z;
    dy = fy.z;
  }
};

// Non-local term of every plane of one column: vq[z] = conj(V_NL t)(ix, iy, z)
// = sum_a F_z K_a + d_z F_z L_a with K_a = H_a conj(W_s + d_x W_px + d_y W_py),
// L_a = H_a conj(W_pz), H_a = F_x(ix) F_y(iy); wt[j] = pn_j E_j P_j.
template <int NZ, typename Col>
__device__ __forceinline__ void sep_ket_column(const CellDev& c, const Col& colf, const float4* fzt,
                                               const float2* wt, int ix, int iy, bool act, bool proj,
                                               float2 (&vq)[NZ]) {
#pragma unroll
  for (int z = 0; z < NZ; ++z) vq[z] = make_float2(0.f, 0.f);
  if (!proj) return;
  for (int a = 0; a < c.n_atoms; ++a) {
    float2 H;
    float dx, dy;
    colf(ix, iy, act, a, H, dx, dy);
    const float2 ws = wt[4 * a], wx = wt[4 * a + 1], wy = wt[4 * a + 2], wz = wt[4 * a + 3];
    const float2 Q = make_float2(ws.x + dx * wx.x + dy * wy.x, ws.y + dx * wx.y + dy * wy.y);
    // K = H conj(Q), Lz = H conj(W_pz)
    const float2 K = make_float2(H.x * Q.x + H.y * Q.y, H.y * Q.x - H.x * Q.y);
    const float2 Lz = make_float2(H.x * wz.x + H.y * wz.y, H.y * wz.x - H.x * wz.y);
    const float2 Kr = sep_rot(K), Lr = sep_rot(Lz);
    const float4* fa = fzt + a * NZ;
    const float4* fda = fzt + (SEP_NA + a) * NZ;
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      vq[z] = sep_cmac(fa[z], K, Kr, vq[z]);
      vq[z] = sep_cmac(fda[z], Lz, Lr, vq[z]);
    }
  }
}

// Warp reduce-scatter: after the call lane l holds in v[i] (i < NV / 32) the
// warp sum of entry sep_rs_base(l, NV) + i.  Fixed order (deterministic).
template <int NV, int H>
__device__ __forceinline__ void sep_rs_level(float (&v)[NV], int lane, int off) {
  const bool up = (lane & off) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const float send = up ? v[i] : v[H + i];
    const float keep = up ? v[H + i] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
  }
}

template <int NV>
__device__ __forceinline__ void sep_reduce_scatter(float (&v)[NV], int lane) {
  static_assert(NV % 32 == 0, "reduce-scatter needs a multiple of 32 entries");
  sep_rs_level<NV, NV / 2>(v, lane, 16);
  sep_rs_level<NV, NV / 4>(v, lane, 8);
  sep_rs_level<NV, NV / 8>(v, lane, 4);
  sep_rs_level<NV, NV / 16>(v, lane, 2);
  sep_rs_level<NV, NV / 32>(v, lane, 1);
}

__device__ __forceinline__ int sep_rs_base(int lane, int nv) {
  return ((lane >> 4) & 1) * (nv / 2) + ((lane >> 3) & 1) * (nv / 4) + ((lane >> 2) & 1) * (nv / 8) +
         ((lane >> 1) & 1) * (nv / 16) + (lane & 1) * (nv / 32);
}

// Projections of one (unit, band) from the column values tq[z] = t(ix, iy, z):
// per atom S = sum_z F_z t, S' = sum_z d_z F_z t, weighted by the column
// factors and reduced over the CTA -> Pout[j] = dV pn_j sum (warps added in
// order in double).  red: [8][2 SEP_NP] floats.
template <int NZ, typename Col>
__device__ __forceinline__ void sep_write_p(const CellDev& c, const Col& colf, const float4* fzt, int ix, int iy,
                                            bool act, const float2 (&tq)[NZ], float (*red)[2 * SEP_NP],
                                            float2* __restrict__ Pout) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 S[SEP_NA], Sd[SEP_NA];
#pragma unroll
  for (int a = 0; a < SEP_NA; ++a) S[a] = Sd[a] = make_float2(0.f, 0.f);
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    const float2 t = tq[z], tr = sep_rot(tq[z]);
#pragma unroll
    for (int a = 0; a < SEP_NA; ++a) {
      S[a] = sep_cmac(fzt[a * NZ + z], t, tr, S[a]);
      Sd[a] = sep_cmac(fzt[(SEP_NA + a) * NZ + z], t, tr, Sd[a]);
    }
  }
  // two halves of four atoms (32 entries each) keep the register footprint small
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    float v[32];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int a = 4 * half + k;
      float2 H;
      float dx, dy;
      colf(ix, iy, act, a, H, dx, dy);
      const float2 hs = sep_cmul(H, S[a]), hd = sep_cmul(H, Sd[a]);
      v[8 * k + 0] = hs.x;
      v[8 * k + 1] = hs.y;
      v[8 * k + 2] = dx * hs.x;
      v[8 * k + 3] = dx * hs.y;
      v[8 * k + 4] = dy * hs.x;
      v[8 * k + 5] = dy * hs.y;
      v[8 * k + 6] = hd.x;
      v[8 * k + 7] = hd.y;
    }
    sep_reduce_scatter<32>(v, lane);
    red[warp][32 * half + sep_rs_base(lane, 32)] = v[0];
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < c.n_proj) {
    double re = 0.0, im = 0.0;
    const int nw = (int)(blockDim.x >> 5);
    for (int w = 0; w < nw; ++w) {
      re += (double)red[w][2 * j];
      im += (double)red[w][2 * j + 1];
    }
    const double sc = c.dv * (double)c.pnormf[j];
    Pout[j] = make_float2((float)(sc * re), (float)(sc * im));
  }
}

// Projections for the current of one (unit, band) from the column values
// tq[z] = u(ix, iy, z): Pa[4 j + 0] = <beta~_j|u>, Pa[4 j + alpha] = <d_alpha beta~_j|u>.
// Column sums U_w = sum_z d_z^w F_z u (w = 0, 1, 2) and the ten distinct column
// weights per atom r0..r5 = {1, d_x, d_y, d_x^2, d_x d_y, d_y^2} H U_0,
// r6..r8 = {1, d_x, d_y} H U_1, r9 = H U_2 give a_s = r0, a_px = r1, a_py = r2,
// a_pz = r6 and c_s = (r1, r2, r6), c_px = (r3, r4, r7), c_py = (r4, r5, r8),
// c_pz = (r7, r8, r9).  fzt holds the three plane tables (w = 0, 1, 2);
// red: [8][2 SEP_NP] floats, res: 20 SEP_NA doubles (shared).
template <int NZ, typename Col>
__device__ __forceinline__ void sep_write_pa(const CellDev& c, const Col& colf, const float4* fzt, int ix, int iy,
                                             bool act, const float2 (&tq)[NZ], float (*red)[2 * SEP_NP],
                                             double* res, float2* __restrict__ Pa) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 A0[SEP_NA], A1[SEP_NA], A2[SEP_NA];
#pragma unroll
  for (int a = 0; a < SEP_NA; ++a) A0[a] = A1[a] = A2[a] = make_float2(0.f, 0.f);
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    const float2 t = tq[z], tr = sep_rot(tq[z]);
#pragma unroll
    for (int a = 0; a < SEP_NA; ++a) {
      A0[a] = sep_cmac(fzt[a * NZ + z], t, tr, A0[a]);
      A1[a] = sep_cmac(fzt[(SEP_NA + a) * NZ + z], t, tr, A1[a]);
      A2[a] = sep_cmac(fzt[(2 * SEP_NA + a) * NZ + z], t, tr, A2[a]);
    }
  }
  float dxa[SEP_NA], dya[SEP_NA];
#pragma unroll
  for (int a = 0; a < SEP_NA; ++a) {
    float2 H;
    colf(ix, iy, act, a, H, dxa[a], dya[a]);
    if (!act) H = make_float2(0.f, 0.f);
    A0[a] = sep_cmul(H, A0[a]);
    A1[a] = sep_cmul(H, A1[a]);
    A2[a] = sep_cmul(H, A2[a]);
  }
  // 80 complex column values in 5 passes of 16
#pragma unroll
  for (int pass = 0; pass < 5; ++pass) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = 16 * pass + i, a = q / 10, r = q % 10;
      const float dx = dxa[a], dy = dya[a];
      float2 w;
      switch (r) {
        case 0: w = A0[a]; break;
        case 1: w = make_float2(dx * A0[a].x, dx * A0[a].y); break;
        case 2: w = make_float2(dy * A0[a].x, dy * A0[a].y); break;
        case 3: w = make_float2(dx * dx * A0[a].x, dx * dx * A0[a].y); break;
        case 4: w = make_float2(dx * dy * A0[a].x, dx * dy * A0[a].y); break;
        case 5: w = make_float2(dy * dy * A0[a].x, dy * dy * A0[a].y); break;
        case 6: w = A1[a]; break;
        case 7: w = make_float2(dx * A1[a].x, dx * A1[a].y); break;
        case 8: w = make_float2(dy * A1[a].x, dy * A1[a].y); break;
        default: w = A2[a]; break;
      }
      v[2 * i] = w.x;
      v[2 * i + 1] = w.y;
    }
    sep_reduce_scatter<32>(v, lane);
    red[warp][sep_rs_base(lane, 32)] = v[0];
    __syncthreads();
    if (threadIdx.x < 32) {
      double s = 0.0;
      const int nw = (int)(blockDim.x >> 5);
      for (int w = 0; w < nw; ++w) s += (double)red[w][threadIdx.x];
      res[32 * pass + threadIdx.x] = s;
    }
    __syncthreads();
  }
  const int j = threadIdx.x;
  if (j < c.n_proj) {
    const int a = j >> 2, t = j & 3;
    // (a, c_x, c_y, c_z) rows of projector type t, one nibble each
    const unsigned rows = t == 0 ? 0x6210u : (t == 1 ? 0x7431u : (t == 2 ? 0x8542u : 0x9876u));
    const double sc = c.dv * (double)c.pnormf[j];
    float2* dst = Pa + 4LL * j;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int q = 10 * a + (int)((rows >> (4 * s)) & 15u);
      dst[s] = make_float2((float)(sc * res[2 * q]), (float)(sc * res[2 * q + 1]));
    }
  }
}

// ----------------------------------------------------------------------------
// Taylor stage m (1..4) on a depth-NZ grid, one CTA per (unit, band), one
// thread per (x, y) column (n1 n2 <= 256), blockIdx.x = unit index * n_bands + band.
//   t_m = (-i dt/m)[h_loc t_{m-1} + V_NL t_{m-1}],  V_NL from P[u][b] (projections
//   of t_{m-1});  m = 2: psi += t_1 + t_2;  m >= 3: psi += t_m;  m < 4: P[u][b] <-
//   projections of t_m (in place: each CTA reads its own entry before it writes).
// ----------------------------------------------------------------------------
template <int NZ>
__global__ void __launch_bounds__(256, 2) k_stage_sep(LaunchSet L, const float2* __restrict__ tin,
                                                      float2* __restrict__ tout, float2* __restrict__ psi,
                                                      float2* __restrict__ P, int m) {
  constexpr int ND = ZM_ND;
  extern __shared__ __align__(128) unsigned char sraw[];
  float2* plane = reinterpret_cast<float2*>(sraw);
  __shared__ float4 fzt[2 * SEP_NA * NZ];
  __shared__ float2 wt[SEP_NP];
  __shared__ float red[8][2 * SEP_NP];
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int n1 = c.n1, n2 = c.n2, n12 = n1 * n2;
  const int col = threadIdx.x;
  const bool act = col < n12;
  const int ix = act ? col % n1 : 0, iy = act ? col / n1 : 0;
  const bool proj = c.use_proj != 0;
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  float2* Pu = P + U.p_off + (long long)b * c.n_proj;
  const float2 zero = make_float2(0.f, 0.f);
  if (proj) {
    sep_load_z<NZ, 2>(fzt, c, ph);
    for (int j = threadIdx.x; j < SEP_NP; j += blockDim.x) {
      float2 w = zero;
      if (j < c.n_proj) {
        const float2 p = Pu[j];
        const float e = c.wkbf[j];
        w = make_float2(e * p.x, e * p.y);
      }
      wt[j] = w;
    }
  }
  __syncthreads();
  // non-local term of every plane of the column: vq[z] = conj(V_NL t_{m-1})(ix, iy, z)
  float2 vq[NZ];
  const SepColG colg{c, ph};
  sep_ket_column<NZ>(c, colg, fzt, wt, ix, iy, act, proj, vq);
  const int W = n1 + 2 * ND;
  const float2* me = plane + (iy + ND) * W + ix + ND;
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const float hdt = (float)(S.dt * L.dt_scale) / (float)m;
  const float* veff = reinterpret_cast<const float*>(S.veff);
  const long long base0 = U.psi_off + (long long)b * c.npts + col;
  const float2* tb = tin + base0;
  const float2 neg1 = make_float2(-1.f, -1.f);
  const bool bra = proj && m < 4;
  float2 tq[NZ];   // t_m of the column, for the projections after the march
  float2 qv[NZ + 2 * ND];   // t(z) for z = -ND .. NZ - 1 + ND (periodic)
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) qv[k] = act ? tb[(long long)((k - ND + NZ) % NZ) * n12] : zero;
  float2 p_cur = (act && m >= 2) ? psi[base0] : zero;
  float e_cur = act ? veff[col] : 0.f;
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    qv[z + 2 * ND] = act ? tb[(long long)((z + ND) % NZ) * n12] : zero;
    float2 p_nxt = zero;
    float e_nxt = 0.f;
    if (act && z + 1 < NZ) {
      if (m >= 2) p_nxt = psi[base0 + (long long)(z + 1) * n12];
      e_nxt = veff[(z + 1) * n12 + col];
    }
    __syncthreads();
    if (act) zpad_store(plane, n1, n2, ix, iy, qv[z + ND]);
    __syncthreads();
    float2 t = zero;
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
      float2 qg = __fmul2_rn(make_float2(q0, q0), gx);
      qg = f2fma(make_float2(q1, q1), gy, qg);
      qg = f2fma(make_float2(q2, q2), gz, qg);
      // h t = h_loc t - i q.grad t + V_NL t, V_NL t = conj(vq)
      const float hr = h.x + qg.y + vq[z].x;
      const float hi = h.y - qg.x - vq[z].y;
      t = make_float2(hdt * hi, -hdt * hr);
      if (m < 4) tout[idx] = t;
      if (m == 2) {
        psi[idx] = __fadd2_rn(p_cur, __fadd2_rn(ce, t));
      } else if (m >= 3) {
        psi[idx] = __fadd2_rn(p_cur, t);
      }
    }
    tq[z] = t;
    p_cur = p_nxt;
    e_cur = e_nxt;
  }
  if (bra) sep_write_p<NZ>(c, colg, fzt, ix, iy, act, tq, red, Pu);
}

// ----------------------------------------------------------------------------
// Projections of float orbitals on a depth-NZ grid, one CTA per (unit, band).
//   WD = 0: P[u][b][j] = <beta~_j|src_b>            (q_half, or q_obs if use_obs)
//   WD = 1: Pa[u][b][j][0..3] = <beta~_j|u>, <d_alpha beta~_j|u>   (for the current)
// With WD the column sums are U_w = sum_z d_z^w F_z u (w = 0, 1, 2) and the ten
// distinct column weights per atom are
//   r0..r5 = {1, d_x, d_y, d_x^2, d_x d_y, d_y^2} H U_0,  r6..r8 = {1, d_x, d_y} H U_1,  r9 = H U_2,
// from which a_s = r0, a_px = r1, a_py = r2, a_pz = r6 and
//   c_s = (r1, r2, r6), c_px = (r3, r4, r7), c_py = (r4, r5, r8), c_pz = (r7, r8, r9).
// ----------------------------------------------------------------------------
template <int NZ, int WD>
__global__ void __launch_bounds__(256) k_bra_sep(LaunchSet L, const float2* __restrict__ src,
                                                 float2* __restrict__ out, int use_obs) {
  constexpr int NW = WD ? 3 : 2;
  __shared__ float4 fzt[NW * SEP_NA * NZ];
  __shared__ float4 colt[SEP_NA * 2 * SEP_CPITCH];
  __shared__ float red[8][2 * SEP_NP];
  __shared__ double res[WD ? 2 * 10 * SEP_NA : 1];
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int n1 = c.n1, n12 = n1 * c.n2;
  const int col = threadIdx.x;
  const bool act = col < n12;
  const int ix = act ? col % n1 : 0, iy = act ? col / n1 : 0;
  const float2* ph = (const float2*)(use_obs ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride;
  const float2 zero = make_float2(0.f, 0.f);
  sep_load_z<NZ, NW>(fzt, c, ph);
  sep_load_cols<SEP_CPITCH>(colt, c, ph);
  const SepColS<SEP_CPITCH> cols{colt};
  const float2* tb = src + U.psi_off + (long long)b * c.npts + col;
  float2 tv[NZ];
#pragma unroll
  for (int z = 0; z < NZ; ++z) tv[z] = act ? tb[(long long)z * n12] : zero;
  __syncthreads();
  if (!WD) {
    sep_write_p<NZ>(c, cols, fzt, ix, iy, act, tv, red, out + U.p_off + (long long)b * c.n_proj);
    return;
  }
  sep_write_pa<NZ>(c, cols, fzt, ix, iy, act, tv, red, res, out + U.pa_off + 4LL * b * c.n_proj);
}

// ----------------------------------------------------------------------------
// Taylor stage m on a cubic N^3 grid (N = 8 or 16), one CTA per (unit, band),
// one thread per (x, y) column.  The band of t_{m-1} (and of psi for m >= 2)
// is brought into shared memory with one bulk copy each (N^3 x 8 bytes,
// completed on an mbarrier) while the CTA builds the non-local term of its
// column; the z-march then reads every stencil neighbour from shared memory
// at a per-thread address plus a compile-time plane offset, with no barrier
// per plane.  Same arithmetic and outputs as k_stage_sep; in addition stage 4
// leaves in P the projections of psi(t_{n+1}) for the next step (phase tables
// ph_next) and in Pa those of the current at t_{n+1} (ph_obs), so a step reads
// the orbitals once per stage and once for rho and the local current.
// ----------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(N * N, (N == 16 ? SEP_BULK_MINB : 8))
    k_stage_bulk(LaunchSet L, const float2* __restrict__ tin, float2* __restrict__ tout, float2* __restrict__ psi,
                 float2* __restrict__ P, float2* __restrict__ Pa, int m) {
  constexpr int ND = ZM_ND, NP = N * N, NPTS = N * N * N;
  static_assert((N & (N - 1)) == 0 && N > ND, "N must be a power of two above the stencil half-width");
  extern __shared__ __align__(128) unsigned char sraw[];
  float2* tbuf = reinterpret_cast<float2*>(sraw);
  float2* pbuf = tbuf + NPTS;
  __shared__ float4 fzt[2 * SEP_NA * N];
  __shared__ float4 colt[SEP_NA * 2 * N];
  __shared__ float2 wt[SEP_NP];
  __shared__ float red[8][2 * SEP_NP];
  __shared__ __align__(8) unsigned long long mbar;
  const CellDev& c = L.cell;
  const int b = blockIdx.x % c.n_bands;
  const int u = L.unit_ids[blockIdx.x / c.n_bands];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int col = threadIdx.x;
  const int ix = col & (N - 1), iy = col / N;
  const bool proj = c.use_proj != 0;
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  float2* Pu = P + U.p_off + (long long)b * c.n_proj;
  const long long base = U.psi_off + (long long)b * NPTS;
  const uint32_t bar = bk_smem(&mbar);
  if (threadIdx.x == 0) bk_mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    bk_mbar_expect_tx(bar, (uint32_t)(NPTS * sizeof(float2)) * (m >= 2 ? 2u : 1u));
    bk_copy_g2s(bk_smem(tbuf), tin + base, NPTS * sizeof(float2), bar);
    if (m >= 2) bk_copy_g2s(bk_smem(pbuf), psi + base, NPTS * sizeof(float2), bar);
  }
  // tables and the non-local term while the copies are in flight
  if (proj) {
    sep_load_z<N, 2>(fzt, c, ph);
    sep_load_cols<N>(colt, c, ph);
    for (int j = threadIdx.x; j < SEP_NP; j += blockDim.x) {
      float2 w = make_float2(0.f, 0.f);
      if (j < c.n_proj) {
        const float2 p = Pu[j];
        const float e = c.wkbf[j];
        w = make_float2(e * p.x, e * p.y);
      }
      wt[j] = w;
    }
  }
  __syncthreads();
  float2 vq[N];
  const SepColS<N> cols{colt};
  sep_ket_column<N>(c, cols, fzt, wt, ix, iy, true, proj, vq);
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const float hdt = (float)(S.dt * L.dt_scale) / (float)m;
  const float* veff = reinterpret_cast<const float*>(S.veff) + col;
  float e_cur = veff[0];
  const bool ok = bk_mbar_wait(bar, 0, BK_WAIT_POLLS);
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) {
      atomicOr(S.status, BK_STATUS_TIMEOUT);
      bk_mbar_wait(bar, 0, BK_WAIT_POLLS);   // let copies in flight land before the CTA exits
    }
    return;
  }
  // neighbour columns of plane 0 (periodic in x and y)
  const float2* cz = tbuf + col;
  const float2* xp[ND];
  const float2* xm[ND];
  const float2* yp[ND];
  const float2* ym[ND];
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) {
    xp[mm - 1] = tbuf + iy * N + ((ix + mm) & (N - 1));
    xm[mm - 1] = tbuf + iy * N + ((ix - mm) & (N - 1));
    yp[mm - 1] = tbuf + ((iy + mm) & (N - 1)) * N + ix;
    ym[mm - 1] = tbuf + ((iy - mm) & (N - 1)) * N + ix;
  }
  const float2 zero = make_float2(0.f, 0.f);
  const float2 neg1 = make_float2(-1.f, -1.f);
  const bool bra = proj && m < 4;
  float2 tq[N];
  float2 qv[N + 2 * ND];   // t(z) for z = -ND .. N - 1 + ND (periodic)
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) qv[k] = cz[((k - ND + N) & (N - 1)) * NP];
#pragma unroll
  for (int z = 0; z < N; ++z) {
    qv[z + 2 * ND] = cz[((z + ND) & (N - 1)) * NP];
    const float e_nxt = (z + 1 < N) ? veff[(z + 1) * NP] : 0.f;
    const float2 ce = qv[z + ND];
    const float dg = dg0 + e_cur;
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
    const float hr = h.x + qg.y + vq[z].x;
    const float hi = h.y - qg.x - vq[z].y;
    const float2 t = make_float2(hdt * hi, -hdt * hr);
    const long long idx = base + (long long)z * NP + col;
    if (m < 4) tout[idx] = t;
    if (m == 2) {
      psi[idx] = __fadd2_rn(pbuf[z * NP + col], __fadd2_rn(ce, t));
      tq[z] = t;
    } else if (m == 3) {
      psi[idx] = __fadd2_rn(pbuf[z * NP + col], t);
      tq[z] = t;
    } else if (m == 4) {
      tq[z] = __fadd2_rn(pbuf[z * NP + col], t);   // psi(t_{n+1})
      psi[idx] = tq[z];
    } else {
      tq[z] = t;
    }
    e_cur = e_nxt;
  }
  if (bra) sep_write_p<N>(c, cols, fzt, ix, iy, true, tq, red, Pu);
  if (m == 4 && proj) {
    // psi(t_{n+1}) of the column is in tq: its projections for the next step
    // (q = k + A(t_{n+1} + dt/2)) and those of the current at t_{n+1}
    // (q = k + A(t_{n+1})), with the tables staged where the band was.
    __syncthreads();
    float4* fz_next = reinterpret_cast<float4*>(sraw);
    float4* col_next = fz_next + 2 * SEP_NA * N;
    float4* fz_obs = col_next + SEP_NA * 2 * N;
    float4* col_obs = fz_obs + 3 * SEP_NA * N;
    double* res = reinterpret_cast<double*>(col_obs + SEP_NA * 2 * N);
    const float2* phn = (const float2*)L.ph_next + (long long)u * L.ph_stride;
    const float2* pho = (const float2*)L.ph_obs + (long long)u * L.ph_stride;
    sep_load_z<N, 2>(fz_next, c, phn);
    sep_load_cols<N>(col_next, c, phn);
    sep_load_z<N, 3>(fz_obs, c, pho);
    sep_load_cols<N>(col_obs, c, pho);
    __syncthreads();
    sep_write_p<N>(c, SepColS<N>{col_next}, fz_next, ix, iy, true, tq, red, Pu);
    __syncthreads();
    sep_write_pa<N>(c, SepColS<N>{col_obs}, fz_obs, ix, iy, true, tq, red, res,
                    Pa + U.pa_off + 4LL * b * c.n_proj);
  }
}
