// CUDA kernels of the propagation step, templated on the real type T of
// the orbital arithmetic (double or float).  Density, current and v_Hxc
// are accumulated in double in both cases.
//
// One time step n -> n+1 of every sub-simulation (Eq. 1 with Eq. 2's h):
//   field   : q_half = k + A(t_n + dt/2), q_obs = k + A(t_{n+1}) and the
//             per-axis projector phase tables exp(i q_ax d_ax)
//   4 stages m = 1..4 of the Taylor recurrence t_m = (-i dt/m) h t_{m-1}:
//     bra   : P_jb = dV sum_r conj(beta~_j(r)) t_b(r)        (projector contraction)
//     stage : t_m = (-i dt/m)[-1/2 lap t - i q.grad t + (q^2/2 + v_eff) t
//                              + sum_j E_j beta~_j P_jb]; psi accumulates sum_m t_m
//   observe : Pa = <beta~_j|u>, <d_a beta~_j|u> at q_obs; per-tile sums of
//             occ |u|^2 (Eq. 3), Re(u* (-i grad) u) and |u_b|^2
//   finalize: per sub-simulation rho (Eq. 3), norms and
//             J = -(1/(Omega N_k)) sum occ <u|pi|u> (Eqs. 5-6) in a fixed order
//   hxc     : v_H = F^-1[4 pi rho(G)/G^2] (G = 0 dropped) + PZ81 v_xc; v_eff = v_loc + v_Hxc
// with beta~_j(r) = beta_j(d) exp(-i q.d), beta separable per axis:
//   beta = pnorm * g_x g_y g_z * {1, d_x, d_y, d_z},  exp(i q.d) = prod_ax exp(i q_ax d_ax).
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include "tsbz_internal.h"

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

template <typename V> __device__ __forceinline__ V cmk(decltype(V().x) a, decltype(V().x) b) { V r; r.x = a; r.y = b; return r; }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V, typename R> __device__ __forceinline__ V cscale(V a, R s) { return cmk<V>(a.x * s, a.y * s); }
// acc += a * b
template <typename V> __device__ __forceinline__ void cfma(V& acc, V a, V b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += s * b (s real)
template <typename V, typename R> __device__ __forceinline__ void rfma(V& acc, R s, V b) {
  acc.x = fma(s, b.x, acc.x);
  acc.y = fma(s, b.y, acc.y);
}

__device__ __forceinline__ int wrap_idx(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Cell tables in the arithmetic type of the kernel (float copies for the
// single-precision path keep double operations out of its inner loops).
template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ const double* g1(const CellDev& c) { return c.g1; }
  static __device__ __forceinline__ const double* d1(const CellDev& c) { return c.d1; }
  static __device__ __forceinline__ const double* pnorm(const CellDev& c) { return c.pnorm; }
  static __device__ __forceinline__ const double* wkb(const CellDev& c) { return c.wkb; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ const float* g1(const CellDev& c) { return c.g1f; }
  static __device__ __forceinline__ const float* d1(const CellDev& c) { return c.d1f; }
  static __device__ __forceinline__ const float* pnorm(const CellDev& c) { return c.pnormf; }
  static __device__ __forceinline__ const float* wkb(const CellDev& c) { return c.wkbf; }
};

// ----------------------------------------------------------------------------
// field: q vectors and phase tables of every unit (k-point) of one cell
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_field(LaunchSet L, int mode) {
  using V = typename Cplx<T>::type;
  const int u = L.unit_ids[blockIdx.x];
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const CellDev& c = L.cell;
  // step budget: a sub-simulation that has done max_steps steps sits out the
  // step (every later kernel of the step reads the flag); the evaluations of
  // J(0-), J(0+) and of a restored state take part whatever the step count
  const bool step_mode = mode == TSBZ_FIELD_STEP || mode == TSBZ_FIELD_STEP_KEEP || mode == TSBZ_FIELD_AT_NOW ||
                         mode == TSBZ_FIELD_AT_NEXT;
  const bool act = !step_mode || *S.step < S.max_steps;
  if (U.kloc == 0 && threadIdx.x == 0) *S.active = act ? 1 : 0;
  if (!act) return;
  double ah[3] = {0.0, 0.0, 0.0}, ao[3] = {0.0, 0.0, 0.0};
  if (step_mode) {
    const int step = *S.step;
    const int jh = 2 * step + (mode == TSBZ_FIELD_AT_NOW ? 0 : (mode == TSBZ_FIELD_AT_NEXT ? 2 : 1));
    const int jo = 2 * step + 2;
    if (jo < S.n_field) {
      for (int ax = 0; ax < 3; ++ax) {
        ah[ax] = S.A[3 * jh + ax];
        ao[ax] = S.A[3 * jo + ax];
      }
    }
  } else if (mode == TSBZ_FIELD_J0PLUS) {
    for (int ax = 0; ax < 3; ++ax) ao[ax] = S.A[ax];
  }
  double qh[3], qo[3];
  for (int ax = 0; ax < 3; ++ax) {
    qh[ax] = L.kcart[3 * u + ax] + ah[ax];
    qo[ax] = L.kcart[3 * u + ax] + ao[ax];
  }
  if (threadIdx.x < 3) {
    L.q_half[3 * u + threadIdx.x] = qh[threadIdx.x];
    L.q_obs[3 * u + threadIdx.x] = qo[threadIdx.x];
    reinterpret_cast<T*>(L.qt_half)[4 * u + threadIdx.x] = (T)qh[threadIdx.x];
  }
  if (threadIdx.x == 3)
    reinterpret_cast<T*>(L.qt_half)[4 * u + 3] = (T)(0.5 * (qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2]));
  // constant field: q and every phase table equal those of the previous step
  if (mode == TSBZ_FIELD_STEP_KEEP) return;
  V* phh = (V*)L.ph_half + (long long)u * L.ph_stride;
  V* pho = (V*)L.ph_obs + (long long)u * L.ph_stride;
  const int tab = c.n_atoms * 3 * c.nmax;
  for (int i = threadIdx.x; i < tab; i += blockDim.x) {
    const int ax = (i / c.nmax) % 3;
    const double d = c.d1[i];
    double s, co;
    sincos(qh[ax] * d, &s, &co);
    phh[i] = cmk<V>((T)co, (T)s);
    sincos(qo[ax] * d, &s, &co);
    pho[i] = cmk<V>((T)co, (T)s);
  }
  if (L.ph_next != nullptr && mode == TSBZ_FIELD_STEP) {
    // q_half of step n + 1, evaluated exactly as that step's field launch will
    const int step = *S.step;
    const int jh = 2 * step + 3, jo = 2 * step + 4;
    double qn[3];
    for (int ax = 0; ax < 3; ++ax) qn[ax] = L.kcart[3 * u + ax] + (jo < S.n_field ? S.A[3 * jh + ax] : 0.0);
    V* phn = (V*)L.ph_next + (long long)u * L.ph_stride;
    for (int i = threadIdx.x; i < tab; i += blockDim.x) {
      const int ax = (i / c.nmax) % 3;
      double s, co;
      sincos(qn[ax] * c.d1[i], &s, &co);
      phn[i] = cmk<V>((T)co, (T)s);
    }
  }
}

// ----------------------------------------------------------------------------
// bra: P[u][b][row] = dV sum_r C_row(r) t_b(r), C = conj(beta~) (times d_a for
// the current rows).  Register-blocked complex GEMM (rows x bands x points)
// with the C tile generated in shared memory from the separable tables.
//   NW = 1: rows j = 0..n_proj-1              (projections for the ket)
//   NW = 4: rows 4 j + a, a = 0 (beta~), 1..3 (d_x, d_y, d_z times beta~)
// grid (row blocks, band blocks, units), 256 threads.
// ----------------------------------------------------------------------------
template <typename T, int NW>
__global__ void __launch_bounds__(256) k_bra(LaunchSet L, const typename Cplx<T>::type* __restrict__ src,
                                             typename Cplx<T>::type* __restrict__ P, int use_obs) {
  using V = typename Cplx<T>::type;
  constexpr int RB = 32, BB = 16;
  constexpr int KT = sizeof(T) == 8 ? 32 : 64;
  constexpr int APB = RB / (4 * NW);
  __shared__ V Cs[KT][RB];
  __shared__ V Us[KT][BB];
  __shared__ V red[RB][BB];
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.z];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int rows = c.n_proj * NW;
  const int a0 = blockIdx.x * APB;
  const int bb0 = blockIdx.y * BB;
  const V* ph = (const V*)(use_obs ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = lane >> 2, bg = lane & 3;
  const int nm = c.nmax;
  const V zero = cmk<V>((T)0, (T)0);
  V acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = zero;
  const V* srcU = src + U.psi_off;
  for (int p0 = 0; p0 < c.npts; p0 += KT) {
    __syncthreads();
    for (int i = tid; i < KT * APB; i += 256) {
      const int kk = i % KT, al = i / KT;
      const int p = p0 + kk, a = a0 + al;
      V vals[4 * NW];
#pragma unroll
      for (int r = 0; r < 4 * NW; ++r) vals[r] = zero;
      if (p < c.npts && a < c.n_atoms) {
        const int ix = p % c.n1, iy = (p / c.n1) % c.n2, iz = p / (c.n1 * c.n2);
        const T* ga = Tab<T>::g1(c) + (long long)a * 3 * nm;
        const T* da = Tab<T>::d1(c) + (long long)a * 3 * nm;
        const T g = ga[ix] * ga[nm + iy] * ga[2 * nm + iz];
        const T d[3] = {da[ix], da[nm + iy], da[2 * nm + iz]};
        const V* pa = ph + (long long)a * 3 * nm;
        const V f = cscale(cmul(cmul(pa[ix], pa[nm + iy]), pa[2 * nm + iz]), g);
        const T* pn = Tab<T>::pnorm(c) + 4 * a;
        const T w[4] = {pn[0], pn[1] * d[0], pn[2] * d[1], pn[3] * d[2]};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (NW == 1) {
            vals[t] = cscale(f, w[t]);
          } else {
            vals[4 * t + 0] = cscale(f, w[t]);
            vals[4 * t + 1] = cscale(f, w[t] * d[0]);
            vals[4 * t + 2] = cscale(f, w[t] * d[1]);
            vals[4 * t + 3] = cscale(f, w[t] * d[2]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4 * NW; ++r) Cs[kk][al * 4 * NW + r] = vals[r];
    }
    for (int i = tid; i < KT * BB; i += 256) {
      const int kk = i % KT, b = i / KT;
      const int p = p0 + kk, band = bb0 + b;
      V v = zero;
      if (p < c.npts && band < c.n_bands) v = srcU[(long long)band * c.npts + p];
      Us[kk][b] = v;
    }
    __syncthreads();
    for (int kk = warp; kk < KT; kk += 8) {
      V cv[4], uv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        cv[i] = Cs[kk][rg * 4 + i];
        uv[i] = Us[kk][bg * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], cv[i], uv[j]);
    }
  }
  for (int w = 0; w < 8; ++w) {
    __syncthreads();
    if (warp == w) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          V prev = (w == 0) ? zero : red[rg * 4 + i][bg * 4 + j];
          red[rg * 4 + i][bg * 4 + j] = cadd(prev, acc[i][j]);
        }
    }
  }
  __syncthreads();
  const long long off = (NW == 1) ? U.p_off : U.pa_off;
  const T dv = (T)c.dv;
  for (int i = tid; i < RB * BB; i += 256) {
    const int r = i % RB, b = i / RB;
    const int row = blockIdx.x * RB + r, band = bb0 + b;
    if (row < rows && band < c.n_bands) P[off + (long long)band * rows + row] = cscale(red[r][b], dv);
  }
}

// ----------------------------------------------------------------------------
// bra on the projector boxes: the same P as k_bra, from the factorisation
// C_row(r) = pn_t F^a_x(ix) F^a_y(iy) F^a_z(iz) d_x^i d_y^j d_z^k (F = g e^{i q d})
// restricted to the atom's box (the Gaussian factor is zero outside it).  One CTA
// per (atom, unit, block of BRA_BOX_BANDS bands), one thread per (x, y) column of
// the box (at most 16 x 16).  Bands go through in sub-blocks of BB_SUB: per
// column the sums Z_k = sum_z F_z d_z^k t (k <= 1, or <= 2 for the current) of
// all bands of the sub-block in one z loop (F_z, d_z read once per plane), then
// the x and y weights give the sub-block's row values, which one warp
// reduce-scatter and one fixed-order sum over the warps add up.
//   NW = 1: rows 4 a + t (t = s, p_x, p_y, p_z);  NW = 4: rows 4 (4 a + t) + alpha.
// ----------------------------------------------------------------------------
#define BRA_BOX_BANDS 8   // bands per CTA of k_bra_box

template <typename T, int NW> struct BraBoxShape {
  static constexpr int NR = 4 * NW;                                // rows of the atom
  static constexpr int KD = NW == 1 ? 2 : 3;                       // powers of d_z in the column sums
  static constexpr int SUB = (sizeof(T) == 8 ? 4 : 8) / NW;      // bands per sub-block (NW = 1 or 4)
  static constexpr int NF = 2 * SUB * NR;                          // real values per thread (32 or 64)
};

// Sum of x[0..NF) over the 32 lanes of a warp, scattered: afterwards lane l holds
// in x[0..NF/32) the sums of the values NF/32 * l + e (fixed butterfly order).
template <typename T, int NF>
__device__ __forceinline__ void warp_reduce_scatter(T (&x)[NF], int lane) {
  static_assert(NF == 32 || NF == 64, "32 or 64 values");
#pragma unroll
  for (int o = 16, n = NF; o > 0; o >>= 1, n >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const T keep = up ? x[n / 2 + i] : x[i];
      const T send = up ? x[i] : x[n / 2 + i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

template <typename T, int NW>
__global__ void __launch_bounds__(256) k_bra_box(LaunchSet L, const typename Cplx<T>::type* __restrict__ src,
                                                 typename Cplx<T>::type* __restrict__ P, int use_obs) {
  using V = typename Cplx<T>::type;
  using SH = BraBoxShape<T, NW>;
  constexpr int NR = SH::NR, KD = SH::KD, SUB = SH::SUB, NF = SH::NF, PL = NF / 32;
  __shared__ T red[8][NF];
  const CellDev& c = L.cell;
  const int a = blockIdx.x;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int* bx = c.pbox + a * 6;
  const int sx = bx[0], lx = bx[1], sy = bx[2], ly = bx[3], sz = bx[4], lz = bx[5];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int n_warps = (int)(blockDim.x >> 5);
  const bool live = t < lx * ly;
  const int ix = (sx + (live ? t % lx : 0)) % c.n1, iy = (sy + (live ? t / lx : 0)) % c.n2;
  const int nm = c.nmax, n12 = c.n1 * c.n2;
  const V* ph = (const V*)(use_obs ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride + (long long)a * 3 * nm;
  const T* ga = Tab<T>::g1(c) + (long long)a * 3 * nm;
  const T* da = Tab<T>::d1(c) + (long long)a * 3 * nm;
  const T* pn = Tab<T>::pnorm(c) + 4 * a;
  // column weights F_x F_y and the displacements of the column
  const V fxy = cscale(cmul(ph[ix], ph[nm + iy]), ga[ix] * ga[nm + iy]);
  const T dx = da[ix], dy = da[nm + iy];
  const int rows = c.n_proj * NW;
  const long long off = (NW == 1) ? U.p_off : U.pa_off;
  const int b_begin = blockIdx.z * BRA_BOX_BANDS;
  const int b_end = min(c.n_bands, b_begin + BRA_BOX_BANDS);
  for (int b0 = b_begin; b0 < b_end; b0 += SUB) {
    const V* tb = src + U.psi_off + (long long)b0 * c.npts + iy * c.n1 + ix;
    V z[SUB][KD];
#pragma unroll
    for (int bl = 0; bl < SUB; ++bl)
#pragma unroll
      for (int k = 0; k < KD; ++k) z[bl][k] = cmk<V>((T)0, (T)0);
    if (live) {
#pragma unroll 2
      for (int kz = 0; kz < lz; ++kz) {
        const int iz = (sz + kz) % c.n3;
        const V fz = cscale(ph[2 * nm + iz], ga[2 * nm + iz]);
        const T dz = da[2 * nm + iz];
#pragma unroll
        for (int bl = 0; bl < SUB; ++bl) {
          if (b0 + bl < b_end) {
            V w = cmul(fz, tb[(long long)bl * c.npts + (long long)iz * n12]);
            z[bl][0] = cadd(z[bl][0], w);
            w = cscale(w, dz);
            z[bl][1] = cadd(z[bl][1], w);
            if (KD > 2) z[bl][KD - 1] = cadd(z[bl][KD - 1], cscale(w, dz));
          }
        }
      }
    }
    // row values of this column, (band, row) in order, as real pairs:
    // monomial d_x^i d_y^j d_z^k times the column sums
    T x[NF];
#pragma unroll
    for (int bl = 0; bl < SUB; ++bl)
#pragma unroll
      for (int tt = 0; tt < 4; ++tt) {
        const int ti = tt == 1, tj = tt == 2, tk = tt == 3;
#pragma unroll
        for (int al = 0; al < NW; ++al) {
          const int i = ti + (NW == 4 && al == 1), j = tj + (NW == 4 && al == 2), k = tk + (NW == 4 && al == 3);
          T wxy = (T)1;
          if (i >= 1) wxy *= dx;
          if (i >= 2) wxy *= dx;
          if (j >= 1) wxy *= dy;
          if (j >= 2) wxy *= dy;
          const V vv = live ? cscale(cmul(fxy, z[bl][k < KD ? k : KD - 1]), wxy) : cmk<V>((T)0, (T)0);
          const int r = bl * NR + tt * NW + al;
          x[2 * r] = vv.x;
          x[2 * r + 1] = vv.y;
        }
      }
    // fixed-order reduction over the columns: warp reduce-scatter, then warps in order
    warp_reduce_scatter<T, NF>(x, lane);
#pragma unroll
    for (int e = 0; e < PL; ++e) red[warp][PL * lane + e] = x[e];
    __syncthreads();
    if (t < NF) {
      T sum = (T)0;
      for (int w = 0; w < n_warps; ++w) sum += red[w][t];
      const int r = (t >> 1) % NR, bl = (t >> 1) / NR, b = b0 + bl;
      if (b < b_end) {
        const T sc = (T)c.dv * pn[r / NW];
        reinterpret_cast<T*>(P + off + (long long)b * rows + a * NR + r)[t & 1] = sum * sc;
      }
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// stage m of the Taylor recurrence for all bands of one unit and TSBZ_PT points
//   t_m = (-i dt/m) [ -1/2 lap t - i q.grad t + (|q|^2/2 + v_eff) t + V_NL t ]
//   m = 1: write t_1                      m = 2: write t_2, psi += t_1 + t_2
//   m = 3: write t_3, psi += t_3          m = 4: psi += t_4
// V_NL t = sum_a conj(phase_a) g_a [W_s + d_x W_px + d_y W_py + d_z W_pz],
// W_j = pnorm E_j P_jb staged in shared memory per band chunk.
// grid (point tiles, units), TSBZ_PT threads, dynamic smem BC * n_proj complex.
// ----------------------------------------------------------------------------
template <typename T, int BC>
__global__ void __launch_bounds__(TSBZ_PT) k_stage(LaunchSet L, const typename Cplx<T>::type* __restrict__ tin,
                                                   typename Cplx<T>::type* __restrict__ tout,
                                                   typename Cplx<T>::type* __restrict__ psi,
                                                   const typename Cplx<T>::type* __restrict__ P, int m) {
  using V = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* Ws = reinterpret_cast<V*>(smraw);
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int p = blockIdx.x * TSBZ_PT + threadIdx.x;
  const bool valid = p < c.npts;
  const int pp = valid ? p : 0;
  const int ix = pp % c.n1, iy = (pp / c.n1) % c.n2, iz = pp / (c.n1 * c.n2);
  const int n12 = c.n1 * c.n2;
  const T* qt = reinterpret_cast<const T*>(L.qt_half) + 4 * u;
  const T q[3] = {qt[0], qt[1], qt[2]};
  const T q2h = qt[3];
  const T v = valid ? reinterpret_cast<const T*>(S.veff)[pp] : (T)0;
  const T diag = q2h + v;
  const T hdt = (T)(S.dt * L.dt_scale) / (T)(m > 0 ? m : 1);
  const V* ph = (const V*)L.ph_half + (long long)u * L.ph_stride;
  const int nm = c.nmax;
  const V zero = cmk<V>((T)0, (T)0);
  // m = 0: filter step of the ground-state solver, tout = c1 h t + c2 t + c3 prev
  // with per-unit coefficients L.filt[3 u ..] and prev passed as psi
  const T fc1 = m == 0 ? (T)L.filt[3 * u] : (T)0, fc2 = m == 0 ? (T)L.filt[3 * u + 1] : (T)0;
  const T fc3 = m == 0 ? (T)L.filt[3 * u + 2] : (T)0;
  __shared__ T lw[3][TSBZ_MAX_ND + 1], gw[3][TSBZ_MAX_ND + 1];
  if (threadIdx.x < 3 * (TSBZ_MAX_ND + 1)) {
    const int ax = threadIdx.x / (TSBZ_MAX_ND + 1), mm = threadIdx.x % (TSBZ_MAX_ND + 1);
    lw[ax][mm] = (T)(-0.5 * c.lapw[ax][mm]);
    gw[ax][mm] = (T)c.gradw[ax][mm];
  }
  // the atoms whose projector box holds the point (bit a), found once for all
  // band chunks when there are at most 64; outside a box the factor is exactly zero
  const bool use_mask = c.use_proj && c.n_atoms <= 64;
  unsigned long long amask = 0ull;
  if (use_mask && valid)
    for (int a = 0; a < c.n_atoms; ++a) {
      const T* ga = Tab<T>::g1(c) + (long long)a * 3 * nm;
      if (ga[ix] * ga[nm + iy] * ga[2 * nm + iz] != (T)0) amask |= 1ull << a;
    }
  for (int b0 = 0; b0 < c.n_bands; b0 += BC) {
    __syncthreads();
    if (c.use_proj) {
      for (int i = threadIdx.x; i < BC * c.n_proj; i += TSBZ_PT) {
        const int bl = i / c.n_proj, j = i % c.n_proj, b = b0 + bl;
        V w = zero;
        if (b < c.n_bands) w = cscale(P[U.p_off + (long long)b * c.n_proj + j], Tab<T>::wkb(c)[j]);
        Ws[i] = w;
      }
    }
    __syncthreads();
    if (!valid) continue;
    V ket[BC];
#pragma unroll
    for (int bl = 0; bl < BC; ++bl) ket[bl] = zero;
    if (c.use_proj) {
      // atoms in increasing order: the set bits of the mask, else every atom with the box test
      unsigned long long mk = amask;
      for (int a = use_mask ? (mk ? __ffsll((long long)mk) - 1 : c.n_atoms) : 0; a < c.n_atoms;
           a = use_mask ? ((mk &= mk - 1) ? __ffsll((long long)mk) - 1 : c.n_atoms) : a + 1) {
        const T* ga = Tab<T>::g1(c) + (long long)a * 3 * nm;
        const T* da = Tab<T>::d1(c) + (long long)a * 3 * nm;
        const T g = ga[ix] * ga[nm + iy] * ga[2 * nm + iz];
        if (g == (T)0) continue;   // outside the atom's projector box the factor is exactly zero
        const T dx = da[ix], dy = da[nm + iy], dz = da[2 * nm + iz];
        const V* pa = ph + (long long)a * 3 * nm;
        const V fph = cmul(cmul(pa[ix], pa[nm + iy]), pa[2 * nm + iz]);
        const V f = cmk<V>(fph.x * g, -fph.y * g);   // g * exp(-i q.d)
#pragma unroll
        for (int bl = 0; bl < BC; ++bl) {
          const V* wb = Ws + bl * c.n_proj + 4 * a;
          V w = wb[0];
          rfma(w, dx, wb[1]);
          rfma(w, dy, wb[2]);
          rfma(w, dz, wb[3]);
          cfma(ket[bl], f, w);
        }
      }
    }
#pragma unroll
    for (int bl = 0; bl < BC; ++bl) {
      const int b = b0 + bl;
      if (b >= c.n_bands) break;
      const long long base = U.psi_off + (long long)b * c.npts;
      const V* tb = tin + base;
      const V ce = tb[pp];
      // h t (local part), lap scaled by -1/2 through lw
      V h = cmk<V>(ce.x * (lw[0][0] + lw[1][0] + lw[2][0] + diag), ce.y * (lw[0][0] + lw[1][0] + lw[2][0] + diag));
      V qg = zero;
      const int rowb = iz * n12 + iy * c.n1;
      for (int mm = 1; mm <= c.nd; ++mm) {
        // x
        {
          const V up = tb[rowb + wrap_idx(ix + mm, c.n1)];
          const V dn = tb[rowb + wrap_idx(ix - mm, c.n1)];
          rfma(h, lw[0][mm], cadd(up, dn));
          rfma(qg, q[0] * gw[0][mm], csub(up, dn));
        }
        // y
        {
          const V up = tb[iz * n12 + wrap_idx(iy + mm, c.n2) * c.n1 + ix];
          const V dn = tb[iz * n12 + wrap_idx(iy - mm, c.n2) * c.n1 + ix];
          rfma(h, lw[1][mm], cadd(up, dn));
          rfma(qg, q[1] * gw[1][mm], csub(up, dn));
        }
        // z
        {
          const V up = tb[wrap_idx(iz + mm, c.n3) * n12 + iy * c.n1 + ix];
          const V dn = tb[wrap_idx(iz - mm, c.n3) * n12 + iy * c.n1 + ix];
          rfma(h, lw[2][mm], cadd(up, dn));
          rfma(qg, q[2] * gw[2][mm], csub(up, dn));
        }
      }
      // -i q.grad t
      h.x += qg.y;
      h.y -= qg.x;
      h = cadd(h, ket[bl]);
      if (m == 0) {
        V o = cmk<V>(fc1 * h.x + fc2 * ce.x, fc1 * h.y + fc2 * ce.y);
        if (fc3 != (T)0) {
          const V pv = psi[base + pp];
          o = cmk<V>(o.x + fc3 * pv.x, o.y + fc3 * pv.y);
        }
        tout[base + pp] = o;
        continue;
      }
      // t_m = (-i dt/m) h
      const V t = cmk<V>(hdt * h.y, -hdt * h.x);
      if (m < 4) tout[base + pp] = t;
      if (m == 2) {
        psi[base + pp] = cadd(psi[base + pp], cadd(ce, t));
      } else if (m >= 3) {
        psi[base + pp] = cadd(psi[base + pp], t);
      }
    }
  }
}

// ----------------------------------------------------------------------------
// stage m with the non-local term supplied: t_m = (-i dt/m)[h_loc t + V]
// (V = sum_j beta~_j E_j P_jb from the tensor-core ket), psi accumulation as
// in k_stage.  Thread per point with its 2 x 3 x ND neighbour offsets
// computed once; grid (point tiles, units), TSBZ_PT threads.
// ----------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(TSBZ_PT) k_stage_v(LaunchSet L, const typename Cplx<T>::type* __restrict__ tin,
                                                     typename Cplx<T>::type* __restrict__ tout,
                                                     typename Cplx<T>::type* __restrict__ psi,
                                                     const typename Cplx<T>::type* __restrict__ V, int m) {
  using VT = typename Cplx<T>::type;
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int p = blockIdx.x * TSBZ_PT + threadIdx.x;
  if (p >= c.npts) return;
  const int n12 = c.n1 * c.n2;
  const int ix = p % c.n1, iy = (p / c.n1) % c.n2, iz = p / n12;
  int off[6 * ND];
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) {
    off[6 * (mm - 1) + 0] = wrap_idx(ix + mm, c.n1) - ix;
    off[6 * (mm - 1) + 1] = wrap_idx(ix - mm, c.n1) - ix;
    off[6 * (mm - 1) + 2] = (wrap_idx(iy + mm, c.n2) - iy) * c.n1;
    off[6 * (mm - 1) + 3] = (wrap_idx(iy - mm, c.n2) - iy) * c.n1;
    off[6 * (mm - 1) + 4] = (wrap_idx(iz + mm, c.n3) - iz) * n12;
    off[6 * (mm - 1) + 5] = (wrap_idx(iz - mm, c.n3) - iz) * n12;
  }
  const T* qt = reinterpret_cast<const T*>(L.qt_half) + 4 * u;
  const T q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const T dg = (T)(c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0]) + qt[3] + reinterpret_cast<const T*>(S.veff)[p];
  const T hdt = (T)(S.dt * L.dt_scale) / (T)m;
  for (int b = 0; b < c.n_bands; ++b) {
    const long long base = U.psi_off + (long long)b * c.npts + p;
    const VT* tb = tin + base;
    const VT ce = tb[0];
    T hx = dg * ce.x, hy = dg * ce.y;
    T gxr = 0, gxi = 0, gyr = 0, gyi = 0, gzr = 0, gzi = 0;
#pragma unroll
    for (int mm = 1; mm <= ND; ++mm) {
      const VT xu = tb[off[6 * (mm - 1) + 0]], xd = tb[off[6 * (mm - 1) + 1]];
      const VT yu = tb[off[6 * (mm - 1) + 2]], yd = tb[off[6 * (mm - 1) + 3]];
      const VT zu = tb[off[6 * (mm - 1) + 4]], zd = tb[off[6 * (mm - 1) + 5]];
      hx = fma((T)c.hlapf[0][mm], xu.x + xd.x, hx);
      hy = fma((T)c.hlapf[0][mm], xu.y + xd.y, hy);
      hx = fma((T)c.hlapf[1][mm], yu.x + yd.x, hx);
      hy = fma((T)c.hlapf[1][mm], yu.y + yd.y, hy);
      hx = fma((T)c.hlapf[2][mm], zu.x + zd.x, hx);
      hy = fma((T)c.hlapf[2][mm], zu.y + zd.y, hy);
      gxr = fma((T)c.gradwf[0][mm], xu.x - xd.x, gxr);
      gxi = fma((T)c.gradwf[0][mm], xu.y - xd.y, gxi);
      gyr = fma((T)c.gradwf[1][mm], yu.x - yd.x, gyr);
      gyi = fma((T)c.gradwf[1][mm], yu.y - yd.y, gyi);
      gzr = fma((T)c.gradwf[2][mm], zu.x - zd.x, gzr);
      gzi = fma((T)c.gradwf[2][mm], zu.y - zd.y, gzi);
    }
    const VT v = V[base];
    const T qgr = fma(q0, gxr, fma(q1, gyr, q2 * gzr));
    const T qgi = fma(q0, gxi, fma(q1, gyi, q2 * gzi));
    const T hr = hx + qgi + v.x;
    const T hi = hy - qgr + v.y;
    const VT t = cmk<VT>(hdt * hi, -hdt * hr);
    if (m < 4) tout[base] = t;
    if (m == 2) {
      psi[base] = cadd(psi[base], cadd(ce, t));
    } else if (m >= 3) {
      psi[base] = cadd(psi[base], t);
    }
  }
}

// ----------------------------------------------------------------------------
// stage m, 2.5-D form: one CTA per (band, unit), one thread per (x, y) column
// marching in z.  Each thread keeps the 2 ND + 1 values of its column around
// the current plane in a register queue; the current plane is also written
// to shared memory for the in-plane neighbours; plane z + ND + 1 is loaded
// one step ahead.  t_m = (-i dt/m)[h_loc t + V], psi accumulation as in
// k_stage.  Requires n1 * n2 <= blockDim.x (one thread per column).
// ----------------------------------------------------------------------------
template <typename T, int ND>
__global__ void __launch_bounds__(256, 4) k_stage_z(LaunchSet L, const typename Cplx<T>::type* __restrict__ tin,
                                                 typename Cplx<T>::type* __restrict__ tout,
                                                 typename Cplx<T>::type* __restrict__ psi,
                                                 const typename Cplx<T>::type* __restrict__ V, int m) {
  using VT = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char zraw[];
  VT* plane = reinterpret_cast<VT*>(zraw);
  const CellDev& c = L.cell;
  const int b = blockIdx.x;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int n1 = c.n1, n2 = c.n2, n3 = c.n3, n12 = n1 * n2;
  const int col = threadIdx.x;
  const bool act = col < n12;
  const int ix = act ? col % n1 : 0, iy = act ? col / n1 : 0;
  const int rowb = iy * n1;
  const T* qt = reinterpret_cast<const T*>(L.qt_half) + 4 * u;
  const T q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const T dg0 = (T)(c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0]) + qt[3];
  const T hdt = (T)(S.dt * L.dt_scale) / (T)m;
  const T* veff = reinterpret_cast<const T*>(S.veff);
  const long long base0 = U.psi_off + (long long)b * c.npts + col;
  const VT* tb = tin + base0;
  // queue[k] = t(z - ND + k) of this column
  VT qv[2 * ND + 1];
  const VT zero = cmk<VT>((T)0, (T)0);
#pragma unroll
  for (int k = 0; k < 2 * ND + 1; ++k) {
    const int zz = wrap_idx(k - ND, n3);
    qv[k] = act ? tb[(long long)zz * n12] : zero;
  }
  // values of the current plane loaded one step ahead: V, psi (m >= 2), v_eff
  VT v_cur = act ? V[base0] : zero;
  VT p_cur = (act && m >= 2) ? psi[base0] : zero;
  T e_cur = act ? veff[col] : (T)0;
  for (int z = 0; z < n3; ++z) {
    // prefetch t(z + ND + 1) and V, psi, v_eff of plane z + 1
    const int zn = wrap_idx(wrap_idx(z + ND + 1, n3), n3);
    const VT nxt = act ? tb[(long long)zn * n12] : zero;
    const bool more = act && z + 1 < n3;
    const long long idx_n = base0 + (long long)(z + 1) * n12;
    const VT v_nxt = more ? V[idx_n] : zero;
    const VT p_nxt = (more && m >= 2) ? psi[idx_n] : zero;
    const T e_nxt = more ? veff[(z + 1) * n12 + col] : (T)0;
    __syncthreads();
    if (act) plane[col] = qv[ND];
    __syncthreads();
    if (act) {
      const VT ce = qv[ND];
      const long long idx = base0 + (long long)z * n12;
      const T dg = dg0 + e_cur;
      T hx = dg * ce.x, hy = dg * ce.y;
      T gxr = 0, gxi = 0, gyr = 0, gyi = 0, gzr = 0, gzi = 0;
#pragma unroll
      for (int mm = 1; mm <= ND; ++mm) {
        const VT xu = plane[rowb + wrap_idx(ix + mm, n1)], xd = plane[rowb + wrap_idx(ix - mm, n1)];
        const VT yu = plane[wrap_idx(iy + mm, n2) * n1 + ix], yd = plane[wrap_idx(iy - mm, n2) * n1 + ix];
        const VT zu = qv[ND + mm], zd = qv[ND - mm];
        hx = fma((T)c.hlapf[0][mm], xu.x + xd.x, hx);
        hy = fma((T)c.hlapf[0][mm], xu.y + xd.y, hy);
        hx = fma((T)c.hlapf[1][mm], yu.x + yd.x, hx);
        hy = fma((T)c.hlapf[1][mm], yu.y + yd.y, hy);
        hx = fma((T)c.hlapf[2][mm], zu.x + zd.x, hx);
        hy = fma((T)c.hlapf[2][mm], zu.y + zd.y, hy);
        gxr = fma((T)c.gradwf[0][mm], xu.x - xd.x, gxr);
        gxi = fma((T)c.gradwf[0][mm], xu.y - xd.y, gxi);
        gyr = fma((T)c.gradwf[1][mm], yu.x - yd.x, gyr);
        gyi = fma((T)c.gradwf[1][mm], yu.y - yd.y, gyi);
        gzr = fma((T)c.gradwf[2][mm], zu.x - zd.x, gzr);
        gzi = fma((T)c.gradwf[2][mm], zu.y - zd.y, gzi);
      }
      const T qgr = fma(q0, gxr, fma(q1, gyr, q2 * gzr));
      const T qgi = fma(q0, gxi, fma(q1, gyi, q2 * gzi));
      const T hr = hx + qgi + v_cur.x;
      const T hi = hy - qgr + v_cur.y;
      const VT t = cmk<VT>(hdt * hi, -hdt * hr);
      if (m < 4) tout[idx] = t;
      if (m == 2) {
        psi[idx] = cadd(p_cur, cadd(ce, t));
      } else if (m >= 3) {
        psi[idx] = cadd(p_cur, t);
      }
    }
    // advance the queue
#pragma unroll
    for (int k = 0; k < 2 * ND; ++k) qv[k] = qv[k + 1];
    qv[2 * ND] = nxt;
    v_cur = v_nxt;
    p_cur = p_nxt;
    e_cur = e_nxt;
  }
}

// ----------------------------------------------------------------------------
// observe: per (unit, point tile, band group) sums for rho, kinetic current
// and band norms.  grid (point tiles, units, band groups), TSBZ_PT threads.
// At one grid point the sums over the bands of the group are formed in T
// (their terms are products of T orbitals); every sum over grid points,
// k-points and sub-simulations is double.  The current's local part is only
// needed summed over the periodic grid, where
//   sum_r Re(u* (-i grad_ax) u) = 2 sum_m w_m sum_r Im(conj(u(r)) u(r + m e_ax)),
// so each point loads its forward neighbours only (the tile partials differ
// from the gradient form's, their total does not).
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(TSBZ_PT) k_observe(LaunchSet L, const typename Cplx<T>::type* __restrict__ psi,
                                                     double* __restrict__ rho_part, double* __restrict__ jk_part,
                                                     double* __restrict__ nrm_part) {
  using V = typename Cplx<T>::type;
  __shared__ T red_n[TSBZ_BG][TSBZ_PT];
  __shared__ double red_j[3][TSBZ_PT / 32];
  __shared__ T gw[3][TSBZ_MAX_ND + 1];
  const CellDev& c = L.cell;
  if (threadIdx.x < 3 * (TSBZ_MAX_ND + 1)) {
    const int ax = threadIdx.x / (TSBZ_MAX_ND + 1), mm = threadIdx.x % (TSBZ_MAX_ND + 1);
    gw[ax][mm] = (T)c.gradw[ax][mm];
  }
  __syncthreads();
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const int tile = blockIdx.x, grp = blockIdx.z;
  const int p = tile * TSBZ_PT + threadIdx.x;
  const bool valid = p < c.npts;
  const int pp = valid ? p : 0;
  const int ix = pp % c.n1, iy = (pp / c.n1) % c.n2, iz = pp / (c.n1 * c.n2);
  const int n12 = c.n1 * c.n2;
  const int b_begin = grp * TSBZ_BG;
  const int b_end = min(c.n_bands, b_begin + TSBZ_BG);
  T rho = (T)0, jx = (T)0, jy = (T)0, jz = (T)0;
  for (int b = b_begin; b < b_end; ++b) {
    T n2 = (T)0;
    if (valid) {
      const V* tb = psi + U.psi_off + (long long)b * c.npts;
      const V ce = tb[pp];
      n2 = ce.x * ce.x + ce.y * ce.y;
      rho += n2;
      T cx = (T)0, cy = (T)0, cz = (T)0;
      const int rowb = iz * n12 + iy * c.n1;
      for (int mm = 1; mm <= c.nd; ++mm) {
        const V xu = tb[rowb + wrap_idx(ix + mm, c.n1)];
        const V yu = tb[iz * n12 + wrap_idx(iy + mm, c.n2) * c.n1 + ix];
        const V zu = tb[wrap_idx(iz + mm, c.n3) * n12 + iy * c.n1 + ix];
        // Im(conj(u) v) = u_r v_i - u_i v_r
        cx += gw[0][mm] * (ce.x * xu.y - ce.y * xu.x);
        cy += gw[1][mm] * (ce.x * yu.y - ce.y * yu.x);
        cz += gw[2][mm] * (ce.x * zu.y - ce.y * zu.x);
      }
      jx += (T)2 * cx;
      jy += (T)2 * cy;
      jz += (T)2 * cz;
    }
    red_n[b - b_begin][threadIdx.x] = n2;
  }
  if (valid) rho_part[U.rho_off + (long long)grp * c.npts + p] = c.occ * (double)rho;
  double djx = jx, djy = jy, djz = jz;
  for (int off = 16; off > 0; off >>= 1) {
    djx += __shfl_xor_sync(0xffffffffu, djx, off);
    djy += __shfl_xor_sync(0xffffffffu, djy, off);
    djz += __shfl_xor_sync(0xffffffffu, djz, off);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    red_j[0][warp] = djx;
    red_j[1][warp] = djy;
    red_j[2][warp] = djz;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0.0;
    for (int w = 0; w < TSBZ_PT / 32; ++w) sum += red_j[threadIdx.x][w];
    jk_part[U.jk_off + ((long long)tile * c.n_bgroups + grp) * 3 + threadIdx.x] = sum;
  }
  // band norms of this tile
  for (int bl = warp; bl < b_end - b_begin; bl += TSBZ_PT / 32) {
    T sum = (T)0;
    for (int i = lane; i < TSBZ_PT; i += 32) sum += red_n[bl][i];
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) nrm_part[U.nrm_off + (long long)tile * c.n_bands + b_begin + bl] = (double)sum;
  }
}

// ----------------------------------------------------------------------------
// finalize: n_tiles CTAs per sub-simulation.  rho (Eq. 3), norms, and the current
// J = -(1/(Omega N_k)) sum_k sum_b occ [ dV Re<u|-i grad u> + q |u|^2
//                                        + 2 sum_j E_j Im(conj(c_j) a_j) ]   (Eqs. 5-6)
// summed in a fixed order.  The inputs are
// read-only here and disjoint from the outputs (restrict), so that the loads of
// a thread's chain of units and bands are issued ahead of the sums and stores.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(const SubDev* __restrict__ subs, const UnitDev* __restrict__ units,
                                                  const CellDev* __restrict__ cells, const double* __restrict__ q_obs,
                                                  const typename Cplx<T>::type* __restrict__ Pa,
                                                  const double* __restrict__ rho_part,
                                                  const double* __restrict__ jk_part,
                                                  const double* __restrict__ nrm_part, const int* __restrict__ mask,
                                                  int mode) {
  using V = typename Cplx<T>::type;
  const int s = blockIdx.x;
  const SubDev S = subs[s];
  if ((mode == TSBZ_FIN_STEP || mode == TSBZ_FIN_RHO) && !*S.active) return;   // budget spent: nothing of this step
  const CellDev c = cells[S.cell];
  // density: point tile blockIdx.y of the sub-simulation (fixed k and band-group order per point)
  const double inv_nk = 1.0 / S.n_k;
  const int chunk = (c.npts + (int)gridDim.y - 1) / (int)gridDim.y;
  const int r_end = min(c.npts, ((int)blockIdx.y + 1) * chunk);
  // the units of a sub-simulation are consecutive, n_bgroups * npts doubles apart
  const double* rho_s = rho_part + units[S.unit0].rho_off;
  const long long ustride = (long long)c.n_bgroups * c.npts;
  for (int r = (int)blockIdx.y * chunk + threadIdx.x; r < r_end; r += blockDim.x) {
    double acc = 0.0;
    if (c.n_bgroups == 1) {
#pragma unroll 8
      for (int kl = 0; kl < S.n_k; ++kl) acc += rho_s[kl * ustride + r];
    } else {
      for (int kl = 0; kl < S.n_k; ++kl)
        for (int g = 0; g < c.n_bgroups; ++g) acc += rho_s[kl * ustride + (long long)g * c.npts + r];
    }
    S.rho[r] = acc * inv_nk;
  }
  // current and norms of the units kl = tile + ntile j.  Small units (few
  // bands x projectors): warp w of the CTA takes every n_warps-th of them, lanes
  // share a unit.  Large units: the CTA takes them one at a time over all its
  // threads (warp w takes the band norms w, w + n_warps, ...).  Either way the
  // partial sums are added in a fixed order (lanes, warps in order, units in
  // increasing kl); the CTA that finishes last adds the tiles' partial currents
  // in tile order, writes J and advances the step.
  const int tile = blockIdx.y, ntile = gridDim.y;
  const int step = *S.step;
  const bool write_j = mode != TSBZ_FIN_RHO &&
                       ((mode == TSBZ_FIN_STEP) || (mask != nullptr && mask[s] != 0 &&
                                                    (mode == TSBZ_FIN_J0MINUS || step == 0)));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, n_warps = (int)(blockDim.x >> 5);
  const bool wide = fin_wide(c);
  const int u_first = wide ? tile : tile + ntile * warp, u_step = wide ? ntile : ntile * n_warps;
  const int b_first = wide ? warp : 0, b_step = wide ? n_warps : 1;
  const int e_first = wide ? (int)threadIdx.x : lane, e_step = wide ? (int)blockDim.x : 32;
  __shared__ double red[8][4];
  double jw[3] = {0.0, 0.0, 0.0};   // this warp's units (small), thread 0: this CTA's units (large)
  for (int kl = u_first; kl < S.n_k; kl += u_step) {
    const UnitDev U = units[S.unit0 + kl];
    const int u = S.unit0 + kl;
    double jk[3] = {0.0, 0.0, 0.0}, jn[3] = {0.0, 0.0, 0.0}, nsum = 0.0;
#pragma unroll 4
    for (int b = b_first; b < c.n_bands; b += b_step) {
      double nb = 0.0;
      for (int t = lane; t < c.n_tiles; t += 32) nb += nrm_part[U.nrm_off + (long long)t * c.n_bands + b];
      for (int off = 16; off > 0; off >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, off);
      nb *= c.dv;
      if (lane == 0) S.norms[kl * c.n_bands + b] = nb;
      nsum += nb;  // identical in every lane
    }
    for (int i = e_first; i < c.n_tiles * c.n_bgroups; i += e_step)
      for (int ax = 0; ax < 3; ++ax) jk[ax] += jk_part[U.jk_off + 3LL * i + ax];
    if (c.use_proj) {
      const int np = c.n_proj;
      if constexpr (sizeof(T) == sizeof(float)) {
        // single-precision projections: each thread forms and sums its own terms
        // in FP32 (the terms carry the projections' own ~1e-6 relative error) and
        // converts the sum once; the FP64 pipe of this GPU is ~1/64 of the FP32 one
        float jf[3] = {0.f, 0.f, 0.f};
#pragma unroll 4
        for (int i = e_first; i < c.n_bands * np; i += e_step) {
          const int j = i % np;
          const V* pr = Pa + U.pa_off + 4LL * i;
          const float ar = pr[0].x, ai = pr[0].y;
          const float e2 = 2.0f * c.ekbf[j];
          for (int ax = 0; ax < 3; ++ax) {
            // Im(conj(c) a) = c_r a_i - c_i a_r
            const float cr = pr[1 + ax].x, ci = pr[1 + ax].y;
            jf[ax] = __fmaf_rn(e2, __fmaf_rn(cr, ai, -ci * ar), jf[ax]);
          }
        }
        for (int ax = 0; ax < 3; ++ax) jn[ax] = (double)jf[ax];
      } else {
#pragma unroll 4
        for (int i = e_first; i < c.n_bands * np; i += e_step) {
          const int j = i % np;
          const V* pr = Pa + U.pa_off + 4LL * i;
          const double ar = pr[0].x, ai = pr[0].y;
          const double e2 = 2.0 * c.ekb[j];
          for (int ax = 0; ax < 3; ++ax) {
            // Im(conj(c) a) = c_r a_i - c_i a_r
            const double cr = pr[1 + ax].x, ci = pr[1 + ax].y;
            jn[ax] += e2 * (cr * ai - ci * ar);
          }
        }
      }
    }
    double v[3];
    for (int ax = 0; ax < 3; ++ax) {
      v[ax] = c.dv * jk[ax] + jn[ax];
      for (int off = 16; off > 0; off >>= 1) v[ax] += __shfl_xor_sync(0xffffffffu, v[ax], off);
    }
    if (!wide) {
      for (int ax = 0; ax < 3; ++ax) jw[ax] += c.occ * (v[ax] + q_obs[3 * u + ax] * nsum);
      continue;
    }
    if (lane == 0) {
      for (int ax = 0; ax < 3; ++ax) red[warp][ax] = v[ax];
      red[warp][3] = nsum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum[4] = {0.0, 0.0, 0.0, 0.0};
      for (int w = 0; w < n_warps; ++w)
        for (int k = 0; k < 4; ++k) sum[k] += red[w][k];
      for (int ax = 0; ax < 3; ++ax) jw[ax] += c.occ * (sum[ax] + q_obs[3 * u + ax] * sum[3]);
    }
    __syncthreads();
  }
  if (!wide) {
    // the warps' sums in warp order
    if (lane == 0)
      for (int ax = 0; ax < 3; ++ax) red[warp][ax] = jw[ax];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int ax = 0; ax < 3; ++ax) {
        double t = 0.0;
        for (int w = 0; w < n_warps; ++w) t += red[w][ax];
        jw[ax] = t;
      }
  }
  __shared__ int last;
  if (threadIdx.x == 0) {
    for (int ax = 0; ax < 3; ++ax) S.jtile[3 * tile + ax] = jw[ax];
    __threadfence();
    last = atomicAdd(S.jcount, 1) == ntile - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double J[3];
  bool finite = true;
  for (int ax = 0; ax < 3; ++ax) {
    double t = 0.0;
    for (int y = 0; y < ntile; ++y) t += __ldcg(S.jtile + 3 * y + ax);
    J[ax] = -t / (c.omega * S.n_k);
    finite = finite && isfinite(J[ax]);
  }
  *S.jcount = 0;
  if (!finite) *S.status |= 1;
  if (write_j) {
    double* dst = (mode == TSBZ_FIN_J0MINUS) ? S.J0m : (mode == TSBZ_FIN_J0PLUS ? S.J : S.J + 3LL * (step + 1));
    for (int ax = 0; ax < 3; ++ax) dst[ax] = J[ax];
  }
  if (mode == TSBZ_FIN_STEP) *S.step = step + 1;
}

// ----------------------------------------------------------------------------
// v_Hxc: rho -> complex work, 1-D DFT passes, Poisson scaling, PZ81, v_eff
// All sub-simulations in the list share one cell (same grid).
// ----------------------------------------------------------------------------
static __global__ void k_hxc_load(const SubDev* subs, const int* sub_ids, int n_subs, int npts, double2* work) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n_subs * npts) return;
  const int sl = (int)(e / npts), r = (int)(e % npts);
  work[e] = make_double2(subs[sub_ids[sl]].rho[r], 0.0);
}

// out = sum_n in[.. n ..] exp(sign * 2 pi i n k / N) along one axis.
static __global__ void k_dft_axis(const double2* __restrict__ in, double2* __restrict__ out, long long total, int npts,
                           int stride, int N, const double2* __restrict__ tw, int sign) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const long long sbase = (e / npts) * npts;
  const int r = (int)(e % npts);
  const int k = (r / stride) % N;
  const int base = r - k * stride;
  double sr = 0.0, si = 0.0;
  int idx = 0;
  for (int n = 0; n < N; ++n) {
    const double2 x = in[sbase + base + n * stride];
    const double2 w = tw[idx];
    const double wi = sign * w.y;
    sr += x.x * w.x - x.y * wi;
    si += x.x * wi + x.y * w.x;
    idx += k;
    if (idx >= N) idx -= N;
  }
  out[e] = make_double2(sr, si);
}

static __global__ void k_poisson(double2* work, long long total, CellDev c) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= total) return;
  const int r = (int)(e % c.npts);
  const int i1 = r % c.n1, i2 = (r / c.n1) % c.n2, i3 = r / (c.n1 * c.n2);
  const int m1 = i1 < (c.n1 + 1) / 2 ? i1 : i1 - c.n1;
  const int m2 = i2 < (c.n2 + 1) / 2 ? i2 : i2 - c.n2;
  const int m3 = i3 < (c.n3 + 1) / 2 ? i3 : i3 - c.n3;
  const double g1 = m1 * c.gsq_scale[0], g2 = m2 * c.gsq_scale[1], g3 = m3 * c.gsq_scale[2];
  const double gg = g1 * g1 + g2 * g2 + g3 * g3;
  const double f = gg > 0.0 ? 4.0 * M_PI / (gg * c.npts) : 0.0;
  const double2 x = work[e];
  work[e] = make_double2(x.x * f, x.y * f);
}

__device__ __forceinline__ double pz81_potential(double rho) {
  // Perdew-Zunger 1981, unpolarised: v_xc = d(rho e_xc)/d rho.
  const double r = fmax(rho, 1e-30);
  const double rs = cbrt(3.0 / (4.0 * M_PI * r));
  const double ex = -0.75 * cbrt(3.0 / M_PI) * cbrt(r);
  const double vx = 4.0 / 3.0 * ex;
  double vc;
  if (rs >= 1.0) {
    const double sq = sqrt(rs);
    const double den = 1.0 + 1.0529 * sq + 0.3334 * rs;
    const double ec = -0.1423 / den;
    vc = ec * (1.0 + 7.0 / 6.0 * 1.0529 * sq + 4.0 / 3.0 * 0.3334 * rs) / den;
  } else {
    const double lr = log(rs);
    vc = 0.0311 * lr + (-0.048 - 0.0311 / 3.0) + 2.0 / 3.0 * 0.0020 * rs * lr + (2.0 * -0.0116 - 0.0020) / 3.0 * rs;
  }
  return vx + vc;
}

template <typename T>
__global__ void k_hxc_final(const SubDev* subs, const int* sub_ids, int n_subs, CellDev c, const double2* work) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n_subs * c.npts) return;
  const int sl = (int)(e / c.npts), r = (int)(e % c.npts);
  const SubDev S = subs[sub_ids[sl]];
  double v = 0.0;
  if (S.hartree) v += work[e].x;
  if (S.xc) v += pz81_potential(S.rho[r]);
  S.vhxc[r] = v;
  reinterpret_cast<T*>(S.veff)[r] = (T)(c.vloc[r] + v);
}

// ----------------------------------------------------------------------------
// Hartree potential of one sub-simulation per CTA on small power-of-two grids
// (each axis 2..16, at most 4096 points): rho -> 3-D FFT in shared memory
// (radix-2 line transforms of each axis, one line per thread in registers),
// Poisson scaling (G = 0 -> 0), inverse FFT, into the work array.  The same
// FP64 arithmetic as the multi-launch path with the O(N^2) line DFTs replaced
// by FFTs; PZ81 and v_eff are then formed point-parallel by k_hxc_final.
// ----------------------------------------------------------------------------
#define HXC_FFT_MAXN 16
#define HXC_FFT_MAXPTS 4096
#define HXC_LINES_MIN_SUBS 8   // sub-simulations of a cell from which the per-axis line kernels take over

// In-place radix-2 transform of the line x (length N, a power of two):
// x[k] <- sum_n x[n] exp(sign 2 pi i n k / N); tw[m] = exp(2 pi i m / N).
// The twiddles exp(0) = 1 and exp(sign i pi / 2) = sign i are applied exactly,
// without a multiplication (22 of the 32 butterflies of a 16-point line).
template <int N>
__device__ __forceinline__ void hxc_fft_line(double2 (&x)[N], const double2* __restrict__ tw, int sign) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    int j = 0;
#pragma unroll
    for (int b = 1, r = i; b < N; b <<= 1, r >>= 1) j = (j << 1) | (r & 1);
    if (j > i) {
      const double2 t = x[i];
      x[i] = x[j];
      x[j] = t;
    }
  }
#pragma unroll
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1, step = N / len;
#pragma unroll
    for (int i = 0; i < N; i += len) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int m = k * step;
        const double2 v = x[i + k + half];
        double2 vw;
        if (m == 0) {
          vw = v;
        } else if (4 * m == N) {
          vw = sign > 0 ? make_double2(-v.y, v.x) : make_double2(v.y, -v.x);
        } else {
          const double2 w = tw[m];
          const double wi = sign * w.y;
          vw = make_double2(v.x * w.x - v.y * wi, v.x * wi + v.y * w.x);
        }
        const double2 u = x[i + k];
        x[i + k] = make_double2(u.x + vw.x, u.y + vw.y);
        x[i + k + half] = make_double2(u.x - vw.x, u.y - vw.y);
      }
    }
  }
}

template <int N>
__device__ __forceinline__ void hxc_fft_axis(double2* w, int npts, int stride, const double2* __restrict__ tw,
                                             int sign) {
  // lines: every r0 whose coordinate on this axis is 0, r0 = outer * (stride * N) + in, in < stride
  const int lines = npts / N;
  for (int l = threadIdx.x; l < lines; l += blockDim.x) {
    const int in = l % stride, outer = l / stride;
    const int r0 = outer * stride * N + in;
    double2 x[N];
#pragma unroll
    for (int n = 0; n < N; ++n) x[n] = w[r0 + n * stride];
    hxc_fft_line<N>(x, tw, sign);
#pragma unroll
    for (int n = 0; n < N; ++n) w[r0 + n * stride] = x[n];
  }
}

__device__ __forceinline__ void hxc_fft_any(double2* w, int npts, int n, int stride, const double2* tw, int sign) {
  switch (n) {
    case 2: hxc_fft_axis<2>(w, npts, stride, tw, sign); break;
    case 4: hxc_fft_axis<4>(w, npts, stride, tw, sign); break;
    case 8: hxc_fft_axis<8>(w, npts, stride, tw, sign); break;
    default: hxc_fft_axis<16>(w, npts, stride, tw, sign); break;
  }
}

static __global__ void __launch_bounds__(256) k_hxc_fft(const SubDev* subs, const int* sub_ids, CellDev c,
                                                  const double2* __restrict__ tw1, const double2* __restrict__ tw2,
                                                  const double2* __restrict__ tw3, double2* __restrict__ work) {
  extern __shared__ __align__(16) double2 hw[];
  const SubDev S = subs[sub_ids[blockIdx.x]];
  const int npts = c.npts, n12 = c.n1 * c.n2;
  for (int r = threadIdx.x; r < npts; r += blockDim.x) hw[r] = make_double2(S.rho[r], 0.0);
  __syncthreads();
  hxc_fft_any(hw, npts, c.n1, 1, tw1, -1);
  __syncthreads();
  hxc_fft_any(hw, npts, c.n2, c.n1, tw2, -1);
  __syncthreads();
  hxc_fft_any(hw, npts, c.n3, n12, tw3, -1);
  __syncthreads();
  for (int r = threadIdx.x; r < npts; r += blockDim.x) {
    const int i1 = r % c.n1, i2 = (r / c.n1) % c.n2, i3 = r / n12;
    const int m1 = i1 < (c.n1 + 1) / 2 ? i1 : i1 - c.n1;
    const int m2 = i2 < (c.n2 + 1) / 2 ? i2 : i2 - c.n2;
    const int m3 = i3 < (c.n3 + 1) / 2 ? i3 : i3 - c.n3;
    const double g1 = m1 * c.gsq_scale[0], g2 = m2 * c.gsq_scale[1], g3 = m3 * c.gsq_scale[2];
    const double gg = g1 * g1 + g2 * g2 + g3 * g3;
    const double f = gg > 0.0 ? 4.0 * M_PI / (gg * npts) : 0.0;
    hw[r] = make_double2(hw[r].x * f, hw[r].y * f);
  }
  __syncthreads();
  hxc_fft_any(hw, npts, c.n3, n12, tw3, +1);
  __syncthreads();
  hxc_fft_any(hw, npts, c.n2, c.n1, tw2, +1);
  __syncthreads();
  hxc_fft_any(hw, npts, c.n1, 1, tw1, +1);
  __syncthreads();
  // v_H of the sub-simulation; PZ81 and v_eff follow in k_hxc_final over all points
  double2* out = work + (long long)blockIdx.x * npts;
  for (int r = threadIdx.x; r < npts; r += blockDim.x) out[r] = hw[r];
}

__host__ __device__ inline bool hxc_fft_ok(int n) { return n == 2 || n == 4 || n == 8 || n == 16; }

// One FFT line per thread along one axis, over the grids of every sub-simulation
// of the list at once (work holds n_subs grids of npts complex values), in
// place: the same line transform as k_hxc_fft, spread over all SMs.
template <int N>
static __global__ void __launch_bounds__(64) k_fft_lines(double2* __restrict__ work, long long total_lines, int npts,
                                                         int stride, const double2* __restrict__ tw, int sign) {
  const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= total_lines) return;
  const int per = npts / N;
  const long long s = l / per;
  const int ll = (int)(l - s * per), in = ll % stride, outer = ll / stride;
  double2* w = work + s * npts + (long long)outer * stride * N + in;
  double2 x[N];
#pragma unroll
  for (int n = 0; n < N; ++n) x[n] = w[(long long)n * stride];
  hxc_fft_line<N>(x, tw, sign);
#pragma unroll
  for (int n = 0; n < N; ++n) w[(long long)n * stride] = x[n];
}

static void launch_fft_lines(double2* work, int n_subs, int npts, int n, int stride, const double2* tw, int sign,
                             cudaStream_t st) {
  const long long lines = (long long)n_subs * (npts / n);
  const unsigned blocks = (unsigned)((lines + 63) / 64);
  switch (n) {
    case 2: k_fft_lines<2><<<blocks, 64, 0, st>>>(work, lines, npts, stride, tw, sign); break;
    case 4: k_fft_lines<4><<<blocks, 64, 0, st>>>(work, lines, npts, stride, tw, sign); break;
    case 8: k_fft_lines<8><<<blocks, 64, 0, st>>>(work, lines, npts, stride, tw, sign); break;
    default: k_fft_lines<16><<<blocks, 64, 0, st>>>(work, lines, npts, stride, tw, sign); break;
  }
}

// v_eff of every sub-simulation of the list: copied to veff_save (swap = 0) or
// exchanged with it (swap = 1).
template <typename T>
__global__ void k_veff_keep(const SubDev* subs, const CellDev* cells, int swap) {
  const SubDev S = subs[blockIdx.y];
  const int npts = cells[S.cell].npts;
  T* a = reinterpret_cast<T*>(S.veff);
  T* b = reinterpret_cast<T*>(S.veff_save);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < npts; r += gridDim.x * blockDim.x) {
    const T v = a[r];
    if (swap) a[r] = b[r];
    b[r] = v;
  }
}

template <typename T> void launch_veff_keep_t(const SubDev* subs, const CellDev* cells, int n_subs, int swap,
                                              void* stream) {
  if (n_subs == 0) return;
  k_veff_keep<T><<<dim3(16, n_subs), 256, 0, (cudaStream_t)stream>>>(subs, cells, swap);
}

template <typename T>
__global__ void k_veff_frozen(const SubDev* subs, int s, CellDev c) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= c.npts) return;
  const SubDev S = subs[s];
  reinterpret_cast<T*>(S.veff)[r] = (T)(c.vloc[r] + S.vhxc[r]);
}

template <typename T>
__global__ void k_convert_in(const double2* __restrict__ src, typename Cplx<T>::type* __restrict__ dst, long long n) {
  using V = typename Cplx<T>::type;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = cmk<V>((T)src[i].x, (T)src[i].y);
}

template <typename T>
__global__ void k_convert_out(const typename Cplx<T>::type* __restrict__ src, double2* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
// Dynamic shared memory above the 48 KiB default needs the kernel's opt-in.
template <typename K> void stage_smem_attr(K* kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T> void launch_field(const LaunchSet& L, int mode, void* stream) {
  if (L.n_units == 0) return;
  k_field<T><<<L.n_units, 128, 0, (cudaStream_t)stream>>>(L, mode);
}

template <typename T>
void launch_bra(const LaunchSet& L, const void* src, void* P, int with_d, int use_obs, void* stream) {
  using V = typename Cplx<T>::type;
  if (L.n_units == 0 || !L.cell.use_proj) return;
  if (L.cell.pbox_ok) {
    // projector boxes of at most 16 x 16 columns: the factorised bra on the boxes
    dim3 gb(L.cell.n_atoms, L.n_units, (L.cell.n_bands + BRA_BOX_BANDS - 1) / BRA_BOX_BANDS);
    if (with_d)
      k_bra_box<T, 4><<<gb, 256, 0, (cudaStream_t)stream>>>(L, (const V*)src, (V*)P, use_obs);
    else
      k_bra_box<T, 1><<<gb, 256, 0, (cudaStream_t)stream>>>(L, (const V*)src, (V*)P, use_obs);
    return;
  }
  const int rows = L.cell.n_proj * (with_d ? 4 : 1);
  dim3 grid((rows + 31) / 32, (L.cell.n_bands + 15) / 16, L.n_units);
  if (with_d)
    k_bra<T, 4><<<grid, 256, 0, (cudaStream_t)stream>>>(L, (const V*)src, (V*)P, use_obs);
  else
    k_bra<T, 1><<<grid, 256, 0, (cudaStream_t)stream>>>(L, (const V*)src, (V*)P, use_obs);
}

template <typename T>
void launch_stage(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* P, int m, void* stream) {
  using V = typename Cplx<T>::type;
  if (L.n_units == 0) return;
  // bands per chunk of the staged projections: 8 (variant 0), 4 (1) or 16 (2)
  const int bc = L.variant == 1 ? 4 : (L.variant == 2 ? 16 : 8);
  dim3 grid(L.cell.n_tiles, L.n_units);
  const size_t sm = (size_t)bc * (L.cell.n_proj > 0 ? L.cell.n_proj : 1) * sizeof(V);
  cudaStream_t st = (cudaStream_t)stream;
  if (bc == 4) {
    stage_smem_attr(k_stage<T, 4>, sm);
    k_stage<T, 4><<<grid, TSBZ_PT, sm, st>>>(L, (const V*)tin, (V*)tout, (V*)psi, (const V*)P, m);
  } else if (bc == 16) {
    stage_smem_attr(k_stage<T, 16>, sm);
    k_stage<T, 16><<<grid, TSBZ_PT, sm, st>>>(L, (const V*)tin, (V*)tout, (V*)psi, (const V*)P, m);
  } else {
    stage_smem_attr(k_stage<T, 8>, sm);
    k_stage<T, 8><<<grid, TSBZ_PT, sm, st>>>(L, (const V*)tin, (V*)tout, (V*)psi, (const V*)P, m);
  }
}

template <typename T>
void launch_observe(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                    void* stream) {
  using V = typename Cplx<T>::type;
  if (L.n_units == 0) return;
  dim3 grid(L.cell.n_tiles, L.n_units, L.cell.n_bgroups);
  k_observe<T><<<grid, TSBZ_PT, 0, (cudaStream_t)stream>>>(L, (const V*)psi, rho_part, jk_part, nrm_part);
}

template <typename T>
void launch_finalize_t(const SubDev* subs, int n_subs, const UnitDev* units, const CellDev* cells_dev,
                       const double* q_obs, const void* Pa, const double* rho_part, const double* jk_part,
                       const double* nrm_part, const int* mask, int mode, int n_tiles, void* stream) {
  using V = typename Cplx<T>::type;
  if (n_subs == 0) return;
  // n_tiles (16 .. TSBZ_FIN_MAX_TILES) tiles per sub-simulation: density points, and units for the
  // current and the norms
  k_finalize<T><<<dim3(n_subs, n_tiles), 256, 0, (cudaStream_t)stream>>>(subs, units, cells_dev, q_obs, (const V*)Pa,
                                                                         rho_part, jk_part, nrm_part, mask, mode);
}

template <typename T>
int launch_hxc_t(const SubDev* subs_dev, const int* sub_ids_dev, int n_subs, const CellDev& c, double2* wa,
                 double2* wb, double2* const tw[3], void* stream) {
  if (n_subs == 0) return 0;
  cudaStream_t st = (cudaStream_t)stream;
  const long long total = (long long)n_subs * c.npts;
  const bool pow2 = hxc_fft_ok(c.n1) && hxc_fft_ok(c.n2) && hxc_fft_ok(c.n3);
  if (pow2 && n_subs >= HXC_LINES_MIN_SUBS) {
    // many sub-simulations: per-axis line kernels over all of them (the FP64
    // work of one grid per CTA would occupy only n_subs SMs)
    const int thr = 256;
    const unsigned blocks = (unsigned)((total + thr - 1) / thr);
    const int nn[3] = {c.n1, c.n2, c.n3};
    const int strides[3] = {1, c.n1, c.n1 * c.n2};
    k_hxc_load<<<blocks, thr, 0, st>>>(subs_dev, sub_ids_dev, n_subs, c.npts, wa);
    for (int ax = 0; ax < 3; ++ax) launch_fft_lines(wa, n_subs, c.npts, nn[ax], strides[ax], tw[ax], -1, st);
    k_poisson<<<blocks, thr, 0, st>>>(wa, total, c);
    for (int ax = 2; ax >= 0; --ax) launch_fft_lines(wa, n_subs, c.npts, nn[ax], strides[ax], tw[ax], +1, st);
    k_hxc_final<T><<<blocks, thr, 0, st>>>(subs_dev, sub_ids_dev, n_subs, c, wa);
    return 9;
  }
  if (pow2 && c.npts <= HXC_FFT_MAXPTS) {
    const size_t sm = (size_t)c.npts * sizeof(double2);
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_hxc_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_hxc_fft<<<n_subs, 256, sm, st>>>(subs_dev, sub_ids_dev, c, tw[0], tw[1], tw[2], wa);
    k_hxc_final<T><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(subs_dev, sub_ids_dev, n_subs, c, wa);
    return 2;
  }
  const int thr = 256;
  const unsigned blocks = (unsigned)((total + thr - 1) / thr);
  int launches = 0;
  k_hxc_load<<<blocks, thr, 0, st>>>(subs_dev, sub_ids_dev, n_subs, c.npts, wa);
  ++launches;
  const int nn[3] = {c.n1, c.n2, c.n3};
  const int strides[3] = {1, c.n1, c.n1 * c.n2};
  double2* a = wa;
  double2* b = wb;
  for (int ax = 0; ax < 3; ++ax) {
    k_dft_axis<<<blocks, thr, 0, st>>>(a, b, total, c.npts, strides[ax], nn[ax], tw[ax], -1);
    double2* t = a; a = b; b = t;
    ++launches;
  }
  k_poisson<<<blocks, thr, 0, st>>>(a, total, c);
  ++launches;
  for (int ax = 0; ax < 3; ++ax) {
    k_dft_axis<<<blocks, thr, 0, st>>>(a, b, total, c.npts, strides[ax], nn[ax], tw[ax], +1);
    double2* t = a; a = b; b = t;
    ++launches;
  }
  k_hxc_final<T><<<blocks, thr, 0, st>>>(subs_dev, sub_ids_dev, n_subs, c, a);
  ++launches;
  return launches;
}

template <typename T> void launch_convert_in_t(const double2* src, void* dst, long long n, void* stream) {
  using V = typename Cplx<T>::type;
  if (n == 0) return;
  k_convert_in<T><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src, (V*)dst, n);
}

template <typename T> void launch_convert_out_t(const void* src, double2* dst, long long n, void* stream) {
  using V = typename Cplx<T>::type;
  if (n == 0) return;
  k_convert_out<T><<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const V*)src, dst, n);
}

template <typename T> void launch_veff_frozen_t(const SubDev* subs_dev, int s, const CellDev& c, void* stream) {
  k_veff_frozen<T><<<(c.npts + 255) / 256, 256, 0, (cudaStream_t)stream>>>(subs_dev, s, c);
}
