// Single-precision Taylor stage for cells whose grid rows hold 32 points and
// whose atoms fall into at most 8 z groups (cell B: 32^3, 64 atoms in 8
// groups): a z-march over slabs of 8 rows.
//
// One CTA per (unit, band, slab of 8 rows), one thread per (x, y) column of the
// slab.  The band of t_{m-1} streams through a ring of 8 plane slabs in shared
// memory: 8 rows plus 4 halo rows on each side (periodic in y), each slot
// filled by bulk copies that complete on its own mbarrier (bounded waits).
// The thread keeps t(z - 4 .. z + 4) of its column in registers, so the z
// neighbours of the star stencil come from registers and the x and y
// neighbours from the staged plane.
//
// Stage m of the Taylor recurrence (Eq. 5 with Eq. 2's h):
//   t_m = (-i dt / m) [ -1/2 lap t - i q.grad t + (|q|^2/2 + v_eff) t + V_NL t ]
//   m = 1: write t_1;  m = 2: write t_2, psi += t_1 + t_2;  m = 3: write t_3,
//   psi += t_3;  m = 4: psi += t_4  (t = t_{m-1}, t_0 = psi).
//
// Non-local term, factorised by z group.  For the atoms a of group g (the same
// z rows of the Gaussian factor g_z, the displacement d_z and the phase ph_z):
//   (V_NL t)(x, y, z) = sum_g f_g(z) [C_g0(x, y) + d_g(z) C_g1(x, y)],
//   f_g(z) = g_z(z) conj(ph_z(z)),
//   C_g0 = sum_{a in g} g_x g_y conj(ph_x ph_y) (W_a,s + d_x W_a,px + d_y W_a,py),
//   C_g1 = sum_{a in g} g_x g_y conj(ph_x ph_y) W_a,pz,
// with W_aj = pnorm_j E_j P_aj and P the projections of t_{m-1}.  The C of the
// thread's column are formed once per stage in registers; f_g and d_g per
// (group, plane) are tabulated in shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "tsbz.h"
#include "tsbz_bulk.cuh"
#include "tsbz_internal.h"
#include "tsbz_zmarch.cuh"

#define SL_N1 32                      // points per grid row
#define SL_SY 8                       // rows per slab
#define SL_ND ZM_ND                   // stencil half-width (4)
#define SL_RY (SL_SY + 2 * SL_ND)     // rows of a staged plane slab
#define SL_PL (SL_RY * SL_N1)         // complex values per staged plane slab
#define SL_R 8                        // ring slots (power of two, >= 8)
#define SL_G 8                        // most z groups
#define SL_MAXZ 64                    // most planes
#define SL_T (SL_SY * SL_N1)          // threads per CTA

namespace {

struct SlSmem {
  float2 ring[SL_R][SL_PL];   // t_{m-1}: the slab's rows with their halo
  float2 pr[SL_R][SL_T];      // psi on the slab's rows (stages m >= 2)
  float vr[SL_R][SL_T];       // v_eff on the slab's rows
  float4 fz[SL_G][SL_MAXZ];   // (Re f_g, Im f_g, d_g, 0) per (group, plane)
  float4 xt[64][SL_N1];       // (Re g_x ph_x, Im g_x ph_x, d_x, g_x) per (atom, x)
  float4 yt[64][SL_SY];       // the same in y on the slab's rows
  float2 wt[64][4];           // W_aj = pnorm_j E_j P_aj
  unsigned long long bar[SL_R];
};

__device__ __forceinline__ float2 sl_cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Ring slot of plane p (p = -SL_ND .. n3 - 1 + SL_ND) and the parity of its fill.
__device__ __forceinline__ int sl_slot(int p) { return (p + SL_ND) & (SL_R - 1); }
__device__ __forceinline__ uint32_t sl_parity(int p) { return (uint32_t)((p + SL_ND) / SL_R) & 1u; }

// Thread 0: stage plane p (periodic in z) of the band into its slot: rows
// slab * SL_SY - SL_ND .. + SL_RY - 1 (periodic in y; n2 >= 16, so at most two
// contiguous pieces, each a whole number of 256-byte rows); for the planes the
// march computes (0 <= p < n3), also v_eff and, when pband is given, psi on
// the slab's own rows.
__device__ __forceinline__ void sl_issue(SlSmem& sm, const float2* band, const float2* pband, const float* veff,
                                         int p, int slab, int n2, int n3) {
  const int s = sl_slot(p);
  const uint32_t bar = bk_smem(&sm.bar[s]);
  const bool own = p >= 0 && p < n3;
  constexpr uint32_t own_c = SL_T * (uint32_t)sizeof(float2), own_v = SL_T * (uint32_t)sizeof(float);
  bk_mbar_expect_tx(bar, SL_PL * (uint32_t)sizeof(float2) + (own ? own_v + (pband ? own_c : 0u) : 0u));
  if (own) {
    const long long o = ((long long)p * n2 + slab * SL_SY) * SL_N1;
    bk_copy_g2s(bk_smem(sm.vr[s]), veff + o, own_v, bar);
    if (pband) bk_copy_g2s(bk_smem(sm.pr[s]), pband + o, own_c, bar);
  }
  const int pz = ((p % n3) + n3) % n3;
  const float2* src = band + (long long)pz * SL_N1 * n2;
  float2* dst = sm.ring[s];
  const int r0 = slab * SL_SY - SL_ND;
  constexpr uint32_t row = SL_N1 * (uint32_t)sizeof(float2);
  if (r0 >= 0 && r0 + SL_RY <= n2) {
    bk_copy_g2s(bk_smem(dst), src + r0 * SL_N1, SL_RY * row, bar);
  } else if (r0 < 0) {
    const int k = -r0;   // rows n2 - k .. n2 - 1, then 0 .. SL_RY - k - 1
    bk_copy_g2s(bk_smem(dst), src + (n2 - k) * SL_N1, k * row, bar);
    bk_copy_g2s(bk_smem(dst + k * SL_N1), src, (SL_RY - k) * row, bar);
  } else {
    const int k = n2 - r0;   // rows r0 .. n2 - 1, then 0 .. SL_RY - k - 1
    bk_copy_g2s(bk_smem(dst), src + r0 * SL_N1, k * row, bar);
    bk_copy_g2s(bk_smem(dst + k * SL_N1), src, (SL_RY - k) * row, bar);
  }
}

// Failure path: record the timeout and give every fill issued so far (planes
// -SL_ND .. last) one more bounded wait, so that no copy lands after the CTA
// has exited.
__device__ __forceinline__ void sl_bail(SlSmem& sm, int last, int* status) {
  if (threadIdx.x == 0) {
    atomicOr(status, BK_STATUS_TIMEOUT);
    for (int s = 0; s < SL_R; ++s) {
      const int p = last - ((last + SL_ND - s) & (SL_R - 1));
      if (p >= -SL_ND) bk_mbar_wait(bk_smem(&sm.bar[s]), sl_parity(p), BK_WAIT_POLLS);
    }
  }
}

// G: z groups covered (compile-time; the cell's groups beyond c.zs_n, if any,
// have no members and contribute zero).
template <int G>
__global__ void __launch_bounds__(SL_T, 2) k_stage_slab(LaunchSet L, const float2* __restrict__ tin,
                                                        float2* __restrict__ tout, float2* __restrict__ psi,
                                                        const float2* __restrict__ P, int m) {
  constexpr int ND = SL_ND;
  extern __shared__ __align__(128) unsigned char slraw[];
  SlSmem& sm = *reinterpret_cast<SlSmem*>(slraw);
  const CellDev& c = L.cell;
  const int n2 = c.n2, n3 = c.n3, nm = c.nmax, n12 = SL_N1 * n2;
  const int n_slabs = n2 / SL_SY;
  const int b = blockIdx.x / n_slabs, slab = blockIdx.x - b * n_slabs;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int tid = threadIdx.x, ix = tid & (SL_N1 - 1), ry = tid / SL_N1, iy = slab * SL_SY + ry;
  const long long base = U.psi_off + (long long)b * c.npts;
  const float2* band = tin + base;
  const float2* pband = m >= 2 ? psi + base : nullptr;
  const float* veff = reinterpret_cast<const float*>(S.veff);
  if (tid == 0) {
    for (int s = 0; s < SL_R; ++s) bk_mbar_init(bk_smem(&sm.bar[s]), 1);
    // planes -4 .. SL_R - 5 (never beyond the last plane the march reads, n3 + 3)
    for (int p = -ND; p < SL_R - ND && p <= n3 - 1 + ND; ++p) sl_issue(sm, band, pband, veff, p, slab, n2, n3);
  }
  // f_g(z), d_g(z) of the unit (the phase rows at q = k + A(t_n + dt/2))
  const float2* ph = (const float2*)L.ph_half + (long long)u * L.ph_stride;
  for (int i = tid; i < SL_G * n3; i += SL_T) {
    const int g = i / n3, z = i - g * n3;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g < c.zs_n) {
      const int a = c.zs_mem[c.zs_off[g]];
      const long long o = (long long)(a * 3 + 2) * nm + z;
      const float gz = c.g1f[o];
      const float2 pz = ph[o];
      e = make_float4(gz * pz.x, -gz * pz.y, c.d1f[o], 0.f);
    }
    sm.fz[g][z] = e;
  }
  // per-atom factor rows in x (all columns) and y (the slab's rows), and W, for
  // the non-local coefficients below (coalesced loads, then shared memory)
  const int na = c.use_proj ? c.n_atoms : 0;
  if (na) {
    const float2* Pb = P + U.p_off + (long long)b * c.n_proj;
    for (int i = tid; i < na * SL_N1; i += SL_T) {
      const int a = i / SL_N1, x = i - a * SL_N1;
      const long long o = (long long)(a * 3) * nm + x;
      const float g = c.g1f[o];
      const float2 q = ph[o];
      sm.xt[a][x] = make_float4(g * q.x, g * q.y, c.d1f[o], g);
    }
    for (int i = tid; i < na * SL_SY; i += SL_T) {
      const int a = i / SL_SY, r = i - a * SL_SY;
      const long long o = (long long)(a * 3 + 1) * nm + slab * SL_SY + r;
      const float g = c.g1f[o];
      const float2 q = ph[o];
      sm.yt[a][r] = make_float4(g * q.x, g * q.y, c.d1f[o], g);
    }
    for (int i = tid; i < 4 * na; i += SL_T) {
      const float2 p = Pb[i];
      const float w = c.wkbf[i];
      sm.wt[i >> 2][i & 3] = make_float2(w * p.x, w * p.y);
    }
  }
  const float* qt = reinterpret_cast<const float*>(L.qt_half) + 4 * u;
  const float q0 = qt[0], q1 = qt[1], q2 = qt[2];
  const float dg0 = c.hlapf[0][0] + c.hlapf[1][0] + c.hlapf[2][0] + qt[3];
  const float hdt = (float)(S.dt * L.dt_scale) / (float)m;
  const long long off = (long long)iy * SL_N1 + ix;
  float2* to = tout + base + off;
  float2* po = psi + base + off;
  const float2 zero = make_float2(0.f, 0.f);
  const int me = (ry + ND) * SL_N1 + ix;   // this column in a staged plane slab
  int xo[2 * ND];                          // x neighbours ix + mm, ix - mm within the row
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) {
    xo[mm - 1] = (ry + ND) * SL_N1 + ((ix + mm) & (SL_N1 - 1));
    xo[ND + mm - 1] = (ry + ND) * SL_N1 + ((ix - mm) & (SL_N1 - 1));
  }
  __syncthreads();   // the barriers are initialised and the tables written before anyone reads them
  // C_g0, C_g1 of this column from the projections of t_{m-1}
  float2 C0[G > 0 ? G : 1], C1[G > 0 ? G : 1];
#pragma unroll
  for (int g = 0; g < (G > 0 ? G : 1); ++g) C0[g] = C1[g] = make_float2(0.f, 0.f);
  if (na) {
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if (g >= c.zs_n) break;
      for (int j = c.zs_off[g]; j < c.zs_off[g + 1]; ++j) {
        const int a = c.zs_mem[j];
        const float4 ey = sm.yt[a][ry];   // the same for the whole warp (one grid row)
        if (ey.w == 0.f) continue;         // the row is outside the atom's projector box
        const float4 ex = sm.xt[a][ix];
        if (ex.w == 0.f) continue;         // the column is outside it in x
        // g_x g_y conj(ph_x ph_y) = conj(e_x e_y), e = g ph
        const float2 exy = sl_cmul(make_float2(ex.x, ex.y), make_float2(ey.x, ey.y));
        const float2 f = make_float2(exy.x, -exy.y);
        const float2 w0 = sm.wt[a][0], w1 = sm.wt[a][1], w2 = sm.wt[a][2], w3 = sm.wt[a][3];
        const float2 w = make_float2(w0.x + ex.z * w1.x + ey.z * w2.x, w0.y + ex.z * w1.y + ey.z * w2.y);
        const float2 a0 = sl_cmul(f, w), a1 = sl_cmul(f, w3);
        C0[g].x += a0.x;
        C0[g].y += a0.y;
        C1[g].x += a1.x;
        C1[g].y += a1.y;
      }
    }
  }
  // the queue t(z - 4 .. z + 4) of this column: planes -4 .. 3 first (slots 0 .. 7, the first fill)
  float2 qv[2 * ND + 1];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 2 * ND; ++k) {
    ok = ok && bk_mbar_wait(bk_smem(&sm.bar[k]), 0, BK_WAIT_POLLS);
    qv[k] = sm.ring[k][me];
  }
  if (!__syncthreads_and(ok)) {
    sl_bail(sm, min(SL_R - ND - 1, n3 - 1 + ND), S.status);
    return;
  }
  // slots 0 .. 3 (planes -4 .. -1, read) take planes SL_R - 4 .. SL_R - 1
  if (tid == 0)
    for (int p = SL_R - ND; p < SL_R && p <= n3 - 1 + ND; ++p) sl_issue(sm, band, pband, veff, p, slab, n2, n3);
  int last = min(SL_R - 1, n3 - 1 + ND);   // last plane issued
  const float2 neg1 = make_float2(-1.f, -1.f);
  static_assert(SL_R == 8, "the unrolled march names ring slots by zz");
#pragma unroll 1
  for (int z0 = 0; z0 < n3; z0 += SL_R) {
#pragma unroll
    for (int zz = 0; zz < SL_R; ++zz) {
      const int z = z0 + zz;
      // plane z + 4 (slot zz: z0 is a multiple of SL_R = 8) completes the queue;
      // plane z (slot zz + 4) gives the x and y neighbours, v_eff and psi
      const int sq = zz, sz = (zz + ND) & (SL_R - 1);
      const bool okw = bk_mbar_wait(bk_smem(&sm.bar[sq]), sl_parity(z + ND), BK_WAIT_POLLS);
      qv[2 * ND] = sm.ring[sq][me];
      const float2* pl = sm.ring[sz];
      const float2 ce = qv[ND];
      const float dg = dg0 + sm.vr[sz][tid];
      float2 h = __fmul2_rn(make_float2(dg, dg), ce);
      float2 gx = zero, gy = zero, gz = zero;
#pragma unroll
      for (int mm = 1; mm <= ND; ++mm) {
        const float2 xu = pl[xo[mm - 1]], xd = pl[xo[ND + mm - 1]];
        const float2 yu = pl[me + mm * SL_N1], yd = pl[me - mm * SL_N1];
        const float2 zu = qv[ND + mm], zd = qv[ND - mm];
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
      // V_NL t at (x, y, z)
      float2 vn = zero;
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const float4 f = sm.fz[g][z];
        const float2 t = make_float2(C0[g].x + f.z * C1[g].x, C0[g].y + f.z * C1[g].y);
        vn.x += f.x * t.x - f.y * t.y;
        vn.y += f.x * t.y + f.y * t.x;
      }
      const float hr = h.x + qg.y + vn.x;
      const float hi = h.y - qg.x + vn.y;
      const float2 t = make_float2(hdt * hi, -hdt * hr);
      const long long o = (long long)z * n12;
      if (m < 4) to[o] = t;
      if (m == 2) {
        po[o] = __fadd2_rn(sm.pr[sz][tid], __fadd2_rn(ce, t));
      } else if (m >= 3) {
        po[o] = __fadd2_rn(sm.pr[sz][tid], t);
      }
#pragma unroll
      for (int k = 0; k < 2 * ND; ++k) qv[k] = qv[k + 1];
      // every thread is done with plane z: its slot takes plane z + SL_R
      if (__syncthreads_or(!okw)) {
        sl_bail(sm, last, S.status);
        return;
      }
      if (z + SL_R <= n3 - 1 + ND) {
        if (tid == 0) sl_issue(sm, band, pband, veff, z + SL_R, slab, n2, n3);
        last = z + SL_R;
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Projections P[u][b][j] of a band on the slab layout (the bra of Eq. 2's
// non-local term, q = k + A(t_n + dt/2)):
//   P_aj = dV pn_j sum_r g(r) ph(r) mono_j(d(r)) t(r),  mono = 1, d_x, d_y, d_z,
// factorised by z group: per column the z sums
//   S_gk(x, y) = sum_z g_z(z) ph_z(z) d_z(z)^k t(x, y, z)   (k = 0, 1),
// then per atom and slab row the x sums
//   R_a,00 = sum_x g_x ph_x S_g0,  R_a,01 = sum_x g_x ph_x d_x S_g0,
//   R_a,10 = sum_x g_x ph_x S_g1,
// then per atom the y sums: P_s = sum_y w R_00, P_px = sum_y w R_01,
// P_py = sum_y w d_y R_00, P_pz = sum_y w R_10 with w = g_y ph_y.  One CTA per
// (unit, band, slab); the slabs of a band form one thread-block cluster, and
// its first CTA adds the slabs' partial projections from distributed shared
// memory in slab order.
// ----------------------------------------------------------------------------
// KD z moments per column: 2 for P (monomials 1, d_x, d_y, d_z), 3 for the
// current's Pa (the monomials of degree <= 2: each projector monomial times
// 1, d_x, d_y, d_z).  NX x sums per (atom, row): the (z power k, x power i)
// with i + k < KD.
template <int KD> struct SbSmem {
  static constexpr int NX = KD == 2 ? 3 : 6;
  static constexpr int NOUT = KD == 2 ? 4 : 16;   // outputs per atom
  float4 fb[SL_G][SL_MAXZ];      // (Re g_z ph_z, Im g_z ph_z, d_z, 0) per (group, plane)
  float2 S[KD * SL_G][SL_T];     // z sums of the columns
  float2 R[64][SL_SY][NX];       // x sums per (atom, slab row)
  float2 Pp[NOUT * 64];          // this slab's partial projections
  int grp[64];                   // z group of each atom
};

// a b in explicitly rounded operations (no contraction left to the compiler)
__device__ __forceinline__ float2 sb_cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}

// x-sum index of (z power k, x power i)
template <int KD> __device__ __forceinline__ int sb_xterm(int k, int i) {
  if (KD == 2) return k == 0 ? i : 2;
  return k == 0 ? i : (k == 1 ? 3 + i : 5);
}

// pnext (three z moments only, may be null): also write the first-weight
// entries Pa_aj,0 = P_aj into P, the projections the next step starts from when
// the field is constant (q at t_{n+1} and at t_{n+1} + dt/2 are then the same,
// and these entries are formed by the same operations as the two-moment pass).
template <int G, int KD>
__global__ void __launch_bounds__(SL_T) k_bra_slab(LaunchSet L, const float2* __restrict__ src,
                                                   float2* __restrict__ out, float2* __restrict__ pnext,
                                                   int use_obs) {
  namespace cg = cooperative_groups;
  using Sm = SbSmem<KD>;
  constexpr int D = 8;   // planes of t loaded ahead
  extern __shared__ __align__(16) unsigned char sbraw[];
  Sm& sm = *reinterpret_cast<Sm*>(sbraw);
  const CellDev& c = L.cell;
  const int n2 = c.n2, n3 = c.n3, nm = c.nmax, n12 = SL_N1 * n2, na = c.n_atoms;
  const int n_slabs = n2 / SL_SY;
  const int b = blockIdx.x / n_slabs, slab = blockIdx.x - b * n_slabs;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;   // the same for every CTA of the cluster (one unit)
  const UnitDev U = L.units[u];
  const int tid = threadIdx.x, ix = tid & (SL_N1 - 1), ry = tid / SL_N1, iy = slab * SL_SY + ry;
  const float2* ph = (const float2*)(use_obs ? L.ph_obs : L.ph_half) + (long long)u * L.ph_stride;
  for (int i = tid; i < SL_G * n3; i += SL_T) {
    const int g = i / n3, z = i - g * n3;
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
    if (g < c.zs_n) {
      const int a = c.zs_mem[c.zs_off[g]];
      const long long o = (long long)(a * 3 + 2) * nm + z;
      const float gz = c.g1f[o];
      const float2 pz = ph[o];
      e = make_float4(gz * pz.x, gz * pz.y, c.d1f[o], 0.f);
    }
    sm.fb[g][z] = e;
  }
  for (int g = 0; g < c.zs_n; ++g)
    for (int j = c.zs_off[g] + tid; j < c.zs_off[g + 1]; j += SL_T) sm.grp[c.zs_mem[j]] = g;
  __syncthreads();
  // z sums of this column: S_gk = sum_z g_z ph_z d_z^k t
  const float2* col = src + U.psi_off + (long long)b * c.npts + (long long)iy * SL_N1 + ix;
  float2 Sk[KD][G];
#pragma unroll
  for (int k = 0; k < KD; ++k)
#pragma unroll
    for (int g = 0; g < G; ++g) Sk[k][g] = make_float2(0.f, 0.f);
  float2 tq[D];
#pragma unroll
  for (int k = 0; k < D; ++k) tq[k] = col[(long long)k * n12];
#pragma unroll 1
  for (int z0 = 0; z0 < n3; z0 += D) {
#pragma unroll
    for (int zz = 0; zz < D; ++zz) {
      const int z = z0 + zz;
      const float2 t = tq[zz];
      if (z + D < n3) tq[zz] = col[(long long)(z + D) * n12];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const float4 f = sm.fb[g][z];
        if (f.x == 0.f && f.y == 0.f) continue;   // plane z is outside the group's box (uniform)
        // every rounding spelled out: the two- and three-moment passes form the
        // moments they share by the same operations, bit for bit
        float2 ft = sb_cmul(make_float2(f.x, f.y), t);
#pragma unroll
        for (int k = 0; k < KD; ++k) {
          Sk[k][g].x = __fadd_rn(Sk[k][g].x, ft.x);
          Sk[k][g].y = __fadd_rn(Sk[k][g].y, ft.y);
          ft = make_float2(__fmul_rn(f.z, ft.x), __fmul_rn(f.z, ft.y));
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < KD; ++k)
#pragma unroll
    for (int g = 0; g < G; ++g) sm.S[k * G + g][tid] = Sk[k][g];
  __syncthreads();
  // x sums per (atom, slab row) over the atom's box columns [sx, sx + lx) (periodic):
  // R_(k,i) = sum_x g_x ph_x d_x^i S_gk
  for (int j = tid; j < na * SL_SY; j += SL_T) {
    const int a = j / SL_SY, r = j - a * SL_SY;
    const int g = sm.grp[a];
    const int* bx = c.pbox + a * 6;
    const int sx = bx[0], lx = bx[1], sy = bx[2], ly = bx[3];
    float2 rr[Sm::NX];
#pragma unroll
    for (int e = 0; e < Sm::NX; ++e) rr[e] = make_float2(0.f, 0.f);
    if (((slab * SL_SY + r - sy) % n2 + n2) % n2 < ly) {   // the row is in the atom's box
      for (int i = 0; i < lx; ++i) {
        const int x = (sx + i) & (SL_N1 - 1);
        const long long ox = (long long)(a * 3) * nm + x;
        const float gx = c.g1f[ox];
        const float2 px = ph[ox];
        const float dx = c.d1f[ox];
#pragma unroll
        for (int k = 0; k < KD; ++k) {
          const float2 sv = sm.S[k * G + g][r * SL_N1 + x];
          const float2 pv = sb_cmul(px, sv);
          float2 w = make_float2(__fmul_rn(gx, pv.x), __fmul_rn(gx, pv.y));
#pragma unroll
          for (int ip = 0; ip + k < KD; ++ip) {
            const int e = sb_xterm<KD>(k, ip);
            rr[e].x = __fadd_rn(rr[e].x, w.x);
            rr[e].y = __fadd_rn(rr[e].y, w.y);
            w = make_float2(__fmul_rn(dx, w.x), __fmul_rn(dx, w.y));
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < Sm::NX; ++e) sm.R[a][r][e] = rr[e];
  }
  __syncthreads();
  // y sums: this slab's part of every output (P_aj, or Pa_aj,alpha)
  for (int j = tid; j < Sm::NOUT * na; j += SL_T) {
    const int a = j / Sm::NOUT, o = j - a * Sm::NOUT;
    const int tt = KD == 2 ? o : o >> 2, al = KD == 2 ? 0 : o & 3;
    // exponents of the monomial: the projector's (tt) plus the weight's (al)
    const int ei = (tt == 1) + (al == 1), ej = (tt == 2) + (al == 2), ek = (tt == 3) + (al == 3);
    const int e = sb_xterm<KD>(ek, ei);
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < SL_SY; ++r) {
      const long long oy = (long long)(a * 3 + 1) * nm + slab * SL_SY + r;
      const float gy = c.g1f[oy];
      if (gy == 0.f) continue;
      const float2 py = ph[oy];
      float wy = gy;
      for (int q = 0; q < ej; ++q) wy = __fmul_rn(wy, c.d1f[oy]);
      const float2 v = sm.R[a][r][e];
      const float2 pv = sb_cmul(py, v);
      acc.x = __fadd_rn(acc.x, __fmul_rn(wy, pv.x));
      acc.y = __fadd_rn(acc.y, __fmul_rn(wy, pv.y));
    }
    const float sc = (float)c.dv * c.pnormf[4 * a + tt];
    sm.Pp[j] = make_float2(sc * acc.x, sc * acc.y);
  }
  // the slabs' parts, added in slab order by the cluster's first CTA
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  if (cl.block_rank() == 0) {
    float2* ob = KD == 2 ? out + U.p_off + (long long)b * c.n_proj : out + U.pa_off + (long long)b * c.n_proj * 4;
    for (int j = tid; j < Sm::NOUT * na; j += SL_T) {
      float2 v = make_float2(0.f, 0.f);
      for (int r = 0; r < n_slabs; ++r) {
        const float2 w = cl.map_shared_rank(sm.Pp, r)[j];
        v.x += w.x;
        v.y += w.y;
      }
      ob[j] = v;
      if (KD == 3 && pnext != nullptr && (j & 3) == 0) pnext[U.p_off + (long long)b * c.n_proj + (j >> 2)] = v;
    }
  }
  cl.sync();   // the other CTAs keep their shared memory until it has been read
}

// ----------------------------------------------------------------------------
// Observation on the slab layout: one CTA per (unit, band group of TSBZ_BG
// bands, slab of 8 rows, block of SO_ZP planes), one thread per column of the
// slab.  The bands of the group stream through a ring of plane slabs (the
// slab's rows and the next 4 rows, periodic in y; the block's planes and the
// next 4, periodic in z) filled by bulk copies in one continuous sequence
// q = band * (SO_ZP + 4) + plane.  Per
// point it adds occ |u|^2 to the group's density (two-sum in float), and for
// the current's local part the forward correlations
//   sum_r Im(conj(u(r)) u(r + m e_ax)),  m = 1 .. 4
// (z neighbours from a register queue, x and y from the staged plane); per band
// the norm.  The density sums over the group's bands in float per point, as the
// point-parallel form does; the current sums over bands with two-sums.
// Outputs: rho_part of the group on the block's points, jk_part and nrm_part of
// point tile slab * (n3 / SO_ZP) + block (zeros in the tiles beyond them).
// ----------------------------------------------------------------------------
#define SO_RY (SL_SY + SL_ND)          // staged rows: the slab's and 4 forward
#define SO_PL (SO_RY * SL_N1)
#define SO_R 8                         // ring slots
#define SO_ZP 8                        // planes per CTA

struct SoSmem {
  float2 ring[SO_R][SO_PL];
  float nrm[SL_T / 32][TSBZ_BG];
  double redj[SL_T / 32][3];
  unsigned long long bar[SO_R];
};

// Thread 0: stage sequence element q (band q / (SO_ZP + 4), plane z0 + q % (SO_ZP + 4)).
__device__ __forceinline__ void so_issue(SoSmem& sm, const float2* gbase, long long q, int slab, int z0, int n2,
                                         int n3, int npts) {
  constexpr int np = SO_ZP + SL_ND;
  const int bl = (int)(q / np), p = z0 + (int)(q - (long long)bl * np);
  const int s = (int)(q & (SO_R - 1));
  const uint32_t bar = bk_smem(&sm.bar[s]);
  constexpr uint32_t row = SL_N1 * (uint32_t)sizeof(float2);
  bk_mbar_expect_tx(bar, SO_RY * row);
  const float2* src = gbase + (long long)bl * npts + (long long)(p % n3) * SL_N1 * n2;
  float2* dst = sm.ring[s];
  const int r0 = slab * SL_SY;
  if (r0 + SO_RY <= n2) {
    bk_copy_g2s(bk_smem(dst), src + r0 * SL_N1, SO_RY * row, bar);
  } else {
    const int k = n2 - r0;   // rows r0 .. n2 - 1, then 0 .. SO_RY - k - 1
    bk_copy_g2s(bk_smem(dst), src + r0 * SL_N1, k * row, bar);
    bk_copy_g2s(bk_smem(dst + k * SL_N1), src, (SO_RY - k) * row, bar);
  }
}

__device__ __forceinline__ uint32_t so_parity(long long q) { return (uint32_t)((q / SO_R) & 1); }

__global__ void __launch_bounds__(SL_T, 3) k_observe_slab(LaunchSet L, const float2* __restrict__ psi,
                                                          double* __restrict__ rho_part, double* __restrict__ jk_part,
                                                          double* __restrict__ nrm_part) {
  constexpr int ND = SL_ND, NZ = SO_ZP, np = SO_ZP + SL_ND;
  extern __shared__ __align__(128) unsigned char soraw[];
  SoSmem& sm = *reinterpret_cast<SoSmem*>(soraw);
  const CellDev& c = L.cell;
  const int n2 = c.n2, n3 = c.n3, n12 = SL_N1 * n2, npts = c.npts;
  const int n_slabs = n2 / SL_SY, n_zb = n3 / SO_ZP, n_pt = n_slabs * n_zb;   // point tiles of the kernel
  const int grp = blockIdx.x / n_pt, pt = blockIdx.x - grp * n_pt;
  const int slab = pt / n_zb, zb = pt - slab * n_zb, z0 = zb * SO_ZP;
  const int u = L.unit_ids[blockIdx.y];
  if (!unit_active(L, u)) return;
  const UnitDev U = L.units[u];
  const SubDev S = L.subs[U.sub];
  const int tid = threadIdx.x, ix = tid & (SL_N1 - 1), ry = tid / SL_N1, lane = tid & 31, warp = tid >> 5;
  const int b0 = grp * TSBZ_BG, nbg = min(TSBZ_BG, c.n_bands - b0);
  const float2* gbase = psi + U.psi_off + (long long)b0 * npts;
  const long long qend = (long long)nbg * np;   // sequence elements of the group
  if (tid == 0) {
    for (int k = 0; k < SO_R; ++k) bk_mbar_init(bk_smem(&sm.bar[k]), 1);
    for (long long q = 0; q < SO_R && q < qend; ++q) so_issue(sm, gbase, q, slab, z0, n2, n3, npts);
  }
  __syncthreads();
  long long issued = qend < SO_R ? qend : SO_R;
  float rho[NZ];   // the group's density per plane of this column (float, as the point-parallel form)
#pragma unroll
  for (int z = 0; z < NZ; ++z) rho[z] = 0.f;
  float js[3] = {0.f, 0.f, 0.f}, je[3] = {0.f, 0.f, 0.f};
  const int me = ry * SL_N1 + ix;
  int xo[ND];
#pragma unroll
  for (int mm = 1; mm <= ND; ++mm) xo[mm - 1] = ry * SL_N1 + ((ix + mm) & (SL_N1 - 1));
  bool ok = true;
  // release the slot of sequence element q (every thread is done with it) and
  // stage element q + SO_R there
  auto release = [&](long long q) -> bool {
    const bool fail = __syncthreads_or(!ok);
    if (fail) return false;
    if (q + SO_R < qend) {
      if (tid == 0) so_issue(sm, gbase, q + SO_R, slab, z0, n2, n3, npts);
      issued = q + SO_R + 1;
    }
    return true;
  };
  bool alive = true;
  for (int bl = 0; bl < nbg && alive; ++bl) {
    const long long q0 = (long long)bl * np;
    float2 qv[2 * ND + 1];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      ok = ok && bk_mbar_wait(bk_smem(&sm.bar[(q0 + k) & (SO_R - 1)]), so_parity(q0 + k), BK_WAIT_POLLS);
      qv[k] = sm.ring[(q0 + k) & (SO_R - 1)][me];
    }
    float nbs = 0.f;
    float cx[ND], cy[ND], cz[ND];
#pragma unroll
    for (int mm = 0; mm < ND; ++mm) cx[mm] = cy[mm] = cz[mm] = 0.f;
    // the plane loop is unrolled, so that rho[z] is a register
#pragma unroll
    for (int z = 0; z < NZ; ++z) {
      {
        const long long qz = q0 + z, qn = qz + ND;
        ok = ok && bk_mbar_wait(bk_smem(&sm.bar[qn & (SO_R - 1)]), so_parity(qn), BK_WAIT_POLLS);
        qv[ND] = sm.ring[qn & (SO_R - 1)][me];
        const float2* pl = sm.ring[qz & (SO_R - 1)];
        const float2 ce = qv[0];
#pragma unroll
        for (int mm = 1; mm <= ND; ++mm) {
          const float2 xu = pl[xo[mm - 1]], yu = pl[me + mm * SL_N1], zu = qv[mm];
          // Im(conj(u) v) = u_r v_i - u_i v_r
          cx[mm - 1] = __fmaf_rn(ce.x, xu.y, __fmaf_rn(-ce.y, xu.x, cx[mm - 1]));
          cy[mm - 1] = __fmaf_rn(ce.x, yu.y, __fmaf_rn(-ce.y, yu.x, cy[mm - 1]));
          cz[mm - 1] = __fmaf_rn(ce.x, zu.y, __fmaf_rn(-ce.y, zu.x, cz[mm - 1]));
        }
        const float n2v = ce.x * ce.x + ce.y * ce.y;
        rho[z] += n2v;
        nbs += n2v;
#pragma unroll
        for (int k = 0; k < 2 * ND; ++k) qv[k] = qv[k + 1];
        if (!release(qz)) alive = false;
      }
      if (!alive) break;
    }
    if (!alive) break;
    // the 4 planes after the block are done too
    for (int k = 0; k < ND && alive; ++k) alive = release(q0 + NZ + k);
    if (!alive) break;
    float bx = 0.f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int mm = 1; mm <= ND; ++mm) {
      bx = __fmaf_rn(2.f * c.gradwf[0][mm], cx[mm - 1], bx);
      by = __fmaf_rn(2.f * c.gradwf[1][mm], cy[mm - 1], by);
      bz = __fmaf_rn(2.f * c.gradwf[2][mm], cz[mm - 1], bz);
    }
    const float bv[3] = {bx, by, bz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const float t = js[ax] + bv[ax], bb = t - js[ax];
      je[ax] += (js[ax] - (t - bb)) + (bv[ax] - bb);
      js[ax] = t;
    }
    for (int off = 16; off > 0; off >>= 1) nbs += __shfl_xor_sync(0xffffffffu, nbs, off);
    if (lane == 0) sm.nrm[warp][bl] = nbs;
  }
  if (!alive || !ok) {
    if (tid == 0) {
      atomicOr(S.status, BK_STATUS_TIMEOUT);
      // let every issued copy land before the CTA's shared memory is released
      for (long long q = issued > SO_R ? issued - SO_R : 0; q < issued; ++q)
        bk_mbar_wait(bk_smem(&sm.bar[q & (SO_R - 1)]), so_parity(q), BK_WAIT_POLLS);
    }
    return;
  }
  // density of the group on the block's points
  const long long pbase = (long long)slab * SL_SY * SL_N1 + me;
#pragma unroll
  for (int z = 0; z < NZ; ++z)
    rho_part[U.rho_off + (long long)grp * npts + (long long)(z0 + z) * n12 + pbase] = c.occ * (double)rho[z];
  // the group's current over the slab's points, in warp order
  double jd[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    jd[ax] = (double)js[ax] + (double)je[ax];
    for (int off = 16; off > 0; off >>= 1) jd[ax] += __shfl_xor_sync(0xffffffffu, jd[ax], off);
  }
  if (lane == 0)
    for (int ax = 0; ax < 3; ++ax) sm.redj[warp][ax] = jd[ax];
  __syncthreads();
  if (tid < 3) {
    double sum = 0.0;
    for (int w = 0; w < SL_T / 32; ++w) sum += sm.redj[w][tid];
    jk_part[U.jk_off + ((long long)pt * c.n_bgroups + grp) * 3 + tid] = sum;
  }
  for (int bl = tid; bl < nbg; bl += SL_T) {
    double sum = 0.0;
    for (int w = 0; w < SL_T / 32; ++w) sum += (double)sm.nrm[w][bl];
    nrm_part[U.nrm_off + (long long)pt * c.n_bands + b0 + bl] = sum;
  }
  // tiles beyond the kernel's hold nothing of this group
  if (pt == 0) {
    for (int i = tid; i < (c.n_tiles - n_pt) * 3; i += SL_T) {
      const int t = n_pt + i / 3, ax = i - (i / 3) * 3;
      jk_part[U.jk_off + ((long long)t * c.n_bgroups + grp) * 3 + ax] = 0.0;
    }
    for (int i = tid; i < (c.n_tiles - n_pt) * nbg; i += SL_T) {
      const int t = n_pt + i / nbg, bl = i - (i / nbg) * nbg;
      nrm_part[U.nrm_off + (long long)t * c.n_bands + b0 + bl] = 0.0;
    }
  }
}

}  // namespace

bool slab_supported(const CellDev& c) {
  return c.n1 == SL_N1 && c.n2 >= 16 && c.n2 <= 8 * SL_SY && c.n2 % SL_SY == 0 && c.n3 % 8 == 0 && c.n3 >= 8 &&
         c.n3 <= SL_MAXZ && c.n_atoms <= 64 &&
         c.nd == SL_ND && (!c.use_proj || (c.zs_n > 0 && c.zs_n <= SL_G));
}

bool launch_stage_slab(const LaunchSet& L, const void* tin, void* tout, void* psi, const void* P, int m,
                       void* stream) {
  if (L.variant != 0 || !slab_supported(L.cell)) return false;
  if (L.n_units == 0) return true;
  const CellDev& c = L.cell;
  const size_t smem = sizeof(SlSmem);
  const dim3 grid(c.n_bands * (c.n2 / SL_SY), L.n_units);
  cudaStream_t st = (cudaStream_t)stream;
  const int g = c.use_proj ? c.zs_n : 0;
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, SL_T, smem, st>>>(L, (const float2*)tin, (float2*)tout, (float2*)psi, (const float2*)P, m);
  };
  if (g == 0) go(k_stage_slab<0>);
  else if (g == 1) go(k_stage_slab<1>);
  else if (g == 2) go(k_stage_slab<2>);
  else if (g <= 4) go(k_stage_slab<4>);
  else go(k_stage_slab<8>);
  return true;
}

bool launch_bra_slab(const LaunchSet& L, const void* src, void* out, int with_d, int use_obs, void* stream,
                     void* pnext) {
  const CellDev& c = L.cell;
  if (L.variant != 0 || !slab_supported(c) || !c.use_proj) return false;
  if (L.n_units == 0) return true;
  const int n_slabs = c.n2 / SL_SY;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.n_bands * n_slabs, L.n_units);
  cfg.blockDim = dim3(SL_T);
  cfg.stream = (cudaStream_t)stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = n_slabs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  auto go = [&](auto kern, size_t smem) {
    cfg.dynamicSmemBytes = smem;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaLaunchKernelEx(&cfg, kern, L, (const float2*)src, (float2*)out, with_d ? (float2*)pnext : nullptr, use_obs);
  };
  const int g = c.zs_n;
  if (with_d) {
    const size_t sm3 = sizeof(SbSmem<3>);
    if (g == 1) go(k_bra_slab<1, 3>, sm3);
    else if (g == 2) go(k_bra_slab<2, 3>, sm3);
    else if (g <= 4) go(k_bra_slab<4, 3>, sm3);
    else go(k_bra_slab<8, 3>, sm3);
  } else {
    const size_t sm2 = sizeof(SbSmem<2>);
    if (g == 1) go(k_bra_slab<1, 2>, sm2);
    else if (g == 2) go(k_bra_slab<2, 2>, sm2);
    else if (g <= 4) go(k_bra_slab<4, 2>, sm2);
    else go(k_bra_slab<8, 2>, sm2);
  }
  return true;
}

bool launch_observe_slab(const LaunchSet& L, const void* psi, double* rho_part, double* jk_part, double* nrm_part,
                         void* stream) {
  const CellDev& c = L.cell;
  const int n_pt = (c.n2 / SL_SY) * (c.n3 / SO_ZP);
  if (!slab_supported(c) || c.n3 % SO_ZP != 0 || c.n_tiles < n_pt) return false;
  if (L.n_units == 0) return true;
  const size_t smem = sizeof(SoSmem);
  cudaFuncSetAttribute(k_observe_slab, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const dim3 grid(c.n_bgroups * n_pt, L.n_units);
  k_observe_slab<<<grid, SL_T, smem, (cudaStream_t)stream>>>(L, (const float2*)psi, rho_part, jk_part, nrm_part);
  return true;
}
