// Kernels of the ground-state solver (FP64): Chebyshev-filtered subspace
// iteration for the n_bands lowest eigenvectors of h_k[v_eff] at A = 0, per
// k-point.  The filter steps run in the point-parallel stage kernel (m = 0);
// the kernels here orthonormalise the filtered block and bound its spectrum.
//
// The filtered block is very ill-conditioned (the filter amplifies the lowest
// occupied states by many orders of magnitude more than the highest), so it
// is orthonormalised by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa,
// Zhang, Yamamoto, SIAM J. Sci. Comput. 42 (2020)): one Cholesky-QR pass of
// the Gram matrix plus a small multiple of its trace on the diagonal, then two
// plain Cholesky-QR passes of the rotated block.  The bound of the block's
// spectrum (the largest Ritz value) comes from h applied to the final
// orthonormal block Q: carried through the ill-conditioned passes by
// congruence, C^H (Y^H h Y) C loses every digit in the directions that the
// filter left small.
//
// Per unit (k-point) with the block Y (n_b columns); the n_b x n_b matrices of
// unit i (row-major, pitch n_b) start at i n_b^2 in each buffer:
//   S = dV Y^H Y (and Hs = dV Y^H (h Y) when h Y is given)
//                                             (k_scf_gram, 32 x 32 band tiles)
//   S + s I = L L^H,  C = L^{-H}  (orthonormalisation pass), or
//   S = L L^H,  lam = largest eigenvalue of L^{-1} Hs L^{-H}  (bound pass)
//                                             (k_scf_ortho, one CTA per unit)
//   Y' = Y C                                  (k_scf_rotate, out of place)
#include <cuda_runtime.h>

#include "tsbz_internal.h"

#define SCF_MAXB 256   // bands a unit may have in the ground-state solver
#define SCF_T 32       // band tile edge of the Gram kernel
#define SCF_CH 16      // points per staged chunk of the Gram kernel
#define SCF_RB 16      // output bands per CTA of the rotation
#define SCF_OT 256     // threads of the factorisation kernel (>= SCF_MAXB)

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// One 32 x 32 tile (rows t1, columns t2) of S (and Hs when WH) of one unit per CTA
// (blockIdx.x = unit, blockIdx.y = t1 T + t2).  Bands t1 of Y and bands t2
// of Y and HY are staged in chunks of SCF_CH points (rows padded by one
// element: the column band varies across a warp); each thread accumulates
// four entries (rows r0, r0 + 8, r0 + 16, r0 + 24, column c) in point order.
template <bool WH>
__global__ void __launch_bounds__(256) k_scf_gram(LaunchSet L, const double2* __restrict__ Y,
                                                  const double2* __restrict__ HY, double2* __restrict__ Sout,
                                                  double2* __restrict__ Hout) {
  __shared__ double2 y1[SCF_T][SCF_CH + 1];
  __shared__ double2 y2[SCF_T][SCF_CH + 1];
  __shared__ double2 h2[SCF_T][SCF_CH + 1];
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  const UnitDev U = L.units[u];
  const int nb = c.n_bands, nt = (nb + SCF_T - 1) / SCF_T;
  const int t1 = blockIdx.y / nt, t2 = blockIdx.y % nt;
  const double2* yb = Y + U.psi_off;
  const double2* hb = HY + U.psi_off;
  const int col = threadIdx.x & 31, r0 = threadIdx.x >> 5;
  double2 sacc[4], hacc[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) sacc[q] = hacc[q] = make_double2(0.0, 0.0);
  const double2 z = make_double2(0.0, 0.0);
  for (int p0 = 0; p0 < c.npts; p0 += SCF_CH) {
    __syncthreads();
    for (int i = threadIdx.x; i < SCF_T * SCF_CH; i += blockDim.x) {
      const int b = i / SCF_CH, k = i % SCF_CH, p = p0 + k;
      const int g1 = t1 * SCF_T + b, g2 = t2 * SCF_T + b;
      const bool in = p < c.npts;
      y1[b][k] = in && g1 < nb ? yb[(long long)g1 * c.npts + p] : z;
      y2[b][k] = in && g2 < nb ? yb[(long long)g2 * c.npts + p] : z;
      if (WH) h2[b][k] = in && g2 < nb ? hb[(long long)g2 * c.npts + p] : z;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < SCF_CH; ++k) {
      const double2 a2 = y2[col][k], g2 = WH ? h2[col][k] : z;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 a1 = zconj(y1[r0 + 8 * q][k]);
        sacc[q] = zadd(sacc[q], zmul(a1, a2));
        if (WH) hacc[q] = zadd(hacc[q], zmul(a1, g2));
      }
    }
  }
  const int b2 = t2 * SCF_T + col;
  if (b2 >= nb) return;
  const long long base = (long long)blockIdx.x * nb * nb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int b1 = t1 * SCF_T + r0 + 8 * q;
    if (b1 >= nb) break;
    const long long o = base + (long long)b1 * nb + b2;
    Sout[o] = make_double2(c.dv * sacc[q].x, c.dv * sacc[q].y);
    if (WH) Hout[o] = make_double2(c.dv * hacc[q].x, c.dv * hacc[q].y);
  }
}

// Sum of part[0..n) in index order by one thread (fixed order: results do
// not depend on scheduling).
__device__ __forceinline__ double ordered_sum(const double* part, int n) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  return s;
}

// One CTA per unit (blockIdx.x): Cholesky S + s I = L L^H (right-looking, in
// W1; s = shift_coef tr S), Li = L^{-1} (one column per thread, in W2) and
// C = L^{-H}; when want_lam is set, also A = L^{-1} Hs L^{-H} over Hs (T =
// Hs L^{-H} in W1 first) and its largest eigenvalue by power iteration on
// A + shift (Gershgorin shift so that A + shift is positive semidefinite).
// The matrices live in global memory (they stay in L2); every sum runs in a
// fixed order.  status bit 4: S + s I not positive definite.
__global__ void __launch_bounds__(SCF_OT) k_scf_ortho(int nb, double shift_coef, int want_lam,
                                                      const double2* __restrict__ Sg, double2* __restrict__ Hg,
                                                      double2* __restrict__ Cg, double2* __restrict__ W1g,
                                                      double2* __restrict__ W2g, double* __restrict__ lam,
                                                      int* __restrict__ bad) {
  __shared__ double2 v[SCF_MAXB], w[SCF_MAXB];
  __shared__ double red[3][SCF_OT];
  __shared__ double sc[3];
  __shared__ int okf;
  const long long o = (long long)blockIdx.x * nb * nb;
  const double2* S = Sg + o;
  double2* A = Hg + o;   // Hs on entry, L^{-1} Hs L^{-H} on exit (want_lam)
  double2* C = Cg + o;
  double2* Lm = W1g + o;
  double2* Li = W2g + o;
  const int tid = threadIdx.x, nt = blockDim.x, n2 = nb * nb;
  const double2 z = make_double2(0.0, 0.0);
  for (int i = tid; i < n2; i += nt) Lm[i] = S[i];
  if (tid == 0) {
    okf = 1;
    double tr = 0.0;
    for (int i = 0; i < nb; ++i) tr += S[i * nb + i].x;
    sc[0] = shift_coef * tr;
  }
  __syncthreads();
  for (int i = tid; i < nb; i += nt) Lm[i * nb + i].x += sc[0];
  __syncthreads();
  // Cholesky, lower triangle of Lm; column j is final after step j
  for (int j = 0; j < nb; ++j) {
    const double d = Lm[j * nb + j].x;
    const double ljj = sqrt(d > 0.0 ? d : 1e-300);
    for (int i = j + 1 + tid; i < nb; i += nt) {
      const double2 x = Lm[i * nb + j];
      Lm[i * nb + j] = make_double2(x.x / ljj, x.y / ljj);
    }
    __syncthreads();
    if (tid == 0) {
      Lm[j * nb + j] = make_double2(ljj, 0.0);
      if (!(d > 0.0)) okf = 0;
    }
    const int m = nb - j - 1;
    for (int idx = tid; idx < m * m; idx += nt) {
      const int i = j + 1 + idx / m, k = j + 1 + idx % m;
      if (k <= i) Lm[i * nb + k] = zsub(Lm[i * nb + k], zmul(Lm[i * nb + j], zconj(Lm[k * nb + j])));
    }
    __syncthreads();
  }
  // Li = L^{-1}: column jj by forward substitution
  for (int jj = tid; jj < nb; jj += nt) {
    for (int i = 0; i < jj; ++i) Li[i * nb + jj] = z;
    Li[jj * nb + jj] = make_double2(1.0 / Lm[jj * nb + jj].x, 0.0);
    for (int i = jj + 1; i < nb; ++i) {
      double2 s = z;
      for (int k = jj; k < i; ++k) s = zadd(s, zmul(Lm[i * nb + k], Li[k * nb + jj]));
      const double lii = Lm[i * nb + i].x;
      Li[i * nb + jj] = make_double2(-s.x / lii, -s.y / lii);
    }
  }
  __syncthreads();
  // C = L^{-H} (upper triangular)
  for (int idx = tid; idx < n2; idx += nt) C[idx] = zconj(Li[(idx % nb) * nb + idx / nb]);
  if (!want_lam) {
    if (tid == 0 && !okf) atomicOr(bad, 4);
    return;
  }
  // T = Hs L^{-H} into Lm (Hs is in A)
  for (int idx = tid; idx < n2; idx += nt) {
    const int i = idx / nb, j = idx % nb;
    double2 s = z;
    for (int k = 0; k <= j; ++k) s = zadd(s, zmul(A[i * nb + k], zconj(Li[j * nb + k])));
    Lm[idx] = s;
  }
  __syncthreads();
  // A = L^{-1} T (Hs was last read in the previous loop)
  for (int idx = tid; idx < n2; idx += nt) {
    const int i = idx / nb, j = idx % nb;
    double2 s = z;
    for (int k = 0; k <= i; ++k) s = zadd(s, zmul(Li[i * nb + k], Lm[k * nb + j]));
    A[idx] = s;
  }
  __syncthreads();
  // Gershgorin lower bound of the Hermitian A
  double gl = 1e300;
  for (int i = tid; i < nb; i += nt) {
    double r = 0.0;
    for (int j = 0; j < nb; ++j)
      if (j != i) r += sqrt(A[i * nb + j].x * A[i * nb + j].x + A[i * nb + j].y * A[i * nb + j].y);
    gl = fmin(gl, A[i * nb + i].x - r);
  }
  red[0][tid] = gl;
  for (int i = tid; i < nb; i += nt) v[i] = make_double2(1.0 + 0.01 * i, 0.0);
  __syncthreads();
  if (tid == 0) {
    double lo = red[0][0];
    for (int i = 1; i < nt; ++i) lo = fmin(lo, red[0][i]);
    sc[0] = -lo;
  }
  __syncthreads();
  const double shift = sc[0];
  double rq = 0.0;
  for (int it = 0; it < 200; ++it) {
    double pn = 0.0, pv = 0.0, pw = 0.0;
    for (int i = tid; i < nb; i += nt) {
      double2 s = make_double2(shift * v[i].x, shift * v[i].y);
      for (int j = 0; j < nb; ++j) s = zadd(s, zmul(A[i * nb + j], v[j]));
      w[i] = s;
      pn += s.x * s.x + s.y * s.y;
      pv += v[i].x * v[i].x + v[i].y * v[i].y;
      pw += v[i].x * s.x + v[i].y * s.y;
    }
    red[0][tid] = pn;
    red[1][tid] = pv;
    red[2][tid] = pw;
    __syncthreads();
    if (tid < 3) sc[tid] = ordered_sum(red[tid], nt);
    __syncthreads();
    const double nrm = sqrt(sc[0]);
    rq = sc[2] / sc[1] - shift;
    for (int i = tid; i < nb; i += nt) v[i] = make_double2(w[i].x / nrm, w[i].y / nrm);
    __syncthreads();
  }
  if (tid == 0) {
    lam[blockIdx.x] = rq;
    if (!okf) atomicOr(bad, 4);
  }
}

// Y'[:, b] = sum_{k <= b} Y[:, k] C[k][b] for the SCF_RB bands of blockIdx.y,
// one point per thread (blockIdx.z selects the point block), out of place.
// The rows of C that the tile needs are staged in shared memory.
__global__ void __launch_bounds__(128) k_scf_rotate(LaunchSet L, const double2* __restrict__ Y,
                                                    const double2* __restrict__ Cg, double2* __restrict__ Yout) {
  extern __shared__ double2 cs[];   // [k][SCF_RB], k < kend
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  const UnitDev U = L.units[u];
  const int nb = c.n_bands, b0 = blockIdx.y * SCF_RB, nbt = min(SCF_RB, nb - b0), kend = b0 + nbt;
  const double2* C = Cg + (long long)blockIdx.x * nb * nb;
  for (int i = threadIdx.x; i < kend * SCF_RB; i += blockDim.x) {
    const int k = i / SCF_RB, j = i % SCF_RB;
    cs[i] = j < nbt ? C[(long long)k * nb + b0 + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int p = blockIdx.z * blockDim.x + threadIdx.x;
  if (p >= c.npts) return;
  const double2* yb = Y + U.psi_off + p;
  double2 s[SCF_RB];
#pragma unroll
  for (int j = 0; j < SCF_RB; ++j) s[j] = make_double2(0.0, 0.0);
  // C is upper triangular with exact zeros below the diagonal, so the sum
  // over all k < kend adds only zeros beyond k = b
  for (int k = 0; k < kend; ++k) {
    const double2 y = yb[(long long)k * c.npts];
#pragma unroll
    for (int j = 0; j < SCF_RB; ++j) s[j] = zadd(s[j], zmul(y, cs[k * SCF_RB + j]));
  }
  double2* ob = Yout + U.psi_off + p;
#pragma unroll
  for (int j = 0; j < SCF_RB; ++j)
    if (j < nbt) ob[(long long)(b0 + j) * c.npts] = s[j];
}

}  // namespace

int scf_max_bands() { return SCF_MAXB; }

void launch_scf_gram(const LaunchSet& L, const void* Y, const void* HY, void* S, void* H, void* stream) {
  if (L.n_units == 0) return;
  const int nt = (L.cell.n_bands + SCF_T - 1) / SCF_T;
  const dim3 grid(L.n_units, nt * nt);
  if (HY)
    k_scf_gram<true><<<grid, 256, 0, (cudaStream_t)stream>>>(L, (const double2*)Y, (const double2*)HY, (double2*)S,
                                                             (double2*)H);
  else
    k_scf_gram<false><<<grid, 256, 0, (cudaStream_t)stream>>>(L, (const double2*)Y, nullptr, (double2*)S, nullptr);
}

void launch_scf_ortho(int n_units, int nb, double shift_coef, int want_lam, const void* S, void* H, void* C,
                      void* W1, void* W2, double* lam, int* bad, void* stream) {
  if (n_units == 0) return;
  k_scf_ortho<<<n_units, SCF_OT, 0, (cudaStream_t)stream>>>(nb, shift_coef, want_lam, (const double2*)S,
                                                            (double2*)H, (double2*)C, (double2*)W1, (double2*)W2,
                                                            lam, bad);
}

void launch_scf_rotate(const LaunchSet& L, const void* Y, const void* C, void* Yout, void* stream) {
  if (L.n_units == 0) return;
  const int nb = L.cell.n_bands;
  const size_t smem = sizeof(double2) * (size_t)nb * SCF_RB;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_scf_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid(L.n_units, (nb + SCF_RB - 1) / SCF_RB, (L.cell.npts + 127) / 128);
  k_scf_rotate<<<grid, 128, smem, (cudaStream_t)stream>>>(L, (const double2*)Y, (const double2*)C, (double2*)Yout);
}
