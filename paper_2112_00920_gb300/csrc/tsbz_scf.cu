// Kernels of the ground-state solver (FP64): Chebyshev-filtered subspace
// iteration for the n_bands lowest eigenvectors of h_k[v_eff] at A = 0, per
// k-point, with Cholesky-QR re-orthonormalisation.  The filter steps run in
// the point-parallel stage kernel (m = 0); the kernels here form the Gram
// matrices, orthonormalise the block and bound the block's spectrum.
//
// Per unit (k-point) with the block Y (n_b columns) and HY = h Y:
//   S = dV Y^H Y,  Hs = dV Y^H (h Y)          (k_scf_gram)
//   S = L L^H,  C = L^{-H},  A = L^{-1} Hs L^{-H}, lam = largest eigenvalue of A
//                                             (k_scf_ortho)
//   Y <- Y C (columns dV-orthonormal)         (k_scf_rotate)
#include <cuda_runtime.h>

#include "tsbz_internal.h"

#define SCF_MAXB 32   // bands a unit may have in the ground-state solver
#define SCF_CH 32     // points per staged chunk of the Gram kernel

namespace {

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// S and Hs of one unit per CTA; the block and h times the block are staged in
// chunks of SCF_CH points; thread pairs (b1, b2) accumulate in a fixed order.
__global__ void __launch_bounds__(256) k_scf_gram(LaunchSet L, const double2* __restrict__ Y,
                                                  const double2* __restrict__ HY, double2* __restrict__ Sout,
                                                  double2* __restrict__ Hout) {
  __shared__ double2 ys[SCF_MAXB][SCF_CH];
  __shared__ double2 hs[SCF_MAXB][SCF_CH];
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.x];
  const UnitDev U = L.units[u];
  const int nb = c.n_bands, np = nb * nb;
  const double2* yb = Y + U.psi_off;
  const double2* hb = HY + U.psi_off;
  double2 sacc[4], hacc[4];   // up to 4 pairs per thread (nb <= 32: 1024 pairs / 256 threads)
  for (int i = 0; i < 4; ++i) sacc[i] = hacc[i] = make_double2(0.0, 0.0);
  for (int p0 = 0; p0 < c.npts; p0 += SCF_CH) {
    __syncthreads();
    for (int i = threadIdx.x; i < nb * SCF_CH; i += blockDim.x) {
      const int b = i / SCF_CH, k = i % SCF_CH, p = p0 + k;
      ys[b][k] = p < c.npts ? yb[(long long)b * c.npts + p] : make_double2(0.0, 0.0);
      hs[b][k] = p < c.npts ? hb[(long long)b * c.npts + p] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int pr = threadIdx.x + q * blockDim.x;
      if (pr >= np) break;
      const int b1 = pr / nb, b2 = pr % nb;
      for (int k = 0; k < SCF_CH; ++k) {
        const double2 a = zconj(ys[b1][k]);
        sacc[q] = zadd(sacc[q], zmul(a, ys[b2][k]));
        hacc[q] = zadd(hacc[q], zmul(a, hs[b2][k]));
      }
    }
  }
  for (int q = 0; q < 4; ++q) {
    const int pr = threadIdx.x + q * blockDim.x;
    if (pr >= np) break;
    const long long o = (long long)blockIdx.x * SCF_MAXB * SCF_MAXB + pr;
    Sout[o] = make_double2(c.dv * sacc[q].x, c.dv * sacc[q].y);
    Hout[o] = make_double2(c.dv * hacc[q].x, c.dv * hacc[q].y);
  }
}

// One thread per unit: Cholesky S = L L^H, C = L^{-H}, A = L^{-1} Hs L^{-H} and the
// largest eigenvalue of A by power iteration on A + shift (Gershgorin shift so
// that A + shift is positive semidefinite).  status bit 4: S not positive definite.
__global__ void k_scf_ortho(int n_units, int nb, const double2* __restrict__ Sg, const double2* __restrict__ Hg,
                            double2* __restrict__ Cg, double* __restrict__ lam, int* __restrict__ bad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_units) return;
  const long long o = (long long)t * SCF_MAXB * SCF_MAXB;
  const double2* S = Sg + o;
  const double2* H = Hg + o;
  double2* C = Cg + o;
  double2 Lm[SCF_MAXB][SCF_MAXB];
  double2 Li[SCF_MAXB][SCF_MAXB];
  // Cholesky (lower)
  bool ok = true;
  for (int j = 0; j < nb; ++j) {
    double d = S[j * nb + j].x;
    for (int k = 0; k < j; ++k) d -= Lm[j][k].x * Lm[j][k].x + Lm[j][k].y * Lm[j][k].y;
    if (!(d > 0.0)) {
      ok = false;
      d = 1e-300;
    }
    const double ljj = sqrt(d);
    Lm[j][j] = make_double2(ljj, 0.0);
    for (int i = j + 1; i < nb; ++i) {
      double2 s = S[i * nb + j];
      for (int k = 0; k < j; ++k) s = zsub(s, zmul(Lm[i][k], zconj(Lm[j][k])));
      Lm[i][j] = make_double2(s.x / ljj, s.y / ljj);
    }
    for (int i = 0; i < j; ++i) Lm[i][j] = make_double2(0.0, 0.0);
  }
  // inverse of the lower-triangular L (column by column, forward substitution)
  for (int j = 0; j < nb; ++j) {
    for (int i = 0; i < nb; ++i) Li[i][j] = make_double2(0.0, 0.0);
    Li[j][j] = make_double2(1.0 / Lm[j][j].x, 0.0);
    for (int i = j + 1; i < nb; ++i) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = j; k < i; ++k) s = zadd(s, zmul(Lm[i][k], Li[k][j]));
      Li[i][j] = make_double2(-s.x / Lm[i][i].x, -s.y / Lm[i][i].x);
    }
  }
  // C = L^{-H}
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) C[i * nb + j] = zconj(Li[j][i]);
  // A = L^{-1} H L^{-H}: first T = H L^{-H} into Lm (no longer needed), then A = L^{-1} T into Lm in place
  // by rows (row i of A needs rows k <= i of T)
  for (int i = 0; i < nb; ++i)
    for (int j = 0; j < nb; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = 0; k <= j; ++k) s = zadd(s, zmul(H[i * nb + k], zconj(Li[j][k])));
      Lm[i][j] = s;
    }
  for (int i = nb - 1; i >= 0; --i)
    for (int j = 0; j < nb; ++j) {
      double2 s = make_double2(0.0, 0.0);
      for (int k = 0; k <= i; ++k) s = zadd(s, zmul(Li[i][k], Lm[k][j]));
      Lm[i][j] = s;
    }
  // largest eigenvalue of the Hermitian A
  double lo = 0.0;
  for (int i = 0; i < nb; ++i) {
    double r = 0.0;
    for (int j = 0; j < nb; ++j)
      if (j != i) r += sqrt(Lm[i][j].x * Lm[i][j].x + Lm[i][j].y * Lm[i][j].y);
    lo = i == 0 ? Lm[i][i].x - r : fmin(lo, Lm[i][i].x - r);
  }
  const double shift = -lo;
  double2 v[SCF_MAXB], w[SCF_MAXB];
  for (int i = 0; i < nb; ++i) v[i] = make_double2(1.0 + 0.01 * i, 0.0);
  double rq = 0.0;
  for (int it = 0; it < 200; ++it) {
    double nrm = 0.0;
    for (int i = 0; i < nb; ++i) {
      double2 s = make_double2(shift * v[i].x, shift * v[i].y);
      for (int j = 0; j < nb; ++j) s = zadd(s, zmul(Lm[i][j], v[j]));
      w[i] = s;
      nrm += s.x * s.x + s.y * s.y;
    }
    double vv = 0.0, vw = 0.0;
    for (int i = 0; i < nb; ++i) {
      vv += v[i].x * v[i].x + v[i].y * v[i].y;
      vw += v[i].x * w[i].x + v[i].y * w[i].y;
    }
    rq = vw / vv - shift;
    nrm = sqrt(nrm);
    for (int i = 0; i < nb; ++i) v[i] = make_double2(w[i].x / nrm, w[i].y / nrm);
  }
  lam[t] = rq;
  if (!ok) atomicOr(bad, 4);
}

// Y <- Y C with C upper triangular, per point of every unit (in place).
__global__ void k_scf_rotate(LaunchSet L, double2* __restrict__ Y, const double2* __restrict__ Cg) {
  const CellDev& c = L.cell;
  const int u = L.unit_ids[blockIdx.y];
  const UnitDev U = L.units[u];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.npts) return;
  const int nb = c.n_bands;
  const double2* C = Cg + (long long)blockIdx.y * SCF_MAXB * SCF_MAXB;
  double2* yb = Y + U.psi_off + p;
  double2 y[SCF_MAXB];
  for (int b = 0; b < nb; ++b) y[b] = yb[(long long)b * c.npts];
  for (int b = 0; b < nb; ++b) {
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k <= b; ++k) s = zadd(s, zmul(y[k], C[k * nb + b]));
    yb[(long long)b * c.npts] = s;
  }
}

}  // namespace

int scf_max_bands() { return SCF_MAXB; }

void launch_scf_gram(const LaunchSet& L, const void* Y, const void* HY, void* S, void* H, void* stream) {
  if (L.n_units == 0) return;
  k_scf_gram<<<L.n_units, 256, 0, (cudaStream_t)stream>>>(L, (const double2*)Y, (const double2*)HY, (double2*)S,
                                                          (double2*)H);
}

void launch_scf_ortho(int n_units, int nb, const void* S, const void* H, void* C, double* lam, int* bad,
                      void* stream) {
  if (n_units == 0) return;
  k_scf_ortho<<<(n_units + 63) / 64, 64, 0, (cudaStream_t)stream>>>(n_units, nb, (const double2*)S,
                                                                    (const double2*)H, (double2*)C, lam, bad);
}

void launch_scf_rotate(const LaunchSet& L, void* Y, const void* C, void* stream) {
  if (L.n_units == 0) return;
  dim3 grid((L.cell.npts + 127) / 128, L.n_units);
  k_scf_rotate<<<grid, 128, 0, (cudaStream_t)stream>>>(L, (double2*)Y, (const double2*)C);
}
