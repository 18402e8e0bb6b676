// Density of a set of orbitals without any device allocation.
//
// This is a variant of the density part of the observation kernel plus the
// fixed-order reduction that tsbz_get_density uses, for callers that cannot
// allocate device memory.  Its per-k partial sums live in a file-scope
// static device array (TSBZ_NOALLOC_SCRATCH_DOUBLES doubles, 2 MiB), which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "tsbz.h"

#define TSBZ_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_scratch[TSBZ_NOALLOC_SCRATCH_DOUBLES];

namespace {

// Device address of g_noalloc_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current and cached.
std::mutex g_mutex;
double* g_scratch_ptr[TSBZ_NOALLOC_MAX_DEVICES] = {nullptr};

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSBZ_ECUDA;
  if (dev < 0 || dev >= TSBZ_NOALLOC_MAX_DEVICES) return TSBZ_EINVAL;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return TSBZ_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return TSBZ_OK;
}

// part[kl][p] = occ * sum_b |u_{k0+kl, b}(p)|^2 for kl < n_kc
__global__ void k_density_partial_noalloc(const double2* __restrict__ psi, int k0, int n_kc, int n_bands,
                                          long long npts, double occ, double* __restrict__ part) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)n_kc * npts) return;
  const int kl = (int)(e / npts);
  const long long p = e % npts;
  const double2* u = psi + ((long long)(k0 + kl) * n_bands) * npts + p;
  double s = 0.0;
  for (int b = 0; b < n_bands; ++b) {
    const double2 v = u[(long long)b * npts];
    s += v.x * v.x + v.y * v.y;
  }
  part[e] = occ * s;
}

// rho[p] (+)= (1/n_k) sum_{kl < n_kc} part[kl][p], k in increasing order
__global__ void k_density_reduce_noalloc(const double* __restrict__ part, int n_kc, long long npts, double inv_nk,
                                         int accumulate, double* __restrict__ rho) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  double s = 0.0;
  for (int kl = 0; kl < n_kc; ++kl) s += part[(long long)kl * npts + p];
  s *= inv_nk;
  rho[p] = accumulate ? rho[p] + s : s;
}

}  // namespace

extern "C" int tsbz_density_noalloc(const double* psi, int n_k, int n_bands, const int n[3], double occ,
                                    double* rho, void* cuda_stream) {
  if (!psi || !rho || !n || n_k < 1 || n_bands < 1) return TSBZ_EINVAL;
  for (int ax = 0; ax < 3; ++ax)
    if (n[ax] < 1) return TSBZ_EINVAL;
  const long long npts = (long long)n[0] * n[1] * n[2];
  if (npts > TSBZ_NOALLOC_SCRATCH_DOUBLES) return TSBZ_EINVAL;  // one k-point must fit the scratch
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int per_chunk = (int)(TSBZ_NOALLOC_SCRATCH_DOUBLES / npts);
  const double inv_nk = 1.0 / n_k;
  for (int k0 = 0; k0 < n_k; k0 += per_chunk) {
    const int n_kc = n_k - k0 < per_chunk ? n_k - k0 : per_chunk;
    const long long total = (long long)n_kc * npts;
    k_density_partial_noalloc<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const double2*>(psi), k0, n_kc, n_bands, npts, occ, scratch);
    k_density_reduce_noalloc<<<(unsigned)((npts + 255) / 256), 256, 0, st>>>(scratch, n_kc, npts, inv_nk,
                                                                               k0 > 0 ? 1 : 0, rho);
  }
  if (cudaGetLastError() != cudaSuccess) return TSBZ_ECUDA;
  return TSBZ_OK;
}
