// Host-side method arithmetic of the library: k-point sets (Eqs. 8, 10),
// Halton shifts (Sec. II.B), the laser pulse (Eq. 15) and the cell tables
// of Eq. 2's Hamiltonian (finite-difference weights, local potential,
// separable projector tables).  Plain C++; no CUDA.
#include <cmath>
#include <cstring>
#include <vector>

#include "tsbz.h"
#include "tsbz_host.h"

namespace tsbz {

static const double kPi = 3.14159265358979323846;

// Centred finite-difference weights of half-width nd (closed form of the
// Lagrange-interpolation derivatives on the points -nd..nd):
//   2nd derivative: c_m = 2 (-1)^{m+1} (nd!)^2 / (m^2 (nd-m)! (nd+m)!), c_0 = -2 sum c_m
//   1st derivative: d_m = (-1)^{m+1} (nd!)^2 / (m (nd-m)! (nd+m)!)
void fd_weights(int nd, double* c, double* d) {
  double s = 0.0;
  d[0] = 0.0;
  for (int m = 1; m <= nd; ++m) {
    // (nd!)^2 / ((nd-m)! (nd+m)!) as a product, exact for small nd
    double r = 1.0;
    for (int j = 1; j <= m; ++j) r *= (double)(nd - m + j) / (double)(nd + j);
    const double sgn = (m % 2 == 1) ? 1.0 : -1.0;
    c[m] = 2.0 * sgn * r / ((double)m * m);
    d[m] = sgn * r / (double)m;
    s += c[m];
  }
  c[0] = -2.0 * s;
}

static inline int fft_index(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

// v_loc(r) = Re sum_G v(G) exp(i G.r) with
//   v(G) = (1/Omega) sum_a exp(-i G.R_a) [-4 pi Z exp(-G^2 re^2/4)/G^2 + C (2 pi s^2)^{3/2} exp(-G^2 s^2/2)]
//   v(0) = (N_at/Omega) [pi Z re^2 + C (2 pi s^2)^{3/2}]
// evaluated by three separable 1-D inverse DFT passes.
void local_potential(const tsbz_cell_desc& d, std::vector<double>& out) {
  const int n1 = d.n[0], n2 = d.n[1], n3 = d.n[2];
  const long long npts = (long long)n1 * n2 * n3;
  out.assign(npts, 0.0);
  if (d.n_atoms == 0) return;
  const double omega = d.a[0] * d.a[1] * d.a[2];
  const double amp = d.c_core * std::pow(2.0 * kPi * d.sigma_core * d.sigma_core, 1.5);
  std::vector<double> re(npts), im(npts);
  for (int i3 = 0; i3 < n3; ++i3)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i1 = 0; i1 < n1; ++i1) {
        const double g[3] = {2.0 * kPi * fft_index(i1, n1) / d.a[0], 2.0 * kPi * fft_index(i2, n2) / d.a[1],
                             2.0 * kPi * fft_index(i3, n3) / d.a[2]};
        const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const long long idx = ((long long)i3 * n2 + i2) * n1 + i1;
        if (gg == 0.0) {
          re[idx] = d.n_atoms * (kPi * d.z_ion * d.r_erf * d.r_erf + amp) / omega;
          im[idx] = 0.0;
          continue;
        }
        const double form = -4.0 * kPi * d.z_ion * std::exp(-gg * d.r_erf * d.r_erf / 4.0) / gg +
                            amp * std::exp(-gg * d.sigma_core * d.sigma_core / 2.0);
        double sr = 0.0, si = 0.0;
        for (int a = 0; a < d.n_atoms; ++a) {
          double gr = 0.0;
          for (int ax = 0; ax < 3; ++ax) gr += g[ax] * d.atom_frac[3 * a + ax] * d.a[ax];
          sr += std::cos(gr);
          si -= std::sin(gr);
        }
        re[idx] = sr * form / omega;
        im[idx] = si * form / omega;
      }
  // inverse transforms along x, y, z: f(r) = sum_n F(n) exp(+2 pi i n r / N)
  const int nn[3] = {n1, n2, n3};
  const long long stride[3] = {1, n1, (long long)n1 * n2};
  std::vector<double> tr, ti;
  for (int ax = 0; ax < 3; ++ax) {
    const int N = nn[ax];
    std::vector<double> cw(N), sw(N);
    for (int m = 0; m < N; ++m) {
      cw[m] = std::cos(2.0 * kPi * m / N);
      sw[m] = std::sin(2.0 * kPi * m / N);
    }
    tr.assign(npts, 0.0);
    ti.assign(npts, 0.0);
    for (long long e = 0; e < npts; ++e) {
      const int k = (int)((e / stride[ax]) % N);
      const long long base = e - (long long)k * stride[ax];
      double sr = 0.0, si = 0.0;
      int idx = 0;
      for (int n = 0; n < N; ++n) {
        const double xr = re[base + n * stride[ax]], xi = im[base + n * stride[ax]];
        sr += xr * cw[idx] - xi * sw[idx];
        si += xr * sw[idx] + xi * cw[idx];
        idx += k;
        if (idx >= N) idx -= N;
      }
      tr[e] = sr;
      ti[e] = si;
    }
    re.swap(tr);
    im.swap(ti);
  }
  out = re;
}

// Separable projector tables.  For atom a and axis ax the minimum-image
// offset in grid units is o(i) = x - n floor((x + n/2)/n), x = i - f_ax n;
// inside the box |o| < proj_half: d = o h, g = exp(-d^2/(2 rc^2)); else 0.
// pnorm = (N_s, N_px, N_py, N_pz) from dV sum beta^2 = 1 (products of 1-D sums).
void projector_tables(const tsbz_cell_desc& d, std::vector<double>& g1, std::vector<double>& d1,
                      std::vector<double>& pnorm, int nmax) {
  const int na = d.n_atoms;
  g1.assign((size_t)na * 3 * nmax, 0.0);
  d1.assign((size_t)na * 3 * nmax, 0.0);
  pnorm.assign((size_t)na * 4, 0.0);
  const double dv = d.a[0] * d.a[1] * d.a[2] / ((double)d.n[0] * d.n[1] * d.n[2]);
  for (int a = 0; a < na; ++a) {
    double s0[3], s2[3];
    for (int ax = 0; ax < 3; ++ax) {
      const int n = d.n[ax];
      const double h = d.a[ax] / n;
      s0[ax] = 0.0;
      s2[ax] = 0.0;
      for (int i = 0; i < n; ++i) {
        const double x = (double)i - d.atom_frac[3 * a + ax] * n;
        const double o = x - n * std::floor((x + n / 2.0) / n);
        double gv = 0.0, dd = 0.0;
        if (std::fabs(o) < d.proj_half) {
          dd = o * h;
          gv = std::exp(-dd * dd / (2.0 * d.r_proj * d.r_proj));
        }
        g1[((size_t)a * 3 + ax) * nmax + i] = gv;
        d1[((size_t)a * 3 + ax) * nmax + i] = dd;
        s0[ax] += gv * gv;
        s2[ax] += dd * dd * gv * gv;
      }
    }
    pnorm[4 * a + 0] = 1.0 / std::sqrt(dv * s0[0] * s0[1] * s0[2]);
    pnorm[4 * a + 1] = 1.0 / std::sqrt(dv * s2[0] * s0[1] * s0[2]);
    pnorm[4 * a + 2] = 1.0 / std::sqrt(dv * s0[0] * s2[1] * s0[2]);
    pnorm[4 * a + 3] = 1.0 / std::sqrt(dv * s0[0] * s0[1] * s2[2]);
  }
}

}  // namespace tsbz

extern "C" {

int tsbz_shifted_kpoints(const double a[3], const int mp[3], const double shift[3], double* k_out, size_t cap) {
  if (!a || !mp || !shift || !k_out) return TSBZ_EINVAL;
  for (int ax = 0; ax < 3; ++ax)
    if (mp[ax] < 1 || !(a[ax] > 0.0)) return TSBZ_EINVAL;
  const size_t n = (size_t)mp[0] * mp[1] * mp[2];
  if (cap < 3 * n) return TSBZ_EINVAL;
  size_t idx = 0;
  for (int i3 = 1; i3 <= mp[2]; ++i3)
    for (int i2 = 1; i2 <= mp[1]; ++i2)
      for (int i1 = 1; i1 <= mp[0]; ++i1) {
        const int ii[3] = {i1, i2, i3};
        for (int ax = 0; ax < 3; ++ax) {
          const double N = mp[ax];
          double f = (2.0 * ii[ax] - N - 1.0 + 2.0 * shift[ax]) / (2.0 * N);
          f -= std::floor(f + 0.5);
          k_out[3 * idx + ax] = f * 2.0 * tsbz::kPi / a[ax];
        }
        ++idx;
      }
  return TSBZ_OK;
}

static double radical_inverse(int m, int base) {
  double f = 1.0, r = 0.0;
  while (m > 0) {
    f /= base;
    r += f * (m % base);
    m /= base;
  }
  return r;
}

int tsbz_halton(int n, double* out, size_t cap) {
  if (n < 0 || !out || cap < 3 * (size_t)n) return TSBZ_EINVAL;
  for (int m = 1; m <= n; ++m) {
    out[3 * (m - 1) + 0] = radical_inverse(m, 2);
    out[3 * (m - 1) + 1] = radical_inverse(m, 3);
    out[3 * (m - 1) + 2] = radical_inverse(m, 5);
  }
  return TSBZ_OK;
}

int tsbz_pulse_samples(double e0, double w0, double t_pulse, const double dir[3], double dt, int n_steps,
                       double* out, size_t cap) {
  if (!dir || !out || n_steps < 0 || !(dt > 0.0) || !(t_pulse > 0.0) || w0 == 0.0) return TSBZ_EINVAL;
  const size_t ns = 2 * (size_t)n_steps + 1;
  if (cap < 3 * ns) return TSBZ_EINVAL;
  for (size_t j = 0; j < ns; ++j) {
    const double t = 0.5 * (double)j * dt;
    double amp = 0.0;
    if (t > 0.0 && t < t_pulse) {
      const double s = std::sin(tsbz::kPi * t / t_pulse);
      amp = -(e0 / w0) * s * s * s * s * std::sin(w0 * (t - t_pulse / 2.0));
    }
    for (int ax = 0; ax < 3; ++ax) out[3 * j + ax] = amp * dir[ax];
  }
  return TSBZ_OK;
}

}  // extern "C"
