"""Spectra, error metrics and the free-electron closed form.

Eqs. 12-14: dJ(w) = int_0^inf dt e^{iwt} W_L(t/T_W) e_a.dJ(t),
W_L(x) = 1 - 3x^2 + 2x^3 on [0, 1] (zero outside), sigma = dJ(w)/k0,
eps = 1 + 4 pi i sigma / w.  The integral is the trapezoid rule on the
propagation samples.  The paper's T_W = 30 fs exceeds the short runs used
here, so T_W is a parameter (the run length by default).

Eqs. 16-17: I(w) = w^2 |int dt e^{iwt} W(t) e_L.J(t)|^2 with
W(t) = sin^4(pi t/T_L) on (0, T_L) (the cos^4 envelope of Eq. 17 with the
argument divided by T_L).
"""
from __future__ import annotations

import numpy as np

from . import fd
from .cell import Grid
from .hxc import pz81


def window_l(x):
    x = np.asarray(x, dtype=np.float64)
    return np.where((x >= 0.0) & (x <= 1.0), 1.0 - 3.0 * x * x + 2.0 * x ** 3, 0.0)


def trapezoid_weights(n_samples):
    w = np.ones(n_samples)
    w[0] = 0.5
    w[-1] = 0.5
    return w


def fourier_current(dj_component, dt, omegas, t_w=None):
    """Eq. 13 with the trapezoid rule; dj_component (n+1,) at t_n = n dt."""
    n1 = dj_component.shape[0]
    t = np.arange(n1) * dt
    t_w = t[-1] if t_w is None else t_w
    w = trapezoid_weights(n1) * window_l(t / t_w) * dj_component
    return dt * np.exp(1j * np.outer(omegas, t)) @ w


def dielectric(dj_component, dt, k0, omegas, t_w=None):
    """eps(w) = 1 + 4 pi i sigma(w)/w with sigma = dJ(w)/k0 (Eqs. 12, 14)."""
    sig = fourier_current(dj_component, dt, omegas, t_w) / k0
    return 1.0 + 4.0j * np.pi * sig / omegas


def dielectric_statistics(dj_components, dt, k0, omegas, t_w=None):
    """Mean and standard error of eps(omega) over N_H shifted sub-simulations
    (Eqs. 12-14 per sub-simulation; error bars of Fig. 6, Sec. III.B).
    eps is affine in dJ, so the mean of the per-shift eps is the eps of the
    averaged dJ (Eq. 9).  The standard error is taken separately for the real
    and imaginary parts: sigma = sqrt(sum (x_m - mean)^2 / (N_H (N_H - 1))).
    dj_components: (N_H, n+1) along the kick.  Returns (mean eps, sigma_re,
    sigma_im)."""
    eps = np.stack([dielectric(d, dt, k0, omegas, t_w) for d in dj_components])
    n = eps.shape[0]
    mean = eps.sum(axis=0) / n
    if n < 2:
        z = np.zeros(mean.shape)
        return mean, z, z
    dev = eps - mean
    sre = np.sqrt((dev.real ** 2).sum(axis=0) / (n * (n - 1)))
    sim = np.sqrt((dev.imag ** 2).sum(axis=0) / (n * (n - 1)))
    return mean, sre, sim


def hhg_spectrum(j_component, dt, t_pulse, omegas):
    """Eqs. 16-17: I(w) = w^2 |dt sum_n w_n e^{i w t_n} W(t_n) J(t_n)|^2 with
    W(t) = sin^4(pi t/T_L) on (0, T_L), zero elsewhere, trapezoid weights w_n
    and t_n = n dt.  Pinned by closed-form transforms of sinusoidal currents
    (tests/test_oracle_analysis.py)."""
    n1 = j_component.shape[0]
    t = np.arange(n1) * dt
    win = np.where((t > 0) & (t < t_pulse), np.sin(np.pi * t / t_pulse) ** 4, 0.0)
    w = trapezoid_weights(n1) * win * j_component
    amp = dt * np.exp(1j * np.outer(omegas, t)) @ w
    return omegas ** 2 * np.abs(amp) ** 2


# ----------------------------------------------------------------------------
# Error metrics
# ----------------------------------------------------------------------------
def err_j(j_test, j_ref):
    return float(np.max(np.linalg.norm(j_test - j_ref, axis=-1)) / np.max(np.linalg.norm(j_ref, axis=-1)))


def err_rho(rho_test, rho_ref):
    return float(np.max(np.abs(rho_test - rho_ref)) / np.max(np.abs(rho_ref)))


def err_norm(n_test, n_ref):
    return float(np.max(np.abs(np.asarray(n_test) - np.asarray(n_ref))))


def err_eps(eps_test, eps_ref):
    return float(np.max(np.abs(eps_test - eps_ref)) / np.max(np.abs(eps_ref)))


# ----------------------------------------------------------------------------
# Free-electron closed form
# ----------------------------------------------------------------------------
def taylor4_factor(z):
    """T_4(z) = sum_{m=0..4} z^m / m!."""
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


def plane_wave_orbitals(grid: Grid, gints):
    """u = exp(i G.r)/sqrt(Omega) for integer triples gints (n_k, n_b, 3)."""
    x, y, z = grid.coords()
    n_k, n_b, _ = gints.shape
    out = np.empty((n_k, n_b) + x.shape, dtype=np.complex128)
    for k in range(n_k):
        for b in range(n_b):
            g = 2.0 * np.pi * gints[k, b] / grid.a
            out[k, b] = np.exp(1j * (g[0] * x + g[1] * y + g[2] * z)) / np.sqrt(grid.omega)
    return out


def lowest_plane_waves(grid: Grid, kcart, n_b, nd: int = 4, span: int = 3):
    """The n_b integer G per k with the lowest FD kinetic energy at q = k
    (ties broken lexicographically on (n_x, n_y, n_z))."""
    rng = range(-span, span + 1)
    cands = np.array([(i, j, l) for i in rng for j in rng for l in rng])
    out = np.empty((kcart.shape[0], n_b, 3), dtype=np.int64)
    for k in range(kcart.shape[0]):
        e = np.array([fd_kinetic(grid, c, kcart[k], nd) for c in cands])
        order = sorted(range(len(cands)), key=lambda i: (round(e[i], 12), tuple(cands[i])))
        out[k] = cands[order[:n_b]]
    return out


def fd_kinetic(grid: Grid, gint, q, nd: int = 4):
    """Eigenvalue of -1/2 lap_FD - i q.grad_FD + |q|^2/2 on exp(i G.r)."""
    e = 0.5 * float(np.dot(q, q))
    for ax in range(3):
        th = 2.0 * np.pi * gint[ax] / grid.n[ax]
        h = grid.h[ax]
        e += -0.5 * float(fd.laplacian_symbol(th, nd)) / (h * h) + q[ax] * float(fd.gradient_symbol(th, nd)) / h
    return e


def fd_velocity(grid: Grid, gint, nd: int = 4):
    """<-i grad_FD> on exp(i G.r): s(theta)/h per axis."""
    return np.array([float(fd.gradient_symbol(2.0 * np.pi * gint[ax] / grid.n[ax], nd)) / grid.h[ax]
                     for ax in range(3)])


def free_electron_current(grid: Grid, occ, kcart, gints, dt, n_steps, a_samples, xc: bool = True, nd: int = 4,
                          propagator: str = "taylor4"):
    """Closed-form J(t_n) for plane-wave orbitals in a cell with no ions.

    Each orbital stays a plane wave, u_n = c_n u_0 with
    c_{n+1} = c_n T_4(-i e_n dt), e_n = kinetic(G, k + A(t_n + dt/2)) + v_xc(rho_n);
    rho_n = f sum |c_n|^2 / (Omega N_k) is uniform so v_H = 0.
    J_n = -(f/(Omega N_k)) sum |c_n|^2 (s(G)/h + k + A(t_n)).
    With propagator "etrs": c_{n+1} = c_n T_4(-i e'' dt/2) T_4(-i e' dt/2),
    e' = kinetic(G, k + A(t_n)) + v_xc(rho_n), e'' = kinetic(G, k + A(t_{n+1}))
    + v_xc(rho~), rho~ the uniform density of the Taylor-4 predictor c_n T_4(-i e_n dt).
    Returns (J (n_steps+1, 3), J0_minus (3,), |c|^2 (n_k, n_b))."""
    n_k, n_b, _ = gints.shape
    c = np.ones((n_k, n_b), dtype=np.complex128)
    vel = np.array([[fd_velocity(grid, gints[k, b], nd) for b in range(n_b)] for k in range(n_k)])

    def cur(cc, a):
        w = np.abs(cc) ** 2
        tot = np.einsum("kb,kbx->x", w, vel) + np.einsum("kb,kx->x", w, kcart + a[None, :])
        return -occ * tot / (grid.omega * n_k)

    j0m = cur(c, np.zeros(3))
    js = [cur(c, a_samples[0])]
    def vxc_of(cc):
        rho = occ * np.sum(np.abs(cc) ** 2) / (grid.omega * n_k)
        return float(pz81(np.array([rho]))[1][0]) if xc else 0.0

    for n in range(n_steps):
        vxc = vxc_of(c)
        a_half = a_samples[2 * n + 1]
        step = np.array([[taylor4_factor(-1j * (fd_kinetic(grid, gints[k, b], kcart[k] + a_half, nd) + vxc) * dt)
                          for b in range(n_b)] for k in range(n_k)])
        if propagator == "etrs":
            vxc_p = vxc_of(c * step)
            for k in range(n_k):
                for b in range(n_b):
                    e1 = fd_kinetic(grid, gints[k, b], kcart[k] + a_samples[2 * n], nd) + vxc
                    e2 = fd_kinetic(grid, gints[k, b], kcart[k] + a_samples[2 * n + 2], nd) + vxc_p
                    c[k, b] *= taylor4_factor(-1j * e1 * 0.5 * dt) * taylor4_factor(-1j * e2 * 0.5 * dt)
        else:
            c = c * step
        js.append(cur(c, a_samples[2 * n + 2]))
    return np.array(js), j0m, np.abs(c) ** 2
