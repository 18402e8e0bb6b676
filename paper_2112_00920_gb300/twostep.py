"""Second sampling with a convergence check.

Sec. II.B (steps 2-4) averages N_H shifted sub-simulations (Eq. 9); the
discussion of Fig. 6 (Sec. III.B) treats them as N_H data sets whose
standard error of the mean measures how far the k-sampling has converged.
``adaptive_two_step`` adds shifted sub-simulations in batches (each batch one
library context, propagated on the GPU) until the standard error of the
two-step eps(omega) is below a tolerance, so no run is spent only on the
convergence check.

Host orchestration and post-processing only: the propagation runs in the
library's kernels, and eps(omega) (Eqs. 12-14) is a host Fourier sum of the
FP64 current history.
"""
from __future__ import annotations

import numpy as np

from ._lib import Propagator, halton, shifted_kpoints


def dielectric(dj, dt, k0, omegas, t_w=None):
    """Eqs. 12-14 on the samples dJ(t_n), t_n = n dt (n = 0..N):
    dJ(w) = dt sum_n c_n e^{i w t_n} W_L(t_n / T_W) dJ(t_n) with trapezoid
    weights c_0 = c_N = 1/2 and W_L(x) = 1 - 3x^2 + 2x^3 on [0, 1];
    sigma = dJ(w) / k0, eps = 1 + 4 pi i sigma / w.  T_W defaults to t_N."""
    dj = np.asarray(dj, dtype=np.float64)
    t = np.arange(dj.shape[-1]) * dt
    tw = t[-1] if t_w is None else t_w
    x = t / tw
    win = np.where((x >= 0.0) & (x <= 1.0), 1.0 - 3.0 * x * x + 2.0 * x ** 3, 0.0)
    c = np.ones_like(t)
    c[0] = c[-1] = 0.5
    om = np.asarray(omegas, dtype=np.float64)
    sig = dt * (np.exp(1j * np.outer(om, t)) @ (c * win * dj)) / k0
    return 1.0 + 4.0j * np.pi * sig / om


def standard_error(samples):
    """Mean over axis 0 and its standard error sqrt(sum (x - mean)^2 / (n (n - 1)))
    (0 for one sample); real and imaginary parts separately for complex data."""
    x = np.asarray(samples)
    n = x.shape[0]
    mean = x.sum(axis=0) / n
    if n < 2:
        return mean, np.zeros(mean.shape), np.zeros(mean.shape)
    d = x - mean
    re = np.sqrt((d.real ** 2).sum(axis=0) / (n * (n - 1)))
    im = np.sqrt((d.imag ** 2).sum(axis=0) / (n * (n - 1))) if np.iscomplexobj(x) else np.zeros(mean.shape)
    return mean, re, im


def halton_source(n_total: int):
    """Shifts m = 1..n_total of the Halton sequence in bases 2, 3, 5 (the paper's choice)."""
    h = halton(n_total)
    return [tuple(float(v) for v in row) for row in h]


def random_source(n_total: int, seed: int):
    """Uniform random shifts in (0,1)^3, for which sigma_E is a true standard error."""
    rng = np.random.default_rng([seed, 11])
    return [tuple(float(v) for v in row) for row in rng.uniform(0.0, 1.0, size=(n_total, 3))]


def adaptive_two_step(cell, mp, shifts, dt, n_steps, k0, omegas, tol, ground_state, batch=8, min_shifts=2,
                      precision="fp32", direction=(1.0, 0.0, 0.0), device=0, hxc="scf"):
    """Run shifted N^3 subgrids (``mp``) of ``cell`` from the list ``shifts`` in
    batches of ``batch`` until max_w sigma_E(Im eps(w)) <= tol with at least
    ``min_shifts`` shifts, or the list is used up.

    ground_state(kcart, shift_index) returns the complex128 orbitals
    (n_k, n_bands, n3, n2, n1) of one shift.  Returns a dict: n_h, eps (mean),
    sigma_re, sigma_im (standard errors of Re / Im eps), dj (n_h, n_steps+1)
    along ``direction``, history [(n_h, max sigma_im)] after each batch."""
    e = np.asarray(direction, dtype=np.float64)
    djs, history = [], []
    used = 0
    eps = sre = sim = None
    while used < len(shifts):
        chunk = shifts[used:used + batch]
        P = Propagator(precision, device=device)
        try:
            cid = P.add_cell_spec(cell, hxc=hxc)
            ks = [shifted_kpoints(cell.a, mp, s) for s in chunk]
            sids = [P.add_subsim(cid, k, dt, n_steps) for k in ks]
            for j, (sid, k) in enumerate(zip(sids, ks)):
                P.load_ground_state(sid, ground_state(k, used + j))
                P.set_kick(sid, k0, direction)
            P.propagate(n_steps)
            for sid in sids:
                J, j0 = P.current(sid)
                djs.append((J - j0[None, :]) @ e)
        finally:
            P.close()
        used += len(chunk)
        eps_m = np.stack([dielectric(d, dt, k0, omegas) for d in djs])
        eps, sre, sim = standard_error(eps_m)
        history.append((used, float(np.max(sim))))
        if used >= min_shifts and np.max(sim) <= tol:
            break
    return dict(n_h=used, eps=eps, sigma_re=sre, sigma_im=sim, dj=np.stack(djs), history=history)
