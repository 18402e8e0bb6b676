"""Hartree-exchange-correlation potential v_Hxc[rho] (Eq. 2).

Hartree: spectral Poisson solve on the FFT grid, v_H(G) = 4 pi rho(G)/G^2,
with the G = 0 term set to zero (neutralising background).

Exchange-correlation: the paper uses the adiabatic LDA (Sec. III); the
functional fixed for this build is Perdew-Zunger 1981 (Phys. Rev. B 23,
5048, App. C, unpolarised), with the Ceperley-Alder parametrisation
    r_s >= 1:  e_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1:  e_c = A ln r_s + B + C r_s ln r_s + D r_s
and Slater exchange e_x = -(3/4)(3/pi)^{1/3} rho^{1/3}; the potentials are
v = d(rho e)/d rho.  rho is floored at 1e-30 before evaluation.
"""
from __future__ import annotations

import numpy as np

from .cell import Grid

PZ_GAMMA = -0.1423
PZ_BETA1 = 1.0529
PZ_BETA2 = 0.3334
PZ_A = 0.0311
PZ_B = -0.048
PZ_C = 0.0020
PZ_D = -0.0116
RHO_FLOOR = 1e-30


def hartree(grid: Grid, rho: np.ndarray) -> np.ndarray:
    gx, gy, gz = grid.g_vectors()
    g2 = gx * gx + gy * gy + gz * gz
    rho_g = np.fft.fftn(rho)
    vg = np.zeros_like(rho_g)
    nz = g2 > 0
    vg[nz] = 4.0 * np.pi * rho_g[nz] / g2[nz]
    return np.real(np.fft.ifftn(vg))


def pz81(rho: np.ndarray):
    """Return (e_xc, v_xc) per electron / potential for the unpolarised LDA."""
    rho = np.maximum(np.asarray(rho, dtype=np.float64), RHO_FLOOR)
    rs = (3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0)
    ex = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * rho ** (1.0 / 3.0)
    vx = 4.0 / 3.0 * ex
    ec = np.empty_like(rho)
    vc = np.empty_like(rho)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[lo] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) / 3.0 * r
    return ex + ec, vx + vc


def v_hxc(grid: Grid, rho: np.ndarray, xc: bool = True, hartree_on: bool = True) -> np.ndarray:
    v = np.zeros_like(rho)
    if hartree_on:
        v = v + hartree(grid, rho)
    if xc:
        v = v + pz81(rho)[1]
    return v
