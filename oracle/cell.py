"""Grid, local ionic potential and Kleinman-Bylander projectors.

Eq. 2: h_k(t) = (p + k + A(t))^2 / 2 + v_ion + v_Hxc[rho], with v_ion a
norm-conserving pseudopotential made of a local part and non-local
(projector) operators.  The paper uses HGH pseudopotentials for Si; the
synthetic stand-in used here (its parameters live in ``workloads.CellSpec``):

local part, defined through its Fourier coefficients on the FFT set of G:
    v(G) = (1/Omega) sum_a exp(-i G.R_a) [ -4 pi Z exp(-G^2 r_e^2 / 4) / G^2
                                          + C (2 pi sigma^2)^{3/2} exp(-G^2 sigma^2 / 2) ]
    v(G=0) = (N_at/Omega) [ pi Z r_e^2 + C (2 pi sigma^2)^{3/2} ]
  i.e. -Z erf(r/r_e)/r + C exp(-r^2/2 sigma^2) per atom with the divergent
  G = 0 Coulomb part removed; v_loc(r_i) = Re sum_G v(G) exp(i G.r_i).

projectors: per atom one s and three p functions
    beta_s = N_s exp(-|d|^2/(2 r_c^2)),   beta_{p,ax} = N_p d_ax exp(-|d|^2/(2 r_c^2)),
  d = minimum-image displacement of the grid point from the atom, zero
  outside the box |o_ax| < proj_half (o = d / h in grid units), normalised so
  that dV sum_r beta^2 = 1.  The k- and A-dependence enters through the
  phased projector  beta~_j(r) = beta_j(d) exp(-i q.d),  q = k + A(t).
"""
from __future__ import annotations

import numpy as np

from workloads import CellSpec


class Grid:
    """Real-space grid of an orthorhombic cell. Arrays are (n3, n2, n1)."""

    def __init__(self, cell: CellSpec):
        self.cell = cell
        self.a = np.asarray(cell.a, dtype=np.float64)
        self.n = tuple(int(v) for v in cell.n)
        self.h = self.a / np.asarray(self.n, dtype=np.float64)
        self.omega = float(np.prod(self.a))
        self.n_pts = int(np.prod(self.n))
        self.dv = self.omega / self.n_pts

    def g_vectors(self):
        """Cartesian components (Gx, Gy, Gz) broadcast to (n3, n2, n1); the
        integer set per axis is [-N/2, N/2) for even N (numpy FFT order)."""
        n1, n2, n3 = self.n
        g1 = 2.0 * np.pi * np.fft.fftfreq(n1, 1.0 / n1) / self.a[0]
        g2 = 2.0 * np.pi * np.fft.fftfreq(n2, 1.0 / n2) / self.a[1]
        g3 = 2.0 * np.pi * np.fft.fftfreq(n3, 1.0 / n3) / self.a[2]
        gz, gy, gx = np.meshgrid(g3, g2, g1, indexing="ij")
        return gx, gy, gz

    def coords(self):
        """Cartesian coordinates of the grid points, (x, y, z) each (n3, n2, n1)."""
        n1, n2, n3 = self.n
        z, y, x = np.meshgrid(np.arange(n3) * self.h[2], np.arange(n2) * self.h[1],
                              np.arange(n1) * self.h[0], indexing="ij")
        return x, y, z


def local_potential(cell: CellSpec) -> np.ndarray:
    """v_loc on the grid (Eq. 2's local ionic part, synthetic form above)."""
    g = Grid(cell)
    gx, gy, gz = g.g_vectors()
    g2 = gx * gx + gy * gy + gz * gz
    vhat = np.zeros(g2.shape, dtype=np.complex128)
    if cell.n_atoms == 0:
        return np.zeros(g2.shape)
    nz = g2 > 0
    gauss_amp = cell.c_core * (2.0 * np.pi * cell.sigma_core ** 2) ** 1.5
    form = np.zeros_like(g2)
    form[nz] = (-4.0 * np.pi * cell.z_ion * np.exp(-g2[nz] * cell.r_erf ** 2 / 4.0) / g2[nz]
                + gauss_amp * np.exp(-g2[nz] * cell.sigma_core ** 2 / 2.0))
    struct = np.zeros(g2.shape, dtype=np.complex128)
    for fr in cell.atom_frac:
        r = fr * g.a
        struct += np.exp(-1j * (gx * r[0] + gy * r[1] + gz * r[2]))
    vhat[nz] = struct[nz] * form[nz] / g.omega
    vhat[~nz] = cell.n_atoms * (np.pi * cell.z_ion * cell.r_erf ** 2 + gauss_amp) / g.omega
    return np.real(np.fft.ifftn(vhat) * g.n_pts)


def atom_offsets(cell: CellSpec, atom: int, axis: int) -> np.ndarray:
    """Grid-unit minimum-image offsets o(i) = wrap(i - f N) in [-N/2, N/2)
    of the grid points along ``axis`` from atom ``atom``."""
    n = cell.n[axis]
    x = np.arange(n, dtype=np.float64) - cell.atom_frac[atom, axis] * n
    return x - n * np.floor((x + n / 2.0) / n)


def projector_tables(cell: CellSpec):
    """Real projector values and displacements on the grid.

    Returns (beta, disp, e_kb): beta (n_proj, n3, n2, n1) real, ordered atom
    by atom as [s, p_x, p_y, p_z]; disp (n_atoms, 3, n3, n2, n1) the
    minimum-image displacement d (bohr, zero outside the box); e_kb (n_proj,).
    """
    g = Grid(cell)
    if not cell.use_projectors or cell.n_atoms == 0:
        return (np.zeros((0,) + g.n[::-1]), np.zeros((0, 3) + g.n[::-1]), np.zeros(0))
    n1, n2, n3 = g.n
    betas, disps, es = [], [], []
    for a in range(cell.n_atoms):
        o = [atom_offsets(cell, a, ax) for ax in range(3)]
        inside = [np.abs(o[ax]) < cell.proj_half for ax in range(3)]
        d1 = [np.where(inside[ax], o[ax] * g.h[ax], 0.0) for ax in range(3)]
        mask = inside[2][:, None, None] & inside[1][None, :, None] & inside[0][None, None, :]
        dz, dy, dx = np.meshgrid(d1[2], d1[1], d1[0], indexing="ij")
        r2 = dx * dx + dy * dy + dz * dz
        gauss = np.where(mask, np.exp(-r2 / (2.0 * cell.r_proj ** 2)), 0.0)
        shapes = [gauss, dx * gauss, dy * gauss, dz * gauss]
        for sh in shapes:
            nrm = np.sqrt(g.dv * np.sum(sh * sh))
            betas.append(sh / nrm)
        es.extend([cell.e_kb_s, cell.e_kb_p, cell.e_kb_p, cell.e_kb_p])
        disps.append(np.stack([np.where(mask, dx, 0.0), np.where(mask, dy, 0.0), np.where(mask, dz, 0.0)]))
    return np.stack(betas), np.stack(disps), np.asarray(es)


def phased_projectors(cell: CellSpec, beta, disp, q):
    """beta~_j(r) = beta_j(d) exp(-i q.d) for one q (3,), shape (n_proj, n_pts)."""
    n_proj = beta.shape[0]
    if n_proj == 0:
        return np.zeros((0, int(np.prod(cell.n))), dtype=np.complex128)
    out = np.empty((n_proj,) + beta.shape[1:], dtype=np.complex128)
    for j in range(n_proj):
        a = j // 4
        d = disp[a]
        ph = np.exp(-1j * (q[0] * d[0] + q[1] * d[1] + q[2] * d[2]))
        out[j] = beta[j] * ph
    return out.reshape(n_proj, -1)
