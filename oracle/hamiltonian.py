"""Application of the Kohn-Sham Hamiltonian h_k(t) of Eq. 2 on the grid.

For the periodic part u of a Bloch orbital and q = k + A(t):
    h u = -1/2 lap_FD u - i q.grad_FD u + 1/2 |q|^2 u + v_eff u
          + sum_j E_j beta~_j <beta~_j | u>,
with <f|u> = dV sum_r conj(f(r)) u(r) and the phased projectors of
``cell.phased_projectors``.  lap_FD, grad_FD are the centred star stencils
of ``fd`` on the periodic grid (the FD form of (p + q)^2/2 with p = -i grad).

Array layout: orbitals (..., n3, n2, n1); axis -1 is x.
"""
from __future__ import annotations

import numpy as np

from . import fd
from .cell import Grid, phased_projectors


def _padded(u, axis, nd):
    """u extended periodically by nd points on both ends of ``axis``."""
    n = u.shape[axis]
    lo = np.take(u, np.arange(n - nd, n), axis=axis)
    hi = np.take(u, np.arange(0, nd), axis=axis)
    return np.concatenate([lo, u, hi], axis=axis)


def _shifted(up, m, axis, nd, n):
    """From the padded array, the values at index i + m along ``axis``."""
    sl = [slice(None)] * up.ndim
    sl[axis] = slice(nd + m, nd + m + n)
    return up[tuple(sl)]


def apply_local(grid: Grid, u, q, v_eff, nd: int = 4):
    """Local part: -1/2 lap u - i q.grad u + (1/2 |q|^2 + v_eff) u.

    u: (..., n3, n2, n1) complex; q: (3,) or broadcastable (..., 3)."""
    c, d = fd.weights_float(nd)
    q = np.asarray(q, dtype=np.float64)
    lap = np.zeros_like(u)
    grad_q = np.zeros_like(u)
    axes = (-1, -2, -3)  # x, y, z
    qx = [q[..., 0], q[..., 1], q[..., 2]]
    for ax in range(3):
        h = grid.h[ax]
        axis = u.ndim + axes[ax]
        n = u.shape[axis]
        up_arr = _padded(u, axis, nd)
        part_l = c[0] * u
        part_g = np.zeros_like(u)
        for m in range(1, nd + 1):
            up = _shifted(up_arr, m, axis, nd, n)
            dn = _shifted(up_arr, -m, axis, nd, n)
            part_l = part_l + c[m] * (up + dn)
            part_g = part_g + d[m] * (up - dn)
        lap = lap + part_l / (h * h)
        qa = np.asarray(qx[ax])
        if qa.ndim:
            qa = qa.reshape(qa.shape + (1,) * (u.ndim - qa.ndim))
        grad_q = grad_q + qa * part_g / h
    q2 = np.sum(q * q, axis=-1)
    if np.ndim(q2):
        q2 = q2.reshape(q2.shape + (1,) * (u.ndim - np.ndim(q2)))
    return -0.5 * lap - 1j * grad_q + (0.5 * q2 + v_eff) * u


def apply_nonlocal(grid: Grid, u, proj, e_kb):
    """sum_j E_j beta~_j <beta~_j|u> for orbitals u (n_b, n3, n2, n1) of one q;
    proj: (n_proj, n_pts) phased projectors."""
    if proj.shape[0] == 0:
        return np.zeros_like(u)
    flat = u.reshape(u.shape[0], -1)
    a = grid.dv * (flat @ proj.conj().T)          # (n_b, n_proj): <beta~_j|u_b>
    return ((a * e_kb[None, :]) @ proj).reshape(u.shape)


def apply_h(grid: Grid, u, q, v_eff, proj, e_kb, nd: int = 4):
    """h_k u for the orbitals u (n_b, n3, n2, n1) sharing one q."""
    return apply_local(grid, u, q, v_eff, nd) + apply_nonlocal(grid, u, proj, e_kb)


def dense_h(cell, q, v_eff, beta, disp, e_kb, nd: int = 4):
    """The Hamiltonian as an explicit (n_pts, n_pts) matrix, built entry by
    entry from the stencil definition (only for tiny grids)."""
    grid = Grid(cell)
    n1, n2, n3 = grid.n
    npts = grid.n_pts
    c, d = fd.weights_float(nd)
    H = np.zeros((npts, npts), dtype=np.complex128)

    def idx(i1, i2, i3):
        return ((i3 % n3) * n2 + (i2 % n2)) * n1 + (i1 % n1)

    q = np.asarray(q, dtype=np.float64)
    vflat = v_eff.reshape(-1)
    for i3 in range(n3):
        for i2 in range(n2):
            for i1 in range(n1):
                r = idx(i1, i2, i3)
                H[r, r] += 0.5 * float(q @ q) + vflat[r]
                for ax in range(3):
                    h = grid.h[ax]
                    H[r, r] += -0.5 * c[0] / (h * h)
                    for m in range(1, nd + 1):
                        for sgn in (1, -1):
                            off = [0, 0, 0]
                            off[ax] = sgn * m
                            col = idx(i1 + off[0], i2 + off[1], i3 + off[2])
                            H[r, col] += -0.5 * c[m] / (h * h)
                            H[r, col] += -1j * q[ax] * sgn * d[m] / h
    proj = phased_projectors(cell, beta, disp, q)
    for j in range(proj.shape[0]):
        H += e_kb[j] * grid.dv * np.outer(proj[j], proj[j].conj())
    return H
