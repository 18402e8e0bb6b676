"""Kohn-Sham ground state for the propagation's initial orbitals.

The paper starts every real-time run from converged Kohn-Sham orbitals
(Sec. II.B, steps 2-3; Sec. III.A: the first sampling provides converged
orbitals and v_Hxc).  It gives no solver; the reading used here:
fixed occupations (the n_bands lowest states of every k, f = 2), h_k at
A = 0, a block LOBPCG eigensolver per k with a kinetic preconditioner,
and Pulay (DIIS) density mixing until dV sum |rho_out - rho_in| / N_e <= tol.

Pinned (tests/test_oracle_scf.py) against results outside this module's
eigensolver and mixing: the free-electron closed form (the lowest plane waves
of the explicit stencil matrix, a constant v_xc, a uniform density) and a
brute-force SCF (explicit Hamiltonian matrix, dense Hermitian eigensolver,
plain linear mixing) on a tiny gapped cell.  No paper values exist for this
synthetic material; tests also check the eigen-residuals with the stencil
Hamiltonian.
"""
from __future__ import annotations

import numpy as np

from workloads import CellSpec, scf_start_vectors
from . import fd
from .cell import Grid, local_potential, phased_projectors, projector_tables
from .hamiltonian import apply_h
from .hxc import v_hxc as build_v_hxc


def _orth_rows(s: np.ndarray, rcond: float = 1e-11) -> np.ndarray:
    """Orthonormal rows spanning the rows of s (rank-revealing SVD)."""
    _, sv, vh = np.linalg.svd(s, full_matrices=False)
    keep = sv > sv[0] * rcond
    return vh[keep]


def kinetic_symbol(grid: Grid, q, nd: int = 4) -> np.ndarray:
    """Plane-wave eigenvalue of the FD kinetic operator -1/2 lap - i q.grad + q^2/2."""
    gx, gy, gz = grid.g_vectors()
    t = np.zeros(gx.shape)
    for ax, g in enumerate((gx, gy, gz)):
        h = grid.h[ax]
        t += -0.5 * fd.laplacian_symbol(g * h, nd) / (h * h) + q[ax] * fd.gradient_symbol(g * h, nd) / h
    return t + 0.5 * float(np.dot(q, q))


def lobpcg(apply, x0: np.ndarray, precond, n_want: int, tol: float, maxiter: int = 400):
    """Lowest eigenpairs of a Hermitian operator; vectors are rows.

    Returns (theta, X, residual_norms) with X orthonormal in the Euclidean
    inner product."""
    x = _orth_rows(x0)
    hx = apply(x)
    hs = x.conj() @ hx.T
    th, c = np.linalg.eigh(0.5 * (hs + hs.conj().T))
    x, hx = c.T @ x, c.T @ hx
    p = hp = None
    nb = x.shape[0]
    rn = np.full(nb, np.inf)
    for _ in range(maxiter):
        r = hx - th[:, None] * x
        rn = np.linalg.norm(r, axis=1)
        if np.max(rn[:n_want]) < tol:
            break
        w = precond(r, th)
        blocks = [x, w] if p is None else [x, w, p]
        q = _orth_rows(np.concatenate(blocks, axis=0))
        hq = apply(q)
        hs = q.conj() @ hq.T
        th_all, c = np.linalg.eigh(0.5 * (hs + hs.conj().T))
        xn = c[:, :nb].T @ q
        hxn = c[:, :nb].T @ hq
        m = x.conj() @ xn.T
        p = xn - m.T @ x
        hp = hxn - m.T @ hx
        x, hx, th = xn, hxn, th_all[:nb]
    return th, x, rn


def density_from(cell: CellSpec, u: np.ndarray) -> np.ndarray:
    """rho(r) = (1/N_k) sum_k sum_b f_b |u_kb(r)|^2 (Eq. 3 with Eq. 7's average)."""
    n_k = u.shape[0]
    return cell.occ * np.sum(np.abs(u) ** 2, axis=(0, 1)) / n_k


def solve_bands(cell, grid, q, v_eff, beta, disp, e_kb, x0, tol, n_want, maxiter=400):
    """Lowest eigenpairs of h_q at a fixed v_eff.

    The solver applies the FD kinetic operator through its exact
    plane-wave symbol (the periodic stencil is a circulant matrix, so FFT,
    multiply by the symbol, inverse FFT is the same operator up to
    rounding); ``ground_state`` re-checks the residuals with the stencil."""
    proj = phased_projectors(cell, beta, disp, q)
    shape = grid.n[::-1]
    tsym = kinetic_symbol(grid, q)
    ax = (-3, -2, -1)

    def apply(rows):
        u = rows.reshape((-1,) + shape)
        kin = np.fft.ifftn(tsym[None] * np.fft.fftn(u, axes=ax), axes=ax)
        out = kin + v_eff[None] * u
        out = out.reshape(rows.shape[0], -1)
        if proj.shape[0]:
            a = grid.dv * (rows @ proj.conj().T)
            out = out + (a * e_kb[None, :]) @ proj
        return out

    def precond(r, th):
        rr = np.fft.fftn(r.reshape((-1,) + shape), axes=ax)
        rr = rr / (1.0 + tsym)[None]
        return np.fft.ifftn(rr, axes=ax).reshape(r.shape[0], -1)

    return lobpcg(apply, x0, precond, n_want, tol, maxiter)


def stencil_residuals(cell, grid, kcart, u, v_eff, eps):
    """max_b || h u_b - eps_b u_b || per k with the stencil Hamiltonian
    (norm in the dV metric, orbitals dV-normalised)."""
    beta, disp, e_kb = projector_tables(cell)
    out = np.zeros(u.shape[0])
    for k in range(u.shape[0]):
        proj = phased_projectors(cell, beta, disp, kcart[k])
        hu = apply_h(grid, u[k], kcart[k], v_eff, proj, e_kb)
        r = hu - eps[k][:, None, None, None] * u[k]
        out[k] = float(np.max(np.sqrt(grid.dv * np.sum(np.abs(r) ** 2, axis=(-3, -2, -1)))))
    return out


def ground_state(cell: CellSpec, kcart: np.ndarray, seed: int = 0, tol: float = 1e-9,
                 eig_tol: float = 1e-8, max_scf: int = 80, n_extra: int = 4, mix: float = 0.35,
                 history: int = 8, hxc: str = "scf", v_hxc_fixed=None, verbose: bool = False):
    """Self-consistent (or fixed-potential) ground state on the k-set ``kcart``.

    Returns dict(u (n_k, n_b, n3, n2, n1), eps (n_k, n_b), rho, v_hxc,
    scf_error, residual)."""
    grid = Grid(cell)
    shape = grid.n[::-1]
    vloc = local_potential(cell)
    beta, disp, e_kb = projector_tables(cell)
    n_k = kcart.shape[0]
    nb = cell.n_bands
    nvec = nb + n_extra
    x = scf_start_vectors(n_k, nvec, grid.n_pts, seed)
    n_e = cell.occ * nb
    rho_in = np.full(shape, n_e / grid.omega)
    if hxc == "frozen":
        v_h = np.zeros(shape) if v_hxc_fixed is None else v_hxc_fixed
    else:
        v_h = build_v_hxc(grid, rho_in)
    hist_in, hist_f = [], []
    err = np.inf
    eps = np.zeros((n_k, nvec))
    resid = np.full(n_k, np.inf)
    iters = 1 if hxc == "frozen" else max_scf
    for it in range(iters):
        v_eff = vloc + v_h
        cur_tol = eig_tol if (hxc == "frozen" or err < 1e2 * tol) else max(eig_tol, min(1e-3, err * 1e-1))
        for k in range(n_k):
            th, xk, rn = solve_bands(cell, grid, kcart[k], v_eff, beta, disp, e_kb, x[k], cur_tol, nb)
            x[k] = xk
            eps[k] = th
            resid[k] = float(np.max(rn[:nb]))
        u = x[:, :nb].reshape((n_k, nb) + shape) / np.sqrt(grid.dv)
        rho_out = density_from(cell, u)
        if hxc == "frozen":
            break
        err = grid.dv * np.sum(np.abs(rho_out - rho_in)) / n_e
        if verbose:
            print(f"scf {it}: err={err:.3e} eig_tol={cur_tol:.1e}")
        if err < tol and cur_tol <= eig_tol:
            break
        f = rho_out - rho_in
        hist_in.append(rho_in.copy())
        hist_f.append(f.copy())
        if len(hist_in) > history:
            hist_in.pop(0)
            hist_f.pop(0)
        m = len(hist_f)
        bmat = np.zeros((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                bmat[i, j] = np.sum(hist_f[i] * hist_f[j])
        bmat[m, :m] = 1.0
        bmat[:m, m] = 1.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        try:
            coef = np.linalg.solve(bmat, rhs)[:m]
        except np.linalg.LinAlgError:
            coef = np.zeros(m)
            coef[-1] = 1.0
        rho_in = sum(coef[i] * (hist_in[i] + mix * hist_f[i]) for i in range(m))
        rho_in = np.maximum(rho_in, 0.0)
        v_h = build_v_hxc(grid, rho_in)
    u = x[:, :nb].reshape((n_k, nb) + shape) / np.sqrt(grid.dv)
    return dict(u=u, eps=eps[:, :nb], eps_all=eps, rho=density_from(cell, u), v_hxc=v_h,
                scf_error=float(err), residual=resid,
                stencil_residual=stencil_residuals(cell, grid, kcart, u, vloc + v_h, eps[:, :nb]))
