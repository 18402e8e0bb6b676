"""Real-time propagation, density, current and the two-step average.

Eq. 1: i du/dt = h_k(t) u.  The paper does not name its propagator; the
reading used here (fixed for this build) is, for step n (t_n = n dt):
  1. v_eff = v_loc + v_Hxc[rho(t_n)], q = k + A(t_n + dt/2)  (fixed in the step)
  2. 4th-order Taylor:  t_0 = u,  t_m = (-i dt / m) h t_{m-1},  u(t_{n+1}) = sum_{m=0..4} t_m
  3. rho(t_{n+1}) (Eq. 3) and, in self-consistent mode, v_Hxc[rho(t_{n+1})]
  4. J(t_{n+1}) (Eqs. 5-6) with q = k + A(t_{n+1})
In frozen mode v_Hxc keeps its initial value.

Fields are given as samples A(j dt/2), j = 0..2n.  Eq. 11's impulsive
distortion is read as E(t) = k0 e delta(t), i.e. A(t) = -k0 e theta(t):
A = 0 before the kick (J(0-)) and A = -k0 e from t = 0+ on.  Eq. 15 is read
with the envelope argument divided by T_L:
A(t) = -(E0/w0) e sin^4(pi t / T_L) sin(w0 (t - T_L/2)) on (0, T_L).

Current (Eqs. 5-6) with pi_q = dh/dq = -i grad_FD + q + d V_NL / dq:
  <u|pi|u> = dV sum Re(u* (-i grad_FD u)) + q dV sum |u|^2
             + 2 sum_j E_j Im(conj(c_j) a_j),
  a_j = <beta~_j|u>, c_j = <d beta~_j|u>;
  J = -(1/Omega) (1/N_k) sum_{k,b} f_b <u|pi|u>.
Two-step (Eq. 9 and Sec. II.B steps 1-4): each shifted sub-simulation m is
propagated on its own; dJ_m = J_m - J_m(0-); J = (1/N_H) sum_m dJ_m.

Propagator variant (the paper leaves the propagator to its TDDFT code):
enforced time-reversal symmetry, step n:
  1. predictor: the step above from u(t_n), giving rho~(t_{n+1}) and
     v~_eff = v_loc + v_Hxc[rho~] (frozen mode: v_eff unchanged);
  2. u(t_{n+1}) = T4(dt/2; q = k + A(t_{n+1}), v~_eff) T4(dt/2; q = k + A(t_n), v_eff(t_n)) u(t_n),
     T4(tau) the 4th-order Taylor polynomial of exp(-i tau h);
  3. rho, v_Hxc and J(t_{n+1}) as above.
"""
from __future__ import annotations

import numpy as np

from workloads import CellSpec, Kick, Pulse
from . import fd
from .cell import Grid, local_potential, phased_projectors, projector_tables
from .hamiltonian import apply_h
from .hxc import v_hxc as build_v_hxc
from .kpoints import kpoints_cartesian
from .scf import density_from


# ----------------------------------------------------------------------------
# Fields
# ----------------------------------------------------------------------------
def vector_potential(field, t):
    """A(t) (3,) for a Kick (A(t>=0) = -k0 e) or a Pulse (Eq. 15)."""
    t = float(t)
    if isinstance(field, Kick):
        e = np.asarray(field.direction, dtype=np.float64)
        return -field.k0 * e if t >= 0.0 else np.zeros(3)
    if isinstance(field, Pulse):
        e = np.asarray(field.direction, dtype=np.float64)
        if t <= 0.0 or t >= field.t_pulse:
            return np.zeros(3)
        env = np.sin(np.pi * t / field.t_pulse) ** 4
        return -(field.e0 / field.omega0) * env * np.sin(field.omega0 * (t - field.t_pulse / 2.0)) * e
    if field is None:
        return np.zeros(3)
    raise TypeError(f"unknown field {field!r}")


def field_samples(field, dt, n_steps):
    """A(j dt/2), j = 0..2 n_steps, shape (2 n_steps + 1, 3); j = 0 is t = 0+."""
    return np.array([vector_potential(field, 0.5 * j * dt) for j in range(2 * n_steps + 1)])


# ----------------------------------------------------------------------------
# Observables
# ----------------------------------------------------------------------------
class Operators:
    """Tables of one cell: grid, v_loc, projectors."""

    def __init__(self, cell: CellSpec, nd: int = 4):
        self.cell = cell
        self.grid = Grid(cell)
        self.nd = nd
        self.vloc = local_potential(cell)
        self.beta, self.disp, self.e_kb = projector_tables(cell)
        self.n_proj = self.beta.shape[0]

    def proj(self, q):
        return phased_projectors(self.cell, self.beta, self.disp, q)

    def dproj(self, q):
        """(3, n_proj, n_pts): d_alpha beta~_j."""
        p = self.proj(q)
        out = np.empty((3,) + p.shape, dtype=np.complex128)
        for j in range(self.n_proj):
            a = j // 4
            for al in range(3):
                out[al, j] = self.disp[a, al].reshape(-1) * p[j]
        return out


def grad_fd(grid: Grid, u, nd: int = 4):
    """(grad_FD u) components (3, ...) on the periodic grid."""
    _, d = fd.weights_float(nd)
    out = []
    for ax, axis in enumerate((-1, -2, -3)):
        g = np.zeros_like(u)
        for m in range(1, nd + 1):
            g = g + d[m] * (np.roll(u, -m, axis=axis) - np.roll(u, m, axis=axis))
        out.append(g / grid.h[ax])
    return np.stack(out)


def momentum_expectation(ops: Operators, u, q):
    """<u_b|pi_q|u_b> (n_b, 3) for the orbitals u (n_b, n3, n2, n1) of one q."""
    grid = ops.grid
    dv = grid.dv
    g = grad_fd(grid, u, ops.nd)                       # (3, n_b, ...)
    kin = np.real(dv * np.sum(np.conj(u)[None] * (-1j) * g, axis=(-3, -2, -1))).T  # (n_b, 3)
    nrm = dv * np.sum(np.abs(u) ** 2, axis=(-3, -2, -1))
    out = kin + nrm[:, None] * np.asarray(q)[None, :]
    if ops.n_proj:
        flat = u.reshape(u.shape[0], -1)
        p = ops.proj(q)
        dp = ops.dproj(q)
        a = dv * flat @ p.conj().T                       # (n_b, n_proj)
        for al in range(3):
            c = dv * flat @ dp[al].conj().T
            out[:, al] += 2.0 * np.sum(ops.e_kb[None, :] * np.imag(np.conj(c) * a), axis=1)
    return out


def current(ops: Operators, u, kcart, A):
    """J (3,) of Eq. 5 for orbitals u (n_k, n_b, ...) at vector potential A."""
    n_k = u.shape[0]
    tot = np.zeros(3)
    for k in range(n_k):
        pe = momentum_expectation(ops, u[k], kcart[k] + A)
        tot += ops.cell.occ * np.sum(pe, axis=0)
    return -tot / (ops.grid.omega * n_k)


def norms(grid: Grid, u):
    return grid.dv * np.sum(np.abs(u) ** 2, axis=(-3, -2, -1))


# ----------------------------------------------------------------------------
# Propagation
# ----------------------------------------------------------------------------
def taylor4(ops: Operators, u, q, v_eff, dt):
    """u(t + dt) = sum_{m=0..4} t_m with t_m = (-i dt/m) h t_{m-1}, for the
    orbitals u (n_b, ...) of one q."""
    proj = ops.proj(q)
    t = u
    acc = u.copy()
    for m in range(1, 5):
        t = (-1j * dt / m) * apply_h(ops.grid, t, q, v_eff, proj, ops.e_kb, ops.nd)
        acc = acc + t
    return acc


def propagate(cell: CellSpec, kcart, u0, dt, n_steps, a_samples, hxc: str = "scf",
              v_hxc_frozen=None, ops: Operators | None = None, keep_state: bool = True,
              propagator: str = "taylor4"):
    """Propagate one (sub-)simulation with the Taylor-4 step ("taylor4") or the
    enforced-time-reversal-symmetry step ("etrs") of the module header.

    Returns dict(J (n_steps+1, 3) at t_0 = 0+ .. t_n, J0_minus (3,), rho,
    norms (n_k, n_b), u, v_hxc)."""
    ops = ops or Operators(cell)
    grid = ops.grid
    kcart = np.asarray(kcart, dtype=np.float64)
    u = np.array(u0, dtype=np.complex128, copy=True)
    rho = density_from(cell, u)
    if hxc == "frozen":
        vh = np.zeros_like(rho) if v_hxc_frozen is None else np.asarray(v_hxc_frozen)
    else:
        vh = build_v_hxc(grid, rho)
    j0m = current(ops, u, kcart, np.zeros(3))
    js = [current(ops, u, kcart, a_samples[0])]
    for n in range(n_steps):
        a_now = a_samples[2 * n]
        a_half = a_samples[2 * n + 1]
        a_next = a_samples[2 * n + 2]
        v_eff = ops.vloc + vh
        if propagator == "etrs":
            # predictor density at t_{n+1}, then the two half steps
            u_pred = np.stack([taylor4(ops, u[k], kcart[k] + a_half, v_eff, dt) for k in range(u.shape[0])])
            vh_pred = vh if hxc == "frozen" else build_v_hxc(grid, density_from(cell, u_pred))
            v_pred = ops.vloc + vh_pred
            for k in range(u.shape[0]):
                w = taylor4(ops, u[k], kcart[k] + a_now, v_eff, 0.5 * dt)
                u[k] = taylor4(ops, w, kcart[k] + a_next, v_pred, 0.5 * dt)
        elif propagator == "taylor4":
            for k in range(u.shape[0]):
                u[k] = taylor4(ops, u[k], kcart[k] + a_half, v_eff, dt)
        else:
            raise ValueError(f"unknown propagator {propagator!r}")
        rho = density_from(cell, u)
        if hxc != "frozen":
            vh = build_v_hxc(grid, rho)
        js.append(current(ops, u, kcart, a_next))
    return dict(J=np.array(js), J0_minus=j0m, rho=rho, norms=norms(grid, u),
                u=u if keep_state else None, v_hxc=vh)


def subsim_kpoints(sub):
    return kpoints_cartesian(sub.cell.a, sub.mp, sub.shift)


def two_step_average(results):
    """Sec. II.B step 4: J(t) = (1/N_H) sum_m (J_m(t) - J_m(0-))."""
    dj = [r["J"] - r["J0_minus"][None, :] for r in results]
    return np.mean(np.stack(dj), axis=0)


def two_step_standard_error(results):
    """Sec. III.B, discussion of the error bars of Fig. 6: the N_H
    sub-simulations are N_H data sets whose mean is the two-step result of
    Eq. 9, so the standard error of that mean is
        sigma_E(t) = sqrt( sum_m (dJ_m(t) - dJ(t))^2 / (N_H (N_H - 1)) ),
    per time sample and component (zero when N_H = 1).  Two passes (mean,
    then squared deviations).  Returns (dJ, sigma_E), each (n_t, 3)."""
    dj = [r["J"] - r["J0_minus"][None, :] for r in results]
    n = len(dj)
    mean = np.zeros_like(dj[0])
    for d in dj:
        mean = mean + d
    mean = mean / n
    if n < 2:
        return mean, np.zeros_like(mean)
    ss = np.zeros_like(mean)
    for d in dj:
        ss = ss + (d - mean) ** 2
    return mean, np.sqrt(ss / (n * (n - 1)))


def _run_one(args):
    sub, u0, hxc, v_frozen = args
    k = subsim_kpoints(sub)
    a = field_samples(sub.field, sub.dt, sub.n_steps)
    return propagate(sub.cell, k, u0, sub.dt, sub.n_steps, a, hxc=hxc, v_hxc_frozen=v_frozen,
                     keep_state=False)


def two_step(run, ground_states, hxc: str | None = None, v_frozen=None, workers: int = 1):
    """Run every sub-simulation of ``run`` from ``ground_states[m]`` (orbital
    arrays) and return (per-subsim results, averaged dJ)."""
    hxc = hxc or run.hxc
    jobs = [(sub, gs, hxc, v_frozen) for sub, gs in zip(run.subsims, ground_states)]
    if workers > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_run_one, jobs)
    else:
        res = [_run_one(j) for j in jobs]
    return res, two_step_average(res)
