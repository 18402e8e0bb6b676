"""Pins of the oracle's propagation, current and two-step average.

* Taylor-4: the recurrence equals the dense-matrix polynomial
  sum_{m<=4} (-i dt H)^m/m! u; an eigenvector's norm changes by
  |T4(-i x)|^2 = 1 - x^6/72 + x^8/576 per step.
* Current (Eqs. 5-6): <u|pi_q|u> equals d<u|h_q|u>/dq by central finite
  differences (checks the kinetic, the q and the non-local commutator term).
* Free electrons: plane waves in an empty cell follow the closed form of
  ``analysis.free_electron_current`` (kick and pulse); the windowed
  transform of the kick response gives the Drude eps = 1 - 4 pi n / w^2.
* Symmetry (diamond, symmetric k-set, kick along x): J_y = J_z = 0 and
  dJ(-k0) = -dJ(k0) (inversion) to the SCF tolerance.
* Gauge: (k, A = -k0 e) and (k - k0 e, A = 0) give the same orbitals.
* Two-step exactness (Eq. 9 at frozen v_Hxc): the average of dJ_m over the
  lattice-shifted subgrids equals the plain full-grid run; same for rho.
"""
import numpy as np
import pytest

import workloads as W
from oracle import analysis, dynamics, kpoints, scf
from oracle import cell as C
from oracle.hamiltonian import dense_h


def _tiny():
    return W.cell_tiny(atoms="pair", n=(6, 6, 6), a=(5.0, 5.0, 5.0), proj_half=3.0, n_bands=3)


def test_taylor_recurrence_equals_dense_polynomial():
    cell = _tiny()
    ops = dynamics.Operators(cell)
    v = ops.vloc + 0.05
    q = np.array([0.1, 0.2, -0.3])
    H = dense_h(cell, q, v, ops.beta, ops.disp, ops.e_kb)
    u = W.random_complex((3, 6, 6, 6), 9)
    dt = 0.08
    got = dynamics.taylor4(ops, u, q, v, dt).reshape(3, -1).T
    M = -1j * dt * H
    poly = np.eye(216) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    np.testing.assert_allclose(got, poly @ u.reshape(3, -1).T, atol=1e-12)


def test_taylor_norm_factor_closed_form():
    x = np.linspace(-2.5, 2.5, 41)
    np.testing.assert_allclose(np.abs(analysis.taylor4_factor(-1j * x)) ** 2,
                               1 - x ** 6 / 72 + x ** 8 / 576, atol=1e-13)
    cell = _tiny()
    ops = dynamics.Operators(cell)
    q = np.array([0.05, 0.0, 0.1])
    H = dense_h(cell, q, ops.vloc, ops.beta, ops.disp, ops.e_kb)
    w, V = np.linalg.eigh(H)
    g = ops.grid
    for idx in (0, 50, 215):
        u = (V[:, idx] / np.sqrt(g.dv)).reshape(1, 6, 6, 6)
        un = dynamics.taylor4(ops, u, q, ops.vloc, 0.08)
        xx = w[idx] * 0.08
        np.testing.assert_allclose(dynamics.norms(g, un), 1 - xx ** 6 / 72 + xx ** 8 / 576, rtol=1e-11)


def test_current_is_energy_derivative():
    cell = W.cell_tiny(atoms="offgrid", n=(8, 8, 8), a=(6.0, 6.0, 6.0))
    ops = dynamics.Operators(cell)
    g = ops.grid
    u = W.random_complex((2, 8, 8, 8), 4)
    u /= np.sqrt(dynamics.norms(g, u))[:, None, None, None]
    q = np.array([0.17, -0.29, 0.41])
    pe = dynamics.momentum_expectation(ops, u, q)
    from oracle.hamiltonian import apply_h

    def energy(qq):
        hu = apply_h(g, u, qq, ops.vloc, ops.proj(qq), ops.e_kb)
        return np.real(g.dv * np.sum(np.conj(u) * hu, axis=(1, 2, 3)))

    h = 1e-5
    for al in range(3):
        e = np.zeros(3)
        e[al] = h
        fdv = (energy(q + e) - energy(q - e)) / (2 * h)
        np.testing.assert_allclose(pe[:, al], fdv, rtol=1e-7, atol=1e-8)
    # the non-local term matters at this size
    ops0 = dynamics.Operators(cell.replace(use_projectors=False))
    assert np.max(np.abs(dynamics.momentum_expectation(ops0, u, q) - pe)) > 1e-3


@pytest.mark.parametrize("field", ["kick", "pulse"])
def test_free_electron_closed_form(field):
    cell = W.free_electron(W.cell_tiny(atoms="none", n=(8, 8, 8), a=(6.0, 6.5, 7.0), n_bands=4))
    g = C.Grid(cell)
    kc = kpoints.kpoints_cartesian(cell.a, (2, 2, 1), (0.0, 0.0, 0.0))
    gints = analysis.lowest_plane_waves(g, kc, 4)
    u0 = analysis.plane_wave_orbitals(g, gints)
    dt, n = 0.1, 12
    f = W.Kick(k0=0.01, direction=(0.6, 0.8, 0.0)) if field == "kick" else W.Pulse(e0=0.05, omega0=0.3, t_pulse=1.2)
    a = dynamics.field_samples(f, dt, n)
    res = dynamics.propagate(cell, kc, u0, dt, n, a)
    jc, j0, w = analysis.free_electron_current(g, cell.occ, kc, gints, dt, n, a)
    np.testing.assert_allclose(res["J"], jc, rtol=0, atol=1e-12 * np.max(np.abs(jc)))
    np.testing.assert_allclose(res["J0_minus"], j0, atol=1e-14)
    np.testing.assert_allclose(res["norms"], w, rtol=1e-12)
    rho_uniform = cell.occ * np.sum(w) / (g.omega * kc.shape[0])
    np.testing.assert_allclose(res["rho"], rho_uniform, rtol=1e-12)


@pytest.mark.parametrize("field", ["kick", "pulse"])
def test_etrs_free_electron_closed_form(field):
    """The ETRS step on plane waves in an empty cell: two half-step Taylor factors
    with the kinetic energy at A(t_n) and A(t_{n+1}) and v_xc of the predictor density."""
    cell = W.free_electron(W.cell_tiny(atoms="none", n=(8, 8, 8), a=(6.0, 6.5, 7.0), n_bands=4))
    g = C.Grid(cell)
    kc = kpoints.kpoints_cartesian(cell.a, (2, 2, 1), (0.0, 0.0, 0.0))
    gints = analysis.lowest_plane_waves(g, kc, 4)
    u0 = analysis.plane_wave_orbitals(g, gints)
    # a long step, so that |T4|^2 departs from 1 and the two schemes differ visibly
    dt, n = 0.45, 12
    f = W.Kick(k0=0.05, direction=(0.6, 0.8, 0.0)) if field == "kick" else W.Pulse(e0=0.3, omega0=0.3, t_pulse=5.4)
    a = dynamics.field_samples(f, dt, n)
    res = dynamics.propagate(cell, kc, u0, dt, n, a, propagator="etrs")
    jc, j0, w = analysis.free_electron_current(g, cell.occ, kc, gints, dt, n, a, propagator="etrs")
    np.testing.assert_allclose(res["J"], jc, rtol=0, atol=1e-12 * np.max(np.abs(jc)))
    np.testing.assert_allclose(res["norms"], w, rtol=1e-12)
    # and it differs from the Taylor-4 step beyond round-off (the pin can tell them apart)
    jt, _, _ = analysis.free_electron_current(g, cell.occ, kc, gints, dt, n, a)
    assert np.max(np.abs(jt - jc)) > 1e-9 * np.max(np.abs(jc))


def test_etrs_constant_h_is_two_half_taylor_steps():
    """Frozen v_Hxc and a constant field: the predictor does not matter and one ETRS
    step is the square of the dense half-step polynomial sum_{m<=4} (-i dt/2 H)^m/m!."""
    cell = _tiny()
    ops = dynamics.Operators(cell)
    kc = np.array([[0.1, 0.2, -0.3]])
    kick = W.Kick(k0=0.02, direction=(0.0, 0.6, 0.8))
    dt = 0.08
    a = dynamics.field_samples(kick, dt, 1)
    u = W.random_complex((1, 3, 6, 6, 6), 13)
    res = dynamics.propagate(cell, kc, u, dt, 1, a, hxc="frozen", v_hxc_frozen=np.zeros((6, 6, 6)),
                             propagator="etrs")
    q = kc[0] + a[1]
    H = dense_h(cell, q, ops.vloc, ops.beta, ops.disp, ops.e_kb)
    M = -0.5j * dt * H
    half = np.eye(216) + M + M @ M / 2 + M @ M @ M / 6 + M @ M @ M @ M / 24
    np.testing.assert_allclose(res["u"][0].reshape(3, -1).T, half @ half @ u[0].reshape(3, -1).T, atol=1e-12)


def test_etrs_second_order_in_dt():
    """Self-consistent v_Hxc under a pulse: the ETRS current at t = 0.96 converges
    at second order or better in dt (error ratio >= 3.5 when dt halves)."""
    cell = W.cell_tiny(atoms="pair", n=(6, 6, 6), a=(5.0, 5.0, 5.0), proj_half=3.0, n_bands=2)
    g = C.Grid(cell)
    kc = kpoints.kpoints_cartesian(cell.a, (1, 1, 1), (0.25, 0.5, 0.0))
    u0 = W.random_orbitals(1, 2, cell.n, g.dv, seed=8)
    pulse = W.Pulse(e0=0.3, omega0=1.5, t_pulse=0.96)
    t_end = 0.96

    def run(n):
        dt = t_end / n
        return dynamics.propagate(cell, kc, u0, dt, n, dynamics.field_samples(pulse, dt, n),
                                  propagator="etrs")["J"][-1]

    ref = run(96)
    e1 = np.linalg.norm(run(6) - ref)
    e2 = np.linalg.norm(run(12) - ref)
    assert e1 / e2 >= 3.5, (e1, e2)


def test_free_electron_drude_limit():
    g = C.Grid(W.free_electron(W.cell_a()))
    n_e = 32.0
    n = n_e / g.omega
    dt, steps, k0 = 0.01, 600000, 0.005   # trapezoid bias (w dt)^2/12 and window edge 12/(w T)^2 stay < 1e-5
    dj = np.full(steps + 1, n * k0)   # ideal free-electron response dJ = n k0 for t > 0
    om = np.linspace(0.5, 1.0, 6)
    eps = analysis.dielectric(dj, dt, k0, om)
    np.testing.assert_allclose(eps, 1 - 4 * np.pi * n / om ** 2, atol=2e-5)
    # and the closed-form FD current reproduces dJ = n k0 (linear regime)
    cell = W.free_electron(W.cell_tiny(atoms="none", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4))
    gg = C.Grid(cell)
    kc = kpoints.kpoints_cartesian(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    gints = analysis.lowest_plane_waves(gg, kc, 4)
    a = dynamics.field_samples(W.Kick(k0=k0), 0.08, 3)
    jc, j0, _ = analysis.free_electron_current(gg, cell.occ, kc, gints, 0.08, 3, a)
    np.testing.assert_allclose((jc - j0)[:, 0], cell.occ * 4 / gg.omega * k0, rtol=1e-6)


@pytest.fixture(scope="module")
def coarse_ground_state():
    cell = W.cell_a_coarse(n=8)
    kc = kpoints.kpoints_cartesian(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    gs = scf.ground_state(cell, kc, seed=3, tol=1e-10, eig_tol=1e-10)
    assert gs["scf_error"] < 1e-10
    assert np.max(gs["stencil_residual"]) < 1e-8
    return cell, kc, gs


def test_symmetry_transverse_current_and_inversion(coarse_ground_state):
    cell, kc, gs = coarse_ground_state
    dt, n = 0.08, 6
    ops = dynamics.Operators(cell)
    out = {}
    for sgn in (1, -1):
        a = dynamics.field_samples(W.Kick(k0=sgn * 0.005), dt, n)
        out[sgn] = dynamics.propagate(cell, kc, gs["u"], dt, n, a, ops=ops)
    djp = out[1]["J"] - out[1]["J0_minus"]
    djm = out[-1]["J"] - out[-1]["J0_minus"]
    scale = np.max(np.abs(djp[:, 0]))
    assert scale > 1e-6
    assert np.max(np.abs(djp[:, 1:])) < 1e-7 * scale
    assert np.max(np.abs(out[1]["J0_minus"])) < 1e-8 * scale / 1e-3
    np.testing.assert_allclose(djm, -djp, atol=1e-7 * scale)


def test_stationary_without_kick(coarse_ground_state):
    cell, kc, gs = coarse_ground_state
    n, dt = 10, 0.08
    a = dynamics.field_samples(W.Kick(k0=0.0), dt, n)
    r = dynamics.propagate(cell, kc, gs["u"], dt, n, a)
    assert np.max(np.abs(r["J"] - r["J0_minus"])) < 1e-9
    # rho changes only by the Taylor-4 norm loss x^6/72 per step (x = eps dt)
    x = np.max(np.abs(gs["eps"])) * dt
    bound = 2 * n * x ** 6 / 72 + 1e-9
    assert np.max(np.abs(r["rho"] - gs["rho"])) < bound * np.max(gs["rho"])


def test_gauge_kick_equals_k_shift(coarse_ground_state):
    cell, kc, gs = coarse_ground_state
    k0 = 0.01
    a = dynamics.field_samples(W.Kick(k0=k0), 0.08, 3)
    r1 = dynamics.propagate(cell, kc, gs["u"], 0.08, 3, a)
    kshift = kc - np.array([k0, 0, 0])
    r2 = dynamics.propagate(cell, kshift, gs["u"], 0.08, 3, np.zeros_like(a))
    np.testing.assert_allclose(r1["u"], r2["u"], atol=1e-13)
    np.testing.assert_allclose(r1["J"][1:], r2["J"][1:], atol=1e-14)


def test_two_step_exactness_frozen_potential():
    """Frozen v_Hxc: (1/N_H) sum_m dJ_m over 8 shifted 2^3 grids = MP 4^3."""
    cell = W.cell_a_coarse(n=8, n_bands=4)
    ops = dynamics.Operators(cell)
    g = ops.grid
    v_fix = 0.02 * np.cos(2 * np.pi * np.arange(8) / 8)[None, None, :] * np.ones((8, 8, 8))
    full_k = kpoints.kpoints_cartesian(cell.a, (4, 4, 4), (0.0, 0.0, 0.0))
    gs = scf.ground_state(cell, full_k, seed=2, hxc="frozen", v_hxc_fixed=v_fix, eig_tol=1e-9)
    key = {tuple(np.round(k, 12)): i for i, k in enumerate(full_k)}
    dt, n = 0.08, 4
    a = dynamics.field_samples(W.Kick(k0=0.005), dt, n)
    full = dynamics.propagate(cell, full_k, gs["u"], dt, n, a, hxc="frozen", v_hxc_frozen=v_fix, ops=ops)
    res = []
    rhos = []
    for s in W.lattice_shifts(2):
        ks = kpoints.kpoints_cartesian(cell.a, (2, 2, 2), s)
        idx = [key[tuple(np.round(k, 12))] for k in ks]
        r = dynamics.propagate(cell, ks, gs["u"][idx], dt, n, a, hxc="frozen", v_hxc_frozen=v_fix, ops=ops)
        res.append(r)
        rhos.append(r["rho"])
    avg = dynamics.two_step_average(res)
    dfull = full["J"] - full["J0_minus"]
    assert np.max(np.abs(dfull[:, 0])) > 1e-6
    np.testing.assert_allclose(avg, dfull, atol=1e-12 * np.max(np.abs(dfull)) + 1e-17)
    np.testing.assert_allclose(np.mean(rhos, axis=0), full["rho"], rtol=1e-12)


def test_local_current_correlation_form():
    """On the periodic grid the kinetic part of <u|pi|u> (Eqs. 5-6), summed over
    the grid, equals 2 sum_m (d_m / h) sum_r Im(conj(u(r)) u(r + m e_ax)): the
    form in which the GPU observation kernels accumulate it (forward neighbours
    only).  Checked per band and axis on a ragged grid with random orbitals."""
    from oracle.cell import Grid
    from oracle.dynamics import grad_fd
    from oracle import fd
    cell = W.cell_tiny(n=(8, 10, 12), a=(6.0, 7.0, 8.0), n_bands=3)
    grid = Grid(cell)
    u = W.random_orbitals(1, 3, cell.n, grid.dv, seed=9)[0]
    g = grad_fd(grid, u)
    kin = np.real(np.sum(np.conj(u)[None] * (-1j) * g, axis=(-3, -2, -1)))   # (3, n_b)
    _, d = fd.weights_float(4)
    corr = np.zeros_like(kin)
    for ax, axis in enumerate((-1, -2, -3)):
        for m in range(1, 5):
            fwd = np.roll(u, -m, axis=axis)                                    # u(r + m e_ax)
            corr[ax] += 2.0 * d[m] / grid.h[ax] * np.sum(np.imag(np.conj(u) * fwd), axis=(-3, -2, -1))
    np.testing.assert_allclose(corr, kin, rtol=0, atol=1e-12 * np.max(np.abs(kin)))
