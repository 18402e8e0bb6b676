"""GPU parity: the library (C ABI) against the oracle on the same seeded inputs.

FP64 bars: err_J <= 1e-10 and err_rho, err_norm <= 1e-12 (element by element
over every time step / grid point / orbital).  FP32 is compared with bars
derived from float rounding (see the FP32 test).  Cases span several point
tiles (128 points) and band groups, a ragged grid (10 x 12 x 14, non-grid
atoms), a pulse and a kick, self-consistent and frozen v_Hxc, the two-step
average, checkpoint/restart, the free-electron closed form and the full
two-step workload of 64 shifted 4^3 subgrids (sampled).
"""
import numpy as np
import pytest

import workloads as W
from oracle import analysis, dynamics, kpoints, scf
from oracle.cell import Grid, local_potential

from gpu_common import (FP32_J_TOL, FP32_NORM_TOL, FP32_RHO_TOL, FP64_J_TOL, FP64_RHO_TOL, compare, gpu_run,
                        oracle_run, random_subsim)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2112_00920_gb300 import build_library
    build_library()


def _tiny_pair():
    return W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4)


def test_cell_tables_match_oracle():
    from paper_2112_00920_gb300 import Propagator
    for cell in (W.cell_a(), W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0))):
        P = Propagator("fp64")
        cid = P.add_cell_spec(cell)
        v, _ = P.cell_tables(cid)
        ref = local_potential(cell)
        assert np.max(np.abs(v - ref)) <= 1e-12 * np.max(np.abs(ref))
        P.close()




@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_parity_fp32_tc_small(case):
    """Tensor-core mode on a tiny cell (4 point tiles) and a ragged 10 x 12 x 14 grid
    (13.1 tiles, non-grid atoms, pulse)."""
    if case == "tiny":
        cell = _tiny_pair()
        subs = [random_subsim(cell, (2, 2, 1), (0.25, 0.5, 0.0), 0.08, 6, W.Kick(k0=0.01), seed=1)]
    else:
        cell = W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0), n_bands=3)
        pulse = W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8, direction=(0.3, 0.4, 0.866))
        subs = [random_subsim(cell, (5, 1, 1), (0.1, 0.2, 0.3), 0.05, 6, pulse, seed=2)]
    _, g = gpu_run(cell, subs, precision="fp32_tc")
    o = oracle_run(cell, subs[0])
    errs = compare(g[0], o, FP32_J_TOL, FP32_RHO_TOL, FP32_NORM_TOL)
    print(f"fp32_tc {case}:", errs)


FP32_CASES = {
    # fused z-march stage, depth 8
    "tiny8": lambda: (_tiny_pair(), (2, 2, 1), (0.25, 0.5, 0.0), 0.08, W.Kick(k0=0.01)),
    # fused stage, depth 16, n1 != n2, non-grid atoms, 120 columns (last warp partly idle), pulse
    "ragged16": lambda: (W.cell_tiny(atoms="offgrid", n=(10, 12, 16), a=(7.0, 8.0, 9.0), n_bands=3), (3, 1, 1),
                         (0.1, 0.2, 0.3), 0.05,
                         W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8, direction=(0.3, 0.4, 0.866))),
    # fused stage without projectors
    "free16": lambda: (W.free_electron(W.cell_tiny(n=(12, 12, 16), a=(7.0, 7.0, 9.0), n_bands=2)), (2, 1, 1),
                       (0.5, 0.0, 0.25), 0.08, W.Kick(k0=0.02)),
    # generic point-parallel kernels (depth 14)
    "ragged14": lambda: (W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0), n_bands=3), (5, 1, 1),
                         (0.1, 0.2, 0.3), 0.05,
                         W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8, direction=(0.3, 0.4, 0.866))),
}


@pytest.mark.parametrize("case", sorted(FP32_CASES))
def test_parity_fp32_small(case):
    """Single-precision mode against the oracle, 6 steps: the fused stage with the
    factorised projector contractions (depths 8 and 16, ragged columns, no
    projectors) and the generic kernels."""
    cell, mp, shift, dt, field = FP32_CASES[case]()
    subs = [random_subsim(cell, mp, shift, dt, 6, field, seed=21)]
    _, g = gpu_run(cell, subs, precision="fp32")
    o = oracle_run(cell, subs[0])
    errs = compare(g[0], o, FP32_J_TOL, FP32_RHO_TOL, FP32_NORM_TOL)
    print(f"fp32 {case}:", errs)


@pytest.mark.parametrize("precision,n,per_step", [("fp32", (8, 8, 8), 9), ("fp32", (16, 16, 16), 6),
                                                  ("fp32", (10, 12, 14), 21),
                                                  ("fp32_tc", (8, 8, 8), 18), ("fp64", (8, 8, 8), 14)])
def test_kernel_launches_per_step(precision, n, per_step):
    """Which kernel sequence a step runs (after the first): the fused single-precision
    stage takes field + 4 stages + observation + finalize + v_Hxc (stage 4 leaves the
    projections of the next step and of the current), and on 16^3 cells whose atoms
    form z groups the four stages are one launch; v_Hxc is two launches on grids of
    power-of-two axes up to 16 (FFT Hartree, then PZ81 and v_eff; 9 otherwise); the generic and FP64 paths take a
    projection before each of the 4 stages and one for the current; the
    tensor-core mode adds a ket launch before each stage."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    cell = W.cell_tiny(atoms="pair", n=n, a=(6.0, 6.0, 6.0), n_bands=4)
    s = random_subsim(cell, (1, 1, 1), (0.25, 0.25, 0.25), 0.08, 4, W.Kick(k0=0.01), seed=5)
    P = Propagator(precision)
    cid = P.add_cell_spec(cell)
    sid = P.add_subsim(cid, shifted_kpoints(cell.a, s["mp"], s["shift"]), s["dt"], 4)
    P.load_ground_state(sid, s["psi"])
    P.set_kick(sid, 0.01, (1.0, 0.0, 0.0))
    P.set_graphs(False)
    P.propagate(1)
    before = P.launches()
    P.propagate(2)
    assert P.launches() - before == 2 * per_step
    P.close()


def test_tc_mode_rejects_unsupported_cells():
    from paper_2112_00920_gb300 import Propagator, TsbzError
    P = Propagator("fp32_tc")
    with pytest.raises(TsbzError) as e:
        P.add_cell_spec(W.cell_tiny(atoms="one", n=(9, 9, 9), n_bands=40, proj_half=4.5))
    assert e.value.code == -1
    P.close()


def test_parity_tiny_fp64_kick():
    cell = _tiny_pair()
    subs = [random_subsim(cell, (2, 2, 1), (0.25, 0.5, 0.0), 0.08, 10, W.Kick(k0=0.01), seed=1)]
    _, g = gpu_run(cell, subs)
    o = oracle_run(cell, subs[0])
    compare(g[0], o, FP64_J_TOL, FP64_RHO_TOL)


def test_parity_ragged_fp64_pulse():
    cell = W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0), n_bands=3)
    pulse = W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8, direction=(0.3, 0.4, 0.866))
    subs = [random_subsim(cell, (5, 1, 1), (0.1, 0.2, 0.3), 0.05, 8, pulse, seed=2)]
    _, g = gpu_run(cell, subs)
    o = oracle_run(cell, subs[0])
    compare(g[0], o, FP64_J_TOL, FP64_RHO_TOL)


def test_parity_many_bands_fp64():
    """40 bands: two band groups of the point kernels and three band blocks of the bra."""
    cell = W.cell_tiny(atoms="one", n=(9, 9, 9), a=(6.0, 6.0, 6.0), n_bands=40, proj_half=4.5)
    subs = [random_subsim(cell, (1, 1, 2), (0.3, 0.3, 0.3), 0.05, 4, W.Kick(k0=0.02, direction=(0, 1, 0)), seed=3)]
    _, g = gpu_run(cell, subs)
    o = oracle_run(cell, subs[0])
    compare(g[0], o, FP64_J_TOL, FP64_RHO_TOL)


def test_parity_frozen_fp64():
    cell = _tiny_pair()
    vf = 0.03 * np.sin(2 * np.pi * np.arange(512).reshape(8, 8, 8) / 37.0)
    subs = [random_subsim(cell, (1, 2, 2), (0.5, 0.25, 0.75), 0.08, 6, W.Kick(k0=0.01), seed=4)]
    _, g = gpu_run(cell, subs, hxc="frozen", v_frozen=vf)
    o = oracle_run(cell, subs[0], hxc="frozen", v_frozen=vf)
    compare(g[0], o, FP64_J_TOL, FP64_RHO_TOL)


@pytest.fixture(scope="module")
def mp2_ground_state():
    run = W.mp2_kick_run()
    sub = run.subsims[0]
    k = kpoints.kpoints_cartesian(sub.cell.a, sub.mp, sub.shift)
    gs = scf.ground_state(sub.cell, k, seed=W.MASTER_SEED, tol=1e-8, eig_tol=1e-8)
    return sub, gs


def test_parity_mp2_fp64(mp2_ground_state):
    """Cell A, MP 2^3, SCF ground state, kick 0.005 x, dt 0.08 (20 of the 100 steps)."""
    sub, gs = mp2_ground_state
    s = dict(mp=sub.mp, shift=sub.shift, psi=gs["u"], dt=sub.dt, n_steps=20, field=sub.field)
    _, g = gpu_run(sub.cell, [s])
    o = oracle_run(sub.cell, s)
    compare(g[0], o, FP64_J_TOL, FP64_RHO_TOL)
    # transverse current vanishes by symmetry on the GPU as well
    dj = g[0]["J"] - g[0]["J0m"]
    assert np.max(np.abs(dj[:, 1:])) < 1e-6 * np.max(np.abs(dj[:, 0]))


def test_gpu_ground_state_mp2(mp2_ground_state):
    """The GPU ground-state solver on the MP 2^3 k-set of cell A (16^3,
    16 bands) from plane-wave starting orbitals: its density matches the oracle's
    SCF (both converged to dV sum |rho_out - rho_in| / N_e <= 1e-8), and so does the
    kicked current propagated from each ground state."""
    import time
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    sub, gs = mp2_ground_state
    cell = sub.cell
    start = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), 8)
    P = Propagator("fp64")
    cid = P.add_cell_spec(cell)
    sid = P.add_subsim(cid, shifted_kpoints(cell.a, sub.mp, sub.shift), sub.dt, 10)
    P.load_ground_state(sid, start)
    t0 = time.perf_counter()
    iters, err = P.ground_state(max_iter=80, tol=1e-8)
    print(f"GPU SCF, cell A MP 2^3: {iters} iterations, error {err:.2e}, {time.perf_counter() - t0:.2f} s")
    rel = np.max(np.abs(P.density(sid) - gs["rho"])) / np.max(gs["rho"])
    assert rel <= 1e-6, rel
    P.set_kick(sid, sub.field.k0, sub.field.direction)
    P.propagate(10)
    J, j0 = P.current(sid)
    P.close()
    o = oracle_run(cell, dict(mp=sub.mp, shift=sub.shift, psi=gs["u"], dt=sub.dt, n_steps=10, field=sub.field))
    dj, djo = J - j0[None, :], o["J"] - o["J0_minus"][None, :]
    e = float(np.max(np.abs(dj - djo)) / np.max(np.abs(djo)))
    print("density", rel, "dJ", e)
    assert e <= 1e-5, e


def test_parity_mp2_fp32(mp2_ground_state):
    """FP32 stencil/Taylor/projectors with FP64 rho/J: errors stay at float
    rounding (~1e-7 per step on each orbital, accumulated over 20 steps)."""
    sub, gs = mp2_ground_state
    s = dict(mp=sub.mp, shift=sub.shift, psi=gs["u"], dt=sub.dt, n_steps=20, field=sub.field)
    _, g = gpu_run(sub.cell, [s], precision="fp32")
    o = oracle_run(sub.cell, s)
    dj_g = g[0]["J"] - g[0]["J0m"]
    dj_o = o["J"] - o["J0_minus"]
    e_dj = float(np.max(np.abs(dj_g - dj_o)) / np.max(np.abs(dj_o)))
    # 20 steps from the SCF ground state: measured err_J 6.1e-7, err_dJ 5.4e-7 (GB300); bars >= 10x
    errs = compare(g[0], o, 7e-6, FP32_RHO_TOL, FP32_NORM_TOL)
    assert e_dj < 7e-6, e_dj
    print("fp32 mp2:", errs, "err_dJ", e_dj)


def test_parity_mp2_fp32_tc(mp2_ground_state):
    """Tensor-core mode on cell A, MP 2^3 (SCF ground state, 20 steps)."""
    sub, gs = mp2_ground_state
    s = dict(mp=sub.mp, shift=sub.shift, psi=gs["u"], dt=sub.dt, n_steps=20, field=sub.field)
    _, g = gpu_run(sub.cell, [s], precision="fp32_tc")
    o = oracle_run(sub.cell, s)
    dj_g = g[0]["J"] - g[0]["J0m"]
    dj_o = o["J"] - o["J0_minus"]
    e_dj = float(np.max(np.abs(dj_g - dj_o)) / np.max(np.abs(dj_o)))
    # measured err_J 1.1e-6, err_dJ 1.2e-6 (GB300); bars 10x
    errs = compare(g[0], o, 1.2e-5, FP32_RHO_TOL, FP32_NORM_TOL)
    assert e_dj < 1.2e-5, e_dj
    print("fp32_tc mp2:", errs, "err_dJ", e_dj)


def test_free_electron_closed_form_gpu():
    """Plane waves in an empty 16^3 cell: J(t) follows the closed form."""
    cell = W.free_electron(W.cell_a(n_bands=16))
    g = Grid(cell)
    k = kpoints.kpoints_cartesian(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    gints = analysis.lowest_plane_waves(g, k, 16)
    psi = analysis.plane_wave_orbitals(g, gints)
    n = 15
    kick = W.Kick(k0=0.005)
    a = dynamics.field_samples(kick, 0.08, n)
    jc, j0, w = analysis.free_electron_current(g, cell.occ, k, gints, 0.08, n, a)
    s = dict(mp=(2, 2, 2), shift=(0, 0, 0), psi=psi, dt=0.08, n_steps=n, field=kick)
    _, out = gpu_run(cell, [s])
    assert np.max(np.abs(out[0]["J"] - jc)) <= 1e-10 * np.max(np.abs(jc))
    np.testing.assert_allclose(out[0]["J0m"], j0, atol=1e-13 * np.max(np.abs(jc)))
    np.testing.assert_allclose(out[0]["norms"], w, rtol=1e-12)


def test_two_step_average_gpu():
    """Sub-simulation id -1 returns (1/N_H) sum_m (J_m - J_m(0-)) (Eq. 9)."""
    cell = _tiny_pair()
    subs = [random_subsim(cell, (1, 1, 2), s, 0.08, 5, W.Kick(k0=0.01), seed=5, tag=i)
            for i, s in enumerate(W.lattice_shifts(2))]
    P, g = gpu_run(cell, subs)
    avg, _ = P.current(-1)
    orcs = [oracle_run(cell, s) for s in subs]
    ref = dynamics.two_step_average(orcs)
    assert np.max(np.abs(avg - ref)) <= FP64_J_TOL * np.max(np.abs(ref))
    for gi, oi in zip(g, orcs):
        compare(gi, oi, FP64_J_TOL, FP64_RHO_TOL)


@pytest.mark.parametrize("precision,n", [("fp64", 8), ("fp32", 8), ("fp32", 16), ("fp32", 32), ("fp32_tc", 8),
                                         ("fp32_tc", 16)])
def test_checkpoint_restart_bitwise(precision, n):
    """propagate(6) == propagate(3) + get_state/load_state + propagate(3), bit for bit
    (8^3, 16^3 and 32 x 16 x 16 grids: each shape's own stage and projection
    kernels; the 16^3 cell is 10 bohr wide so that dt E_max of the FD kinetic
    stays inside the Taylor-4 stability range, about 2.8).  On the 32-point rows
    (slab kernels) a continuing run starts each step from the projections that
    the last observation left in P, a restarted one from a fresh projection
    pass: the two must agree bit for bit."""
    if n == 32:
        cell = W.cell_tiny(atoms="pair", n=(32, 16, 16), a=(20.0, 10.0, 10.0), n_bands=4)
    else:
        side = 6.0 if n == 8 else 10.0
        cell = W.cell_tiny(atoms="pair", n=(n, n, n), a=(side, side, side), n_bands=4)
    subs = [random_subsim(cell, (2, 1, 1), (0.5, 0.5, 0.5), 0.08, 6, W.Kick(k0=0.01), seed=6, tag=i) for i in range(2)]
    P1, g1 = gpu_run(cell, subs, precision=precision)
    P2, _ = gpu_run(cell, subs, precision=precision, steps=3)
    states = [P2.get_state(i) for i in range(2)]
    for i, (st, step) in enumerate(states):
        assert step == 3
        P2.load_state(i, st, step)
    P2.propagate(3)
    for i in range(2):
        J2, _ = P2.current(i)
        np.testing.assert_array_equal(J2, g1[i]["J"])
        np.testing.assert_array_equal(P2.density(i), g1[i]["rho"])
        np.testing.assert_array_equal(P2.get_state(i)[0], P1.get_state(i)[0])


def test_error_paths():
    from paper_2112_00920_gb300 import Propagator, TsbzError
    cell = _tiny_pair()
    P = Propagator("fp64")
    cid = P.add_cell_spec(cell)
    sid = P.add_subsim(cid, np.zeros((2, 3)), 0.08, 3)
    with pytest.raises(TsbzError) as e:
        P.propagate(1)
    assert e.value.code == -6
    with pytest.raises(TsbzError) as e:
        P.load_ground_state(sid, np.zeros((2, 4, 8, 8, 7), dtype=np.complex128))
    assert e.value.code == -1
    bad = np.full((2, 4, 8, 8, 8), np.nan, dtype=np.complex128)
    P.load_ground_state(sid, bad)
    with pytest.raises(TsbzError) as e:
        P.propagate(1)
    assert e.value.code == -5
    # step budget (max_steps = 3): the sub-simulation stops at 3 steps, not an error
    # in itself; the non-finite status of the earlier step is still reported
    with pytest.raises(TsbzError) as e:
        P.propagate(5)
    assert e.value.code == -5
    assert P.step(sid) == 3
    with pytest.raises(TsbzError) as e:
        P.propagate(-1)
    assert e.value.code == -1
    P.close()


def test_bounded_wait_times_out_without_fault():
    """Failure detection without a GPU fault: a bulk-copy barrier that no copy
    completes makes the bounded device wait run out; the kernel records the
    timeout and returns, the call reports TSBZ_ETIMEOUT, and the device keeps
    working (the delivered case and a propagation afterwards succeed)."""
    from paper_2112_00920_gb300 import _lib
    rc, st = _lib.selftest_bounded_wait(0, polls=1000, deliver=False)
    assert rc == -4 and (st & 2)
    rc, st = _lib.selftest_bounded_wait(0, polls=1 << 20, deliver=True)
    assert rc == 0 and st == 0
    cell = _tiny_pair()
    subs = [random_subsim(cell, (2, 1, 1), (0.25, 0.5, 0.0), 0.08, 2, W.Kick(k0=0.01), seed=3)]
    _, g = gpu_run(cell, subs, precision="fp32")
    compare(g[0], oracle_run(cell, subs[0]), FP32_J_TOL, FP32_RHO_TOL, FP32_NORM_TOL)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_tc"])
def test_full_two_step_workload_sampled(precision):
    """The benchmark's launch configuration: 64 shifted 4^3 subgrids of cell A
    (4096 k, 65 536 orbitals), plane-wave start, kick; two steps.  Sub-simulations
    are independent, so sampled ones are checked against the oracle run alone."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    run = W.twostep_kick_run(n_steps=2)
    cell = run.subsims[0].cell
    gints = W.plane_wave_set(cell.n_bands)
    psi = W.plane_wave_orbitals(cell.a, cell.n, gints, 64)
    P = Propagator(precision)
    cid = P.add_cell_spec(cell)
    sids = [P.add_subsim(cid, shifted_kpoints(cell.a, s.mp, s.shift), s.dt, 2) for s in run.subsims]
    for sid in sids:
        P.load_ground_state(sid, psi)
    P.set_kick(-1, 0.005, (1.0, 0.0, 0.0))
    P.propagate(2)
    for m in (0, 37, 63):
        sub = run.subsims[m]
        s = dict(mp=sub.mp, shift=sub.shift, psi=psi, dt=sub.dt, n_steps=2, field=sub.field)
        o = oracle_run(cell, s)
        J, j0 = P.current(sids[m])
        g = dict(J=J, J0m=j0, rho=P.density(sids[m]), norms=P.norms(sids[m]))
        if precision == "fp64":
            compare(g, o, FP64_J_TOL, FP64_RHO_TOL)
        else:
            # two steps from plane waves: measured err_J 4.2e-7 (fp32), 2.8e-6 (fp32_tc) on GB300; bars 10x
            print(precision, m, compare(g, o, 5e-6 if precision == "fp32" else 3e-5, FP32_RHO_TOL, FP32_NORM_TOL))


def _eps(j, j0, dt, k0, omegas):
    return analysis.dielectric((j - j0[None, :])[:, 0], dt, k0, omegas)


def test_eps_error_vs_oracle():
    """eps(omega) over 0.1-20 eV (Eqs. 12-14) from each GPU path against the
    complex128 oracle: cell A on an 8^3 grid, MP 2^3, SCF ground state,
    kick 0.005 x, 600 steps of dt = 0.08 (T_W = run length).  Bar for the
    single-precision and tensor-core paths: err_eps <= 1e-4."""
    cell = W.cell_a_coarse(n=8)
    k = kpoints.kpoints_cartesian(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    gs = scf.ground_state(cell, k, seed=7, tol=1e-10, eig_tol=1e-10)
    n, dt, k0 = 600, 0.08, 0.005
    s = dict(mp=(2, 2, 2), shift=(0, 0, 0), psi=gs["u"], dt=dt, n_steps=n, field=W.Kick(k0=k0))
    o = oracle_run(cell, s)
    om = np.linspace(0.1, 20.0, 400) / 27.211386245988
    e_ref = _eps(o["J"], o["J0_minus"], dt, k0, om)
    errs = {}
    for prec in ("fp64", "fp32", "fp32_tc"):
        _, g = gpu_run(cell, [s], precision=prec)
        errs[prec] = analysis.err_eps(_eps(g[0]["J"], g[0]["J0m"], dt, k0, om), e_ref)
    print("err_eps vs oracle:", errs)
    assert errs["fp64"] <= 1e-10
    assert errs["fp32_tc"] <= 1e-4
    assert errs["fp32"] <= 1e-4


def test_eps_single_vs_fp64_gpu_16():
    """eps(omega) over 0.1-20 eV of the single-precision paths on the 16^3 cell A
    (the grid of the two-step workload, where the fused stage and the
    tensor-core projections run) against the FP64 GPU path, which the tests
    above pin to the oracle at err_J <= 1e-10.  MP 2^3, plane-wave start,
    kick 0.005 x, 600 steps of dt = 0.08.  Bar: 1e-4."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    cell = W.cell_a()
    n, dt, k0 = 600, 0.08, 0.005
    k = shifted_kpoints(cell.a, (2, 2, 2), (0.0, 0.0, 0.0))
    psi = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), 8)
    om = np.linspace(0.1, 20.0, 400) / 27.211386245988
    eps = {}
    for prec in ("fp64", "fp32", "fp32_tc"):
        P = Propagator(prec)
        cid = P.add_cell_spec(cell)
        sid = P.add_subsim(cid, k, dt, n)
        P.load_ground_state(sid, psi)
        P.set_kick(sid, k0, (1.0, 0.0, 0.0))
        P.propagate(n)
        J, j0 = P.current(sid)
        P.close()
        eps[prec] = _eps(J, j0, dt, k0, om)
    errs = {p: analysis.err_eps(eps[p], eps["fp64"]) for p in ("fp32", "fp32_tc")}
    print("err_eps vs fp64 GPU (16^3):", errs)
    assert errs["fp32"] <= 1e-4
    assert errs["fp32_tc"] <= 1e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_tc"])
def test_graph_replay_bitwise(precision):
    """Steps replayed from the captured CUDA graph equal direct launches bit for bit."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    cell = _tiny_pair()
    subs = [random_subsim(cell, (2, 1, 1), (0.5, 0.25, 0.5), 0.08, 7, W.Kick(k0=0.01), seed=8, tag=i) for i in range(2)]
    out = []
    for graphs in (False, True):
        P = Propagator(precision)
        cid = P.add_cell_spec(cell)
        sids = [P.add_subsim(cid, shifted_kpoints(cell.a, s["mp"], s["shift"]), s["dt"], 7) for s in subs]
        for sid, s in zip(sids, subs):
            P.load_ground_state(sid, s["psi"])
            P.set_kick(sid, 0.01, (1.0, 0.0, 0.0))
        P.set_graphs(graphs)
        P.propagate(3)
        P.propagate(4)
        out.append([(P.current(sid)[0], P.get_state(sid)[0]) for sid in sids])
        P.close()
    for (ja, sa), (jb, sb) in zip(out[0], out[1]):
        np.testing.assert_array_equal(ja, jb)
        np.testing.assert_array_equal(sa, sb)
