"""GPU: the standard error of the two-step mean (error bars of Fig. 6,
Sec. III.B) and the adaptive second sampling built on it, against the oracle
on the same seeded inputs (FP64 path)."""
import numpy as np
import pytest

import workloads as W
from oracle import analysis, dynamics, kpoints
from oracle.cell import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2112_00920_gb300 import build_library
    build_library()


CELL = W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4)
DT, K0 = 0.08, 0.01


def _psi(index):
    return W.random_orbitals(1, CELL.n_bands, CELL.n, Grid(CELL).dv, seed=100 + index)


def _oracle_shift(shift, index, n_steps):
    k = kpoints.kpoints_cartesian(CELL.a, (1, 1, 1), shift)
    a = dynamics.field_samples(W.Kick(k0=K0), DT, n_steps)
    return dynamics.propagate(CELL, k, _psi(index), DT, n_steps, a, keep_state=False)


def test_current_stats_match_oracle():
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    shifts = [(0.125, 0.5, 0.75), (0.6, 0.1, 0.3), (0.9, 0.8, 0.2), (0.35, 0.45, 0.55), (0.7, 0.25, 0.95)]
    n = 12
    P = Propagator("fp64")
    cid = P.add_cell_spec(CELL)
    sids = [P.add_subsim(cid, shifted_kpoints(CELL.a, (1, 1, 1), s), DT, n) for s in shifts]
    for i, sid in enumerate(sids):
        P.load_ground_state(sid, _psi(i))
        P.set_kick(sid, K0, (1.0, 0.0, 0.0))
    P.propagate(n)
    mean, se = P.current_stats()
    avg, _ = P.current(-1)
    P.close()
    ref_mean, ref_se = dynamics.two_step_standard_error([_oracle_shift(s, i, n) for i, s in enumerate(shifts)])
    scale = np.max(np.abs(ref_mean))
    assert np.max(np.abs(mean - ref_mean)) <= 1e-10 * scale
    assert np.array_equal(mean, avg)
    assert np.max(ref_se) > 1e-6 * scale          # the shifts really differ
    assert np.max(np.abs(se - ref_se)) <= 1e-9 * scale


def test_adaptive_second_sampling_matches_oracle_loop():
    """Halton shifts in batches of 4 until max sigma_E(Im eps) <= tol: the GPU
    driver stops at the same N_H as the same loop run on the oracle, with the
    same eps and error bars."""
    from paper_2112_00920_gb300 import twostep
    n_steps, batch, n_max = 150, 4, 12
    om = np.linspace(0.05, 1.0, 60)
    shifts = twostep.halton_source(n_max)
    np.testing.assert_array_equal(np.array(shifts), np.array(kpoints.halton_shifts(n_max)))
    orc = [_oracle_shift(s, i, n_steps) for i, s in enumerate(shifts)]
    dj = np.stack([(r["J"] - r["J0_minus"][None, :])[:, 0] for r in orc])
    hist = [float(np.max(analysis.dielectric_statistics(dj[:m], DT, K0, om)[2])) for m in (4, 8, 12)]
    if hist[1] < hist[0]:
        tol, expect = np.sqrt(hist[0] * hist[1]), 8
    else:
        tol, expect = 1.5 * hist[0], 4
    res = twostep.adaptive_two_step(CELL, (1, 1, 1), shifts, DT, n_steps, K0, om, tol,
                                    lambda k, i: _psi(i), batch=batch, precision="fp64")
    assert res["n_h"] == expect
    mean, sre, sim = analysis.dielectric_statistics(dj[:expect], DT, K0, om)
    assert np.max(np.abs(res["eps"] - mean)) <= 1e-9 * np.max(np.abs(mean))
    assert np.max(np.abs(res["sigma_im"] - sim)) <= 1e-8 * np.max(np.abs(mean))
    assert np.max(np.abs(res["sigma_re"] - sre)) <= 1e-8 * np.max(np.abs(mean))
    print("history", res["history"], "oracle", hist, "tol", tol)
