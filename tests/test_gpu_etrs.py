"""GPU: the enforced-time-reversal-symmetry step (a Taylor-4 predictor for
rho(t_{n+1}), then two Taylor-4 half steps with h at t_n and at t_{n+1})
against the oracle's, on the same seeded inputs."""
import numpy as np
import pytest

import workloads as W

from gpu_common import FP32_J_TOL, FP32_RHO_TOL, FP64_J_TOL, FP64_RHO_TOL, compare, gpu_run, oracle_run, random_subsim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built_library():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2112_00920_gb300 import build_library
    build_library()


BARS = {"fp64": (FP64_J_TOL, FP64_RHO_TOL), "fp32": (FP32_J_TOL, FP32_RHO_TOL)}

CASES = {
    # 8^3 pair cell, self-consistent v_Hxc, a pulse (A changes within every step)
    "tiny_pulse": lambda: (W.cell_tiny(atoms="pair", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=4), (2, 1, 1),
                           (0.25, 0.5, 0.0), 0.08, W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8,
                                                            direction=(0.3, 0.4, 0.866))),
    # cell A on its 16^3 grid (the whole-step kernel in single precision), kick
    "cellA_kick": lambda: (W.cell_a(), (2, 1, 1), (0.125, 0.375, 0.625), 0.08, W.Kick(k0=0.005)),
    # generic point-parallel kernels (depth 14), pulse
    "ragged14": lambda: (W.cell_tiny(atoms="offgrid", n=(10, 12, 14), a=(7.0, 8.0, 9.0), n_bands=3), (3, 1, 1),
                         (0.1, 0.2, 0.3), 0.05, W.Pulse(e0=0.05, omega0=0.3, t_pulse=0.8,
                                                        direction=(0.3, 0.4, 0.866))),
}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_etrs_parity(precision, case):
    cell, mp, shift, dt, field = CASES[case]()
    s = random_subsim(cell, mp, shift, dt, 5, field, seed=61)
    _, g = gpu_run(cell, [s], precision=precision, propagator="etrs")
    o = oracle_run(cell, s, propagator="etrs")
    jt, rt = BARS[precision]
    errs = compare(g[0], o, jt, rt)
    # and the step is not the Taylor-4 one: the oracle's two propagators differ beyond the bar
    t4 = oracle_run(cell, s)
    assert np.max(np.abs(t4["J"] - o["J"])) > 10 * jt * np.max(np.abs(o["J"]))
    print(precision, case, errs)


def test_etrs_graph_replay_bitwise_and_budgets():
    """Two sub-simulations with budgets 3 and 5 under ETRS: graph replay equals
    direct launches bit for bit, and each stops at its budget."""
    cell, mp, shift, dt, field = CASES["tiny_pulse"]()
    s0 = random_subsim(cell, mp, shift, dt, 3, field, seed=62)
    s1 = random_subsim(cell, (1, 2, 1), (0.5, 0.25, 0.75), dt, 5, field, seed=63)
    out = []
    for graphs in (False, True):
        P, g = gpu_run(cell, [s0, s1], precision="fp32", propagator="etrs", graphs=graphs, steps=5)
        assert [P.step(0), P.step(1)] == [3, 5]
        out.append(g)
        P.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a["J"], b["J"]) and np.array_equal(a["rho"], b["rho"])
    for gres, s in zip(out[0], (s0, s1)):
        compare(gres, oracle_run(cell, s, propagator="etrs"), *BARS["fp32"])
