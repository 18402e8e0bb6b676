"""The library's propagation of the 16^3 linear-response run against the
stored oracle result (tests/golden/cellA16_mp2_kick600_*, written by
tests/golden/make_golden.py from oracle/ alone).

Run: the 8-atom cell on its 16^3 grid, Monkhorst-Pack 2^3 (Eq. 8),
plane-wave start orbitals, the kick of Eq. 11 (k0 = 0.005 along x),
dt = 0.08, 600 Taylor-4 steps with self-consistent v_Hxc.
  * FP64 path: err_J <= 1e-10 over all 601 samples, J(0-), and the final
    density and norms <= 1e-12.
  * single-precision paths, among them the whole-step kernel of the
    benchmark (k_step_fused, FP32 mode on 16^3 cells): eps(omega) of
    Eqs. 12-14 over 0.1-20 eV within 1e-4 of the oracle's (relative to its
    maximum), and err_J within a bar 10x above the measured error.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import analysis

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "cellA16_mp2_kick600")
N_STEPS, DT, K0 = 600, 0.08, 0.005
OMEGAS = np.linspace(0.1, 20.0, 400) / W.HARTREE_EV


@pytest.fixture(scope="module")
def golden():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2112_00920_gb300 import build_library
    build_library()
    jt = np.loadtxt(GOLD + "_J.txt")
    return dict(t=jt[:, 0], J=jt[:, 1:], J0m=np.loadtxt(GOLD + "_J0minus.txt"),
                norms=np.loadtxt(GOLD + "_norms.txt"), rho=np.loadtxt(GOLD + "_rho.txt"))


def _run(precision):
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints
    cell = W.cell_a()
    psi = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), 8)
    P = Propagator(precision)
    cid = P.add_cell_spec(cell)
    sid = P.add_subsim(cid, shifted_kpoints(cell.a, (2, 2, 2), (0.0, 0.0, 0.0)), DT, N_STEPS)
    P.load_ground_state(sid, psi)
    P.set_kick(sid, K0, (1.0, 0.0, 0.0))
    P.propagate(1)
    l0 = P.launches()
    P.propagate(1)
    per_step = P.launches() - l0
    P.propagate(N_STEPS - 2)
    J, j0 = P.current(sid)
    out = dict(J=J, J0m=j0, rho=P.density(sid).reshape(-1), norms=P.norms(sid), variant=P.variant(cid),
               per_step=per_step)
    P.close()
    return out


def _eps(J, j0):
    return analysis.dielectric((J - j0[None, :])[:, 0], DT, K0, OMEGAS)


def test_golden_files_shape(golden):
    assert golden["J"].shape == (N_STEPS + 1, 3)
    np.testing.assert_allclose(golden["t"], np.arange(N_STEPS + 1) * DT, rtol=0, atol=1e-12)
    assert golden["norms"].shape == (8, 16) and golden["rho"].shape == (4096,)


def test_fp64_matches_oracle_600_steps(golden):
    g = _run("fp64")
    ej = analysis.err_j(g["J"], golden["J"])
    ej0 = float(np.max(np.abs(g["J0m"] - golden["J0m"])) / np.max(np.abs(golden["J"])))
    er = analysis.err_rho(g["rho"], golden["rho"])
    en = analysis.err_norm(g["norms"], golden["norms"])
    ee = analysis.err_eps(_eps(g["J"], g["J0m"]), _eps(golden["J"], golden["J0m"]))
    print(f"fp64 vs oracle, 600 steps: err_J {ej:.2e} err_J0 {ej0:.2e} err_rho {er:.2e} err_norm {en:.2e} "
          f"err_eps {ee:.2e}")
    assert ej <= 1e-10 and ej0 <= 1e-10
    assert er <= 1e-12 and en <= 1e-12


# errors measured over the 600 steps on GB300 (fp32: err_J 2.7e-7, err_eps 3.4e-7;
# fp32_tc: err_J 2.5e-6, err_eps 3.1e-6): the bars sit 10x above them, well inside
# the 1e-4 target for eps(omega)
SINGLE_BARS = {"fp32": dict(err_j=2.7e-6, err_eps=3.4e-6), "fp32_tc": dict(err_j=2.5e-5, err_eps=3.1e-5)}


@pytest.mark.parametrize("precision", ["fp32", "fp32_tc"])
def test_single_precision_eps_vs_oracle(golden, precision):
    g = _run(precision)
    if precision == "fp32":
        # the benchmark's kernel: the whole time step in one launch with the z
        # contractions on tcgen05 (variant 0 of four on 16^3 cells with z groups):
        # field, step, observation, finalize, FFT Hartree and PZ81 per step
        assert g["variant"][0] == 0 and g["variant"][1] == 4
        assert g["per_step"] == 6, g["per_step"]
    ej = analysis.err_j(g["J"], golden["J"])
    dj_g, dj_o = g["J"] - g["J0m"][None, :], golden["J"] - golden["J0m"][None, :]
    edj = float(np.max(np.abs(dj_g - dj_o)) / np.max(np.abs(dj_o)))
    ee = analysis.err_eps(_eps(g["J"], g["J0m"]), _eps(golden["J"], golden["J0m"]))
    print(f"{precision} vs oracle, 600 steps: err_J {ej:.2e} err_dJ {edj:.2e} err_eps {ee:.2e}")
    bars = SINGLE_BARS[precision]
    assert ee <= bars["err_eps"], ee
    assert ej <= bars["err_j"], ej
