"""Write the stored oracle results under tests/golden/ (calls only oracle/ and
the seeded inputs of workloads/; nothing from the GPU library).

cellA16_mp2_kick600: the linear-response run of Sec. III.A on the 16^3 grid
of the 8-atom cell: Monkhorst-Pack 2^3 (Eq. 8), the plane-wave start
orbitals of workloads.plane_wave_orbitals, the impulsive kick of Eq. 11
(k0 = 0.005 along x, read as A(t) = -k0 e theta(t)), dt = 0.08, 600 steps of
the Taylor-4 step with self-consistent v_Hxc (oracle.dynamics).  Stored:
J(t_n) for n = 0..600 (Eqs. 5-6), J(0-), the final orbital norms and the
final density (Eq. 3), every value with 17 significant digits.

nk1_tiny8: the one-k-point-per-sub-simulation study of Sec. III.A (discussion
of Fig. 4) on the small cell of tests/nk1_common.py: the two-step averages
dJ(t) of the Monkhorst-Pack 4^3 reference, of 8 shifted 2^3 subgrids and of
64 single k-points, each sub-simulation from its own oracle SCF ground state.

    python tests/golden/make_golden.py          # about ten minutes on one core
    python tests/golden/make_golden.py nk1      # the second set only
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import dynamics, kpoints  # noqa: E402

NAME = "cellA16_mp2_kick600"
N_STEPS, DT, K0 = 600, 0.08, 0.005
MP, SHIFT = (2, 2, 2), (0.0, 0.0, 0.0)


def inputs():
    """The run's inputs: (cell, k-points of Eq. 8, start orbitals, kick)."""
    cell = W.cell_a()
    k = kpoints.kpoints_cartesian(cell.a, MP, SHIFT)
    psi = W.plane_wave_orbitals(cell.a, cell.n, W.plane_wave_set(cell.n_bands), MP[0] * MP[1] * MP[2])
    return cell, k, psi, W.Kick(k0=K0)


def write_nk1():
    sys.path.insert(0, os.path.dirname(HERE))
    import nk1_common as NK
    t0 = time.perf_counter()
    curves = NK.oracle_curves(workers=max(1, min(8, len(os.sched_getaffinity(0)))))
    head = ("nk1_tiny8: oracle (complex128) two-step averages dJ(t) of tests/nk1_common.py (8^3 cell with two "
            f"off-grid ions, 2 bands, kick k0={NK.K0} x, dt={NK.DT}, {NK.N_STEPS} Taylor-4 steps, self-consistent "
            "v_Hxc, every sub-simulation from its own SCF ground state); written by tests/golden/make_golden.py")
    t = np.arange(NK.N_STEPS + 1) * NK.DT
    cols = [t] + [curves[name][:, ax] for name in ("mp4", "nk8", "nk1") for ax in range(3)]
    np.savetxt(os.path.join(HERE, "nk1_tiny8_dJ.txt"), np.column_stack(cols), fmt="%.17e",
               header=head + "\ncolumns: t, then dJx, dJy, dJz of mp4 (MP 4^3), nk8 (8 x 2^3), nk1 (64 x 1)")
    print(f"nk1_tiny8: {time.perf_counter() - t0:.1f} s")


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "nk1":
        write_nk1()
        return
    write_nk1()
    cell, k, psi, kick = inputs()
    t0 = time.perf_counter()
    res = dynamics.propagate(cell, k, psi, DT, N_STEPS, dynamics.field_samples(kick, DT, N_STEPS),
                             keep_state=False)
    wall = time.perf_counter() - t0
    head = (f"{NAME}: oracle (complex128), cell A 16^3, MP 2^3, plane-wave start, kick k0={K0} x, dt={DT}, "
            f"{N_STEPS} Taylor-4 steps, self-consistent v_Hxc; written by tests/golden/make_golden.py")
    t = np.arange(N_STEPS + 1) * DT
    np.savetxt(os.path.join(HERE, NAME + "_J.txt"), np.column_stack([t, res["J"]]), fmt="%.17e",
               header=head + "\ncolumns: t, Jx, Jy, Jz (J(t_n), Eqs. 5-6; row 0 is t = 0+)")
    np.savetxt(os.path.join(HERE, NAME + "_J0minus.txt"), res["J0_minus"][None, :], fmt="%.17e",
               header=head + "\nJ(0-) (Eqs. 5-6 at A = 0, before the kick)")
    np.savetxt(os.path.join(HERE, NAME + "_norms.txt"), res["norms"], fmt="%.17e",
               header=head + "\nfinal orbital norms dV sum |u|^2, rows k, columns bands")
    np.savetxt(os.path.join(HERE, NAME + "_rho.txt"), res["rho"].reshape(-1), fmt="%.17e",
               header=head + "\nfinal density (Eq. 3) on the grid, x fastest ([z][y][x] flattened)")
    print(f"{NAME}: {wall:.1f} s")


if __name__ == "__main__":
    main()
