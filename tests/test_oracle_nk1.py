"""The failure of one k-point per sub-simulation (Sec. III.A, discussion of
Fig. 4) in the oracle: see tests/nk1_common.py for the set-up and the
criterion.  A frozen potential removes the failure: with v_Hxc fixed at the
full-grid ground state's and each k-point starting from the full grid's
orbitals, the 64 one-point sub-simulations average to the full-grid result
to rounding (Eq. 9 is an exact re-indexing of the k sum), so what goes wrong
with N_k = 1 is the self-consistent density of each sub-simulation."""
import os

import numpy as np

import nk1_common as NK
import workloads as W
from oracle import dynamics, kpoints, scf


def test_one_kpoint_per_subsimulation_fails():
    workers = max(1, min(8, len(os.sched_getaffinity(0))))
    curves = NK.oracle_curves(workers)
    e = NK.check_failure(curves)
    print("oracle err_eps vs MP 4^3:", e)


def test_one_kpoint_exact_with_frozen_potential():
    c = NK.cell()
    kf = kpoints.kpoints_cartesian(c.a, (4, 4, 4), (0.0, 0.0, 0.0))
    gs = scf.ground_state(c, kf, seed=100, tol=1e-10, eig_tol=1e-10)
    a = dynamics.field_samples(W.Kick(k0=NK.K0), NK.DT, 40)
    full = dynamics.propagate(c, kf, gs["u"], NK.DT, 40, a, hxc="frozen", v_hxc_frozen=gs["v_hxc"],
                              keep_state=False)
    ref = full["J"] - full["J0_minus"][None, :]
    djs = []
    for s in W.lattice_shifts(4):
        k = kpoints.kpoints_cartesian(c.a, (1, 1, 1), s)
        i = int(np.argmin(np.linalg.norm(kf - k[0][None, :], axis=1)))
        assert np.linalg.norm(kf[i] - k[0]) < 1e-14
        r = dynamics.propagate(c, k, gs["u"][i:i + 1], NK.DT, 40, a, hxc="frozen", v_hxc_frozen=gs["v_hxc"],
                               keep_state=False)
        djs.append(r["J"] - r["J0_minus"][None, :])
    avg = np.mean(djs, axis=0)
    assert np.max(np.abs(avg - ref)) <= 1e-12 * np.max(np.abs(ref))
