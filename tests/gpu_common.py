"""Shared set-up of the GPU parity tests: run the same seeded inputs through
the library (C ABI via the Python binding) and through the oracle."""
from __future__ import annotations

import numpy as np

import workloads as W
from oracle import analysis, dynamics, kpoints

FP64_J_TOL = 1e-10      # err_J bar of the FP64 path
FP64_RHO_TOL = 1e-12    # err_rho and err_norm bars of the FP64 path
# Single-precision bars of the short runs (2-6 steps from random orthonormal
# orbitals or plane waves, every single-precision kernel family): 10x the
# largest errors measured on GB300 (err_J 7.3e-8, err_rho 3.7e-7, err_norm
# 8.5e-8), so that a tenfold regression of any of these kernels fails a test.
FP32_J_TOL, FP32_RHO_TOL, FP32_NORM_TOL = 8e-7, 4e-6, 1e-6


def gpu_run(cell, subs, precision="fp64", hxc="scf", v_frozen=None, fd_nd=4, steps=None, propagator="taylor4",
            graphs=None):
    """subs: list of dict(mp, shift, psi=(n_k,n_b,...), dt, n_steps, field=Kick|Pulse|samples).
    The library computes its own k-points (Eq. 10) from (mp, shift).
    Returns (propagator, list of dict(J, J0m, rho, norms))."""
    from paper_2112_00920_gb300 import Propagator, shifted_kpoints

    P = Propagator(precision)
    if propagator != "taylor4":
        P.set_propagator(propagator)
    if graphs is not None:
        P.set_graphs(graphs)
    cid = P.add_cell_spec(cell, hxc=hxc, fd_nd=fd_nd)
    sids = [P.add_subsim(cid, s.get("k_gpu", shifted_kpoints(cell.a, s["mp"], s["shift"])), s["dt"], s["n_steps"])
            for s in subs]
    for sid, s in zip(sids, subs):
        P.load_ground_state(sid, s["psi"], v_hxc_frozen=v_frozen)
        f = s["field"]
        if isinstance(f, W.Kick):
            P.set_kick(sid, f.k0, f.direction)
        elif isinstance(f, W.Pulse):
            from paper_2112_00920_gb300 import pulse_samples
            P.set_field(sid, pulse_samples(f.e0, f.omega0, f.t_pulse, f.direction, s["dt"], s["n_steps"]))
        elif f is not None:
            P.set_field(sid, f)
    n = steps if steps is not None else subs[0]["n_steps"]
    P.propagate(n)
    out = []
    for sid in sids:
        J, j0 = P.current(sid)
        out.append(dict(J=J, J0m=j0, rho=P.density(sid), norms=P.norms(sid)))
    return P, out


def oracle_run(cell, s, hxc="scf", v_frozen=None, steps=None, propagator="taylor4"):
    n = steps if steps is not None else s["n_steps"]
    f = s["field"]
    a = dynamics.field_samples(f, s["dt"], n) if isinstance(f, (W.Kick, W.Pulse)) else np.asarray(f)[: 2 * n + 1]
    k = s.get("k_orc", kpoints.kpoints_cartesian(cell.a, s["mp"], s["shift"]))
    return dynamics.propagate(cell, k, s["psi"], s["dt"], n, a, hxc=hxc, v_hxc_frozen=v_frozen,
                              keep_state=False, propagator=propagator)


def compare(gpu, orc, j_tol, rho_tol, norm_tol=None):
    norm_tol = rho_tol if norm_tol is None else norm_tol
    ej = analysis.err_j(gpu["J"], orc["J"])
    ej0 = float(np.max(np.abs(gpu["J0m"] - orc["J0_minus"])) / max(np.max(np.abs(orc["J"])), 1e-300))
    er = analysis.err_rho(gpu["rho"], orc["rho"])
    en = analysis.err_norm(gpu["norms"], orc["norms"])
    print(f"[parity] err_J {ej:.3e} err_J0 {ej0:.3e} err_rho {er:.3e} err_norm {en:.3e} "
          f"(bars {j_tol:.0e} {rho_tol:.0e} {norm_tol:.0e})")
    assert ej <= j_tol, f"err_J {ej:.3e} > {j_tol:.1e}"
    assert ej0 <= j_tol, f"err_J(0-) {ej0:.3e} > {j_tol:.1e}"
    assert er <= rho_tol, f"err_rho {er:.3e} > {rho_tol:.1e}"
    assert en <= norm_tol, f"err_norm {en:.3e} > {norm_tol:.1e}"
    return dict(err_J=ej, err_rho=er, err_norm=en)


def random_subsim(cell, mp, shift, dt, n_steps, field, seed, tag=0):
    from oracle.cell import Grid
    g = Grid(cell)
    n_k = int(mp[0] * mp[1] * mp[2])
    psi = W.random_orbitals(n_k, cell.n_bands, cell.n, g.dv, seed, tag)
    return dict(mp=mp, shift=shift, psi=psi, dt=dt, n_steps=n_steps, field=field)
