"""Pins of the oracle's ground-state solver (``oracle/scf.py``, Sec. II.B step 2)
against results that go through neither its block eigensolver (which applies
the kinetic operator through its plane-wave symbol) nor its Pulay mixing.

* Free electrons (no ions, no projectors): any set of plane waves has a uniform
  density, for which v_H = 0 (the G = 0 term is dropped) and v_xc is a constant,
  so the ground state is the n_b lowest plane waves of the FD kinetic operator:
  eigenvalues = those of the explicit stencil matrix + v_xc(rho_0), occupied
  space = their span, rho = f n_b / Omega.
* With ions: a brute-force self-consistent field on a tiny grid -- the
  Hamiltonian as an explicit matrix built entry by entry from the stencil and
  the projector outer products, numpy's dense Hermitian eigensolver, plain
  linear density mixing -- reaches the same fixed point.
"""
import numpy as np

import workloads as W
from oracle import hamiltonian, hxc, kpoints, scf
from oracle.cell import Grid, local_potential, projector_tables


def _projector(u, dv):
    """Orthogonal projector onto the span of the (dV-normalised) orbitals u (n_b, ...)."""
    m = u.reshape(u.shape[0], -1).T * np.sqrt(dv)   # orthonormal columns in the plain metric
    return m @ m.conj().T


def test_free_electron_ground_state_is_lowest_plane_waves():
    cell = W.free_electron(W.cell_tiny(n=(8, 8, 8), a=(6.0, 6.5, 7.0), n_bands=4))
    kc = np.array([[0.11, 0.07, 0.05]])
    gs = scf.ground_state(cell, kc, seed=1, tol=1e-11, eig_tol=1e-11)
    grid = Grid(cell)
    shape = grid.n[::-1]
    nb = cell.n_bands
    rho0 = np.full(shape, cell.occ * nb / grid.omega)
    vxc0 = hxc.v_hxc(grid, rho0)
    assert np.ptp(vxc0) < 1e-14                      # uniform density: constant potential
    beta, disp, e_kb = projector_tables(cell)
    h0 = hamiltonian.dense_h(cell, kc[0], np.zeros(shape), beta, disp, e_kb)
    w, v = np.linalg.eigh(h0)
    assert w[nb] - w[nb - 1] > 1e-2                  # a gap: the occupied space is unique
    np.testing.assert_allclose(gs["eps"][0], w[:nb] + vxc0.flat[0], rtol=0, atol=1e-9)
    np.testing.assert_allclose(gs["rho"], rho0, rtol=0, atol=1e-10 * rho0.flat[0])
    p_ref = v[:, :nb] @ v[:, :nb].conj().T
    assert np.max(np.abs(_projector(gs["u"][0], grid.dv) - p_ref)) < 1e-8


def _brute_force_scf(cell, kc, tol=1e-12, mix=0.5, max_iter=200):
    """Dense-matrix SCF: h as an explicit matrix (the v_eff-independent part
    built once per k, v_eff added on the diagonal), numpy eigh, linear mixing."""
    grid = Grid(cell)
    shape = grid.n[::-1]
    nb = cell.n_bands
    vloc = local_potential(cell)
    beta, disp, e_kb = projector_tables(cell)
    h_fixed = [hamiltonian.dense_h(cell, k, np.zeros(shape), beta, disp, e_kb) for k in kc]
    n_e = cell.occ * nb
    rho = np.full(shape, n_e / grid.omega)
    for _ in range(max_iter):
        v_eff = vloc + hxc.v_hxc(grid, rho)
        rho_out = np.zeros(shape)
        eps, vecs = [], []
        for h in h_fixed:
            w, v = np.linalg.eigh(h + np.diag(v_eff.reshape(-1)))
            eps.append(w[:nb])
            vecs.append(v[:, :nb])
            rho_out += cell.occ * np.sum(np.abs(v[:, :nb]) ** 2, axis=1).reshape(shape) / grid.dv / len(kc)
        err = grid.dv * np.sum(np.abs(rho_out - rho)) / n_e
        if err < tol:
            return dict(rho=rho_out, eps=np.array(eps), vecs=vecs, err=err)
        rho = rho + mix * (rho_out - rho)
    raise AssertionError(f"brute-force SCF did not converge (err {err:.2e})")


def test_ground_state_matches_brute_force_scf():
    # two ions off the grid points, neutral filling (2 bands for Z = 2 x 2): a
    # 0.26 Ha gap above the occupied bands, so the fixed point is unique and
    # plain linear mixing reaches it
    cell = W.cell_tiny(atoms="offgrid", n=(8, 8, 8), a=(6.0, 6.0, 6.0), n_bands=2)
    kc = kpoints.kpoints_cartesian(cell.a, (2, 1, 1), (0.25, 0.5, 0.125))
    gs = scf.ground_state(cell, kc, seed=5, tol=1e-12, eig_tol=1e-11)
    bf = _brute_force_scf(cell, kc)
    grid = Grid(cell)
    assert gs["scf_error"] < 1e-11
    assert np.max(np.abs(gs["rho"] - bf["rho"])) < 1e-8 * np.max(bf["rho"])
    np.testing.assert_allclose(gs["eps"], bf["eps"], rtol=0, atol=1e-8)
    for k in range(len(kc)):
        p_bf = bf["vecs"][k] @ bf["vecs"][k].conj().T
        assert np.max(np.abs(_projector(gs["u"][k], grid.dv) - p_bf)) < 1e-7
