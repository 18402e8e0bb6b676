"""Pins of the oracle's potentials and Hamiltonian (Eq. 2).

* Hartree: rho = cos(G.r) has v_H = 4 pi cos(G.r)/G^2 exactly.
* PZ81: Slater exchange -0.458165/r_s; continuity of e_c and v_c at r_s = 1
  (to the published constants' rounding); v = d(rho e)/d rho by finite
  differences on both branches.
* v_loc: an isolated atom in a large cell equals -Z erf(r/r_e)/r +
  C exp(-r^2/2 sigma^2) - (2 pi Z / 3 Omega) r^2 + const near the atom (the
  last two terms are the neutralising background of the dropped G = 0 term:
  lap v = 4 pi Z (delta - 1/Omega) gives the -r^2 term).
* projectors: normalisation, box support, parity, diamond inversion symmetry;
  covariance V_NL(q + G) e^{-iG.r} = e^{-iG.r} V_NL(q) (the sign of the phase
  relative to the Bloch convention psi = e^{ik.r} u).
* h: the stencil/projector application equals an entry-by-entry dense matrix,
  which is Hermitian.
"""
import numpy as np
import pytest
from scipy.special import erf

import workloads as W
from oracle import cell as C
from oracle import hxc
from oracle.hamiltonian import apply_h, apply_nonlocal, dense_h


def test_hartree_cosine_exact():
    cell = W.cell_tiny(atoms="none", n=(12, 10, 8), a=(7.0, 6.0, 5.0))
    g = C.Grid(cell)
    x, y, z = g.coords()
    gv = 2 * np.pi * np.array([2, -1, 3]) / g.a
    rho = np.cos(gv[0] * x + gv[1] * y + gv[2] * z)
    v = hxc.hartree(g, rho)
    np.testing.assert_allclose(v, 4 * np.pi * rho / (gv @ gv), atol=1e-13)
    np.testing.assert_allclose(hxc.hartree(g, np.full(rho.shape, 0.3)), 0.0, atol=1e-15)


def test_pz81_exchange_and_continuity():
    rs = np.array([0.5, 1.0, 2.0, 4.0])
    rho = 3 / (4 * np.pi * rs ** 3)
    # Slater exchange of the uniform gas: e_x = -(3/4)(9/(4 pi^2))^{1/3}/r_s = -0.458165/r_s
    ex = -0.75 * (9 / (4 * np.pi ** 2)) ** (1 / 3) / rs
    np.testing.assert_allclose(ex, -0.4581652932831429 / rs, rtol=1e-14)
    exc, _ = hxc.pz81(rho)
    assert np.all(exc < ex)  # correlation is negative
    eps = 1e-10
    r_lo = 3 / (4 * np.pi * (1 - eps) ** 3)
    r_hi = 3 / (4 * np.pi * (1 + eps) ** 3)
    e_lo, v_lo = hxc.pz81(np.array([r_lo]))
    e_hi, v_hi = hxc.pz81(np.array([r_hi]))
    assert abs(e_lo[0] - e_hi[0]) < 5e-5
    assert abs(v_lo[0] - v_hi[0]) < 5e-5
    # correlation energy at r_s = 2 from the high-r_s form by hand
    ec2 = -0.1423 / (1 + 1.0529 * np.sqrt(2) + 0.3334 * 2)
    e2, _ = hxc.pz81(np.array([3 / (4 * np.pi * 8)]))
    np.testing.assert_allclose(e2[0], -0.4581652932831429 / 2 + ec2, rtol=1e-13)


@pytest.mark.parametrize("rs", [0.3, 0.8, 1.5, 3.0, 8.0])
def test_pz81_potential_is_derivative(rs):
    rho = 3 / (4 * np.pi * rs ** 3)
    h = rho * 1e-5
    f = lambda r: r * hxc.pz81(np.array([r]))[0][0]
    dfd = (f(rho + h) - f(rho - h)) / (2 * h)
    v = hxc.pz81(np.array([rho]))[1][0]
    np.testing.assert_allclose(v, dfd, rtol=1e-8)


def test_local_potential_isolated_atom():
    cell = W.CellSpec(name="iso", a=(16.0, 16.0, 16.0), n=(48, 48, 48),
                      atom_frac=np.array([[0.5, 0.5, 0.5]]), n_bands=1, e_kb_s=1.0, e_kb_p=1.0)
    g = C.Grid(cell)
    v = C.local_potential(cell)
    x, y, z = g.coords()
    r = np.sqrt((x - 8) ** 2 + (y - 8) ** 2 + (z - 8) ** 2)
    sel = r < 2.2
    rr = r[sel]
    with np.errstate(invalid="ignore", divide="ignore"):
        coul = np.where(rr > 0, -cell.z_ion * erf(rr / cell.r_erf) / rr, -2 * cell.z_ion / (np.sqrt(np.pi) * cell.r_erf))
    model = coul + cell.c_core * np.exp(-rr ** 2 / (2 * cell.sigma_core ** 2)) - 2 * np.pi * cell.z_ion / (3 * g.omega) * rr ** 2
    diff = v[sel] - model
    assert np.ptp(diff) < 1e-3, np.ptp(diff)
    # the potential itself varies by several Ha over this region
    assert np.ptp(v[sel]) > 3.0


def test_projectors_normalised_and_symmetric():
    cell = W.cell_a_coarse(n=16)
    g = C.Grid(cell)
    beta, disp, e = C.projector_tables(cell)
    assert beta.shape == (32, 16, 16, 16)
    np.testing.assert_allclose(g.dv * np.sum(beta ** 2, axis=(1, 2, 3)), 1.0, rtol=1e-13)
    # box support: offsets -7..7 -> 15 non-zero planes per axis for the s function
    s0 = beta[0]
    assert np.count_nonzero(np.any(s0 != 0, axis=(0, 1))) == 15
    # p_x of atom 0 (at the origin) is odd in x: beta(-x) = -beta(x)
    px = beta[1]
    np.testing.assert_allclose(px, -np.roll(px[:, :, ::-1], 1, axis=2), atol=1e-15)
    # diamond inversion through the bond centre (2,2,2): total s density symmetric
    tot = np.sum(beta[0::4] ** 2, axis=0)
    inv = np.roll(np.roll(np.roll(tot[::-1, ::-1, ::-1], 5, 0), 5, 1), 5, 2)
    np.testing.assert_allclose(tot, inv, atol=1e-14)
    np.testing.assert_allclose(e[:4], [cell.e_kb_s, cell.e_kb_p, cell.e_kb_p, cell.e_kb_p])


def test_nonlocal_bloch_covariance():
    """V_NL(q + G)[e^{-iG.r} u] = e^{-iG.r} V_NL(q)[u] for reciprocal-lattice G."""
    cell = W.cell_tiny(atoms="offgrid", n=(8, 8, 8), a=(6.0, 6.0, 6.0))
    g = C.Grid(cell)
    beta, disp, e = C.projector_tables(cell)
    u = W.random_complex((2,) + g.n[::-1], 3)
    q = np.array([0.2, -0.1, 0.33])
    x, y, z = g.coords()
    gv = 2 * np.pi * np.array([1, -2, 1]) / g.a
    ph = np.exp(-1j * (gv[0] * x + gv[1] * y + gv[2] * z))
    lhs = apply_nonlocal(g, ph * u, C.phased_projectors(cell, beta, disp, q + gv), e)
    rhs = ph * apply_nonlocal(g, u, C.phased_projectors(cell, beta, disp, q), e)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    # the opposite phase convention breaks it
    bad = apply_nonlocal(g, ph * u, C.phased_projectors(cell, beta, disp, -(q + gv)), e)
    badr = ph * apply_nonlocal(g, u, C.phased_projectors(cell, beta, disp, -q), e)
    assert np.max(np.abs(bad - badr)) > 1e-3


def test_apply_h_equals_dense_matrix():
    cell = W.cell_tiny(atoms="pair", n=(6, 6, 6), a=(5.0, 5.0, 5.0), proj_half=3.0)
    g = C.Grid(cell)
    beta, disp, e = C.projector_tables(cell)
    v = C.local_potential(cell) + 0.1 * np.cos(np.arange(216).reshape(6, 6, 6))
    q = np.array([0.31, -0.12, 0.05])
    H = dense_h(cell, q, v, beta, disp, e)
    np.testing.assert_allclose(H, H.conj().T, atol=1e-12)
    u = W.random_complex((3, 6, 6, 6), 5)
    hu = apply_h(g, u, q, v, C.phased_projectors(cell, beta, disp, q), e)
    np.testing.assert_allclose(hu.reshape(3, -1), (H @ u.reshape(3, -1).T).T, atol=1e-11)
