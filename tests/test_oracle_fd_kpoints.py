"""Pins of the oracle's finite-difference weights and k-point sets.

* FD weights: the textbook centred-difference rationals (Fornberg 1988,
  Table 1) for half-widths 1..4; plane-wave symbols approach -theta^2 and
  theta with the stencil's order; the stencil acts on exp(iG.r) as its symbol.
* k-points (Eqs. 8, 10): exact-rational identity "union of the lattice-shifted
  subgrids = full MP grid"; Halton radical inverses on small indices.
"""
from fractions import Fraction as F

import numpy as np
import pytest

import workloads as W
from oracle import fd, kpoints
from oracle.cell import Grid
from oracle.hamiltonian import apply_local

TEXTBOOK_D2 = {
    1: [F(-2), F(1)],
    2: [F(-5, 2), F(4, 3), F(-1, 12)],
    3: [F(-49, 18), F(3, 2), F(-3, 20), F(1, 90)],
    4: [F(-205, 72), F(8, 5), F(-1, 5), F(8, 315), F(-1, 560)],
}
TEXTBOOK_D1 = {
    1: [F(1, 2)],
    2: [F(2, 3), F(-1, 12)],
    3: [F(3, 4), F(-3, 20), F(1, 60)],
    4: [F(4, 5), F(-1, 5), F(4, 105), F(-1, 280)],
}


@pytest.mark.parametrize("nd", [1, 2, 3, 4])
def test_fornberg_matches_textbook(nd):
    c, d = fd.central_weights(nd)
    assert c == TEXTBOOK_D2[nd]
    assert d[1:] == TEXTBOOK_D1[nd]


def test_symbol_order_of_accuracy():
    th = np.array([0.05, 0.1, 0.2])
    lam = fd.laplacian_symbol(th)
    s = fd.gradient_symbol(th)
    # 8th-order: error ~ theta^10 (lap) and theta^9 (grad)
    assert np.all(np.abs(lam + th ** 2) < 1e-2 * th ** 10)
    assert np.all(np.abs(s - th) < 1e-2 * th ** 9)
    # A 2nd-order stencil would miss these bounds by orders of magnitude.
    assert np.abs(fd.laplacian_symbol(0.2, 1) + 0.04) > 1e-5


def test_stencil_on_plane_wave_is_symbol():
    cell = W.cell_tiny(atoms="none", n=(10, 8, 12), a=(7.0, 6.0, 8.0))
    g = Grid(cell)
    x, y, z = g.coords()
    q = np.array([0.13, -0.21, 0.07])
    for gint in [(1, 0, 0), (0, -2, 3), (2, 3, -5), (5, 4, 6)]:
        gv = 2 * np.pi * np.array(gint) / g.a
        u = np.exp(1j * (gv[0] * x + gv[1] * y + gv[2] * z))
        hu = apply_local(g, u[None], q, 0.0)[0]
        e = 0.5 * q @ q
        for ax in range(3):
            th = 2 * np.pi * gint[ax] / g.n[ax]
            e += -0.5 * fd.laplacian_symbol(th) / g.h[ax] ** 2 + q[ax] * fd.gradient_symbol(th) / g.h[ax]
        np.testing.assert_allclose(hu, e * u, atol=1e-11 * max(1, abs(e)))


@pytest.mark.parametrize("n_full,r", [(16, 4), (16, 2), (4, 2), (6, 3), (9, 3)])
def test_shift_lattice_union_is_full_mp_grid_exact(n_full, r):
    """Eq. 9/10: r^3 shifted (n_full/r)^3 grids tile the plain n_full^3 MP
    grid exactly (rational arithmetic).  Matching Eq. 10 to Eq. 8 term by
    term gives the shifts s = (2j + 1 - r)/(2r) mod 1, which for even r is
    the set (2i+1)/(2r) that ``workloads.lattice_shifts`` produces."""
    n = n_full // r
    vals = [F(2 * j + 1 - r, 2 * r) % 1 for j in range(r)]
    if r % 2 == 0:
        assert sorted(vals) == sorted(F(v[0]).limit_denominator(64) for v in W.lattice_shifts(r)[:r])
    union = []
    for sz in vals:
        for sy in vals:
            for sx in vals:
                union.extend(kpoints.shifted_mp_fractions((n, n, n), (sx, sy, sz), exact=True))
    full = kpoints.shifted_mp_fractions((n_full,) * 3, (F(0),) * 3, exact=True)
    assert len(union) == len(full) == n_full ** 3
    assert sorted(union) == sorted(full)
    assert len(set(union)) == len(union)


def test_mp_grid_symmetric_and_wrapped():
    fr = np.array(kpoints.shifted_mp_fractions((4, 4, 4), (0, 0, 0)))
    assert np.all(fr >= -0.5) and np.all(fr < 0.5)
    s = {tuple(np.round(v, 12)) for v in fr}
    assert all(tuple(np.round(-v, 12)) in s for v in fr)
    # Eq. 8 for N = 2: +-1/4
    fr2 = kpoints.shifted_mp_fractions((2, 1, 1), (0, 0, 0))
    assert [v[0] for v in fr2] == [-0.25, 0.25]


def test_halton_small_indices():
    assert [kpoints.radical_inverse(m, 2) for m in range(1, 6)] == [0.5, 0.25, 0.75, 0.125, 0.625]
    np.testing.assert_allclose([kpoints.radical_inverse(m, 3) for m in range(1, 6)],
                               [1 / 3, 2 / 3, 1 / 9, 4 / 9, 7 / 9], rtol=1e-15)
    np.testing.assert_allclose([kpoints.radical_inverse(m, 5) for m in range(1, 7)],
                               [0.2, 0.4, 0.6, 0.8, 1 / 25, 6 / 25], rtol=1e-15)
    h = kpoints.halton_shifts(3)
    assert h[0] == (0.5, 1 / 3, 0.2)


def test_kpoints_cartesian_units():
    k = kpoints.kpoints_cartesian((10.0, 5.0, 4.0), (2, 1, 1), (0.5, 0.0, 0.0))
    # shifted by half a step: (2n - 3 + 1)/4 -> 0, 1/2 -> wrapped to -1/2
    np.testing.assert_allclose(k[:, 0], [0.0, -0.5 * 2 * np.pi / 10.0])
