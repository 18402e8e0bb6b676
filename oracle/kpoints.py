"""k-point sets of the plain and two-step Brillouin-zone samplings.

Eq. 8 (Monkhorst-Pack): k = sum_j (2 n_j - N_j - 1)/(2 N_j) b_j, n_j = 1..N_j.
Eq. 10 (shifted grids): k = sum_j (2 n_j - N_j - 1 + 2 s_j)/(2 N_j) b_j with a
shift s = (q_m, p_m, r_m) in (0,1)^3.
Sec. II.B: the shifts come from the Halton sequence in bases 2, 3, 5.

Reading (the paper is silent on it): every fractional coordinate is
wrapped into [-1/2, 1/2) by an integer, because the finite-difference
kinetic operator is not invariant under k -> k + G.  Order of the returned
list: n_1 fastest, then n_2, then n_3.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def wrap_half(f):
    """Map a fractional coordinate into [-1/2, 1/2)."""
    return f - math.floor(f + 0.5) if not isinstance(f, Fraction) else f - math.floor(f + Fraction(1, 2))


def shifted_mp_fractions(mp, shift, exact: bool = False):
    """Fractional coordinates (units of b_j) of the shifted MP grid, Eq. 10.

    ``shift`` = (0,0,0) gives the plain MP grid of Eq. 8.  With ``exact``
    the coordinates are Fractions (shift entries must then be Fractions).
    """
    out = []
    n1, n2, n3 = mp
    for i3 in range(1, n3 + 1):
        for i2 in range(1, n2 + 1):
            for i1 in range(1, n1 + 1):
                row = []
                for n_j, N_j, s_j in ((i1, n1, shift[0]), (i2, n2, shift[1]), (i3, n3, shift[2])):
                    if exact:
                        f = Fraction(2 * n_j - N_j - 1, 2 * N_j) + Fraction(s_j) / N_j
                    else:
                        f = (2.0 * n_j - N_j - 1.0 + 2.0 * s_j) / (2.0 * N_j)
                    row.append(wrap_half(f))
                out.append(tuple(row))
    return out


def kpoints_cartesian(a, mp, shift):
    """Cartesian k (bohr^-1) of the (shifted) MP grid of an orthorhombic
    cell with edges ``a``: b_j = (2 pi / a_j) e_j."""
    fr = np.array(shifted_mp_fractions(mp, shift), dtype=np.float64)
    return fr * (2.0 * np.pi / np.asarray(a, dtype=np.float64))[None, :]


def radical_inverse(m: int, base: int) -> float:
    """Van der Corput radical inverse of the integer m in ``base``."""
    f = 1.0
    r = 0.0
    while m > 0:
        f /= base
        r += f * (m % base)
        m //= base
    return r


def halton_shifts(n: int):
    """First n Halton points in bases (2, 3, 5); index m = 1..n (m = 0 gives
    the origin, which is not in the open cube (0,1)^3)."""
    return [(radical_inverse(m, 2), radical_inverse(m, 3), radical_inverse(m, 5)) for m in range(1, n + 1)]
