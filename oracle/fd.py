"""Finite-difference operators on the periodic real-space grid.

The paper discretises h_k(t) on a real-space grid (Sec. III, 15^3 grid in
Octopus) but does not state the stencil.  The reading used here: a centred
star stencil of half-width Nd = 4 (8th order), weights from Fornberg's
algorithm (B. Fornberg, Math. Comp. 51, 699 (1988)) evaluated in exact
rational arithmetic.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache

import numpy as np


def fornberg_weights(x0, nodes, max_order):
    """Weights w[k][j] of the k-th derivative at x0 from values at ``nodes``
    (Fornberg 1988, the recursive algorithm), exact when the inputs are
    Fractions or ints."""
    n = len(nodes)
    x0 = Fraction(x0)
    xs = [Fraction(x) for x in nodes]
    w = [[Fraction(0)] * n for _ in range(max_order + 1)]
    w[0][0] = Fraction(1)
    c1 = Fraction(1)
    c4 = xs[0] - x0
    for i in range(1, n):
        mn = min(i, max_order)
        c2 = Fraction(1)
        c5 = c4
        c4 = xs[i] - x0
        for j in range(i):
            c3 = xs[i] - xs[j]
            c2 *= c3
            if j == i - 1:
                for k in range(mn, 0, -1):
                    w[k][i] = c1 * (k * w[k - 1][i - 1] - c5 * w[k][i - 1]) / c2
                w[0][i] = -c1 * c5 * w[0][i - 1] / c2
            for k in range(mn, 0, -1):
                w[k][j] = (c4 * w[k][j] - k * w[k - 1][j]) / c3
            w[0][j] = c4 * w[0][j] / c3
        c1 = c2
    return w


@lru_cache(maxsize=None)
def central_weights(nd: int = 4):
    """Centred weights for the 2nd and 1st derivatives on offsets -nd..nd.

    Returns (c, d) as Fractions: c[m], m = 0..nd, with the 2nd derivative
    f'' ~ (1/h^2)(c0 f0 + sum_m c_m (f_m + f_-m)); d[m], m = 1..nd (d[0] = 0),
    with f' ~ (1/h) sum_m d_m (f_m - f_-m).
    """
    nodes = list(range(-nd, nd + 1))
    w = fornberg_weights(0, nodes, 2)
    c = [w[2][nd + m] for m in range(nd + 1)]
    d = [Fraction(0)] + [w[1][nd + m] for m in range(1, nd + 1)]
    return c, d


def weights_float(nd: int = 4):
    c, d = central_weights(nd)
    return np.array([float(v) for v in c]), np.array([float(v) for v in d])


def laplacian_symbol(theta, nd: int = 4):
    """lambda_2(theta) * h^2: the 1-D second-difference eigenvalue on exp(i theta j)."""
    c, _ = weights_float(nd)
    out = np.full_like(np.asarray(theta, dtype=np.float64), c[0])
    for m in range(1, nd + 1):
        out = out + 2.0 * c[m] * np.cos(m * np.asarray(theta))
    return out


def gradient_symbol(theta, nd: int = 4):
    """s(theta) * h: the 1-D first difference acts on exp(i theta j) as i*s."""
    _, d = weights_float(nd)
    out = np.zeros_like(np.asarray(theta, dtype=np.float64))
    for m in range(1, nd + 1):
        out = out + 2.0 * d[m] * np.sin(m * np.asarray(theta))
    return out
