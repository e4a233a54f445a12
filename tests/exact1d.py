"""Exact rational 1D B-spline element integrals, for pinning the oracle.

Independent of the oracle: the B-splines of one span are built as exact
polynomials (Fraction coefficients) from the Cox--de Boor recursion of the
paper (Sec. 2.3, eqs. cox1/cox2), and the element integrals are taken exactly
by integrating the polynomials.  Slow; small p and few knots only.
"""
from fractions import Fraction

import numpy as np


def _padd(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)]


def _pmul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _pder(a):
    return [a[i] * i for i in range(1, len(a))] or [Fraction(0)]


def _pint(a, lo, hi):
    s = Fraction(0)
    for i, c in enumerate(a):
        s += c * (hi ** (i + 1) - lo ** (i + 1)) / (i + 1)
    return s


def span_polys(t, p, s):
    """Polynomials of B_{s-p+r;p} restricted to [t_s, t_{s+1}], r = 0..p."""
    t = [Fraction(x) for x in t]
    m = len(t)
    # degree 0: indicator of span s
    B = {i: ([Fraction(1)] if i == s else [Fraction(0)]) for i in range(m - 1)}
    for r in range(1, p + 1):
        nb = {}
        for i in range(m - r - 1):
            out = [Fraction(0)]
            d1 = t[i + r] - t[i]
            if d1 != 0:
                out = _padd(out, _pmul([-t[i] / d1, 1 / d1], B[i]))
            d2 = t[i + r + 1] - t[i + 1]
            if d2 != 0:
                out = _padd(out, _pmul([t[i + r + 1] / d2, -1 / d2], B[i + 1]))
            nb[i] = out
        B = nb
    return [B[s - p + r] for r in range(p + 1)], t[s], t[s + 1]


def element_matrices_1d(t, p, s):
    """Exact 1D mass M[a][b] = int B_a B_b and stiffness K = int B'_a B'_b and the
    mixed integrals X[a][b] = int B'_a B_b on span s (as float arrays)."""
    polys, lo, hi = span_polys(t, p, s)
    n = p + 1
    M = np.zeros((n, n)); K = np.zeros((n, n)); X = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            M[a, b] = float(_pint(_pmul(polys[a], polys[b]), lo, hi))
            K[a, b] = float(_pint(_pmul(_pder(polys[a]), _pder(polys[b])), lo, hi))
            X[a, b] = float(_pint(_pmul(_pder(polys[a]), polys[b]), lo, hi))
    return M, K, X


def rational_open_uniform(K, p):
    return [Fraction(0)] * (p + 1) + [Fraction(i, K) for i in range(1, K)] + [Fraction(1)] * (p + 1)
