"""The axes-directed non-negative six-point scheme A-NN of Sec. 4.1 (Remark
rem:WG), FP64 with exact rational decisions.  TEST INFRASTRUCTURE (see the
package header of oracle/).

For D = [[a, b], [b, c]] (symmetric positive definite):
* b = 0: the four-point stencil {(+-1, 0), (0, +-1)} with 2 gamma(+-1, 0) = a
  and 2 gamma(0, +-1) = c;
* otherwise the stencil {(+-1, 0), (0, +-1), +-(p, q)}, where p, q are
  non-zero integers with b p q >= 0 and |b| / c <= |p / q| <= a / |b| (Eq.
  ineqPQ) and max(|p|, |q|) minimal, with 2 gamma(+-1, 0) = a - (p/q) b,
  2 gamma(0, +-1) = c - (q/p) b and 2 gamma(+-(p, q)) = b / (p q).

The interval [|b|/c, a/|b|] lies in (0, inf) and is non-empty because
a/|b| - |b|/c = (a c - b^2) / (|b| c) > 0.  Among the fractions p'/q' > 0 it
contains, the one of smallest denominator also has the smallest numerator
(the Stern-Brocot tree: every fraction of an interval descends from its
simplest one), so it is the unique minimiser of max(p', q'); the oracle finds
it by the continued-fraction recursion below, on the exact rational values of
the FP64 entries (fractions.Fraction), so every decision is exact.

Output follows the canonical order of oracle.build2d: an offset whose weight
is exactly zero is written as (0, 0) with weight 0, every other offset has
its first non-zero coordinate positive, and the three pairs are sorted
lexicographically.
"""
from fractions import Fraction
from math import floor

import numpy as np


def simplest_fraction(lo, hi):
    """The fraction of smallest denominator (and numerator) in the closed
    interval [lo, hi], 0 < lo <= hi, as (p, q)."""
    n = floor(lo)
    if n == lo:
        return int(n), 1
    if n + 1 <= hi:
        return int(n) + 1, 1
    # lo, hi in (n, n + 1): x = n + 1 / y with y in [1 / (hi - n), 1 / (lo - n)]
    p, q = simplest_fraction(1 / (hi - n), 1 / (lo - n))
    return int(n) * p + q, p


def ann_pq(a, b, c):
    """(p, q) of Eq. ineqPQ for FP64 entries a, b != 0, c (sign: b p q > 0)."""
    A, B, C = Fraction(a), Fraction(b), Fraction(c)
    p, q = simplest_fraction(abs(B) / C, A / abs(B))
    return (p, q) if B > 0 else (p, -q)


def _canonical(offs, w):
    items = []
    for (x, y), g in zip(offs, w):
        if g == 0.0:
            x, y, g = 0, 0, 0.0
        elif x < 0 or (x == 0 and y < 0):
            x, y = -x, -y
        items.append(((x, y), g))
    items.sort(key=lambda t: t[0])
    return [o for o, _ in items], [g for _, g in items]


def build2d_ann(Dxx, Dxy, Dyy):
    """A-NN stencils (Remark rem:WG) for arrays of tensor entries.  Returns
    (offs int32 [N, 3, 2] canonical half-stencil, w float64 [N, 3])."""
    a = np.ravel(np.asarray(Dxx, np.float64))
    b = np.ravel(np.asarray(Dxy, np.float64))
    c = np.ravel(np.asarray(Dyy, np.float64))
    n = a.size
    offs = np.zeros((n, 3, 2), np.int32)
    w = np.zeros((n, 3), np.float64)
    for i in range(n):
        ai, bi, ci = float(a[i]), float(b[i]), float(c[i])
        if bi == 0.0:
            o = [(1, 0), (0, 1), (0, 0)]
            g = [0.5 * ai, 0.5 * ci, 0.0]
        else:
            p, q = ann_pq(ai, bi, ci)
            A, B, C = Fraction(ai), Fraction(bi), Fraction(ci)
            # the weights from their exact rational values, rounded once
            g = [float((A - Fraction(p, q) * B) / 2), float((C - Fraction(q, p) * B) / 2),
                 float(B / (2 * p * q))]
            o = [(1, 0), (0, 1), (p, q)]
        o, g = _canonical(o, g)
        offs[i] = o
        w[i] = g
    return offs, w
