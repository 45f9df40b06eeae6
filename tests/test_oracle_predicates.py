"""Pins the oracle's exact predicate against exact rational arithmetic.

Every stencil decision of the construction (Sec. 2) is the sign of
sum_k n_k x_k with integer n_k and FP64 x_k; the oracle evaluates it with
floating-point expansions.  Python's Fraction gives the exact value
independently."""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def _exact(x, n):
    return sum(Fraction(int(a)) * Fraction(float(b)) for a, b in zip(n, x))


def _sign(v):
    return (v > 0) - (v < 0)


def test_sign_random_and_cancelling():
    g = np.random.default_rng(11)
    for trial in range(3000):
        K = int(g.integers(1, 7))
        x = g.normal(size=K) * 2.0 ** g.integers(-40, 40, size=K)
        n = g.integers(-20000, 20000, size=K)
        if K >= 2 and trial % 2 == 0:
            # force near-cancellation: choose x[-1] so the sum nearly vanishes
            part = sum(float(n[k]) * x[k] for k in range(K - 1))
            if n[-1] == 0:
                n[-1] = 1
            x[-1] = -part / float(n[-1])
        ex = _exact(x, n)
        assert oracle.exact_sign(x, n) == _sign(ex)
        v = oracle.exact_value(x, n)
        if ex != 0:
            assert abs(Fraction(v) - ex) <= abs(ex) * Fraction(1, 2 ** 50)
        else:
            assert v == 0.0


def test_sign_exact_zero_and_tiny():
    # 3 * 0.1 - 0.3 is not zero in binary; 1e-300 scaled cases stay exact
    x = np.array([0.1, 0.3])
    n = np.array([3, -1])
    assert oracle.exact_sign(x, n) == _sign(_exact(x, n))
    x = np.array([0.5, 0.25])
    n = np.array([1, -2])
    assert oracle.exact_sign(x, n) == 0
    x = np.array([1e-300, 3e-300, 1.0])
    n = np.array([3, -1, 0])
    assert oracle.exact_sign(x, n) == _sign(_exact(x, n))
