"""Pin of the implicit step by the analytic restoration problem (Sec. 5, "A
test case with an explicit solution", Eqs. restoration / elliptic): the
discretisation (stencils, operator, CG) of -lambda div(D grad u) + u = v on
[0,1)^2 with h = 1/N, i.e. (I + lambda N^2 A) u = v, against the exact
solution u = u0 o f of the infinite-domain problem.  u0 solves the 1D problem
-lambda kappa^-2 u'' + u = 1_{y < 1/2}: u0 = 1 - exp(-(1/2 - y)/l)/2 below the
stripe edge and exp(-(y - 1/2)/l)/2 above it, l = sqrt(lambda)/kappa.  The
schemes are first order: the errors must fall with N (the paper plots them,
it does not tabulate them)."""
import numpy as np
import pytest

import oracle
import synth

LAM = 1e-3


def exact(Yf, kappa):
    ell = np.sqrt(LAM) / kappa
    return np.where(Yf < 0.5, 1.0 - 0.5 * np.exp(-(0.5 - Yf) / ell), 0.5 * np.exp(-(Yf - 0.5) / ell))


def errors(x, u, N):
    """Relative L2 and H1-seminorm errors (forward differences on the grid)."""
    l2 = np.sqrt(np.mean((x - u) ** 2) / np.mean(u ** 2))
    g = lambda a: (np.diff(a, axis=1) * N, np.diff(a, axis=0) * N)
    (ex, ey), (ux, uy) = g(x - u), g(u)
    h1 = np.sqrt((np.mean(ex ** 2) + np.mean(ey ** 2)) / (np.mean(ux ** 2) + np.mean(uy ** 2)))
    return l2, h1


def test_exact_solution_solves_the_1d_problem():
    """u0 satisfies -lambda kappa^-2 u0'' + u0 = 1_{y<1/2} away from the edge
    and is C^1 across it (second differences of the closed form)."""
    kappa, h = 5.0, 1e-4
    y = np.array([0.3, 0.45, 0.55, 0.7])
    u = lambda t: exact(t, kappa)
    upp = (u(y + h) - 2 * u(y) + u(y - h)) / h ** 2
    res = -LAM * kappa ** -2 * upp + u(y) - (y < 0.5)
    assert np.abs(res).max() <= 1e-5
    assert abs(u(0.5 - 1e-12) - u(0.5 + 1e-12)) <= 1e-9                    # continuous
    d = lambda t: (u(t + 1e-7) - u(t - 1e-7)) / 2e-7
    assert abs(d(0.5 - 1e-5) - d(0.5 + 1e-5)) <= 1e-2 * abs(d(0.5 - 1e-5))  # C^1


@pytest.mark.parametrize("kappa", [2.0, 10.0])
def test_oracle_converges_to_exact_solution(kappa):
    errs = []
    for N in (100, 200):
        D, v, Yf = synth.restoration_problem(N, kappa)
        offs, w, st, _ = oracle.build2d(*D)
        assert np.all(st == 0)
        x, _, _ = oracle.cg((N, N), oracle.NEUMANN, offs, w, v, v, LAM * N * N, rtol=1e-9)
        errs.append(errors(x, exact(Yf, kappa), N))
    (l2a, h1a), (l2b, h1b) = errs
    assert l2a <= 2e-2 and h1a <= 0.2, errs
    assert l2a / l2b >= 1.8 and h1a / h1b >= 1.6, errs      # first order (or better) in N
