"""Pins of the A-NN oracle (oracle/ann.py; Sec. 4.1, Remark rem:WG)."""
import os
from fractions import Fraction

import numpy as np

import oracle
import synth
from oracle import ann, spectral

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random(n, seed, kmax):
    return synth.random_spd2(n, seed, kmax)


def test_consistency_and_nonnegativity():
    """sum over the stencil of gamma(e) e e^T = D (Eq. DSum), weights >= 0."""
    D = _random(400, 1, 30.0)
    offs, w = ann.build2d_ann(*D)
    assert np.all(w >= 0)
    rec = np.einsum("nk,nki,nkj->nij", 2 * w, offs.astype(np.float64), offs.astype(np.float64))
    Dm = np.stack([np.stack([D[0], D[1]], -1), np.stack([D[1], D[2]], -1)], -2)
    assert np.abs(rec - Dm).max() <= 1e-12 * np.abs(Dm).max()


def test_pq_minimal_and_unique_by_brute_force():
    """(p, q) satisfies Eq. ineqPQ and b p q >= 0, and no other admissible
    pair has max(|p|, |q|) as small (exhaustive over |p|, |q| <= 40)."""
    D = _random(120, 2, 8.0)
    for a, b, c in D.T:
        if b == 0:
            continue
        A, B, C = Fraction(float(a)), Fraction(float(b)), Fraction(float(c))
        lo, hi = abs(B) / C, A / abs(B)
        best, arg = None, []
        for p in range(-40, 41):
            for q in range(-40, 41):
                if p == 0 or q == 0 or B * p * q < 0:
                    continue
                if lo <= abs(Fraction(p, q)) <= hi:
                    m = max(abs(p), abs(q))
                    if best is None or m < best:
                        best, arg = m, [(p, q)]
                    elif m == best:
                        arg.append((p, q))
        p, q = ann.ann_pq(float(a), float(b), float(c))
        assert best is not None and max(abs(p), abs(q)) == best
        # the minimiser is unique up to the sign of the pair
        assert {(abs(x), abs(y)) for x, y in arg} == {(abs(p), abs(q))}
        assert B * p * q > 0 and lo <= Fraction(p, q) * (1 if q > 0 else -1) * (1 if p > 0 else -1) <= hi


def test_coincides_with_adlbr_for_small_anisotropy():
    """Table 1's caption: for kappa <= 1 + sqrt(2), AD-LBR = A-NN (any
    orientation: |b| <= min(a, c), so p / q = 1 and the stencil is an obtuse
    superbase)."""
    g = np.random.default_rng(3)
    th = g.uniform(0, np.pi, 500)
    k = g.uniform(1.0, 1.0 + np.sqrt(2.0), 500)
    D = synth.D_from_angle(th, k) * np.exp(g.uniform(-2, 2, 500))
    oa, wa = ann.build2d_ann(*D)
    ol, wl, st, _ = oracle.build2d(*D)
    assert np.all(st == 0)
    assert np.array_equal(oa, ol)
    assert np.abs(wa - wl).max() <= 1e-13 * np.abs(wl).max()


def test_fig_eigen_tensor_by_hand():
    """D = [[19/2, 6], [6, 4]] (Fig. Eigen): |b|/c = 3/2 <= p/q <= 19/12, so
    (p, q) = (3, 2); 2 gamma(1, 0) = 19/2 - 9 = 1/2, 2 gamma(0, 1) = 4 - 4 = 0,
    2 gamma(3, 2) = 6/6 = 1."""
    offs, w = ann.build2d_ann([9.5], [6.0], [4.0])
    assert offs[0].tolist() == [[0, 0], [1, 0], [3, 2]]
    assert w[0].tolist() == [0.0, 0.25, 0.5]


def test_axis_aligned_tensor_gives_four_points():
    offs, w = ann.build2d_ann([2.0], [0.0], [0.5])
    assert offs[0].tolist() == [[0, 0], [0, 1], [1, 0]]
    assert w[0].tolist() == [0.0, 0.25, 1.0]


def test_radius_grows_like_kappa_squared():
    """Remark "Stencil radius": for D = [[1, 1 - 2e], [1 - 2e, 1 - 3e]],
    1 + e <= p/q + O(e^2) <= 1 + 2e, so q is of order 1/e."""
    for eps in (1e-2, 1e-3):
        p, q = ann.ann_pq(1.0, 1.0 - 2 * eps, 1.0 - 3 * eps)
        assert abs(q) >= 0.4 / eps
        assert 1 + eps - 2 * eps ** 2 <= p / q <= 1 + 2 * eps + 5 * eps ** 2


def test_fig_radius():
    """Fig. Radius: kappa = 10, eigenvector (cos theta, sin theta) over 3600
    orientations (0.05 degree steps): the A-NN radius reaches the printed
    36.1 (the offset (26, 25)), AD-LBR stays at the printed 5.1."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig_radius_ann.txt")) if l.strip() and l[0] != "#"]
    kappa, r_ann, r_adlbr = (float(x) for x in rows[0])
    th = np.linspace(0, np.pi, 3600, endpoint=False)
    D = synth.D_from_angle(th, kappa)
    oa, _ = ann.build2d_ann(*D)
    ol, _, _, _ = oracle.build2d(*D)
    ra = np.sqrt((oa.astype(float) ** 2).sum(-1)).max()
    rl = np.sqrt((ol.astype(float) ** 2).sum(-1)).max()
    assert round(ra, 1) == r_ann and round(rl, 1) == r_adlbr


def test_fig_eigen_oscillation():
    """Fig. Eigen: on n x n periodic grids (4 <= n <= 12) the smallest
    eigenvalues of the A-NN discretisation of D = [[19/2, 6], [6, 4]]
    oscillate with n -- here the second one is 0 for even n (a spurious zero
    mode: the stencil (1, 0), (3, 2) of weights 1/4, 1/2 does not connect the
    grid) -- while AD-LBR's n^2 lambda_2 increases towards the continuous
    4 pi^2 <m, D m> = 59.2."""
    D = np.array([[9.5, 6.0], [6.0, 4.0]])
    oa, wa = ann.build2d_ann([9.5], [6.0], [4.0])
    ol, wl, _, _ = oracle.build2d([9.5], [6.0], [4.0])
    cont = spectral.continuous_smallest(D, 2)[1]
    la = [spectral.periodic_symbol(oa[0], wa[0], (n, n))[1] * n * n for n in range(4, 13)]
    ll = [spectral.periodic_symbol(ol[0], wl[0], (n, n))[1] * n * n for n in range(4, 13)]
    assert all(abs(v) < 1e-9 for v in la[0::2]) and all(v > 15 for v in la[1::2])
    assert all(b > a for a, b in zip(ll, ll[1:])) and ll[-1] < cont and cont - ll[-1] < 0.03 * cont
