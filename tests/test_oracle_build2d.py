"""Pins for the oracle's 2D stencil construction (Sec. 2, Eqs. GaussAlgo,
def:Vz, def:GammaZ) against what the paper prints and what the mathematics
fixes."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(t) for t in line.split()])
    return rows


def _D_test(kappa2):
    """Eq. def:DTest with theta = pi/6."""
    return synth.D_from_angle(np.pi / 6, np.sqrt(kappa2))


def _stencil_matrix(offs, w):
    """Coefficients of -div(D grad) for a constant tensor: centre
    sum_{e in V} 2 gamma(e), off-centre -2 gamma(e) (each pair counted once)."""
    coef = {(0, 0): 4.0 * w.sum()}
    for (x, y), g in zip(offs, w):
        if g > 0:
            coef[(int(x), int(y))] = coef.get((int(x), int(y)), 0.0) - 2.0 * g
    return coef


def test_tables_1_2():
    rows = _load("table1_2_adlbr_stencils.txt")
    by_k = {}
    for k2, ex, ey, c in rows:
        by_k.setdefault(k2, {})[(int(ex), int(ey))] = c
    for k2, printed in by_k.items():
        D = _D_test(k2)
        offs, w, st, _ = oracle.build2d(*D)
        assert st[0] == 0
        coef = _stencil_matrix(offs[0], w[0])
        # every printed coefficient is reproduced to the printed 2 decimals
        for key, c in printed.items():
            got = coef.get(key, 0.0)
            assert abs(got - c) <= 0.005 + 1e-12, (k2, key, got, c)
        # and the stencil has no entry the table does not print (above 1e-9)
        for key, c in coef.items():
            if key not in printed:
                assert abs(c) < 1e-9, (k2, key, c)


def _lambda_max(offs, w):
    """sup over xi of the symbol sum_{e in V} 2 gamma(e) (1 - cos xi.e) of the
    constant-coefficient operator (periodic Fourier modes)."""
    from scipy.optimize import minimize

    t = np.linspace(-np.pi, np.pi, 401)
    X, Y = np.meshgrid(t, t)

    def sym(xi0, xi1):
        s = 0.0
        for (ex, ey), g in zip(offs, w):
            s = s + 4.0 * g * (1.0 - np.cos(xi0 * ex + xi1 * ey))
        return s

    S = sym(X, Y)
    i = np.unravel_index(np.argmax(S), S.shape)
    res = minimize(lambda v: -sym(v[0], v[1]), [X[i], Y[i]], method="Nelder-Mead",
                   options={"xatol": 1e-10, "fatol": 1e-12})
    return max(-res.fun, S[i])


def test_table_3_lambda_max():
    for k2, lam in _load("table3_lambda_max.txt"):
        offs, w, st, _ = oracle.build2d(*_D_test(k2))
        got = _lambda_max(offs[0], w[0])
        assert abs(got - lam) <= 0.005 + 1e-9, (k2, got, lam)


def test_fig_radius_kappa10():
    (kappa, printed), = _load("fig_radius.txt")
    th = np.linspace(0, np.pi, 20001)
    offs, w, st, _ = oracle.build2d(*synth.D_from_angle(th, kappa))
    assert np.all(st == 0)
    rad = np.sqrt((offs.astype(float) ** 2).sum(-1)).max(axis=1)
    assert rad.max() <= printed
    assert rad.max() <= kappa                     # Remark "Stencil radius"
    assert rad.max() > printed - 0.1              # the bound is attained (sqrt 26)


def test_radius_bound_random_tensors():
    """Remark "Stencil radius": the offsets of non-zero weight satisfy
    |e| <= kappa(D) once kappa(D) >= sqrt 2; below, the third superbase
    vector (length sqrt 2) can carry a small positive weight, so the bound
    read for every tensor is max(kappa, sqrt 2).  Random orientations and
    scales, kappa log-uniform in [1, 1000]."""
    rng = np.random.default_rng(11)
    n = 100000
    th = rng.uniform(0, np.pi, n)
    kap = np.exp(rng.uniform(0, np.log(1000.0), n))
    D = synth.D_from_angle(th, kap) * rng.uniform(0.1, 10.0, n)
    offs, w, st, _ = oracle.build2d(*D)
    assert np.all(st == 0)
    r = np.sqrt((offs.astype(float) ** 2).sum(-1)).max(axis=1)   # zero-weight offsets are (0, 0)
    assert np.all(r <= np.maximum(kap, np.sqrt(2.0)) * (1 + 1e-9))
    big = kap >= np.sqrt(2.0)
    assert np.all(r[big] <= kap[big] * (1 + 1e-9))
    assert np.any(r[~big] > kap[~big])   # the sqrt 2 case does occur


def test_fig_eigen_tensor_exact_weights():
    """D = [[19/2, 6], [6, 4]] (Fig. Eigen).  Worked by hand: the superbase
    (1,1), (-3,-2), (2,1) has det 1 and, with S = adj D = [[4,-6],[-6,19/2]],
    <e1,Se2> = -1, <e2,Se0> = -1/2, <e0,Se1> = -1, so the weights of Eq.
    def:GammaZ are 1/2 on (1,1), 1/4 on (3,2) and 1/2 on (2,1); they are
    binary fractions, hence exact in FP64."""
    offs, w, st, _ = oracle.build2d(9.5, 6.0, 4.0)
    assert st[0] == 0
    got = {tuple(o): g for o, g in zip(offs[0].tolist(), w[0])}
    assert got == {(1, 1): 0.5, (2, 1): 0.5, (3, 2): 0.25}


def _recon(offs, w):
    o = offs.astype(np.float64)
    return np.einsum("nk,nki,nkj->nij", 2.0 * w, o, o)


def test_consistency_reconstruction_and_sign():
    """Eq. DSum: D = sum_{e in V} gamma(e) e e^T, gamma >= 0 (Lemma Sum)."""
    D = synth.random_spd2(4000, seed=5, kappa_max=1000.0)
    offs, w, st, _ = oracle.build2d(*D)
    assert np.all(st == 0)
    assert np.all(w >= 0)
    R = _recon(offs, w)
    Dm = np.stack([np.stack([D[0], D[1]], -1), np.stack([D[1], D[2]], -1)], -2)
    rel = np.abs(R - Dm).max(axis=(1, 2)) / np.abs(Dm).max(axis=(1, 2))
    assert rel.max() < 1e-12
    # each offset is primitive and nonzero-weight offsets are canonical
    for o, g in zip(offs.reshape(-1, 2), w.reshape(-1)):
        if g > 0:
            assert np.gcd(abs(o[0]), abs(o[1])) == 1
            assert o[0] > 0 or (o[0] == 0 and o[1] > 0)
        else:
            assert o[0] == 0 and o[1] == 0


def _brute_obtuse_sets(D, R=6):
    """All S-obtuse superbases (e, f, -e-f) with |coords| <= R, and the
    positive-weight parts of their stencils."""
    a, b, c = D
    S = np.array([[c, -b], [-b, a]])
    vecs = [np.array(v) for v in itertools.product(range(-R, R + 1), repeat=2) if v != (0, 0)]
    sets = set()
    for e in vecs:
        for f in vecs:
            if e[0] * f[1] - e[1] * f[0] != 1:
                continue
            g = -e - f
            sb = [e, f, g]
            sp = [sb[(i + 1) % 3] @ S @ sb[(i + 2) % 3] for i in range(3)]
            if max(sp) > 1e-12 * np.abs(S).max() * 4 * R * R:
                continue
            st = []
            for i in range(3):
                wgt = -0.5 * sp[i]
                if wgt > 1e-12:
                    o = sb[i] if (sb[i][0] > 0 or (sb[i][0] == 0 and sb[i][1] > 0)) else -sb[i]
                    st.append((int(o[0]), int(o[1]), round(wgt, 9)))
            sets.add(tuple(sorted(st)))
    return sets


def test_brute_force_uniqueness_2d():
    """Lemma indepBasis: the positive weights do not depend on the obtuse
    superbase; brute force over all small superbases gives one stencil, the
    oracle's."""
    D = synth.random_spd2(60, seed=9, kappa_max=8.0)
    D = np.concatenate([D, np.array([[1.0, 0, 1], [2.0, 0, 1], [9.5, 6, 4], [2, 1, 2]]).T], axis=1)
    offs, w, st, _ = oracle.build2d(*D)
    for i in range(D.shape[1]):
        sets = _brute_obtuse_sets(D[:, i])
        assert len(sets) == 1, (D[:, i], sets)
        mine = tuple(sorted((int(o[0]), int(o[1]), round(g, 9))
                            for o, g in zip(offs[i], w[i]) if g > 0))
        assert sets.pop() == mine


def test_degenerate_mu_zero():
    """mu(M) = 0 (Lemma indepBasis, second case): the third weight is exactly
    zero and the offset is stored as (0, 0)."""
    offs, w, st, _ = oracle.build2d(np.array([1.0, 3.0]), np.array([0.0, 0.0]),
                                    np.array([1.0, 0.5]))
    assert st.tolist() == [0, 0]
    assert offs[0].tolist() == [[0, 0], [0, 1], [1, 0]]
    assert w[0].tolist() == [0.0, 0.5, 0.5]
    assert offs[1].tolist() == [[0, 0], [0, 1], [1, 0]]
    assert w[1].tolist() == [0.0, 0.25, 1.5]


def _canon(o):
    o = [tuple(v) if (v[0] > 0 or (v[0] == 0 and v[1] > 0)) else (-v[0], -v[1]) for v in o]
    return o


def test_symmetries():
    """Equivariance: scaling D scales the weights; swapping the axes or
    reflecting x maps the stencil accordingly."""
    D = synth.random_spd2(500, seed=21, kappa_max=200.0)
    o0, w0, _, _ = oracle.build2d(*D)
    o1, w1, _, _ = oracle.build2d(*(D * 4.0))
    assert np.array_equal(o0, o1) and np.allclose(w1, 4.0 * w0, rtol=1e-14, atol=0)
    o2, w2, _, _ = oracle.build2d(D[2], D[1], D[0])       # swap x and y
    o3, w3, _, _ = oracle.build2d(D[0], -D[1], D[2])      # reflect x
    for i in range(D.shape[1]):
        ref = {tuple(v): g for v, g in zip(o0[i].tolist(), w0[i]) if g > 0}
        sw = {v: g for v, g in zip(_canon([(b, a) for a, b in o0[i].tolist()]), w0[i]) if g > 0}
        got = {tuple(v): g for v, g in zip(o2[i].tolist(), w2[i]) if g > 0}
        assert sw.keys() == got.keys()
        assert all(abs(sw[k] - got[k]) <= 1e-13 * abs(D[:, i]).max() for k in sw)
        rf = {v: g for v, g in zip(_canon([(-a, b) for a, b in o0[i].tolist()]), w0[i]) if g > 0}
        got = {tuple(v): g for v, g in zip(o3[i].tolist(), w3[i]) if g > 0}
        assert rf.keys() == got.keys()
        assert len(ref) >= 2


def test_status_codes():
    offs, w, st, _ = oracle.build2d(np.array([1.0, -1.0, np.nan, 1.0]),
                                    np.array([0.0, 0.0, 0.0, 1.0]),
                                    np.array([1.0, 1.0, 1.0, 1.0]))
    assert st.tolist() == [0, 3, 4, 3]


def test_iterations_logarithmic():
    """Sec. 1 'Complexity': O(ln kappa) iterations of Eq. GaussAlgo."""
    th = np.linspace(0, np.pi, 2000)
    for kappa in (10.0, 100.0, 1000.0):
        _, _, st, it = oracle.build2d(*synth.D_from_angle(th, kappa))
        assert np.all(st == 0)
        assert it.max() <= 3 + 2.0 * np.log2(kappa)
