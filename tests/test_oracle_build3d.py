"""Pins for the oracle's 3D stencil construction (Sec. 2: Def. ReducedBasis,
Prop. MakeObtuse, Lemma Selling / Eq. DSum3D)."""
import itertools

import numpy as np

import oracle
import synth


def _mat(d):
    xx, yy, zz, xy, xz, yz = d
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def _recon(offs, w):
    o = offs.astype(np.float64)
    return np.einsum("nk,nki,nkj->nij", 2.0 * w, o, o)


def test_selling_reconstruction_random():
    """Eq. DSum3D: D = sum_{e in V} gamma(e) e e^T with gamma >= 0, 12 offsets."""
    D = synth.random_spd3(3000, seed=3, kappa_max=50.0)
    offs, w, st, it = oracle.build3d(D)
    assert np.all(st == 0)
    assert np.all(w >= 0)
    M = np.stack([_mat(D[:, i]) for i in range(D.shape[1])])
    rel = np.abs(_recon(offs, w) - M).max(axis=(1, 2)) / np.abs(M).max(axis=(1, 2))
    assert rel.max() < 1e-12
    # canonical form: nonzero weight -> first nonzero coordinate positive
    for o, g in zip(offs.reshape(-1, 3), w.reshape(-1)):
        if g > 0:
            nz = o[np.nonzero(o)[0][0]]
            assert nz > 0
        else:
            assert not o.any()
    assert it.max() <= 12


def _cross(a, b):
    return np.cross(a, b)


def _brute_selling_sets(M, R=1):
    """Positive parts of Selling's stencil for every D-obtuse superbase whose
    basis vectors have coordinates in [-R, R]."""
    vecs = np.array([v for v in itertools.product(range(-R, R + 1), repeat=3) if any(v)])
    sets = set()
    n = len(vecs)
    for i in range(n):
        e1 = vecs[i]
        for j in range(n):
            e2 = vecs[j]
            c12 = np.cross(e1, e2)
            dets = vecs @ c12
            for k in np.nonzero(dets == 1)[0]:
                e3 = vecs[k]
                e = [-(e1 + e2 + e3), e1, e2, e3]
                ok = True
                sp = {}
                for a, b in itertools.combinations(range(4), 2):
                    s = e[a] @ M @ e[b]
                    if s > 1e-12 * np.abs(M).max() * 16:
                        ok = False
                        break
                    sp[(a, b)] = s
                if not ok:
                    continue
                st = []
                for (a, b), s in sp.items():
                    kl = [t for t in range(4) if t not in (a, b)]
                    c = np.cross(e[kl[0]], e[kl[1]])
                    g = -0.5 * s
                    if g > 1e-12:
                        nz = c[np.nonzero(c)[0][0]]
                        if nz < 0:
                            c = -c
                        st.append((int(c[0]), int(c[1]), int(c[2]), round(g, 9)))
                sets.add(tuple(sorted(st)))
    return sets


def test_brute_force_uniqueness_3d():
    """Every D-obtuse superbase found by exhaustive search gives the same
    positive-weight Selling stencil, equal to the oracle's -- including
    degenerate tensors where several Selling weights vanish."""
    cases = [np.eye(3), np.diag([1.0, 2.0, 3.0]),
             np.array([[2.0, 1, 0], [1, 2, 0], [0, 0, 1]]),
             np.array([[2.0, 1, 1], [1, 2, 1], [1, 1, 2]]),
             np.array([[3.0, 1, 1], [1, 3, -1], [1, -1, 3]]),
             np.array([[2.0, -1, 0], [-1, 2, -1], [0, -1, 2]])]
    g = np.random.default_rng(4)
    for _ in range(6):
        Q, _r = np.linalg.qr(g.normal(size=(3, 3)))
        cases.append((Q * g.uniform(0.6, 1.6, 3)) @ Q.T)
    D6 = np.array([[M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]] for M in cases]).T
    offs, w, st, _ = oracle.build3d(D6)
    assert np.all(st == 0)
    for i, M in enumerate(cases):
        sets = _brute_selling_sets(M)
        assert len(sets) == 1, (M, sets)
        mine = tuple(sorted((int(o[0]), int(o[1]), int(o[2]), round(gw, 9))
                            for o, gw in zip(offs[i], w[i]) if gw > 0))
        assert sets.pop() == mine, (M, mine)


def test_identity_and_axis_cases():
    offs, w, st, _ = oracle.build3d(np.array([1.0, 1, 1, 0, 0, 0])[:, None])
    pos = sorted((tuple(o), g) for o, g in zip(offs[0].tolist(), w[0]) if g > 0)
    assert pos == [((0, 0, 1), 0.5), ((0, 1, 0), 0.5), ((1, 0, 0), 0.5)]
    assert sum(1 for g in w[0] if g == 0) == 3


def test_permutation_equivariance():
    D = synth.random_spd3(300, seed=8, kappa_max=20.0)
    o0, w0, _, _ = oracle.build3d(D)
    # swap x and z: (xx,yy,zz,xy,xz,yz) -> (zz,yy,xx,yz,xz,xy)
    Dp = D[[2, 1, 0, 5, 4, 3]]
    o1, w1, _, _ = oracle.build3d(Dp)
    for i in range(D.shape[1]):
        a = {}
        for o, g in zip(o0[i].tolist(), w0[i]):
            if g > 0:
                v = np.array(o[::-1])
                if v[np.nonzero(v)[0][0]] < 0:
                    v = -v
                a[tuple(v)] = g
        b = {tuple(o): g for o, g in zip(o1[i].tolist(), w1[i]) if g > 0}
        assert a.keys() == b.keys()
        assert all(abs(a[k] - b[k]) <= 1e-13 for k in a)


def test_status_codes_3d():
    D = np.array([[1.0, 1, 1, 0, 0, 0], [1.0, 1, -1, 0, 0, 0], [1.0, 1, 1, np.inf, 0, 0],
                  [1.0, 1, 1, 1, 0, 0]]).T
    _, _, st, _ = oracle.build3d(D)
    assert st.tolist() == [0, 3, 4, 3]
