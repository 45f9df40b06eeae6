"""Pins of the oracle's 3D coherence-enhancing tensor (Sec. 5, 3D experiments)."""
import numpy as np

import synth

from oracle import ced


def test_blur3_matches_scipy():
    from scipy.ndimage import gaussian_filter
    a = np.random.default_rng(1).normal(size=(9, 13, 11))
    for s in (0.5, 1.5):
        ref = gaussian_filter(a, s, mode="reflect", truncate=3.0)
        assert np.abs(ced.blur3(a, s) - ref).max() <= 1e-13


def test_gradient3_linear():
    z, y, x = np.mgrid[0:7, 0:8, 0:9].astype(float)
    gx, gy, gz = ced.gradient3(2.0 * x - 3.0 * y + 0.5 * z)
    assert np.allclose(gx[:, :, 1:-1], 2.0) and np.allclose(gy[:, 1:-1, :], -3.0)
    assert np.allclose(gz[1:-1], 0.5)


def test_tensor_planar_and_isotropic_closed_forms():
    """J = g g^T (one direction): mu2 = mu3 = 0, so D = alpha g^ g^T +
    lam (I - g^ g^T) with lam = alpha + (1 - alpha) exp(-C / |g|^4).
    J = 0: D = alpha I."""
    rng = np.random.default_rng(2)
    alpha, C = 1e-2, 1e-3
    g = rng.normal(size=(50, 3)) * 0.3
    J = (g[:, 0] ** 2, g[:, 1] ** 2, g[:, 2] ** 2, g[:, 0] * g[:, 1], g[:, 0] * g[:, 2], g[:, 1] * g[:, 2])
    D = ced.tensor_from_J3(J, alpha, C)
    n2 = (g ** 2).sum(1)
    gh = g / np.sqrt(n2)[:, None]
    lam = alpha + (1 - alpha) * np.exp(-C / n2 ** 2)
    P = gh[:, :, None] * gh[:, None, :]
    ref = alpha * P + lam[:, None, None] * (np.eye(3) - P)
    got = np.stack([np.stack([D[0], D[3], D[4]], -1), np.stack([D[3], D[1], D[5]], -1),
                    np.stack([D[4], D[5], D[2]], -1)], -2)
    assert np.abs(got - ref).max() <= 1e-12
    Z = tuple(np.zeros(4) for _ in range(6))
    D0 = ced.tensor_from_J3(Z, alpha, C)
    assert np.allclose(D0[:3], alpha) and np.allclose(D0[3:], 0.0)


def test_tensor_eigenvalues_and_anisotropy_bound():
    """D's eigenvalues lie in [alpha, 1], the smallest one on J's leading
    eigenvector, so kappa(D) <= 1 / sqrt(alpha)."""
    alpha = 1e-2
    z, y, x = np.mgrid[0:20, 0:20, 0:20] / 19.0 - 0.5
    r = np.sqrt(x * x + y * y + z * z)
    u = np.cos(2 * (r / 0.5) ** 3) + 0.3 * np.random.default_rng(3).normal(size=r.shape)
    D = ced.ced_tensor3(u, 0.5, 2.0, alpha, 1e-5)
    M = np.stack([np.stack([D[0], D[3], D[4]], -1), np.stack([D[3], D[1], D[5]], -1),
                  np.stack([D[4], D[5], D[2]], -1)], -2)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= alpha * (1 - 1e-9) and ev.max() <= 1 + 1e-9
    J = ced.structure_tensor3(u, 0.5, 2.0)
    JM = np.stack([np.stack([J[0], J[3], J[4]], -1), np.stack([J[3], J[1], J[5]], -1),
                   np.stack([J[4], J[5], J[2]], -1)], -2)
    mu, V = np.linalg.eigh(JM)
    v1 = V[..., :, 2]
    assert np.abs(np.einsum("...i,...ij,...j->...", v1, M, v1) - alpha).max() <= 1e-9


def _mat(D):
    return np.stack([np.stack([D[0], D[3], D[4]], -1), np.stack([D[3], D[1], D[5]], -1),
                     np.stack([D[4], D[5], D[2]], -1)], -2)


def _rotations(n, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(n, 3, 3)))
    return q


def test_eed_tensor_rank_two_closed_form():
    """Edge-enhancing D (Sec. 5, 3D MRI experiment) for J = Q diag(a, b, 0) Q^T
    with a > b > 0 and a random rotation Q: D = Q diag(l(a), l(b), 1) Q^T,
    l(m) = 1 - exp(-C / m^2), written here from the eigen-structure of J (the
    columns of Q), not from the oracle's eigensolver.  A swap of lambda1 and
    lambda3, mu in place of mu^2, or differences of eigenvalues as in CED
    fail it."""
    C = 3e-3
    Q = _rotations(40, 11)
    rng = np.random.default_rng(12)
    a = rng.uniform(0.05, 0.3, 40)
    b = a * rng.uniform(0.1, 0.9, 40)
    J3 = np.einsum("nik,nk,njk->nij", Q, np.stack([a, b, 0 * a], -1), Q)
    J = (J3[:, 0, 0], J3[:, 1, 1], J3[:, 2, 2], J3[:, 0, 1], J3[:, 0, 2], J3[:, 1, 2])
    got = _mat(ced.tensor_from_J3_eed(J, C))
    la, lb = 1.0 - np.exp(-C / a ** 2), 1.0 - np.exp(-C / b ** 2)
    ref = (la[:, None, None] * Q[:, :, 0, None] * Q[:, None, :, 0]
           + lb[:, None, None] * Q[:, :, 1, None] * Q[:, None, :, 1]
           + Q[:, :, 2, None] * Q[:, None, :, 2])
    assert np.abs(got - ref).max() <= 1e-12
    # J = 0: D = I; planar J = g g^T: D = l(|g|^2) g^ g^T + (I - g^ g^T)
    D0 = ced.tensor_from_J3_eed(tuple(np.zeros(3) for _ in range(6)), C)
    assert np.allclose(D0[:3], 1.0) and np.allclose(D0[3:], 0.0)
    g = rng.normal(size=(30, 3)) * 0.4
    n2 = (g ** 2).sum(1)
    gh = g / np.sqrt(n2)[:, None]
    P = gh[:, :, None] * gh[:, None, :]
    ref = (1 - np.exp(-C / n2 ** 2))[:, None, None] * P + (np.eye(3) - P)
    Jg = (g[:, 0] ** 2, g[:, 1] ** 2, g[:, 2] ** 2, g[:, 0] * g[:, 1], g[:, 0] * g[:, 2], g[:, 1] * g[:, 2])
    assert np.abs(_mat(ced.tensor_from_J3_eed(Jg, C)) - ref).max() <= 1e-12


def test_eed_tensor_invariants_and_limits():
    """Rotation equivariance D(Q J Q^T) = Q D(J) Q^T; eigenvalues in (0, 1]
    with 1 on J's null direction and the smallest on J's leading
    eigenvector; C -> infinity gives I; small C / mu^2 gives lambda close
    to C / mu^2 (no cancellation in 1 - exp)."""
    rng = np.random.default_rng(13)
    G = rng.normal(size=(50, 3, 2)) * 0.3
    J3 = G @ G.transpose(0, 2, 1)                          # rank 2, PSD
    J = (J3[:, 0, 0], J3[:, 1, 1], J3[:, 2, 2], J3[:, 0, 1], J3[:, 0, 2], J3[:, 1, 2])
    C = 1e-3
    D = _mat(ced.tensor_from_J3_eed(J, C))
    Q = _rotations(50, 14)
    JQ = Q @ J3 @ Q.transpose(0, 2, 1)
    JQt = (JQ[:, 0, 0], JQ[:, 1, 1], JQ[:, 2, 2], JQ[:, 0, 1], JQ[:, 0, 2], JQ[:, 1, 2])
    DQ = _mat(ced.tensor_from_J3_eed(JQt, C))
    assert np.abs(DQ - Q @ D @ Q.transpose(0, 2, 1)).max() <= 1e-12
    ev = np.linalg.eigvalsh(D)
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12
    mu, V = np.linalg.eigh(J3)
    v3, v1 = V[:, :, 0], V[:, :, 2]
    assert np.abs(np.einsum("ni,nij,nj->n", v3, D, v3) - 1.0).max() <= 1e-12
    assert np.abs(np.einsum("ni,nij,nj->n", v1, D, v1) - ev[:, 0]).max() <= 1e-12
    Dinf = _mat(ced.tensor_from_J3_eed(J, 1e6))
    assert np.abs(Dinf - np.eye(3)).max() <= 1e-12
    # lambda1 for C / mu1^2 = 1e-14: 1 - exp(-1e-14) = 1e-14 (1 - 5e-15)
    Jd = (np.array([1.0]), np.array([0.0]), np.array([0.0]), np.zeros(1), np.zeros(1), np.zeros(1))
    Dd = ced.tensor_from_J3_eed(Jd, 1e-14)
    assert abs(Dd[0][0] - 1e-14) <= 1e-27


def test_eed_tensor_of_an_image():
    """On a noisy volume: D is symmetric positive definite with eigenvalues
    in (0, 1], and the largest is 1."""
    _, noisy = synth.radial3d(16, 3)
    D = _mat(ced.eed_tensor3(noisy, 0.5, 4.0, 1e-4))
    ev = np.linalg.eigvalsh(D)
    assert ev.min() > 0 and np.abs(ev[..., 2] - 1.0).max() <= 1e-12
