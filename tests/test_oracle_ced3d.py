"""Pins of the oracle's 3D coherence-enhancing tensor (Sec. 5, 3D experiments)."""
import numpy as np

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
