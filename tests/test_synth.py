"""The seeded synthetic inputs follow the recipes stated for them: each
generator is checked against a property its recipe fixes exactly (eigenvalues,
traces, angles, ranges) or statistically (the fingerprint's frequency band and
noise level, the 3D image's noise variance), and against its seed."""
import numpy as np
import pytest

import synth


def _eig2(D):
    """Eigenvalues (ascending) and the leading eigenvector angle of (3, ...) planes."""
    a, b, c = D
    tr, det = a + c, a * c - b * b
    disc = np.sqrt(np.maximum((a - c) ** 2 / 4 + b * b, 0.0))
    lo, hi = tr / 2 - disc, tr / 2 + disc
    theta = 0.5 * np.arctan2(2 * b, a - c)
    return lo, hi, theta, det


def _angle_diff(t1, t2):
    d = np.mod(t1 - t2 + np.pi / 2, np.pi) - np.pi / 2   # orientations modulo pi
    return np.abs(d)


def test_u_uniform_range_and_seed():
    u = synth.u_uniform((64, 48), 3)
    assert u.shape == (64, 48) and u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.02
    assert np.array_equal(u, synth.u_uniform((64, 48), 3))
    assert not np.array_equal(u, synth.u_uniform((64, 48), 4))


@pytest.mark.parametrize("kappa", [1.0, 10.0, 100.0])
def test_D_from_angle_eigen(kappa):
    th = np.linspace(-3, 3, 41)
    lo, hi, theta, _ = _eig2(synth.D_from_angle(th, kappa))
    assert np.allclose(hi, 1.0, atol=1e-14) and np.allclose(lo, kappa ** -2, atol=1e-14)
    if kappa > 1:
        assert _angle_diff(theta, th).max() < 1e-12


def test_spiral_field_recipe():
    n, kappa = 64, 10.0
    lo, hi, theta, _ = _eig2(synth.spiral_field(n, kappa))
    assert np.allclose(hi, 1.0, atol=1e-14) and np.allclose(lo, 0.01, atol=1e-14)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    c = (n - 1) / 2.0
    want = np.arctan2(y - c, x - c) + np.pi / 2 + 2 * np.pi * np.hypot(x - c, y - c) / 32.0
    assert _angle_diff(theta, want).max() < 1e-12


def test_fingerprint_band_and_noise():
    n, sigma = 512, 0.2
    img = synth.fingerprint(n, 1)
    assert np.array_equal(img, synth.fingerprint(n, 1))
    F = np.fft.fft2(img - img.mean())
    P = np.abs(F) ** 2 / n ** 2   # white noise of variance s^2 has E[P] = s^2 in every bin
    f = np.hypot(*np.meshgrid(np.fft.fftfreq(n), np.fft.fftfreq(n)))
    band = (f >= 1 / 12.5) & (f <= 1 / 5.5)
    # far from the band of the 8 sinusoids (periods 6-12 px) the spectrum is
    # the noise floor: |F|^2 / n^2 is exponentially distributed with mean
    # sigma^2, so median / ln 2 = sigma^2
    hi = f > 0.35
    s2 = np.median(P[hi]) / np.log(2.0)
    assert abs(np.sqrt(s2) - sigma) < 0.01, np.sqrt(s2)
    # the power above the noise floor lies in the band
    excess_band = P[band].sum() - s2 * band.sum()
    excess_all = P.sum() - s2 * (n * n - 1)
    assert excess_band > 0.95 * excess_all


def test_smooth_field2d_recipe():
    D = synth.smooth_field2d(256, 192, 3, 1.0, 50.0, 16)
    assert D.shape == (3, 256, 192)
    lo, hi, _, det = _eig2(D)
    assert np.allclose(hi, 1.0, atol=1e-12) and (det > 0).all()
    kappa = np.sqrt(hi / lo)
    assert kappa.min() >= 1.0 - 1e-9 and kappa.max() <= 50.0 + 1e-9
    assert kappa.min() < 3.0 and kappa.max() > 20.0   # the log-uniform draws span the range
    assert np.array_equal(D, synth.smooth_field2d(256, 192, 3, 1.0, 50.0, 16))


def test_needle_field3d_recipe():
    kappa, eps = 20.0, 1.0 / 400.0
    # trace of an interpolated projector is 1, so trace D = 1 + 2 eps everywhere
    D = synth.needle_field3d(24, 2, kappa=kappa, lattice=16)
    assert D.shape == (6, 24, 24, 24)
    assert np.abs(D[0] + D[1] + D[2] - (1 + 2 * eps)).max() < 1e-12
    # on a grid whose points are the lattice nodes, D = eps I + (1 - eps) v v^T
    D = synth.needle_field3d(16, 2, kappa=kappa, lattice=16)
    M = np.zeros((16 ** 3, 3, 3))
    for k, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        M[:, a, b] = M[:, b, a] = D[k].ravel()
    ev = np.linalg.eigvalsh(M)
    assert np.allclose(ev[:, 2], 1.0, atol=1e-12) and np.allclose(ev[:, :2], eps, atol=1e-12)


def test_radial3d_recipe():
    n, var = 32, 0.5
    u0, noisy = synth.radial3d(n, 5)
    c = (np.arange(n) + 0.5) / n
    r = np.sqrt(c[:, None, None] ** 2 + c[None, :, None] ** 2 + c[None, None, :] ** 2)
    assert np.allclose(u0, np.cos(2.0 * (r / 0.5) ** 3), atol=1e-15)
    e = noisy - u0
    assert abs(e.mean()) < 0.02 and abs(e.var() - var) < 0.02


def test_shells3d_recipe():
    u0, noisy = synth.shells3d((20, 32, 28), 5)
    assert u0.shape == (20, 32, 28)
    # the layers' intensities, the outside, and the blobs' values in (0.1, 0.9)
    vals = set(np.unique(u0).round(12))
    assert {0.0, 0.6, 1.0} <= vals and all(0.0 <= v <= 1.0 for v in vals)
    assert abs(np.std(noisy - u0) - 0.15) < 0.01
    a, b = synth.shells3d((20, 32, 28), 5)
    assert np.array_equal(a, u0) and np.array_equal(b, noisy)


def test_batch_items_recipe():
    items = synth.batch_items()
    img = [it for it in items if it["dim"] == 2]
    vol = [it for it in items if it["dim"] == 3]
    assert len(img) == 64 and len(vol) == 8
    assert all(256 <= it["shape"][0] <= 2048 and it["shape"][0] == it["shape"][1] for it in img)
    assert all(64 <= it["shape"][0] <= 192 and len(set(it["shape"])) == 1 for it in vol)
    assert all(5.0 <= it["kappa"] <= 100.0 for it in items)
    assert len({it["seed"] for it in items}) == len(items)


def test_random_spd_recipes():
    lo, hi, _, det = _eig2(synth.random_spd2(2000, 1, kappa_max=100.0))
    kappa = np.sqrt(hi / lo)
    assert (det > 0).all() and kappa.max() <= 100.0 * (1 + 1e-9) and kappa.min() >= 1.0 - 1e-9
    D6 = synth.random_spd3(300, 2, kappa_max=20.0)
    M = np.zeros((300, 3, 3))
    for k, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
        M[:, a, b] = M[:, b, a] = D6[k]
    ev = np.linalg.eigvalsh(M)
    assert np.allclose(ev[:, 2], 1.0, atol=1e-12)
    assert (ev[:, 0] >= 1.0 / 400.0 * (1 - 1e-9)).all()
