"""Pins for the oracle's CED tensor stage (Sec. 4.4) and its U-Net
preconditioner network (forward and hand-written backward)."""
import numpy as np
import pytest

import synth
from oracle import ced, unet


def test_blur_matches_scipy():
    from scipy.ndimage import gaussian_filter1d

    g = np.random.default_rng(1)
    a = g.normal(size=(37, 53))
    for s in (0.5, 1.0, 4.0):
        ref = gaussian_filter1d(gaussian_filter1d(a, s, axis=1, mode="reflect", truncate=3.0),
                                s, axis=0, mode="reflect", truncate=3.0)
        assert np.abs(ced.blur(a, s) - ref).max() <= 1e-13


def test_gradient_linear_ramp():
    y, x = np.mgrid[0:20, 0:30].astype(float)
    gx, gy = ced.gradient(3.0 * x - 2.0 * y + 1.0)
    assert np.allclose(gx[:, 1:-1], 3.0, atol=1e-14) and np.allclose(gy[1:-1, :], -2.0, atol=1e-14)
    assert np.allclose(gx[:, 0], 1.5) and np.allclose(gy[0, :], -1.0)   # reflected border


def test_tensor_matches_eigh():
    """D(J) built from numpy's eigen-decomposition with the lambda1 / lambda2
    of Sec. 4.4 equals the closed form."""
    g = np.random.default_rng(2)
    n = 500
    A = g.normal(size=(n, 2, 2)) * 10.0 ** g.uniform(-3, 0, (n, 1, 1))
    J = A @ np.transpose(A, (0, 2, 1))
    alpha, C = 1e-4, 1e-5
    Dxx, Dxy, Dyy = ced.tensor_from_J(J[:, 0, 0], J[:, 0, 1], J[:, 1, 1], alpha, C)
    mu, V = np.linalg.eigh(J)             # ascending: mu[:,1] = mu1 >= mu[:,0] = mu2
    lam1 = alpha
    lam2 = alpha + (1 - alpha) * np.exp(-C / (mu[:, 1] - mu[:, 0]) ** 2)
    v1, v2 = V[:, :, 1], V[:, :, 0]
    ref = lam1 * v1[:, :, None] * v1[:, None, :] + lam2[:, None, None] * v2[:, :, None] * v2[:, None, :]
    assert np.abs(Dxx - ref[:, 0, 0]).max() <= 1e-12
    assert np.abs(Dxy - ref[:, 0, 1]).max() <= 1e-12
    assert np.abs(Dyy - ref[:, 1, 1]).max() <= 1e-12


def test_constant_image_and_anisotropy_bound():
    alpha = 1e-2
    D = ced.ced_tensor(np.full((16, 16), 0.3), 1.0, 4.0, alpha, 1e-5)
    assert np.allclose(D[0], alpha) and np.allclose(D[1], 0) and np.allclose(D[2], alpha)
    u = synth.fingerprint(64, 3)
    Dxx, Dxy, Dyy = ced.ced_tensor(u, 1.0, 4.0, alpha, 1e-5)
    tr, det = Dxx + Dyy, Dxx * Dyy - Dxy ** 2
    disc = np.sqrt(np.maximum(tr * tr / 4 - det, 0))
    kappa = np.sqrt((tr / 2 + disc) / (tr / 2 - disc))
    assert kappa.max() <= 1 / np.sqrt(alpha) * (1 + 1e-9)     # kappa <= 1/sqrt(alpha)
    assert kappa.max() > 0.5 / np.sqrt(alpha)


def _tiny():
    cin, kw = 3, dict(c1=2, c2=3, c3=4)
    theta = unet.init_params(cin, seed=0, **kw)
    theta += 0.05 * np.random.default_rng(1).normal(size=theta.size)  # nonzero biases
    x = np.random.default_rng(2).normal(size=(cin, 8, 12))
    return cin, kw, theta, x


def test_unet_backward_finite_differences():
    cin, kw, theta, x = _tiny()
    gy = np.random.default_rng(3).normal(size=(8, 12))
    y, cache = unet.forward(theta, x, **kw)
    gth, gx = unet.backward(theta, cache, gy, **kw)
    f = lambda th, xx: float(np.sum(gy * unet.forward(th, xx, **kw)[0]))
    g = np.random.default_rng(4)
    h = 1e-6
    for idx in g.choice(theta.size, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        fd = (f(tp, x) - f(tm, x)) / (2 * h)
        assert abs(fd - gth[idx]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(20):
        c, i, j = g.integers(0, cin), g.integers(0, 8), g.integers(0, 12)
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (f(theta, xp) - f(theta, xm)) / (2 * h)
        assert abs(fd - gx[c, i, j]) <= 1e-6 * max(1.0, abs(fd))


def test_unet_matches_torch_autograd():
    torch = pytest.importorskip("torch")
    import torch.nn.functional as F

    cin, kw, theta, x = _tiny()
    y, cache = unet.forward(theta, x, **kw)
    gy = np.random.default_rng(5).normal(size=y.shape)
    gth, gx = unet.backward(theta, cache, gy, **kw)

    th = torch.tensor(theta, requires_grad=True)
    xt = torch.tensor(x[None], requires_grad=True)
    P, o = {}, 0
    for name, co, ci, k in unet.layer_shapes(cin, **kw):
        W = th[o:o + co * ci * k * k].view(co, ci, k, k)
        o += co * ci * k * k
        P[name] = (W, th[o:o + co])
        o += co

    def cr(n, a):
        return F.relu(F.conv2d(a, P[n][0], P[n][1], padding=P[n][0].shape[-1] // 2))

    s1 = cr("enc1b", cr("enc1a", xt))
    s2 = cr("enc2b", cr("enc2a", F.avg_pool2d(s1, 2)))
    a = cr("mid_b", cr("mid_a", F.avg_pool2d(s2, 2)))
    a = cr("dec2b", cr("dec2a", torch.cat([F.interpolate(a, scale_factor=2, mode="nearest"), s2], 1)))
    a = cr("dec1b", cr("dec1a", torch.cat([F.interpolate(a, scale_factor=2, mode="nearest"), s1], 1)))
    yt = F.conv2d(a, P["out"][0], P["out"][1])[0, 0]
    assert np.abs(yt.detach().numpy() - y).max() <= 1e-12
    (yt * torch.tensor(gy)).sum().backward()
    assert np.abs(th.grad.numpy() - gth).max() <= 1e-11
    assert np.abs(xt.grad.numpy()[0] - gx).max() <= 1e-11


def test_unet_param_count():
    # ~100k parameters with the preconditioner's input channels and the default widths
    assert 100_000 <= unet.n_params(unet.N_FEATURES) <= 130_000


def test_space_to_depth_index_map():
    """Channel dy * RF + dx at coarse (I, J) holds fine value (I RF + dy, J RF + dx)."""
    RF = unet.RF
    a = np.random.default_rng(6).normal(size=(3 * RF, 5 * RF))
    s = unet.space_to_depth(a)
    assert s.shape == (RF * RF, 3, 5)
    for I in range(3):
        for J in range(5):
            for dy in range(RF):
                for dx in range(RF):
                    assert s[dy * RF + dx, I, J] == a[I * RF + dy, J * RF + dx]
    assert np.allclose(s.mean(axis=0), unet.restrict(a[None])[0], atol=1e-15)


def _stencil_field(shape, seed):
    import oracle

    g = np.random.default_rng(seed)
    n = shape[0] * shape[1]
    D = synth.random_spd2(n, seed, kappa_max=20.0)
    offs, w, st = oracle.build2d(*D)[:3]
    assert np.all(st == 0)
    return offs, w, oracle.diag(shape, oracle.NEUMANN, offs, w), g


def test_preconditioner_features_and_jacobi_limit():
    RF = unet.RF
    shape = (4 * RF, 8 * RF)           # coarse grid divisible by 4 for the U-Net
    offs, w, diag, g = _stencil_field(shape, 9)
    dt = 0.7
    r = g.normal(size=shape)
    f, s = unet.coarse_features(offs, w, dt, r)
    assert abs(s - np.sqrt((r ** 2).sum() / r.size)) <= 1e-15 * s
    assert f.shape == (unet.N_FEATURES, 4, 8)
    # static channels: block means, by explicit loops over each block
    for I in range(4):
        for J in range(8):
            idx = [(I * RF + dy) * shape[1] + J * RF + dx for dy in range(RF) for dx in range(RF)]
            for k in range(3):
                want = np.mean([np.log1p(dt * w[i, k]) for i in idx])
                assert abs(f[RF * RF + k, I, J] - want) <= 1e-14
                for c in range(2):
                    want = np.mean([offs[i, k, c] / 8.0 for i in idx])
                    assert abs(f[RF * RF + 3 + 2 * k + c, I, J] - want) <= 1e-14
            assert abs(f[RF + 2, I, J] - r[I * RF + 1, J * RF + 2] / s) <= 1e-14
    # output layer zeroed: the network adds nothing and M(r) = r / (1 + dt A_zz)
    theta = unet.init_params(unet.N_FEATURES, seed=1)
    theta[-17:] = 0.0
    z = unet.precondition(theta, offs, w, dt, diag, r)
    assert np.array_equal(z, r / (1.0 + dt * diag))
    assert np.array_equal(unet.precondition(theta, offs, w, dt, diag, np.zeros(shape)),
                          np.zeros(shape))


def test_training_target_inverts_the_correction():
    """If the error is r / d + s P(c), the target is c (R P = identity)."""
    RF = unet.RF
    shape = (3 * RF, 2 * RF)
    offs, w, diag, g = _stencil_field(shape, 10)
    dt = 2.5
    r = g.normal(size=shape)
    s = np.sqrt(np.mean(r ** 2))
    c = g.normal(size=(3, 2))
    e = r / (1.0 + dt * diag) + s * unet.prolong(c)
    assert np.abs(unet.training_target(offs, w, dt, diag, r, e) - c).max() <= 1e-13
