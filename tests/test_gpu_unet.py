"""Parity of the CUDA U-Net forward / backward / Adam with the FP64 numpy
oracle (the learned preconditioner's network; not in the paper)."""
import numpy as np
import pytest

from oracle import unet as ou
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cin,c,B,H,W", [(3, (4, 6, 8), 2, 16, 24), (10, (16, 32, 64), 1, 32, 32)])
def test_unet_forward_backward_match_oracle(cin, c, B, H, W):
    t = torch()
    kw = dict(c1=c[0], c2=c[1], c3=c[2])
    g = np.random.default_rng(0)
    theta = ou.init_params(cin, seed=1, **kw) + 0.05 * g.normal(size=ou.n_params(cin, **kw))
    x = g.normal(size=(B, cin, H, W))
    gy = g.normal(size=(B, H, W))
    net = ab.adlbr_unet_create(cin, c[0], c[1], c[2], B, H, W)
    try:
        assert ab.adlbr_unet_num_params(net) == theta.size
        th = dev(theta, t.float32)
        xd = dev(x.ravel(), t.float32)
        y = t.empty(B * H * W, dtype=t.float32, device="cuda")
        ab.adlbr_unet_forward(net, th, xd, y)
        gth = t.empty_like(th)
        gx = t.empty_like(xd)
        ab.adlbr_unet_backward(net, th, dev(gy.ravel(), t.float32), gth, gx)
        t.cuda.synchronize()
        yg = y.double().cpu().numpy().reshape(B, H, W)
        gthg = gth.double().cpu().numpy()
        gxg = gx.double().cpu().numpy().reshape(B, cin, H, W)
    finally:
        ab.adlbr_unet_destroy(net)
    # the oracle sees the FP32-rounded parameters and inputs
    th32 = theta.astype(np.float32).astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    gy32 = gy.astype(np.float32).astype(np.float64)
    gth_ref = np.zeros_like(theta)
    for b in range(B):
        yo, cache = ou.forward(th32, x32[b], **kw)
        assert np.abs(yg[b] - yo).max() <= 1e-4 * max(1.0, np.abs(yo).max())
        gt, gxo = ou.backward(th32, cache, gy32[b], **kw)
        gth_ref += gt
        assert np.abs(gxg[b] - gxo).max() <= 1e-4 * max(1.0, np.abs(gxo).max())
    # FP32 sums over up to B*H*W terms
    assert np.abs(gthg - gth_ref).max() <= 2e-4 * max(1.0, np.abs(gth_ref).max())


def test_adam_step_matches_formula():
    t = torch()
    g = np.random.default_rng(3)
    n = 1000
    th, gr, m, v = (g.normal(size=n) for _ in range(4))
    v = np.abs(v)
    tt = 7
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    d = [dev(a, t.float32) for a in (th, gr, m, v)]
    ab.adlbr_adam_step(d[0], d[1], d[2], d[3], n, lr, b1, b2, eps, tt)
    t.cuda.synchronize()
    a32 = [a.astype(np.float32).astype(np.float64) for a in (th, gr, m, v)]
    m2 = b1 * a32[2] + (1 - b1) * a32[1]
    v2 = b2 * a32[3] + (1 - b2) * a32[1] ** 2
    th2 = a32[0] - lr * (m2 / (1 - b1 ** tt)) / (np.sqrt(v2 / (1 - b2 ** tt)) + eps)
    assert np.abs(d[0].double().cpu().numpy() - th2).max() <= 1e-6
    assert np.abs(d[2].double().cpu().numpy() - m2).max() <= 1e-6


def _forward(net, th, xd, n_out):
    t = torch()
    y = t.empty(n_out, dtype=t.float32, device="cuda")
    ab.adlbr_unet_forward(net, th, xd, y)
    t.cuda.synchronize()
    return y.double().cpu().numpy()


# widths that leave partial 128-pixel tiles at every level; channel mixes
# with each of the 16 / 32 / 64-output kernels in the encoder and decoder
@pytest.mark.parametrize("cin,c,B,H,W", [(25, (16, 32, 64), 1, 20, 200), (7, (64, 32, 16), 2, 12, 36),
                                         (25, (16, 32, 64), 1, 256, 384)])
def test_unet_tensor_core_forward_matches_fp32_and_oracle(cin, c, B, H, W):
    t = torch()
    kw = dict(c1=c[0], c2=c[1], c3=c[2])
    g = np.random.default_rng(5)
    theta = ou.init_params(cin, seed=2, **kw) + 0.05 * g.normal(size=ou.n_params(cin, **kw))
    x = g.normal(size=(B, cin, H, W))
    net = ab.adlbr_unet_create(cin, c[0], c[1], c[2], B, H, W)
    try:
        th = dev(theta, t.float32)
        xd = dev(x.ravel(), t.float32)
        y32 = _forward(net, th, xd, B * H * W).reshape(B, H, W)
        ab.adlbr_unet_set_tensor_cores(net, True)
        ytc = _forward(net, th, xd, B * H * W).reshape(B, H, W)
        # a backward needs the FP32 activations
        with pytest.raises(ab.AdlbrError):
            ab.adlbr_unet_backward(net, th, t.zeros(B * H * W, dtype=t.float32, device="cuda"), t.empty_like(th))
        ab.adlbr_unet_set_tensor_cores(net, False)
        yback = _forward(net, th, xd, B * H * W).reshape(B, H, W)
        # after an FP32 forward the backward runs again
        gth = t.empty_like(th)
        ab.adlbr_unet_backward(net, th, t.ones(B * H * W, dtype=t.float32, device="cuda"), gth)
        t.cuda.synchronize()
        assert t.isfinite(gth).all()
    finally:
        ab.adlbr_unet_destroy(net)
    assert np.isfinite(ytc).all()
    assert np.array_equal(y32, yback)
    scale = np.abs(y32).max()
    # BF16 operands (8 significant bits) through 10 layers, FP32 accumulation
    assert np.abs(ytc - y32).max() <= 3e-2 * scale
    assert np.abs(ytc - y32).mean() <= 3e-3 * scale
    if H * W <= 4096:
        th32 = theta.astype(np.float32).astype(np.float64)
        x32 = x.astype(np.float32).astype(np.float64)
        for b in range(B):
            yo, _ = ou.forward(th32, x32[b], **kw)
            assert np.abs(ytc[b] - yo).max() <= 3e-2 * max(1e-30, np.abs(yo).max())


def test_unet_tensor_cores_reject_unsupported_widths():
    net = ab.adlbr_unet_create(3, 4, 6, 8, 1, 16, 16)
    try:
        with pytest.raises(ab.AdlbrError):
            ab.adlbr_unet_set_tensor_cores(net, True)
    finally:
        ab.adlbr_unet_destroy(net)


@pytest.mark.parametrize("n", [1, 1000, 1 << 20])
def test_mse_grad_matches_formula(n):
    """adlbr_mse_grad: loss = mean((y - t)^2) (FP64 reduction), gy = 2 (y - t) / n."""
    t = torch()
    g = np.random.default_rng(n)
    y, tt = g.normal(size=n), g.normal(size=n)
    yd, td = dev(y, t.float32), dev(tt, t.float32)
    gy = t.empty_like(yd)
    loss = ab.adlbr_mse_grad(yd, td, n, gy)
    t.cuda.synchronize()
    y32, t32 = y.astype(np.float32).astype(np.float64), tt.astype(np.float32).astype(np.float64)
    d = y32 - t32
    assert abs(loss - np.mean(d * d)) <= 1e-6 * max(1.0, np.mean(d * d))
    assert np.abs(gy.double().cpu().numpy() - 2 * d / n).max() <= 1e-6 * (2 * np.abs(d).max() / n)
