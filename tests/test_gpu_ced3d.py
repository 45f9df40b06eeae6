"""The 3D coherence-enhancing tensor (Sec. 5, 3D experiments) on the GPU
against the FP64 oracle, and the 3D CED pipeline (tensor, 3D stencils,
implicit step); the same for the edge-enhancing tensor of the 3D MRI
experiment."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ced
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import dev, torch

pytestmark = pytest.mark.gpu

P3 = dict(sigma=0.5, rho=4.0, alpha=1e-2, C=1e-5)


def _gpu_tensor3(u_np, p=P3):
    t = torch()
    g = ab.grid(u_np.shape)
    u = dev(u_np.ravel(), t.float32)
    N = u.numel()
    D = t.empty(6 * N, dtype=t.float32, device="cuda")
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    ab.adlbr_ced_tensor(g, u, D, p["sigma"], p["rho"], p["alpha"], p["C"], scratch)
    t.cuda.synchronize()
    return D.double().cpu().numpy().reshape(6, *u_np.shape), u.double().cpu().numpy().reshape(u_np.shape)


@pytest.mark.parametrize("shape,p", [((20, 24, 28), P3), ((17, 9, 13), dict(sigma=1.0, rho=2.0, alpha=1e-3, C=1e-4))])
def test_tensor3d_matches_oracle(shape, p):
    _, noisy = synth.radial3d(max(shape), 4)
    u = noisy[:shape[0], :shape[1], :shape[2]]
    Dg, useen = _gpu_tensor3(u, p)
    Do = ced.ced_tensor3(useen, p["sigma"], p["rho"], p["alpha"], p["C"])
    err = np.abs(Dg - Do).max()
    assert err <= 5e-5, err


def test_tensor3d_constant_image():
    Dg, _ = _gpu_tensor3(np.full((6, 7, 8), 0.3))
    a = P3["alpha"]
    assert np.allclose(Dg[:3], a, rtol=1e-6) and np.all(np.abs(Dg[3:]) <= 1e-12)


def test_tensor3d_full_size_samples():
    """The 100^3 workload of the 3D experiment: sampled points against the
    oracle on 40^3 windows (the support of K_sigma, the gradient and K_rho
    keeps the centre exact)."""
    n, h = 100, 20
    _, noisy = synth.radial3d(n, 5)
    Dg, useen = _gpu_tensor3(noisy)
    rng = np.random.default_rng(6)
    for _ in range(4):
        z, y, x = rng.integers(h, n - h, 3)
        win = useen[z - h:z + h, y - h:y + h, x - h:x + h]
        Do = ced.ced_tensor3(win, P3["sigma"], P3["rho"], P3["alpha"], P3["C"])
        assert np.abs(Dg[:, z, y, x] - Do[:, h, h, h]).max() <= 5e-5


def test_ced3d_implicit_steps_match_oracle_and_denoise():
    """Three steps of the 3D CED pipeline on 32^3 (tensor and stencils from
    the current u, then (I + dt A) u_new = u by CG), dt = 1e-3 on [0,1]^3,
    i.e. 1e-3 n^2 in grid units; against the same steps in the oracle.  The
    error to the clean image falls."""
    t = torch()
    n, steps = 32, 3
    dt = 1e-3 * n * n
    u0, noisy = synth.radial3d(n, 7)
    g = ab.grid((n, n, n))
    u = dev(noisy.ravel(), t.float32)
    useen = u.double().cpu().numpy().reshape(n, n, n)
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    h = None
    try:
        for _ in range(steps):
            h = ab.adlbr_ced_stencils(h, g, u, scratch, P3["sigma"], P3["rho"], P3["alpha"], P3["C"],
                                      ab.F32)
            x = u.clone()
            ab.adlbr_step_implicit(h, u, x, dt, 1e-7, 4000)
            u.copy_(x)
        ug = u.double().cpu().numpy().reshape(n, n, n)
    finally:
        if h:
            ab.adlbr_stencils_destroy(h)
    uo = useen
    for _ in range(steps):
        D = ced.ced_tensor3(uo, P3["sigma"], P3["rho"], P3["alpha"], P3["C"])
        offs, w, st, _ = oracle.build3d(D.reshape(6, -1))
        assert np.all(st == 0)
        uo, _, _ = oracle.cg((n, n, n), oracle.NEUMANN, offs, w, uo, uo, dt, rtol=1e-10)
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    assert err <= 1e-3, err
    assert np.sqrt(np.mean((ug - u0) ** 2)) < 0.5 * np.sqrt(np.mean((noisy - u0) ** 2))


def _gpu_eed(u_np, sigma, rho, C):
    t = torch()
    g = ab.grid(u_np.shape)
    u = dev(u_np.ravel(), t.float32)
    D = t.empty(6 * u.numel(), dtype=t.float32, device="cuda")
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    ab.adlbr_eed_tensor(g, u, D, sigma, rho, C, scratch)
    t.cuda.synchronize()
    return D.double().cpu().numpy().reshape(6, *u_np.shape), u.double().cpu().numpy().reshape(u_np.shape)


@pytest.mark.parametrize("shape,sigma,rho,C", [((20, 24, 28), 0.5, 4.0, 1e-5), ((17, 9, 13), 1.0, 2.0, 1e-4),
                                               ((40, 40, 16), 0.5, 4.0, 7.7e-6)])
def test_eed_tensor_matches_oracle(shape, sigma, rho, C):
    """Edge-enhancing tensor (Sec. 5, 3D MRI experiment) on the shell volume
    that stands in for the MRI scan, ragged shapes, against the oracle."""
    _, noisy = synth.shells3d(shape, 8)
    Dg, useen = _gpu_eed(noisy, sigma, rho, C)
    Do = ced.eed_tensor3(useen, sigma, rho, C)
    err = np.abs(Dg - Do).max()
    assert err <= 5e-5, err


def test_eed_tensor_constant_image_and_arguments():
    """J = 0: D = I.  A 2D grid, C = 0 and a negative sigma are refused."""
    t = torch()
    Dg, _ = _gpu_eed(np.full((6, 7, 8), 0.3), 0.5, 4.0, 1e-4)
    assert np.allclose(Dg[:3], 1.0, rtol=0, atol=1e-7) and np.all(np.abs(Dg[3:]) <= 1e-7)
    u = t.zeros(64, dtype=t.float32, device="cuda")
    D = t.empty(6 * 64, dtype=t.float32, device="cuda")
    sc = t.empty(ab.adlbr_ced_scratch_bytes(ab.grid((4, 4, 4))), dtype=t.uint8, device="cuda")
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_eed_tensor(ab.grid((8, 8)), u, D, 0.5, 4.0, 1e-4, sc)
    assert ei.value.status == 2
    for sigma, C in ((0.5, 0.0), (-1.0, 1e-4)):
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_eed_tensor(ab.grid((4, 4, 4)), u, D, sigma, 4.0, C, sc)
        assert ei.value.status == 1


def test_eed_pipeline_stencils_and_implicit_steps_match_oracle():
    """Two steps of the 3D edge-enhancing pipeline on a 24 x 28 x 20 shell
    volume: the GPU tensor, its 3D stencils (offsets bit for bit against the
    oracle's construction on the same tensor), then (I + dt A) u_new = u by
    CG; against the same steps in the oracle."""
    t = torch()
    shape, steps, C = (20, 28, 24), 2, 1e-5
    dt = 2.0
    _, noisy = synth.shells3d(shape, 9)
    g = ab.grid(shape)
    u = dev(noisy.ravel(), t.float32)
    uo = u.double().cpu().numpy().reshape(shape)
    N = u.numel()
    D = t.empty(6 * N, dtype=t.float32, device="cuda")
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    h = None
    try:
        for k in range(steps):
            ab.adlbr_eed_tensor(g, u, D, 0.5, 4.0, C, scratch)
            h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32, out=h)
            ab.adlbr_stencils_check(h)
            if k == 0:
                from gpu_helpers import export
                go, _ = export(h, shape, ab.F32)
                Dseen = D.double().cpu().numpy().reshape(6, -1)
                oo, _, st, _ = oracle.build3d(Dseen)
                assert np.all(st == 0) and np.array_equal(go, oo)
            x = u.clone()
            ab.adlbr_step_implicit(h, u, x, dt, 1e-7, 4000)
            u.copy_(x)
        ug = u.double().cpu().numpy().reshape(shape)
    finally:
        if h:
            ab.adlbr_stencils_destroy(h)
    for _ in range(steps):
        Do = ced.eed_tensor3(uo, 0.5, 4.0, C)
        offs, w, st, _ = oracle.build3d(Do.reshape(6, -1))
        assert np.all(st == 0)
        uo, _, _ = oracle.cg(shape, oracle.NEUMANN, offs, w, uo, uo, dt, rtol=1e-10)
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    assert err <= 1e-3, err
