"""Parity of the CUDA coherence-enhancing-diffusion stages (Sec. 4.4) with the
FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ced
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import dev, torch

pytestmark = pytest.mark.gpu

P = dict(sigma=1.0, rho=4.0, alpha=1e-4, C=1e-5)


def _gpu_tensor(u_np, p=P):
    t = torch()
    shape = u_np.shape
    g = ab.grid(shape)
    u = dev(u_np.ravel(), t.float32)
    N = u.numel()
    D = t.empty(3 * N, dtype=t.float32, device="cuda")
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    ab.adlbr_ced_tensor(g, u, D, p["sigma"], p["rho"], p["alpha"], p["C"], scratch)
    t.cuda.synchronize()
    return D.double().cpu().numpy().reshape(3, *shape), u.double().cpu().numpy().reshape(shape)


@pytest.mark.parametrize("shape,p", [((203, 317), P), ((64, 48), dict(sigma=0.5, rho=4.0, alpha=1e-2, C=1e-5))])
def test_ced_tensor_matches_oracle(shape, p):
    img = synth.fingerprint(max(shape), 5)[:shape[0], :shape[1]]
    Dg, useen = _gpu_tensor(img, p)
    Do = np.stack(ced.ced_tensor(useen, p["sigma"], p["rho"], p["alpha"], p["C"]))
    # FP32 chain: blur, gradient, products, blur, eigen, exp.  Entries are in
    # [0, 1]; the bound is 2e-5 absolute (about 200 FP32 ulps of 1).
    err = np.abs(Dg - Do).max()
    assert err <= 2e-5, err


def test_ced_tensor_constant_image():
    Dg, _ = _gpu_tensor(np.full((40, 56), 0.25))
    a = P["alpha"]
    assert np.allclose(Dg[0], a, rtol=1e-6) and np.all(Dg[1] == 0) and np.allclose(Dg[2], a, rtol=1e-6)


def test_ced_steps_match_oracle():
    """Three full CED steps (tensor, stencils, explicit step) at 160 x 192."""
    t = torch()
    shape = (160, 192)
    img = synth.fingerprint(192, 7)[:160, :192]
    g = ab.grid(shape)
    u = dev(img.ravel(), t.float32)
    u0 = u.double().cpu().numpy().reshape(shape)
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    h = ab.adlbr_ced_step(None, g, u, scratch, P["sigma"], P["rho"], P["alpha"], P["C"], 0.02, 3,
                          ab.F32)
    try:
        ab.adlbr_stencils_check(h)
    finally:
        ab.adlbr_stencils_destroy(h)
    ug = u.double().cpu().numpy().reshape(shape)
    uo = u0
    for _ in range(3):
        D = ced.ced_tensor(uo, P["sigma"], P["rho"], P["alpha"], P["C"])
        offs, w, st, _ = oracle.build2d(*D)
        assert np.all(st == 0)
        uo = oracle.step_explicit(shape, oracle.NEUMANN, offs, w, uo, 0.02, 1)
    # the GPU's D differs from the oracle's by FP32 rounding, which can move a
    # stencil decision at near-ties; the changed offsets carry near-zero
    # weight, so u stays within a small multiple of FP32 resolution
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    assert err <= 1e-4, err
    # maximum principle of the non-negative scheme
    assert ug.min() >= u0.min() - 1e-5 and ug.max() <= u0.max() + 1e-5


def _export(h, shape):
    t = torch()
    N = int(np.prod(shape))
    offs = t.zeros((N, 3, 2), dtype=t.int16, device="cuda")
    w = t.zeros((N, 3), dtype=t.float32, device="cuda")
    ab.adlbr_stencils_export(h, offs, w)
    t.cuda.synchronize()
    return offs.cpu().numpy(), w.cpu().numpy()


@pytest.mark.parametrize("sigma", [1.0, 0.5, 2.0])
def test_fused_stencils_equal_tensor_then_build(sigma):
    """adlbr_ced_stencils (tensor stage fused with the construction) gives
    exactly the stencils of adlbr_build_stencils on adlbr_ced_tensor's D
    (sigma = 2 exercises the multi-kernel path for other radii)."""
    t = torch()
    shape = (150, 230)
    p = dict(P, sigma=sigma)
    img = synth.fingerprint(230, 9)[:150, :230]
    g = ab.grid(shape)
    u = dev(img.ravel(), t.float32)
    N = u.numel()
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    D = t.empty(3 * N, dtype=t.float32, device="cuda")
    ab.adlbr_ced_tensor(g, u, D, p["sigma"], p["rho"], p["alpha"], p["C"], scratch)
    h1 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
    h2 = ab.adlbr_ced_stencils(None, g, u, scratch, p["sigma"], p["rho"], p["alpha"], p["C"], ab.F16)
    try:
        ab.adlbr_stencils_check(h1)
        ab.adlbr_stencils_check(h2)
        o1, w1 = _export(h1, shape)
        o2, w2 = _export(h2, shape)
    finally:
        ab.adlbr_stencils_destroy(h1)
        ab.adlbr_stencils_destroy(h2)
    assert np.array_equal(o1, o2)
    assert np.array_equal(w1, w2)
    # and the D of the tensor stage matches the oracle's
    Do = np.stack(ced.ced_tensor(u.double().cpu().numpy().reshape(shape), p["sigma"], p["rho"],
                                 p["alpha"], p["C"]))
    assert np.abs(D.double().cpu().numpy().reshape(3, *shape) - Do).max() <= 2e-5


@pytest.mark.parametrize("shape,p", [((203, 317), P), ((64, 64), P), ((130, 97), P),
                                     ((160, 256), dict(sigma=2.0, rho=6.0, alpha=1e-3, C=1e-5)),
                                     ((96, 160), dict(sigma=0.5, rho=1.5, alpha=1e-2, C=1e-4))])
def test_fused_tensor_equals_separable(shape, p, monkeypatch):
    """The fused tile kernel reproduces the separable passes bit for bit
    (reflected borders, shifted last tiles, several radii)."""
    img = synth.fingerprint(max(shape), 9)[:shape[0], :shape[1]]
    Df, _ = _gpu_tensor(img, p)
    monkeypatch.setenv("ADLBR_CED_PATH", "separable")
    Ds, _ = _gpu_tensor(img, p)
    assert np.array_equal(Df, Ds), np.abs(Df - Ds).max()


def test_fused_tensor_full_size_samples():
    """4096^2 fingerprint (the benchmark image): fused == separable on the
    whole field, and sampled points against the FP64 oracle evaluated on
    small windows (the Gaussian support keeps a 64 x 64 window around a point
    exact away from the border)."""
    import os
    n = 4096
    img = synth.fingerprint(n, 1).astype(np.float32)
    Df, useen = _gpu_tensor(img)
    os.environ["ADLBR_CED_PATH"] = "separable"
    try:
        Ds, _ = _gpu_tensor(img)
    finally:
        del os.environ["ADLBR_CED_PATH"]
    assert np.array_equal(Df, Ds)
    rng = np.random.default_rng(3)
    for _ in range(6):
        y, x = rng.integers(40, n - 40, 2)
        win = useen[y - 32:y + 32, x - 32:x + 32]
        Do = np.stack(ced.ced_tensor(win, P["sigma"], P["rho"], P["alpha"], P["C"]))
        assert np.abs(Df[:, y, x] - Do[:, 32, 32]).max() <= 2e-5


def test_ced_stencils_bitexact_on_gpu_tensor_4096():
    """The benchmark's 4096^2 CED step: the GPU's own tensor D(u) is fed to
    the oracle's construction (Sec. 2), at 200,000 sampled points and at every
    point where D is exactly alpha I (the degenerate tensors of flat regions):
    offsets bit-exact, F16 weights within their storage precision.  The fused
    tensor + stencil kernel (adlbr_ced_stencils) gives the same stencils."""
    from gpu_helpers import weight_tol
    t = torch()
    n = 4096
    N = n * n
    g = ab.grid((n, n))
    u = t.from_numpy(synth.fingerprint(n, 1).astype(np.float32).ravel()).cuda()
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    D = t.empty(3 * N, dtype=t.float32, device="cuda")
    ab.adlbr_ced_tensor(g, u, D, P["sigma"], P["rho"], P["alpha"], P["C"], scratch)
    h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
    hf = ab.adlbr_ced_stencils(None, g, u, scratch, P["sigma"], P["rho"], P["alpha"], P["C"], ab.F16)
    try:
        ab.adlbr_stencils_check(h)
        ab.adlbr_stencils_check(hf)
        Dp = D.view(3, N)
        iso = ((Dp[1] == 0) & (Dp[0] == Dp[2])).nonzero().flatten()
        rng = np.random.default_rng(3)
        samp = t.from_numpy(rng.choice(N, 200000, replace=False)).cuda()
        idx = t.unique(t.cat([samp, iso]))
        outs = []
        for hh in (h, hf):
            offs = t.zeros((N, 3, 2), dtype=t.int16, device="cuda")
            w = t.zeros((N, 3), dtype=t.float32, device="cuda")
            ab.adlbr_stencils_export(hh, offs, w)
            outs.append((offs[idx].cpu().numpy().astype(np.int32), w[idx].double().cpu().numpy()))
            del offs, w
        Ds = Dp[:, idx].double().cpu().numpy()
    finally:
        ab.adlbr_stencils_destroy(h)
        ab.adlbr_stencils_destroy(hf)
    assert iso.numel() > 0, "no exactly isotropic tensor in the workload"
    oo, ow, st, _ = oracle.build2d(Ds[0], Ds[1], Ds[2])
    assert np.all(st == 0)
    go, gw = outs[0]
    assert np.array_equal(go, oo), np.argwhere(np.any(go != oo, axis=(1, 2)))[:5]
    assert np.all(np.abs(gw - ow) <= weight_tol(ow, ab.F16, np.abs(Ds).max()))
    assert np.array_equal(outs[1][0], go) and np.array_equal(outs[1][1], gw)


def _ced_D(shape, seed):
    img = synth.fingerprint(max(shape), seed)[:shape[0], :shape[1]]
    return np.stack(ced.ced_tensor(img, 1.0, 4.0, 1e-4, 1e-5)).reshape(3, -1), img


BUILD_STEP_CASES = {
    # (shape, bc, D dtype, weight type): the first takes the fused kernel
    "fused": ((96, 160), ab.NEUMANN, "float32", ab.F16),
    "ragged_fused": ((77, 132), ab.NEUMANN, "float32", ab.F16),
    "periodic": ((96, 160), ab.PERIODIC, "float32", ab.F16),
    "nx_not_4": ((96, 158), ab.NEUMANN, "float32", ab.F16),
    "f32_weights": ((96, 160), ab.NEUMANN, "float32", ab.F32),
    "f64_tensor": ((96, 160), ab.NEUMANN, "float64", ab.F16),
}


@pytest.mark.parametrize("case", list(BUILD_STEP_CASES))
def test_build_step_equals_build_then_step(case):
    """adlbr_build_step_explicit against adlbr_build_stencils followed by
    adlbr_step_explicit on the same CED tensor: stencils bit for bit, u to
    FP32 rounding, for the fused kernel and for every fallback."""
    from gpu_helpers import export
    t = torch()
    shape, bc, ddt, wt = BUILD_STEP_CASES[case]
    Dn, img = _ced_D(shape, 13)
    g = ab.grid(shape, bc)
    D = dev(Dn, getattr(t, ddt))
    Dt = ab.F32 if ddt == "float32" else ab.F64
    dt = 0.02
    u1 = dev(img.ravel(), t.float32)
    u2 = u1.clone()
    h1 = h2 = None
    try:
        h1 = ab.adlbr_build_stencils(g, D, Dt, wt)
        sc1 = t.empty(ab.adlbr_step_scratch_bytes(h1, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h1, u1, sc1, ab.F32, dt, 1)
        sc2 = t.empty_like(sc1)
        h2 = ab.adlbr_build_step_explicit(g, D, Dt, wt, None, u2, sc2, dt)
        h2 = ab.adlbr_build_step_explicit(g, D, Dt, wt, h2, u2, sc2, dt)   # a second step, in place
        ab.adlbr_step_explicit(h1, u1, sc1, ab.F32, dt, 1)
        ab.adlbr_stencils_check(h1)
        ab.adlbr_stencils_check(h2)
        o1, w1 = export(h1, shape, wt)
        o2, w2 = export(h2, shape, wt)
    finally:
        for h in (h1, h2):
            if h:
                ab.adlbr_stencils_destroy(h)
    assert np.array_equal(o1, o2)
    assert np.array_equal(w1, w2)
    err = (u1 - u2).abs().max().item() / u1.abs().max().item()
    assert err <= 1e-6, err


WARM_CASES = {
    # the tensor the handle's stencils were built from, then the next one
    "same_tensor": (13, "same"),
    "after_ced_steps": (13, "steps"),
    "unrelated_image": (13, "other"),
    "bad_points_before": (13, "bad_first"),
}


@pytest.mark.parametrize("case", list(WARM_CASES))
def test_build_step_warm_start_equals_cold_build(case):
    """A handle that already holds stencils: the fused build-and-step kernel
    starts each point from its previous stencil (certified and repaired, or
    built from scratch where that fails).  The stencils must be those of a
    fresh build of the new tensor, offsets and F16 weights bit for bit after
    the canonical export, and u that of build-then-step, whether the new
    tensor is the same, a few CED steps later, from an unrelated image, or
    follows a build whose points were partly invalid (zero stencils)."""
    from gpu_helpers import export
    t = torch()
    shape = (96, 160)
    seed, kind = WARM_CASES[case]
    g = ab.grid(shape)
    D1n, img = _ced_D(shape, seed)
    if kind == "same":
        D2n = D1n
    elif kind == "other":
        D2n, _ = _ced_D(shape, seed + 1)
    else:
        D2n = D1n
    D1 = dev(D1n, t.float32)
    if kind == "bad_first":
        D1 = D1.clone().reshape(3, -1)
        D1[:, ::7] = float("nan")   # these points get the zero stencil and an error bit
        D1 = D1.reshape(-1)
    u = dev(img.ravel(), t.float32)
    sc = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    if kind == "steps":
        # the tensor three CED steps later, from the GPU's own loop
        u3 = u.clone()
        h3 = ab.adlbr_ced_step(None, g, u3, sc, 1.0, 4.0, 1e-4, 1e-5, 0.5, 3, ab.F16)
        ab.adlbr_stencils_destroy(h3)
        D2 = t.empty(3 * u.numel(), dtype=t.float32, device="cuda")
        ab.adlbr_ced_tensor(g, u3, D2, 1.0, 4.0, 1e-4, 1e-5, sc)
    else:
        D2 = dev(D2n, t.float32)
    h = hc = None
    try:
        h = ab.adlbr_build_step_explicit(g, D1, ab.F32, ab.F16, None, u.clone(), sc, 0.02)
        if kind == "bad_first":
            with pytest.raises(ab.AdlbrError):
                ab.adlbr_stencils_check(h)
        u_w = u.clone()
        h = ab.adlbr_build_step_explicit(g, D2, ab.F32, ab.F16, h, u_w, sc, 0.02)
        ab.adlbr_stencils_check(h)
        hc = ab.adlbr_build_stencils(g, D2, ab.F32, ab.F16)
        u_c = u.clone()
        sc2 = t.empty(ab.adlbr_step_scratch_bytes(hc, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(hc, u_c, sc2, ab.F32, 0.02, 1)
        ab.adlbr_stencils_check(hc)
        o_w, w_w = export(h, shape, ab.F16)
        o_c, w_c = export(hc, shape, ab.F16)
    finally:
        for hh in (h, hc):
            if hh:
                ab.adlbr_stencils_destroy(hh)
    assert np.array_equal(o_w, o_c)
    assert np.array_equal(w_w, w_c)
    err = (u_w - u_c).abs().max().item() / u_c.abs().max().item()
    assert err <= 1e-6, err


def test_build_step_reports_a_bad_tensor():
    """A tensor that is not positive definite at one point: the fused kernel
    reports it as the build does (ADLBR_E_NOT_SPD from adlbr_stencils_check),
    gives that point the zero stencil, and steps every other point."""
    t = torch()
    shape = (64, 96)
    Dn, img = _ced_D(shape, 17)
    Dn = Dn.copy()
    Dn[0, 700] = -1.0
    g = ab.grid(shape)
    D = dev(Dn, t.float32)
    u1 = dev(img.ravel(), t.float32)
    u2 = u1.clone()
    h1 = h2 = None
    try:
        h1 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
        sc1 = t.empty(ab.adlbr_step_scratch_bytes(h1, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h1, u1, sc1, ab.F32, 0.02, 1)
        h2 = ab.adlbr_build_step_explicit(g, D, ab.F32, ab.F16, None, u2, t.empty_like(sc1), 0.02)
        for h in (h1, h2):
            with pytest.raises(ab.AdlbrError) as ei:
                ab.adlbr_stencils_check(h)
            assert ei.value.status == 3
    finally:
        for h in (h1, h2):
            if h:
                ab.adlbr_stencils_destroy(h)
    err = (u1 - u2).abs().max().item() / u1.abs().max().item()
    assert err <= 1e-6, err


def test_build_step_full_size_4096():
    """The benchmark's timed launch: the 4096^2 CED tensor, then the build
    fused into the operator (F16 weights, FP32 u), against the build and the
    stand-alone step: stencils bit for bit over the whole grid, u to 1e-6, and
    u at 20,000 sampled points against the oracle's explicit step on the
    exported stencils."""
    from gpu_helpers import export
    t = torch()
    n = 4096
    g = ab.grid((n, n))
    img = synth.fingerprint(n, 1).astype(np.float32)
    u1 = t.from_numpy(img.ravel().copy()).cuda()
    u2 = u1.clone()
    N = n * n
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    D = t.empty(3 * N, dtype=t.float32, device="cuda")
    ab.adlbr_ced_tensor(g, u1, D, 1.0, 4.0, 1e-4, 1e-5, scratch)
    acc1 = t.empty(N, dtype=t.float32, device="cuda")
    acc2 = t.empty_like(acc1)
    h1 = h2 = None
    try:
        h1 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
        ab.adlbr_step_explicit(h1, u1, acc1, ab.F32, 0.02, 1)
        h2 = ab.adlbr_build_step_explicit(g, D, ab.F32, ab.F16, None, u2, acc2, 0.02)
        ab.adlbr_stencils_check(h1)
        ab.adlbr_stencils_check(h2)
        o1, w1 = export(h1, (n, n), ab.F16)
        o2, w2 = export(h2, (n, n), ab.F16)
    finally:
        for h in (h1, h2):
            if h:
                ab.adlbr_stencils_destroy(h)
    assert np.array_equal(o1, o2)
    assert np.array_equal(w1, w2)
    a, b = u1.double().cpu().numpy(), u2.double().cpu().numpy()
    scale = np.abs(a).max()
    assert np.abs(a - b).max() <= 1e-6 * scale
    # sampled points against the oracle's step: u - dt (A u) from own and
    # incoming terms of the exported stencils
    from test_gpu_gather import _rows
    uu = img.astype(np.float64).reshape(n, n)
    zs = np.random.default_rng(3).integers(0, N, 20000)
    ref = uu.ravel()[zs] - 0.02 * _rows(o2, w2, uu, zs, n)
    assert np.abs(b[zs] - ref).max() <= 1e-6 * scale


def test_build_step_warm_start_full_size_4096():
    """The benchmark's loop: four CED steps at 4096^2 through the tensor
    stage and the fused build-and-step (every step after the first starts
    from the previous stencils).  The handle's stencils after the last step
    must equal a fresh build of the last tensor over the whole grid, and u
    the build-then-step of the same tensor."""
    from gpu_helpers import export
    t = torch()
    n = 4096
    g = ab.grid((n, n))
    N = n * n
    u = t.from_numpy(synth.fingerprint(n, 1).astype(np.float32).ravel().copy()).cuda()
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    D = t.empty(3 * N, dtype=t.float32, device="cuda")
    acc = t.empty(N, dtype=t.float32, device="cuda")
    h = hc = None
    try:
        for step in range(4):
            ab.adlbr_ced_tensor(g, u, D, 1.0, 4.0, 1e-4, 1e-5, scratch)
            if step == 3:
                u_c = u.clone()
            h = ab.adlbr_build_step_explicit(g, D, ab.F32, ab.F16, h, u, acc, 0.02)
        ab.adlbr_stencils_check(h)
        hc = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
        ab.adlbr_step_explicit(hc, u_c, acc, ab.F32, 0.02, 1)
        ab.adlbr_stencils_check(hc)
        o_w, w_w = export(h, (n, n), ab.F16)
        o_c, w_c = export(hc, (n, n), ab.F16)
    finally:
        for hh in (h, hc):
            if hh:
                ab.adlbr_stencils_destroy(hh)
    assert np.array_equal(o_w, o_c)
    assert np.array_equal(w_w, w_c)
    a, b = u.double().cpu().numpy(), u_c.double().cpu().numpy()
    assert np.abs(a - b).max() <= 1e-6 * np.abs(b).max()


def test_build_step_3d_equals_build_then_step():
    """The 3D grid takes the two-call path inside adlbr_build_step_explicit:
    same stencils bit for bit, same u to FP32 rounding."""
    from gpu_helpers import export
    t = torch()
    shape = (20, 24, 28)
    D = dev(synth.needle_field3d(28, seed=9, kappa=15.0)[:, :20, :24, :28].reshape(6, -1), t.float32)
    g = ab.grid(shape)
    u1 = dev(synth.u_uniform(shape, 4).ravel(), t.float32)
    u2 = u1.clone()
    h1 = h2 = None
    try:
        h1 = ab.adlbr_build_stencils(g, D, ab.F32, ab.F16)
        dt = 0.5 / ab.adlbr_stencils_max_diag(h1)
        sc = t.empty(ab.adlbr_step_scratch_bytes(h1, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h1, u1, sc, ab.F32, dt, 1)
        h2 = ab.adlbr_build_step_explicit(g, D, ab.F32, ab.F16, None, u2, t.empty_like(sc), dt)
        o1, w1 = export(h1, shape, ab.F16)
        o2, w2 = export(h2, shape, ab.F16)
    finally:
        for h in (h1, h2):
            if h:
                ab.adlbr_stencils_destroy(h)
    assert np.array_equal(o1, o2) and np.array_equal(w1, w2)
    assert (u1 - u2).abs().max().item() <= 1e-6 * u1.abs().max().item()
