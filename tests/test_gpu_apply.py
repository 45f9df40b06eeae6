"""Parity of the CUDA operator and explicit step with the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, dev, export, torch

pytestmark = pytest.mark.gpu


def _gpu_apply(h, u_np, u_dtype):
    t = torch()
    u = dev(u_np.ravel(), u_dtype)
    acc = t.float64 if u_dtype == t.float64 else t.float32
    Au = t.empty(u.numel(), dtype=acc, device="cuda")
    ab.adlbr_apply(h, u, Au, ab.dtype_code(u_dtype))
    t.cuda.synchronize()
    return Au.double().cpu().numpy().reshape(u_np.shape), u.double().cpu().numpy().reshape(u_np.shape)


def _oracle_stencils(seen, dim):
    if dim == 2:
        oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
    else:
        oo, ow, st, _ = oracle.build3d(seen.reshape(6, -1))
    assert np.all(st == 0)
    return oo, ow


@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
@pytest.mark.parametrize("dim", [2, 3])
def test_apply_fp64(bc, dim):
    t = torch()
    if dim == 2:
        shape = (45, 67)
        D = synth.smooth_field2d(*shape, seed=3, kappa_min=1, kappa_max=60, lattice=6)
    else:
        shape = (13, 17, 19)
        D = synth.needle_field3d(19, seed=5, kappa=15.0)[:, :13, :17, :19]
    h, seen, _ = build(D, shape, t.float64, ab.F64, bc)
    try:
        u = synth.u_uniform(shape, 1)
        Au, _ = _gpu_apply(h, u, t.float64)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = _oracle_stencils(seen, dim)
    ref = oracle.apply(shape, bc, oo, ow, u)
    assert np.abs(Au - ref).max() <= 1e-13 * np.abs(ref).max()


THIN = [(1, 37), (37, 1), (2, 130), (130, 3), (5, 9), (1, 1, 50), (3, 1, 40), (40, 2, 1), (2, 3, 70)]


@pytest.mark.parametrize("shape", THIN, ids=["x".join(map(str, s)) for s in THIN])
@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
@pytest.mark.parametrize("u_dtype", ["float64", "float32"])
def test_apply_thin_grids(shape, bc, u_dtype):
    """Grids thinner than a tile or its halo in some direction (one point
    wide, fewer points than an offset is long, x not a multiple of 4, so no
    TMA window): FP64 to rounding, FP32 to 1e-5 relative, both boundary
    rules, with anisotropic fields whose offsets leave the grid."""
    t = torch()
    dt_ = getattr(t, u_dtype)
    if len(shape) == 2:
        D = synth.smooth_field2d(*shape, seed=7, kappa_min=1, kappa_max=40, lattice=4)
    else:
        n = max(shape)
        D = synth.needle_field3d(n, seed=8, kappa=15.0)[:, :shape[0], :shape[1], :shape[2]]
    w_t = ab.F64 if u_dtype == "float64" else ab.F32
    h, seen, _ = build(D, shape, dt_, w_t, bc)
    try:
        u = synth.u_uniform(shape, 3)
        Au, useen = _gpu_apply(h, u, dt_)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = _oracle_stencils(seen, len(shape))
    ref = oracle.apply(shape, bc, oo, ow, useen)
    tol = 1e-13 if u_dtype == "float64" else 1e-5
    assert np.abs(Au - ref).max() <= tol * max(np.abs(ref).max(), 1e-300)


@pytest.mark.parametrize("dim", [2, 3])
def test_apply_fp32_within_1e5(dim):
    """FP32 u, FP32 weights, FP32 accumulation: relative L-inf error <= 1e-5."""
    t = torch()
    if dim == 2:
        shape = (64, 96)
        D = synth.smooth_field2d(*shape, seed=4, kappa_min=1, kappa_max=100, lattice=8)
    else:
        shape = (20, 24, 28)
        D = synth.needle_field3d(28, seed=6, kappa=20.0)[:, :20, :24, :28]
    h, seen, _ = build(D, shape, t.float32, ab.F32)
    try:
        u = synth.u_uniform(shape, 2)
        Au, useen = _gpu_apply(h, u, t.float32)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = _oracle_stencils(seen, dim)
    ref = oracle.apply(shape, ab.NEUMANN, oo, ow, useen)
    assert np.abs(Au - ref).max() <= 1e-5 * np.abs(ref).max()


def test_explicit_64x64_fp64_10_steps():
    """64x64 FP64, spiral field kappa = 10, u0 ~ U[0,1] (seed 0), 10 explicit
    steps at dt = 1 / max A_zz, zero-flux boundary: GPU == oracle to 1e-12."""
    t = torch()
    D = synth.spiral_field(64, 10.0)
    h, seen, _ = build(D, (64, 64), t.float64, ab.F64)
    oo, ow = _oracle_stencils(seen, 2)
    dt = oracle.dt_limit((64, 64), oracle.NEUMANN, oo, ow)
    u0 = synth.u_uniform((64, 64), 0)
    try:
        u = dev(u0.ravel(), t.float64)
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F64), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.F64, dt, 10)
        t.cuda.synchronize()
        ug = u.cpu().numpy().reshape(64, 64)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.step_explicit((64, 64), oracle.NEUMANN, oo, ow, u0, dt, 10)
    assert np.abs(ug - ref).max() <= 1e-12 * np.abs(ref).max()
    # discrete maximum principle and mass conservation hold on the GPU too
    assert ug.min() >= u0.min() - 1e-12 and ug.max() <= u0.max() + 1e-12
    assert abs(ug.sum() - u0.sum()) <= 1e-9


@pytest.mark.parametrize("u_name,w_t,tol", [("float32", ab.F32, 1e-5), ("float32", ab.F16, 1e-3),
                                            ("bfloat16", ab.F16, 2e-2), ("float16", ab.F16, 4e-3)])
def test_explicit_step_error_per_step(u_name, w_t, tol):
    """Per-step relative L-inf error of one explicit step from the same u^n,
    against the FP64 oracle fed the same (rounded) u^n and D."""
    t = torch()
    shape = (96, 128)
    D = synth.smooth_field2d(*shape, seed=8, kappa_min=1, kappa_max=100, lattice=8)
    h, seen, _ = build(D, shape, t.float32, w_t)
    oo, ow = _oracle_stencils(seen, 2)
    dt = oracle.dt_limit(shape, oracle.NEUMANN, oo, ow)
    u0 = synth.u_uniform(shape, 3)
    ud = getattr(t, u_name)
    try:
        u = dev(u0.ravel(), ud)
        useen = u.double().cpu().numpy().reshape(shape)
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.dtype_code(ud)), dtype=t.uint8,
                          device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.dtype_code(ud), dt, 1)
        t.cuda.synchronize()
        ug = u.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.step_explicit(shape, oracle.NEUMANN, oo, ow, useen, dt, 1)
    err = np.abs(ug - ref).max() / np.abs(ref).max()
    assert err <= tol, err


def test_apply_full_size_4096():
    """4096^2 FP32 field, kappa up to 100 (CED-sized), FP32 weights and u:
    every output against the oracle, plus Neumann mass conservation."""
    t = torch()
    n = 4096
    D = synth.smooth_field2d(n, n, seed=9, kappa_min=1, kappa_max=100, lattice=64)
    h, seen, _ = build(D, (n, n), t.float32, ab.F32)
    try:
        u = synth.u_uniform((n, n), 4)
        Au, useen = _gpu_apply(h, u, t.float32)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = _oracle_stencils(seen, 2)
    ref = oracle.apply((n, n), oracle.NEUMANN, oo, ow, useen)
    assert np.abs(Au - ref).max() <= 1e-5 * np.abs(ref).max()
    assert abs(Au.sum()) <= 1e-6 * np.abs(Au).sum()


@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
@pytest.mark.parametrize("dim", [2, 3])
def test_max_diag_matches_oracle(bc, dim):
    """max_z A_zz (the explicit limit dt = 1 / max A_zz) against the oracle's
    diagonal; FP32 accumulation on the device."""
    t = torch()
    if dim == 2:
        shape = (45, 67)
        D = synth.smooth_field2d(*shape, seed=3, kappa_min=1, kappa_max=60, lattice=6)
    else:
        shape = (13, 17, 19)
        D = synth.needle_field3d(19, seed=5, kappa=15.0)[:, :13, :17, :19]
    h, seen, _ = build(D, shape, t.float32, ab.F32, bc)
    try:
        m = ab.adlbr_stencils_max_diag(h)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = _oracle_stencils(seen, dim)
    ref = oracle.diag(shape, bc, oo, ow).max()
    assert abs(m - ref) <= 1e-5 * ref, (m, ref)


def test_apply3d_full_size_sampled():
    """256^3 needle stencils (F16 weights), FP32 u, the launch the benchmark
    times: Au at sampled points against the oracle on a crop around each
    point (the crop's half width exceeds the longest offset, so every pair
    that touches the centre lies inside the crop)."""
    t = torch()
    n = 256
    D = synth.needle_field3d(n, 2, kappa=20.0, dtype=np.float32)
    h, seen, _ = build(D, (n, n, n), t.float32, ab.F16)
    try:
        go, gw = export(h, (n, n, n), ab.F16)
        u = synth.u_uniform((n, n, n), 7)
        Au, useen = _gpu_apply(h, u, t.float32)
    finally:
        ab.adlbr_stencils_destroy(h)
    half = int(np.abs(go).max()) + 1     # crop half width beyond the longest offset
    assert half <= 24
    go = go.reshape(n, n, n, 6, 3)
    gw = gw.reshape(n, n, n, 6)
    scale = np.abs(Au).max()
    rng = np.random.default_rng(2)
    pts = [tuple(rng.integers(half, n - half, 3)) for _ in range(6)] + [(0, 0, 0), (n - 1, 5, n - 1)]
    for z, y, x in pts:
        z0, y0, x0 = (max(0, c - half) for c in (z, y, x))
        z1, y1, x1 = (min(n, c + half + 1) for c in (z, y, x))
        cs = (z1 - z0, y1 - y0, x1 - x0)
        oo = go[z0:z1, y0:y1, x0:x1].reshape(-1, 6, 3)
        ow = gw[z0:z1, y0:y1, x0:x1].reshape(-1, 6)
        ref = oracle.apply(cs, oracle.NEUMANN, oo, ow, useen[z0:z1, y0:y1, x0:x1])
        assert abs(Au[z, y, x] - ref[z - z0, y - y0, x - x0]) <= 1e-5 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_fourier_modes_are_eigenvectors(dim):
    """Constant D on a periodic grid: the Fourier mode cos(xi . z) is an
    eigenvector of A with eigenvalue sigma(xi) = sum over the stencil V (both
    signs of every offset) of 2 gamma(e) (1 - cos(xi . e)), i.e. four times
    the sum over the stored half-stencil (the symbol of the scheme; Fig.
    Eigen of the paper studies it), on the GPU operator in FP64."""
    t = torch()
    if dim == 2:
        shape = (48, 64)
        D1 = synth.D_from_angle(np.array(0.37), np.array(7.0))
    else:
        shape = (16, 20, 24)
        D1 = synth.random_spd3(1, 9, kappa_max=6.0)[:, 0]
    Dfield = np.broadcast_to(D1.reshape(-1, *([1] * dim)), (D1.shape[0],) + shape).copy()
    h, seen, _ = build(Dfield, shape, t.float64, ab.F64, ab.PERIODIC)
    try:
        oo, ow = export(h, shape, ab.F64)
        k = (3, 5) if dim == 2 else (2, 3, 1)
        grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")   # [z, y, x] order
        xi = [2 * np.pi * k[i] / shape[i] for i in range(dim)]
        phase = sum(xi[i] * grids[i] for i in range(dim))
        u = np.cos(phase)
        Au, _ = _gpu_apply(h, u, t.float64)
    finally:
        ab.adlbr_stencils_destroy(h)
    # symbol from the (constant) stencil of point 0; offsets are (x, y[, z])
    e = oo[0]
    xi_xyz = xi[::-1]
    sig = sum(4 * ow[0, j] * (1 - np.cos(sum(xi_xyz[c] * e[j, c] for c in range(dim))))
              for j in range(e.shape[0]))
    assert np.abs(Au - sig * u).max() <= 1e-12 * max(1.0, sig)


@pytest.mark.parametrize("u_name", ["float16", "bfloat16"])
@pytest.mark.parametrize("nx", [32, 28])
def test_apply3d_half_vectors(u_name, nx):
    """3D operator on 16-bit u (F16 weights), against the oracle fed the same
    rounded u: nx = 32 takes the TMA window (16-bit staging box widened in
    shared memory), nx = 28 the plain loads; then two explicit steps (the
    vectorised 16-bit finalize) against the oracle's."""
    t = torch()
    shape = (20, 24, nx)
    D = synth.needle_field3d(32, seed=6, kappa=20.0)[:, :20, :24, :nx]
    h, seen, _ = build(D, shape, t.float32, ab.F16)
    ud = getattr(t, u_name)
    try:
        oo, ow = export(h, shape, ab.F16)
        u = dev(synth.u_uniform(shape, 2).ravel(), ud)
        useen = u.double().cpu().numpy().reshape(shape)
        Au, _ = _gpu_apply(h, useen, ud)
        dt = oracle.dt_limit(shape, oracle.NEUMANN, oo, ow)
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.dtype_code(ud)), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.dtype_code(ud), dt, 1)
        t.cuda.synchronize()
        u1 = u.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, ab.NEUMANN, oo, ow, useen)
    assert np.abs(Au - ref).max() <= 1e-5 * np.abs(ref).max()
    # one step, rounded once to the storage type (half an ulp of 1: 2^-11 / 2^-8)
    step = oracle.step_explicit(shape, oracle.NEUMANN, oo, ow, useen, dt, 1)
    tol = {"float16": 2.0 ** -11, "bfloat16": 2.0 ** -8}[u_name]
    assert np.abs(u1 - step).max() <= tol * np.abs(step).max() + 1e-6
