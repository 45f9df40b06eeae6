"""Parity of the CUDA stencil construction with the FP64 oracle: offsets bit
for bit (canonical form), weights within the storage precision."""
import numpy as np
import pytest

import oracle
import synth
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, export, torch, weight_tol

pytestmark = pytest.mark.gpu


def _compare(D, shape, D_dtype, w_t, dim):
    t = torch()
    h, seen, _ = build(D, shape, D_dtype, w_t)
    try:
        ab.adlbr_stencils_check(h)
        go, gw = export(h, shape, w_t)
    finally:
        ab.adlbr_stencils_destroy(h)
    if dim == 2:
        oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
    else:
        oo, ow, st, _ = oracle.build3d(seen.reshape(6, -1))
    assert np.all(st == 0)
    mism = np.nonzero((go != oo).any(axis=(1, 2)))[0]
    assert mism.size == 0, ("offset mismatch", mism[:5], go[mism[:2]], oo[mism[:2]])
    scale = np.abs(seen.reshape(seen.shape[0], -1)).max(axis=0)[:, None]
    tol = weight_tol(ow, w_t, scale)
    err = np.abs(gw - ow)
    assert np.all(err <= tol), (err.max(), np.unravel_index(np.argmax(err - tol), err.shape))


@pytest.mark.parametrize("D_dtype,w_t", [("float64", ab.F64), ("float32", ab.F32),
                                         ("float32", ab.F16), ("float64", ab.F32)])
def test_build2d_random_tensors(D_dtype, w_t):
    t = torch()
    D = synth.random_spd2(37 * 53, seed=1, kappa_max=1000.0).reshape(3, 37, 53)
    _compare(D, (37, 53), getattr(t, D_dtype), w_t, 2)


def test_build2d_spiral_64_fp64():
    """64x64 FP64 spiral field, kappa = 10 (the small FP64 configuration)."""
    D = synth.spiral_field(64, 10.0)
    _compare(D, (64, 64), torch().float64, ab.F64, 2)


def test_build2d_degenerate_and_exact():
    t = torch()
    D = np.array([[1.0, 0, 1], [2.0, 0, 1], [1.0, 0, 3], [9.5, 6, 4], [2, 1, 2], [2, -1, 2],
                  [1, 0.5, 1], [5, 0, 1e-4], [1e-4, 0, 5], [1, 1 - 1e-6, 1]]).T
    D = np.concatenate([D, np.repeat(D[:, :1], 6, axis=1)], axis=1)   # 16 points
    for dt in (t.float64, t.float32):
        _compare(D.reshape(3, 4, 4), (4, 4), dt, ab.F64 if dt == t.float64 else ab.F32, 2)


def test_build2d_status_codes():
    t = torch()
    for bad, code in [((1.0, 0.0, -1.0), 3), ((1.0, 2.0, 1.0), 3), ((np.nan, 0.0, 1.0), 4)]:
        D = np.ones((3, 2, 2))
        D[1] = 0.0
        D[:, 1, 1] = bad
        h, _, _ = build(D, (2, 2), t.float32, ab.F32)
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_stencils_check(h)
        assert ei.value.status == code
        ab.adlbr_stencils_check(h)  # sticky flag was cleared
        ab.adlbr_stencils_destroy(h)


@pytest.mark.parametrize("D_dtype,w_t", [("float64", ab.F64), ("float32", ab.F32),
                                         ("float32", ab.F16)])
def test_build3d_random_tensors(D_dtype, w_t):
    t = torch()
    D = synth.random_spd3(9 * 10 * 11, seed=2, kappa_max=40.0).reshape(6, 9, 10, 11)
    _compare(D, (9, 10, 11), getattr(t, D_dtype), w_t, 3)


def test_build3d_needle_field_and_degenerate():
    t = torch()
    D = synth.needle_field3d(24, seed=2, kappa=20.0)
    _compare(D, (24, 24, 24), t.float32, ab.F32, 3)
    cases = [np.eye(3), np.diag([1.0, 2.0, 3.0]), np.array([[2.0, 1, 1], [1, 2, 1], [1, 1, 2]]),
             np.array([[2.0, -1, 0], [-1, 2, -1], [0, -1, 2]])]
    D6 = np.array([[M[0, 0], M[1, 1], M[2, 2], M[0, 1], M[0, 2], M[1, 2]] for M in cases]).T
    D6 = np.repeat(D6, 2, axis=1).reshape(6, 2, 2, 2)
    _compare(D6, (2, 2, 2), t.float64, ab.F64, 3)


def test_build2d_full_size_sampled():
    """4096^2 FP32 field with kappa up to 100 (the size of the CED workload),
    built in one launch; a random sample of points is checked against the
    oracle point by point."""
    t = torch()
    n = 4096
    D = synth.smooth_field2d(n, n, seed=7, kappa_min=1.0, kappa_max=100.0, lattice=64)
    h, seen, _ = build(D, (n, n), t.float32, ab.F16)
    try:
        ab.adlbr_stencils_check(h)
        go, gw = export(h, (n, n), ab.F16)
    finally:
        ab.adlbr_stencils_destroy(h)
    idx = np.random.default_rng(0).choice(n * n, 200_000, replace=False)
    oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1)[:, idx])
    assert np.all(st == 0)
    assert np.array_equal(go[idx], oo)
    assert np.all(np.abs(gw[idx] - ow) <= weight_tol(ow, ab.F16, None))


def test_build3d_full_size_sampled():
    """256^3 needle field (the 3D workload, FP32 D, F16 weights) built in one
    launch; a random sample of points against the oracle point by point."""
    t = torch()
    n = 256
    D = synth.needle_field3d(n, 2, kappa=20.0, dtype=np.float32)
    h, seen, _ = build(D, (n, n, n), t.float32, ab.F16)
    try:
        ab.adlbr_stencils_check(h)
        go, gw = export(h, (n, n, n), ab.F16)
    finally:
        ab.adlbr_stencils_destroy(h)
    idx = np.random.default_rng(1).choice(n ** 3, 50_000, replace=False)
    oo, ow, st, _ = oracle.build3d(seen.reshape(6, -1)[:, idx])
    assert np.all(st == 0)
    assert np.array_equal(go[idx], oo)
    assert np.all(np.abs(gw[idx] - ow) <= weight_tol(ow, ab.F16, None))
