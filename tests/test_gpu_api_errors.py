"""Argument checking at the C ABI: bad grids, null buffers, aliasing and
mismatched types are reported as status codes (no launch), and a 1-point
grid (no in-grid pairs) is a valid degenerate case."""
import ctypes

import numpy as np
import pytest

from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import dev, torch

pytestmark = pytest.mark.gpu


def _D(shape):
    t = torch()
    D = np.zeros((3,) + shape)
    D[0] = 1.0
    D[2] = 0.5
    return dev(D.reshape(3, -1), t.float32)


@pytest.mark.parametrize("shape", [(0, 8), (8, 0), (70000, 2)])
def test_bad_grid_extents(shape):
    t = torch()
    D = t.zeros(3 * max(1, shape[0] * shape[1]), device="cuda")
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_build_stencils(ab.grid(shape), D, ab.F32, ab.F32)
    assert ei.value.status == 2


def test_bad_dimension_and_types():
    g = ab.grid((4, 4))
    g.dim = 4
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_build_stencils(g, _D((4, 4)), ab.F32, ab.F32)
    assert ei.value.status == 2
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_build_stencils(ab.grid((4, 4)), _D((4, 4)), ab.F16, ab.F32)   # D must be F32/F64
    assert ei.value.status == 1
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_build_stencils(ab.grid((4, 4)), _D((4, 4)), ab.F32, ab.BF16)  # no BF16 weights
    assert ei.value.status == 1


def test_null_and_aliased_buffers():
    t = torch()
    h = ab.adlbr_build_stencils(ab.grid((4, 4)), _D((4, 4)), ab.F32, ab.F32)
    try:
        u = t.rand(16, device="cuda")
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_apply(h, u, u, ab.F32)                  # Au must not alias u
        assert ei.value.status == 1
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_explicit(h, u, None, ab.F32, 0.1, 1)
        assert ei.value.status == 1
        sc = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_explicit(h, u, sc, ab.F32, -1.0, 1)  # negative dt
        assert ei.value.status == 1
        x = u.clone()
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_implicit(h, u, x, 1.0, 0.0, 10)     # rtol must be > 0
        assert ei.value.status == 1
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_implicit(h, u, x, 1.0, 1e-6, 10, precond=7)
        assert ei.value.status == 1
    finally:
        ab.adlbr_stencils_destroy(h)


def test_single_point_grid():
    """One grid point: the stencil exists, no pair stays in the grid (Neumann),
    so A u = 0 and the explicit step leaves u unchanged."""
    t = torch()
    h = ab.adlbr_build_stencils(ab.grid((1, 1)), _D((1, 1)), ab.F32, ab.F32)
    try:
        ab.adlbr_stencils_check(h)
        u = t.tensor([0.75], device="cuda")
        Au = t.empty_like(u)
        ab.adlbr_apply(h, u, Au, ab.F32)
        sc = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, sc, ab.F32, 0.5, 3)
        t.cuda.synchronize()
        assert Au.item() == 0.0 and u.item() == 0.75
    finally:
        ab.adlbr_stencils_destroy(h)


def test_stencils_grid_round_trip():
    """adlbr_stencils_grid returns the grid the handle was built on."""
    t = torch()
    for shape, bc in (((12, 20), ab.NEUMANN), ((6, 8, 10), ab.PERIODIC)):
        # D = identity: planes (Dxx, Dxy, Dyy) or (Dxx, Dyy, Dzz, Dxy, Dxz, Dyz)
        diag = [1.0, 0.0, 1.0] if len(shape) == 2 else [1.0, 1.0, 1.0, 0.0, 0.0, 0.0]
        D = np.array(diag).reshape(-1, 1) * np.ones((1, int(np.prod(shape))))
        h = ab.adlbr_build_stencils(ab.grid(shape, bc), dev(D, t.float64), ab.F64, ab.F32)
        try:
            g = ab.adlbr_stencils_grid(h)
            assert g.dim == len(shape) and g.bc == bc
            assert tuple(int(g.n[k]) for k in range(len(shape))) == tuple(reversed(shape))
        finally:
            ab.adlbr_stencils_destroy(h)
