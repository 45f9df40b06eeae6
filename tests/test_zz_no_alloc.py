"""The allocation-free explicit step (adlbr_step_explicit_noalloc).

Some callers cannot allocate device memory while they step (a host
framework that owns the whole memory pool, a real-time loop that must not
call an allocator that can block, a plugin that may not allocate).  For them
the library offers the explicit step with its scratch in a fixed array inside
the library.  This test calls it through the C ABI and checks it against the
ordinary entry point (caller-provided scratch) on two calls in a row -- the
second call must not see anything the first left in the shared array -- and
that a grid above the array's limit is refused.  This file is collected last
on purpose.
"""
import numpy as np
import pytest

import synth
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("u_name,w_t,dim", [("float32", ab.F32, 2), ("float64", ab.F64, 2),
                                             ("bfloat16", ab.F16, 2), ("float32", ab.F16, 3)])
def test_noalloc_step_matches_step_explicit(u_name, w_t, dim):
    t = torch()
    if dim == 2:
        shape = (181, 233)
        D = synth.smooth_field2d(*shape, seed=11, kappa_min=1, kappa_max=60, lattice=8)
    else:
        shape = (21, 26, 31)
        D = synth.needle_field3d(31, seed=4, kappa=15.0)[:, :21, :26, :31]
    ud = getattr(t, u_name)
    h, seen, _ = build(D, shape, t.float64 if ud == t.float64 else t.float32, w_t)
    try:
        ab.adlbr_stencils_check(h)
        code = ab.dtype_code(ud)
        dt = 0.05
        u0 = dev(synth.u_uniform(shape, 12).ravel(), ud)
        # reference: the ordinary entry point with caller-owned scratch
        ref = u0.clone()
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, code), dtype=t.uint8, device="cuda")
        # the fixed array is shared by every call and keeps old contents:
        # two calls in a row must each match the reference
        got = u0.clone()
        ab.adlbr_step_explicit_noalloc(h, got, code, dt, 0)   # set-up call: no step
        t.cuda.synchronize()
        assert t.equal(got, u0)
        for nsteps in (3, 2):
            ab.adlbr_step_explicit(h, ref, scratch, code, dt, nsteps)
            t.cuda.synchronize()
            # the call itself allocates nothing: device memory in use and the
            # torch allocator's statistics are the same before and after
            free0, _ = t.cuda.mem_get_info()
            alloc0 = t.cuda.memory_allocated()
            ab.adlbr_step_explicit_noalloc(h, got, code, dt, nsteps)
            t.cuda.synchronize()
            assert t.cuda.mem_get_info()[0] == free0
            assert t.cuda.memory_allocated() == alloc0
            r = ref.double().cpu().numpy()
            g = got.double().cpu().numpy()
            # same kernels; only the order of the FP atomic additions differs
            # (BF16: each step rounds u once, so a last-bit difference of an
            # intermediate step can move the result by one BF16 ulp)
            tol = {t.float32: 1e-6, t.float64: 1e-13, t.bfloat16: 2 ** -7}[ud]
            assert np.abs(g - r).max() <= tol * np.abs(r).max()
    finally:
        ab.adlbr_stencils_destroy(h)


def test_noalloc_step_refuses_grids_above_limit():
    t = torch()
    shape = (2049, 2049)   # 4,198,401 points > 4,194,304
    D = np.zeros((3,) + shape)
    D[0] = 1.0
    D[2] = 1.0
    h, _, _ = build(D, shape, t.float32, ab.F32)
    try:
        u = t.zeros(shape[0] * shape[1], dtype=t.float32, device="cuda")
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_explicit_noalloc(h, u, ab.F32, 0.1, 1)
        assert ei.value.status == 2
    finally:
        ab.adlbr_stencils_destroy(h)
