"""The A-NN comparison scheme (Sec. 4.1, Remark rem:WG) on the GPU against its
oracle (oracle/ann.py): stencils bit-exact, the operator, the explicit and
implicit steps on A-NN handles, and the periodic spectrum of Fig. Eigen."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ann, spectral
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import dev, torch, weight_tol

pytestmark = pytest.mark.gpu


def _build(D, shape, D_dtype, w_t, bc=ab.NEUMANN):
    t = torch()
    Dd = dev(D.reshape(3, -1), D_dtype)
    h = ab.adlbr_build_stencils_scheme(ab.grid(shape, bc), Dd, ab.dtype_code(D_dtype), w_t, ab.SCHEME_ANN)
    return h, Dd.double().cpu().numpy()


def _export(h, N, w_t):
    t = torch()
    offs = t.zeros((N, 3, 2), dtype=t.int16, device="cuda")
    w = t.zeros((N, 3), dtype=t.float64 if w_t == ab.F64 else t.float32, device="cuda")
    ab.adlbr_stencils_export(h, offs, w)
    t.cuda.synchronize()
    return offs.cpu().numpy().astype(np.int32), w.double().cpu().numpy()


def _tensors():
    D = synth.random_spd2(3000, 21, 20.0)
    special = np.array([[9.5, 6.0, 4.0], [2.0, 0.0, 0.5], [1.0, 0.98, 0.97], [1.0, -0.98, 0.97],
                        [1.0, 1 - 2e-3, 1 - 3e-3], [3.0, -1.0, 3.0]]).T
    return np.concatenate([D, special], axis=1)


@pytest.mark.parametrize("D_name,w_t", [("float64", ab.F64), ("float64", ab.F32), ("float32", ab.F16)])
def test_ann_stencils_match_oracle(D_name, w_t):
    t = torch()
    D = _tensors()
    N = D.shape[1]
    h, seen = _build(D.reshape(3, 1, N), (1, N), getattr(t, D_name), w_t)
    try:
        ab.adlbr_stencils_check(h)
        assert ab.adlbr_stencils_scheme(h) == ab.SCHEME_ANN
        go, gw = _export(h, N, w_t)
    finally:
        ab.adlbr_stencils_destroy(h)
    oo, ow = ann.build2d_ann(*seen)
    assert np.array_equal(go, oo), np.argwhere(np.any(go != oo, axis=(1, 2)))[:5]
    assert np.all(np.abs(gw - ow) <= weight_tol(ow, w_t, np.abs(seen).max()))


@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
def test_ann_apply_and_steps(bc):
    """A u (scatter operator, long A-NN offsets through L2) against the
    oracle's operator on the A-NN stencils; explicit steps keep the maximum
    principle; the implicit step by CG and Jacobi-PCG converges."""
    t = torch()
    shape = (72, 90)
    D = synth.smooth_field2d(*shape, seed=5, kappa_min=1, kappa_max=12, lattice=6)
    h, seen = _build(D, shape, t.float64, ab.F64, bc)
    try:
        oo, ow = _export(h, shape[0] * shape[1], ab.F64)
        u0 = synth.u_uniform(shape, 4)
        u = dev(u0.ravel(), t.float64)
        Au = t.empty_like(u)
        ab.adlbr_apply(h, u, Au, ab.F64)
        t.cuda.synchronize()
        ref = oracle.apply(shape, bc, oo, ow, u0).ravel()
        assert np.abs(Au.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
        dt = 1.0 / ab.adlbr_stencils_max_diag(h)
        assert abs(dt - oracle.dt_limit(shape, bc, oo, ow)) <= 1e-5 * dt
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F64), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.F64, dt, 5)
        t.cuda.synchronize()
        ug = u.cpu().numpy()
        assert ug.min() >= u0.min() - 1e-12 and ug.max() <= u0.max() + 1e-12
        assert np.abs(ug - oracle.step_explicit(shape, bc, oo, ow, u0, dt, 5).ravel()).max() <= 1e-12
    finally:
        ab.adlbr_stencils_destroy(h)
    h, _ = _build(D, shape, t.float32, ab.F32, bc)
    try:
        dt = 50.0 / ab.adlbr_stencils_max_diag(h)
        b = dev(u0.ravel(), t.float32)
        for pc in (0, 2):
            x = b.clone()
            it, rel = ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 3000, precond=pc)
            assert rel <= 2e-5, (pc, it, rel)
        # the gather form is AD-LBR-only: on an A-NN handle the scatter form runs
        ab.adlbr_stencils_set_operator(h, ab.OP_GATHER)
        ab.adlbr_apply(h, b, t.empty_like(b), ab.F32)
        assert ab.adlbr_stencils_get_operator(h)[1] == 0
    finally:
        ab.adlbr_stencils_destroy(h)


def test_ann_periodic_spectrum_fig_eigen():
    """Fig. Eigen on the GPU: the A-NN operator of D = [[19/2, 6], [6, 4]] on
    periodic n x n grids, assembled column by column through adlbr_apply
    (FP64), has the spectrum of the oracle's closed-form symbol of the A-NN
    stencil, which oscillates with n (a zero second eigenvalue on even n)."""
    t = torch()
    oa, wa = ann.build2d_ann([9.5], [6.0], [4.0])
    for n in (7, 8):
        N = n * n
        planes = t.tensor([9.5, 6.0, 4.0], dtype=t.float64, device="cuda")[:, None].expand(3, N).contiguous()
        h = ab.adlbr_build_stencils_scheme(ab.grid((n, n), ab.PERIODIC), planes, ab.F64, ab.F64, ab.SCHEME_ANN)
        try:
            A = np.zeros((N, N))
            e = t.zeros(N, dtype=t.float64, device="cuda")
            col = t.empty_like(e)
            for j in range(N):
                e.zero_()
                e[j] = 1.0
                ab.adlbr_apply(h, e, col, ab.F64)
                A[:, j] = col.cpu().numpy()
        finally:
            ab.adlbr_stencils_destroy(h)
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        lam = np.linalg.eigvalsh(A)
        sym = spectral.periodic_symbol(oa[0], wa[0], (n, n))
        assert np.abs(lam - sym).max() <= 1e-12 * sym.max()
        assert (abs(lam[1]) < 1e-12) == (n % 2 == 0)
