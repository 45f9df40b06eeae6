"""Parity of the CUDA implicit step (CG on (I + dt A) x = b) with the oracle."""
import numpy as np
import pytest

import oracle
import synth
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, dev, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
def test_cg_matches_oracle(bc):
    t = torch()
    shape = (96, 112)
    D = synth.smooth_field2d(*shape, seed=3, kappa_min=1, kappa_max=50, lattice=8)
    h, seen, _ = build(D, shape, t.float32, ab.F32, bc)
    oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
    dt = 200.0 * oracle.dt_limit(shape, bc, oo, ow)
    b = synth.u_uniform(shape, 3)
    try:
        bd = dev(b.ravel(), t.float32)
        x = bd.clone()
        it, rel = ab.adlbr_step_implicit(h, bd, x, dt, 1e-6, 2000)
        xg = x.double().cpu().numpy().reshape(shape)
        bs = bd.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    # true residual of the FP32 solution, by the oracle in FP64: x stored in
    # FP32 bounds it near eps32 |I + dt A| (|I + dt A| ~ 400 here, so a few
    # 1e-6 -- the recursive residual is the stop test, 1e-6)
    res = bs - (xg + dt * oracle.apply(shape, bc, oo, ow, xg))
    true_rel = np.linalg.norm(res) / np.linalg.norm(bs)
    assert true_rel <= 1e-5, true_rel
    assert abs(rel - true_rel) <= 0.05 * true_rel + 1e-9   # the library reports it
    xo, ito, relo = oracle.cg(shape, bc, oo, ow, bs, bs, dt, rtol=1e-10)
    assert np.abs(xg - xo).max() <= 1e-4 * np.abs(xo).max()
    # same Krylov method: the first CG round takes about the iterations of FP64
    # CG at 1e-6; a refinement round from the true residual may add a few
    _, ito6, _ = oracle.cg(shape, bc, oo, ow, bs, bs, dt, rtol=1e-6)
    assert ito6 - 3 <= it <= ito6 + max(10, 0.15 * ito6), (it, ito6)


def test_cg_iteration_limit_reports_not_converged():
    t = torch()
    shape = (64, 64)
    D = synth.smooth_field2d(*shape, seed=4, kappa_min=1, kappa_max=50, lattice=8)
    h, seen, _ = build(D, shape, t.float32, ab.F32)
    try:
        b = dev(synth.u_uniform(shape, 5).ravel(), t.float32)
        x = b.clone()
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_implicit(h, b, x, 500.0, 1e-8, 3)
        assert ei.value.status == 5
    finally:
        ab.adlbr_stencils_destroy(h)


def test_cg_full_size_2048():
    """The benchmark's implicit step: 2048^2, kappa <= 50, dt = 200 / max A_zz,
    tolerance 1e-6.  The true residual of the returned x is recomputed by the
    oracle in FP64 with the library's own stencils (exported)."""
    from gpu_helpers import export
    t = torch()
    n = 2048
    D = synth.smooth_field2d_torch(n, n, 3, 1.0, 50.0, 16).reshape(3, -1).contiguous()
    g = ab.grid((n, n))
    h = ab.adlbr_build_stencils(g, D, ab.F32, ab.F32)
    try:
        dt = 200.0 / ab.adlbr_stencils_max_diag(h)
        b = dev(synth.u_uniform((n, n), 3).ravel(), t.float32)
        x = b.clone()
        it, rel = ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 4000)
        oo, ow = export(h, (n, n), ab.F32)
        xs = x.double().cpu().numpy().reshape(n, n)
        bs = b.double().cpu().numpy().reshape(n, n)
    finally:
        ab.adlbr_stencils_destroy(h)
    res = bs - (xs + dt * oracle.apply((n, n), oracle.NEUMANN, oo, ow, xs))
    true_rel = np.linalg.norm(res) / np.linalg.norm(bs)
    assert true_rel <= 1e-5, true_rel
    assert abs(rel - true_rel) <= 0.05 * true_rel + 1e-9
    assert 50 <= it <= 400, it


def test_restoration_against_exact_solution():
    """The analytic restoration problem (Sec. 5) solved through the library:
    F32 tensor, F32 weights, CG to 1e-6 at lambda N^2.  At N = 200 the errors
    to the exact solution equal the oracle's (same scheme); they fall with N
    (first order) up to N = 800."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_restoration import LAM, errors, exact
    t = torch()
    kappa = 10.0
    errs = {}
    for N in (200, 400, 800):
        D, v, Yf = synth.restoration_problem(N, kappa)
        h, seen, _ = build(D, (N, N), t.float32, ab.F32)
        try:
            vd = dev(v.ravel(), t.float32)
            x = vd.clone()
            ab.adlbr_step_implicit(h, vd, x, LAM * N * N, 1e-6, 5000)
            xs = x.double().cpu().numpy().reshape(N, N)
        finally:
            ab.adlbr_stencils_destroy(h)
        errs[N] = errors(xs, exact(Yf, kappa), N)
        if N == 200:
            oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
            xo, _, _ = oracle.cg((N, N), oracle.NEUMANN, oo, ow, v, v, LAM * N * N, rtol=1e-9)
            eo = errors(xo, exact(Yf, kappa), N)
            assert np.allclose(errs[N], eo, rtol=1e-2), (errs[N], eo)
    # L2 falls at first order or faster; the H1 error sits in the transition
    # layer of width sqrt(lambda)/kappa ~ 0.003, resolved only from N ~ 800,
    # and falls more slowly there (pre-asymptotic)
    for a, b in ((200, 400), (400, 800)):
        assert errs[a][0] / errs[b][0] >= 1.6 and errs[a][1] / errs[b][1] >= 1.3, errs


def test_cg_non_finite_rhs_is_an_error():
    """A NaN in the right-hand side makes the residual non-finite: the solve
    stops and reports ADLBR_E_NONFINITE instead of a converged result."""
    t = torch()
    shape = (64, 64)
    D = synth.smooth_field2d(*shape, seed=4, kappa_min=1, kappa_max=20, lattice=8)
    h, seen, _ = build(D, shape, t.float32, ab.F32)
    try:
        bn = synth.u_uniform(shape, 5).ravel()
        bn[100] = np.nan
        b = dev(bn, t.float32)
        x = b.clone()
        with pytest.raises(ab.AdlbrError) as ei:
            ab.adlbr_step_implicit(h, b, x, 50.0, 1e-6, 500)
        assert ei.value.status == 4
    finally:
        ab.adlbr_stencils_destroy(h)


@pytest.mark.parametrize("shape", [(96, 112), (12, 14, 16)])
def test_jacobi_pcg_matches_cg_with_fewer_iterations(shape):
    """precond = 2: CG preconditioned by 1 + dt A_zz reaches the same solution
    as plain CG (same true-residual test), in fewer iterations on an
    anisotropic field with varying kappa."""
    t = torch()
    if len(shape) == 2:
        D = synth.smooth_field2d(*shape, seed=4, kappa_min=1, kappa_max=50, lattice=6)
    else:
        D = synth.needle_field3d(max(shape), seed=2, kappa=12.0)[:, :shape[0], :shape[1], :shape[2]]
    h, _, _ = build(D, shape, t.float32, ab.F32)
    try:
        dt = 200.0 / ab.adlbr_stencils_max_diag(h)
        b = dev(synth.u_uniform(shape, 7).ravel(), t.float32)
        x1 = b.clone()
        it_cg, rel_cg = ab.adlbr_step_implicit(h, b, x1, dt, 1e-6, 4000)
        x2 = b.clone()
        it_j, rel_j = ab.adlbr_step_implicit(h, b, x2, dt, 1e-6, 4000, precond=2)
        d = ((x1 - x2).abs().max() / x1.abs().max()).item()
    finally:
        ab.adlbr_stencils_destroy(h)
    assert rel_j <= 2e-5 and rel_cg <= 2e-5, (rel_j, rel_cg)
    assert d <= 5e-5, d
    assert it_j < it_cg, (it_j, it_cg)


def test_residual_met_flag():
    """adlbr_last_residual_met: 1 when the true residual of the returned x is
    at or below rtol; 0 when rtol lies below the FP32 floor of x (the solve
    still returns OK once its last refinement round converged)."""
    t = torch()
    shape = (64, 80)
    D = synth.smooth_field2d(*shape, seed=3, kappa_min=1, kappa_max=20, lattice=8)
    h, seen, _ = build(D, shape, t.float32, ab.F32)
    oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
    try:
        bd = dev(synth.u_uniform(shape, 3).ravel(), t.float32)
        dt = 2.0 * oracle.dt_limit(shape, ab.NEUMANN, oo, ow)
        for precond in (0, 2):
            x = bd.clone()
            _, rel = ab.adlbr_step_implicit(h, bd, x, dt, 1e-5, 2000, precond=precond)
            assert rel <= 1e-5 and ab.adlbr_last_residual_met() == 1
            x = bd.clone()
            try:
                _, rel = ab.adlbr_step_implicit(h, bd, x, 200.0 * dt, 1e-9, 4000, precond=precond)
                assert rel > 1e-9, rel
            except ab.AdlbrError as e:   # the recursive residual may not reach 1e-9 either
                assert e.status == 5, e
            assert ab.adlbr_last_residual_met() == 0
    finally:
        ab.adlbr_stencils_destroy(h)
