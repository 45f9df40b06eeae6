"""The spectral study (Sec. 4, Fig. Eigen) on the GPU operator: LOBPCG's
smallest eigenvalues against the closed-form symbol of the periodic scheme
(constant D of the paper's figure) and against the oracle's dense
eigensolve (variable D)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import spectral as osp
from paper_1301_3925_gb300 import adlbr as ab
from paper_1301_3925_gb300 import spectral

from gpu_helpers import build, export, torch

pytestmark = pytest.mark.gpu

D_FIG = np.array([[19 / 2, 6.0], [6.0, 4.0]])


def _constant(shape, D):
    planes = np.array([D[0, 0], D[0, 1], D[1, 1]]).reshape(3, 1, 1)
    return np.broadcast_to(planes, (3,) + shape).copy()


@pytest.mark.parametrize("shape,precondition", [((64, 64), True), ((48, 80), True), ((24, 24), False)])
def test_lobpcg_matches_symbol(shape, precondition):
    t = torch()
    h, _, _ = build(_constant(shape, D_FIG), shape, t.float64, ab.F64, ab.PERIODIC)
    try:
        oo, ow = export(h, shape, ab.F64)
        k = 7
        theta, X, its = spectral.lobpcg_smallest(h, shape[0] * shape[1], k, precondition=precondition,
                                                 tol=1e-10, maxit=400)
        # the Ritz vectors are orthonormal and satisfy A x = theta x
        G = (X @ X.T).cpu().numpy()
        assert np.abs(G - np.eye(k)).max() <= 1e-10
    finally:
        ab.adlbr_stencils_destroy(h)
    sym = osp.periodic_symbol(oo[0], ow[0], shape)[:k]
    assert np.abs(theta - sym).max() <= 1e-8 * sym[-1], (theta, sym)
    n2 = shape[0] * shape[1]
    assert its < 400


def test_lobpcg_matches_dense_variable_field():
    t = torch()
    shape = (12, 14)
    D = synth.smooth_field2d(*shape, seed=5, kappa_min=1, kappa_max=30, lattice=4)
    h, seen, _ = build(D, shape, t.float64, ab.F64, ab.PERIODIC)
    try:
        oo, ow = export(h, shape, ab.F64)
        theta, _, _ = spectral.lobpcg_smallest(h, shape[0] * shape[1], 6, tol=1e-10)
    finally:
        ab.adlbr_stencils_destroy(h)
    # the oracle's own stencils of the same D (bit-exact offsets, FP64 weights)
    offs, w, st, _ = oracle.build2d(*seen)
    assert (st == 0).all() and np.array_equal(offs, oo)
    dense = osp.dense_smallest(shape, oracle.PERIODIC, offs, w, 6)
    assert np.abs(theta - dense).max() <= 1e-8 * max(dense[-1], 1.0), (theta, dense)


def test_scheme_eigenvalues_converge_on_gpu():
    """n^2 lambda of the GPU operator approaches 4 pi^2 <m, D m> as n grows."""
    t = torch()
    cont = osp.continuous_smallest(D_FIG, 7)
    errs = []
    for n in (32, 64):
        shape = (n, n)
        h, _, _ = build(_constant(shape, D_FIG), shape, t.float64, ab.F64, ab.PERIODIC)
        try:
            theta, _, _ = spectral.lobpcg_smallest(h, n * n, 7, tol=1e-10)
        finally:
            ab.adlbr_stencils_destroy(h)
        errs.append(np.abs(theta * n * n - cont)[1:].max() / cont[1:].max())
    assert errs[1] < errs[0] / 3 and errs[1] < 5e-3, errs


@pytest.mark.parametrize("ma,mb,n", [(5, 7, 1037), (21, 21, 256), (64, 3, 5000), (1, 1, 1)])
def test_block_kernels_match_their_definitions(ma, mb, n):
    """The eigensolver's block kernels against their plain definitions in
    FP64 (numpy): G = A B^T, C^T S, and R = AX - theta X with its row norms,
    on ragged lengths and the largest block (64 rows); twice, to check that
    the fixed-order sums give the same bits."""
    t = torch()
    rng = np.random.default_rng(ma * 1000 + n)
    A = rng.standard_normal((ma, n))
    B = rng.standard_normal((mb, n))
    C = rng.standard_normal((ma, mb))
    th = rng.standard_normal(ma)
    Ad, Bd = t.from_numpy(A).cuda(), t.from_numpy(B).cuda()
    G = t.empty((ma, mb), dtype=t.float64, device="cuda")
    ab.adlbr_block_dot(Ad, Bd, G)
    G1 = G.cpu().numpy()
    ab.adlbr_block_dot(Ad, Bd, G)
    assert np.array_equal(G.cpu().numpy(), G1)
    ref = A @ B.T
    assert np.abs(G1 - ref).max() <= 1e-13 * max(1.0, np.abs(A).max() * np.abs(B).max() * n)
    out = t.empty((mb, n), dtype=t.float64, device="cuda")
    ab.adlbr_block_combine(t.from_numpy(C).cuda(), Ad, out)
    assert np.abs(out.cpu().numpy() - C.T @ A).max() <= 1e-13 * ma * np.abs(C).max() * np.abs(A).max()
    AX = Bd[:1].repeat(ma, 1)
    AXn = AX.cpu().numpy()
    R = t.empty_like(Ad)
    rn = t.empty(ma, dtype=t.float64, device="cuda")
    ab.adlbr_block_residual(AX, Ad, t.from_numpy(th).cuda(), R, rn)
    Rref = AXn - th[:, None] * A
    scale = (np.abs(AXn) + np.abs(th[:, None] * A)).max()
    assert np.abs(R.cpu().numpy() - Rref).max() <= 4e-16 * scale
    assert np.allclose(rn.cpu().numpy(), np.linalg.norm(Rref, axis=1), rtol=1e-13, atol=0)
    # in place: R = AX
    ab.adlbr_block_residual(AX, Ad, t.from_numpy(th).cuda(), AX, rn)
    assert np.array_equal(AX.cpu().numpy(), R.cpu().numpy())


def test_block_kernels_refuse_bad_shapes():
    t = torch()
    A = t.zeros((65, 8), dtype=t.float64, device="cuda")
    G = t.empty((65, 65), dtype=t.float64, device="cuda")
    with pytest.raises(ab.AdlbrError) as ei:
        ab.adlbr_block_dot(A, A, G)
    assert ei.value.status == 1
    C = t.zeros((65, 2), dtype=t.float64, device="cuda")
    out = t.empty((2, 8), dtype=t.float64, device="cuda")
    with pytest.raises(ab.AdlbrError):
        ab.adlbr_block_combine(C, A, out)
