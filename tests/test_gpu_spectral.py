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
