"""Pins of the spectral reference values (Sec. 4, Fig. Eigen): the closed-form
symbol of the periodic constant-coefficient scheme against a dense
eigensolve of the oracle's assembled operator, the continuous eigenvalues
4 pi^2 <m, D m> against values worked out by hand, and the convergence of
n^2 lambda towards them."""
import numpy as np
import pytest

import oracle
from oracle import spectral as osp

# The tensor of the paper's spectral figure.
D_FIG = np.array([[19 / 2, 6.0], [6.0, 4.0]])


def _stencil(D):
    offs, w, st, _ = oracle.build2d(np.array([D[0, 0]]), np.array([D[0, 1]]), np.array([D[1, 1]]))
    assert st[0] == 0
    return offs[0], w[0]


@pytest.mark.parametrize("shape", [(4, 4), (5, 5), (8, 8), (12, 12), (6, 10)])
def test_symbol_equals_dense_spectrum(shape):
    offs1, w1 = _stencil(D_FIG)
    N = shape[0] * shape[1]
    offs = np.broadcast_to(offs1, (N, 3, 2)).copy()
    w = np.broadcast_to(w1, (N, 3)).copy()
    dense = osp.dense_smallest(shape, oracle.PERIODIC, offs, w, N)
    sym = osp.periodic_symbol(offs1, w1, shape)
    assert np.abs(dense - sym).max() <= 1e-11 * sym.max()


def test_continuous_values_by_hand():
    # <m, D m> = 19/2 m_x^2 + 12 m_x m_y + 4 m_y^2: 0 at m = 0; 3/2 at
    # +-(1, -1) and +-(1, -2); 2 at +-(2, -3); 4 at +-(0, 1)
    want = 4 * np.pi ** 2 * np.array([0, 1.5, 1.5, 1.5, 1.5, 2, 2, 4, 4])
    assert np.allclose(osp.continuous_smallest(D_FIG, 9), want, rtol=1e-14, atol=1e-12)


def test_scheme_eigenvalues_approach_the_continuous_ones():
    """n^2 lambda_j(n) -> 4 pi^2 <m_j, D m_j> with error O(n^-2) (the scheme is
    consistent of order 2 on smooth modes: 1 - cos x = x^2/2 - x^4/24 + ...)."""
    offs1, w1 = _stencil(D_FIG)
    cont = osp.continuous_smallest(D_FIG, 9)
    errs = []
    for n in (12, 24, 48, 96):
        lam = osp.periodic_symbol(offs1, w1, (n, n))[:9] * n * n
        errs.append(np.abs(lam - cont)[1:].max() / cont[1:].max())
    assert errs[-1] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0, errs


def test_dense_smallest_variable_field_is_psd_with_constant_kernel():
    """Variable D on a periodic grid: A is symmetric positive semi-definite
    with the constants as its kernel (zero row sums, non-negative weights)."""
    import synth
    shape = (10, 12)
    D = synth.smooth_field2d(*shape, seed=4, kappa_min=1, kappa_max=20, lattice=4)
    offs, w, st, _ = oracle.build2d(*D)
    assert (st == 0).all()
    lam = osp.dense_smallest(shape, oracle.PERIODIC, offs, w, 4)
    assert abs(lam[0]) <= 1e-12 and lam[1] > 1e-6
