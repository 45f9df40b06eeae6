"""Pins for the oracle's operator A = (1/2) grad E_h (Eq. def:E*, h = 1), its
explicit step and its CG solver."""
import numpy as np
import pytest

import oracle
import synth


def _field2d(shape, seed, kmax=20.0):
    ny, nx = shape
    D = synth.smooth_field2d(ny, nx, seed, 1.0, kmax, lattice=4)
    offs, w, st, _ = oracle.build2d(*D)
    assert np.all(st == 0)
    return offs, w


def _field3d(n, seed):
    D = synth.needle_field3d(n, seed, kappa=6.0, lattice=3)
    offs, w, st, _ = oracle.build3d(D)
    assert np.all(st == 0)
    return offs, w


def _dense(shape, bc, offs, w):
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        A[:, j] = oracle.apply(shape, bc, offs, w, e.reshape(shape)).ravel()
    return A


@pytest.mark.parametrize("bc", [oracle.NEUMANN, oracle.PERIODIC])
def test_apply_is_half_gradient_of_energy_2d(bc):
    """Rebuild the quadratic form E_h(u) = u^T Q u by polarisation from the
    energy alone and check that the oracle's A equals Q."""
    shape = (7, 9)
    offs, w = _field2d(shape, 1)
    N = int(np.prod(shape))
    A = _dense(shape, bc, offs, w)
    E = lambda v: oracle.energy(shape, bc, offs, w, v.reshape(shape))
    g = np.random.default_rng(0)
    for _ in range(40):
        i, j = g.integers(0, N, 2)
        ei = np.zeros(N)
        ei[i] = 1
        ej = np.zeros(N)
        ej[j] = 1
        q = 0.5 * (E(ei + ej) - E(ei) - E(ej)) if i != j else E(ei)
        assert abs(A[i, j] - q) <= 1e-12 * max(1.0, abs(q))
    # and the gradient identity on random vectors: E(u) = u^T A u
    for _ in range(5):
        u = g.normal(size=N)
        assert abs(E(u) - u @ A @ u) <= 1e-10 * abs(E(u))


@pytest.mark.parametrize("bc", [oracle.NEUMANN, oracle.PERIODIC])
def test_matrix_properties_2d_3d(bc):
    """Sec. 1 'Non-negativity': A symmetric, off-diagonal <= 0, diagonal > 0,
    A 1 = 0 (so mass sum(A u) = 0)."""
    for shape, (offs, w) in [((8, 8), _field2d((8, 8), 2, 50.0)), ((5, 5, 5), _field3d(5, 3))]:
        A = _dense(shape, bc, offs, w)
        assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
        off = A - np.diag(np.diag(A))
        assert off.max() <= 0.0
        assert np.diag(A).min() > 0
        assert np.abs(A.sum(axis=1)).max() <= 1e-13 * np.abs(A).max()
        d = oracle.diag(shape, bc, offs, w).ravel()
        assert np.allclose(d, np.diag(A), rtol=1e-14, atol=0)


def test_periodic_fourier_modes_constant_D():
    """Constant D on a periodic grid: exp(i xi.z), xi = 2 pi k / n, is an exact
    eigenvector with eigenvalue sum_{e in V} 2 gamma(e) (1 - cos xi.e)."""
    n = 12
    D = synth.D_from_angle(np.pi / 6, np.sqrt(10.0))
    offs1, w1, _, _ = oracle.build2d(*D)
    offs = np.broadcast_to(offs1, (n * n, 3, 2)).copy()
    w = np.broadcast_to(w1, (n * n, 3)).copy()
    y, x = np.mgrid[0:n, 0:n]
    for k in [(0, 1), (1, 2), (3, 5), (6, 6)]:
        xi = 2 * np.pi * np.array(k) / n
        for f in (np.cos, np.sin):
            u = f(xi[0] * x + xi[1] * y)
            lam = sum(4 * g * (1 - np.cos(xi @ o)) for o, g in zip(offs1[0], w1[0]))
            Au = oracle.apply((n, n), oracle.PERIODIC, offs, w, u)
            assert np.abs(Au - lam * u).max() <= 1e-12


def test_explicit_step_max_principle_and_mass():
    """Non-negative scheme => discrete maximum principle for dt <= 1/max A_zz
    (Sec. 4.1); Neumann => sum of u conserved."""
    shape = (24, 24)
    offs, w = _field2d(shape, 4, 100.0)
    u0 = synth.u_uniform(shape, 0)
    dt = oracle.dt_limit(shape, oracle.NEUMANN, offs, w)
    u = oracle.step_explicit(shape, oracle.NEUMANN, offs, w, u0, dt, nsteps=10)
    assert u.min() >= u0.min() - 1e-14 and u.max() <= u0.max() + 1e-14
    assert abs(u.sum() - u0.sum()) <= 1e-11 * u0.size
    # and the range strictly contracts
    assert u.max() - u.min() < u0.max() - u0.min()


def test_cg_matches_dense_solve():
    shape = (10, 12)
    offs, w = _field2d(shape, 6, 30.0)
    b = synth.u_uniform(shape, 1)
    dt = 200.0 * oracle.dt_limit(shape, oracle.NEUMANN, offs, w)
    A = _dense(shape, oracle.NEUMANN, offs, w)
    xref = np.linalg.solve(np.eye(A.shape[0]) + dt * A, b.ravel())
    x, it, res = oracle.cg(shape, oracle.NEUMANN, offs, w, b, b, dt, rtol=1e-12)
    assert res <= 1e-11
    assert np.abs(x.ravel() - xref).max() <= 1e-9 * np.abs(xref).max()
    # flexible PCG with the identity preconditioner is CG
    x2, it2, res2 = oracle.fcg(shape, oracle.NEUMANN, offs, w, b, b, dt, lambda r: r, rtol=1e-12)
    assert abs(it2 - it) <= 1 and np.abs(x2 - x).max() <= 1e-9
