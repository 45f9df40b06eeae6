"""Spectrum of the AD-LBR operator on periodic grids (Sec. 4, Fig. Eigen):
the reference values for the spectral study.  Test infrastructure only (see
the package header of oracle/).

Three independent routes to the smallest eigenvalues of A = 1/2 grad E_h
(h = 1, pixel units):

* periodic_symbol: for a constant stencil on a periodic n_y x n_x grid the
  Fourier modes exp(i xi . z), xi = 2 pi (k_x / n_x, k_y / n_y), are
  eigenvectors, with eigenvalue sum over V (both signs of every stored offset)
  of 2 gamma(e) (1 - cos xi . e) = 4 sum_i gamma_i (1 - cos xi . e_i);
* dense_smallest: the operator assembled column by column from the oracle's
  apply and handed to a dense symmetric eigensolver;
* continuous_smallest: the eigenvalues 4 pi^2 <k, D k>, k in Z^2, of
  -div(D grad) on the periodic unit square, which the scheme approaches as
  n^2 lambda (h = 1/n) for n -> infinity (the consistency the figure shows).
"""
import numpy as np

import oracle


def periodic_symbol(offs1, w1, shape):
    """All eigenvalues, ascending, of the constant-stencil periodic operator.
    offs1: (3, 2) half-stencil offsets (x, y); w1: (3,) weights; shape (ny, nx)."""
    ny, nx = shape
    ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xi_x = 2 * np.pi * kx / nx
    xi_y = 2 * np.pi * ky / ny
    lam = np.zeros(shape)
    for e, g in zip(np.asarray(offs1, dtype=np.float64), np.asarray(w1, dtype=np.float64)):
        lam += 4 * g * (1 - np.cos(xi_x * e[0] + xi_y * e[1]))
    return np.sort(lam.ravel())


def dense_matrix(shape, bc, offs, w):
    """The operator as a dense N x N matrix (column j = A applied to unit vector j)."""
    N = int(np.prod(shape))
    A = np.zeros((N, N))
    for j in range(N):
        u = np.zeros(N)
        u[j] = 1.0
        A[:, j] = oracle.apply(shape, bc, offs, w, u.reshape(shape)).ravel()
    return A


def dense_smallest(shape, bc, offs, w, k):
    """The k smallest eigenvalues of the assembled operator (symmetric)."""
    A = dense_matrix(shape, bc, offs, w)
    return np.linalg.eigvalsh(0.5 * (A + A.T))[:k]


def continuous_smallest(D, k, kmax=8):
    """The k smallest values of 4 pi^2 <m, D m> over m in Z^2, |m_i| <= kmax
    (D = [[Dxx, Dxy], [Dxy, Dyy]] acting on m = (m_x, m_y))."""
    D = np.asarray(D, dtype=np.float64)
    r = np.arange(-kmax, kmax + 1)
    mx, my = np.meshgrid(r, r, indexing="ij")
    q = D[0, 0] * mx ** 2 + 2 * D[0, 1] * mx * my + D[1, 1] * my ** 2
    return np.sort(4 * np.pi ** 2 * q.ravel())[:k]
