"""Smallest eigenvalues of the AD-LBR operator by LOBPCG on the library's
operator: the periodic spectral study of Sec. 4 (Fig. Eigen).

A X is adlbr_apply on each block vector (FP64 u; the handle's weights).  The
preconditioner is T = (I + tau A)^-1, one loose solve by the library's CG
(adlbr_step_implicit, FP32) per vector: it keeps the low end of the spectrum
and compresses the high end to about 1 / tau.

Each iteration is the locally optimal block step of Knyazev's LOBPCG: the
Rayleigh-Ritz problem on span[X, T R, P] (R the block residual, P the
previous update).  Every device-side operation is a library kernel: the
block residual and its norms (adlbr_block_residual), the Gram matrices
S S^T and S (A S)^T of the search block S (adlbr_block_dot), and the new
X, A X and P as combinations of its rows (adlbr_block_combine).  The
projected problem (at most 3b x 3b) is solved on the host in FP64, with the
rows of S scaled to unit norm through the Gram diagonal and basis directions
dropped whose Gram eigenvalue is below 1e-13 of the largest.  torch only
holds the device buffers (allocation, concatenation, FP64 <-> FP32 copies
for the FP32 solver).
"""
import numpy as np

from . import adlbr as ab


def _torch():
    import torch
    return torch


def _apply(h, X, AX):
    for j in range(X.shape[0]):
        ab.adlbr_apply(h, X[j], AX[j], ab.F64)


def _precondition(h, R, tau, rtol, maxit):
    """T R row by row: (I + tau A) w = r by the library's FP32 CG (the
    relative stopping test makes the solve independent of the scale of r)."""
    t = _torch()
    out = t.empty_like(R)
    r32 = t.empty(R.shape[1], dtype=t.float32, device=R.device)
    x32 = t.empty_like(r32)
    for j in range(R.shape[0]):
        r32.copy_(R[j])
        x32.copy_(r32)
        ab.adlbr_step_implicit(h, r32, x32, tau, rtol, maxit)
        out[j].copy_(x32)
    return out


def _gram(A, B):
    t = _torch()
    G = t.empty((A.shape[0], B.shape[0]), dtype=t.float64, device=A.device)
    ab.adlbr_block_dot(A, B, G)
    return G.cpu().numpy()


def _combine(C, S):
    """C^T S for a host coefficient matrix C (m x k) and a device block S."""
    t = _torch()
    Cd = t.as_tensor(np.ascontiguousarray(C), dtype=t.float64, device=S.device)
    out = t.empty((C.shape[1], S.shape[1]), dtype=t.float64, device=S.device)
    ab.adlbr_block_combine(Cd, S, out)
    return out


def lobpcg_smallest(h, n_points, k, block=None, tau=None, precondition=True, tol=1e-9, maxit=300,
                    seed=0, pc_rtol=1e-2, pc_maxit=2000):
    """The k smallest eigenvalues of the operator of handle h (n_points grid
    points), ascending, with their vectors.

    block: block size (default k + 3; extra vectors speed up convergence and
    hold eigenvalue clusters); tau: preconditioner shift (default, at every
    iteration, 1 / the largest Ritz value of the block); tol: convergence when every
    wanted residual ||A x - theta x|| <= tol * ||A||, ||A|| bounded by
    2 max_z A_zz (Gershgorin with zero row sums).

    Returns (theta [k], X [k, n_points] on the device, iterations)."""
    t = _torch()
    b = block or k + 3
    if not (1 <= k <= b < n_points) or 3 * b > 64:
        raise ValueError("need 1 <= k <= block < n_points and block <= 21")
    g = t.Generator(device="cuda").manual_seed(seed)
    # a random start block; the first Rayleigh-Ritz step orthonormalises it
    X = t.randn((b, n_points), dtype=t.float64, device="cuda", generator=g)
    AX = t.empty_like(X)
    _apply(h, X, AX)
    anorm = 2.0 * ab.adlbr_stencils_max_diag(h)
    P = AP = None
    theta = None
    R = t.empty_like(X)
    rn = t.empty(b, dtype=t.float64, device="cuda")
    for it in range(1, maxit + 1):
        # Rayleigh-Ritz on span[X, W, P]
        parts, aparts = [X], [AX]
        if theta is not None:
            ab.adlbr_block_residual(AX, X, t.as_tensor(theta, device="cuda"), R, rn)
            if bool((rn[:k] <= tol * anorm).all()):
                return theta[:k], X[:k], it - 1
            # shift 1 / (largest Ritz value of the block), unless given
            sh = tau if tau is not None else 1.0 / max(float(theta[b - 1]), 1e-30)
            W = _precondition(h, R, sh, pc_rtol, pc_maxit) if precondition else R.clone()
            AW = t.empty_like(W)
            _apply(h, W, AW)
            parts.append(W)
            aparts.append(AW)
            if P is not None:
                parts.append(P)
                aparts.append(AP)
        S = t.cat(parts, 0)
        AS = t.cat(aparts, 0)
        G = _gram(S, S)
        H = _gram(S, AS)
        # rows of S scaled to unit norm (a zero row stays out of the basis)
        gd = np.diag(G).copy()
        d = np.where(gd > 0, 1.0 / np.sqrt(np.where(gd > 0, gd, 1.0)), 0.0)
        G = d[:, None] * G * d[None, :]
        H = d[:, None] * H * d[None, :]
        H = 0.5 * (H + H.T)
        gv, gV = np.linalg.eigh(0.5 * (G + G.T))
        keep = gv > 1e-13 * gv[-1]
        T = gV[:, keep] / np.sqrt(gv[keep])
        if T.shape[1] < b:
            raise RuntimeError("LOBPCG: the basis lost rank")
        ev, Y = np.linalg.eigh(T.T @ H @ T)
        C = d[:, None] * (T @ Y[:, :b])   # coefficients on the unscaled rows of S
        Xn = _combine(C, S)
        AXn = _combine(C, AS)
        if len(parts) > 1:
            P = _combine(C[b:], S[b:])
            AP = _combine(C[b:], AS[b:])
        X, AX = Xn, AXn
        theta = ev[:b].copy()
    raise RuntimeError("LOBPCG: no convergence in %d iterations" % maxit)
