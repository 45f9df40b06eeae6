"""Smallest eigenvalues of the AD-LBR operator by LOBPCG on the library's
operator: the periodic spectral study of Sec. 4 (Fig. Eigen).

A X is adlbr_apply on each block vector (FP64 u; the handle's weights).  The
preconditioner is T = (I + tau A)^-1, one loose solve by the library's CG
(adlbr_step_implicit, FP32) per vector: it keeps the low end of the spectrum
and compresses the high end to about 1 / tau.

Each iteration is the locally optimal block step of Knyazev's LOBPCG: the
Rayleigh-Ritz problem on span[X, T R, P] (R the block residual, P the
previous update).  Block inner products are device GEMMs; the projected
problem (at most 3b x 3b) is solved on the host in FP64, after discarding
basis directions whose Gram eigenvalue is below 1e-13 of the largest.
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
    t = _torch()
    out = t.empty_like(R)
    r32 = t.empty(R.shape[1], dtype=t.float32, device=R.device)
    x32 = t.empty_like(r32)
    for j in range(R.shape[0]):
        s = float(R[j].abs().max())
        if s == 0.0:
            out[j].zero_()
            continue
        r32.copy_(R[j] / s)
        x32.copy_(r32)
        ab.adlbr_step_implicit(h, r32, x32, tau, rtol, maxit)
        out[j].copy_(x32.double() * s)
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
    if not (1 <= k <= b < n_points):
        raise ValueError("need 1 <= k <= block < n_points")
    g = t.Generator(device="cuda").manual_seed(seed)
    X = t.randn((b, n_points), dtype=t.float64, device="cuda", generator=g)
    X = t.linalg.qr(X.T)[0].T.contiguous()
    AX = t.empty_like(X)
    _apply(h, X, AX)
    anorm = 2.0 * ab.adlbr_stencils_max_diag(h)
    P = AP = None
    theta = None
    for it in range(1, maxit + 1):
        # Rayleigh-Ritz on span[X, W, P]
        parts, aparts = [X], [AX]
        if theta is not None:
            R = AX - theta[:, None] * X
            rn = t.linalg.vector_norm(R, dim=1)
            if bool((rn[:k] <= tol * anorm).all()):
                return theta[:k].cpu().numpy(), X[:k], it - 1
            # shift 1 / (largest Ritz value of the block), unless given
            sh = tau if tau is not None else 1.0 / max(float(theta[b - 1]), 1e-30)
            W = _precondition(h, R, sh, pc_rtol, pc_maxit) if precondition else R.clone()
            W /= t.linalg.vector_norm(W, dim=1, keepdim=True).clamp_min(1e-300)
            AW = t.empty_like(W)
            _apply(h, W, AW)
            parts.append(W)
            aparts.append(AW)
            if P is not None:
                nP = t.linalg.vector_norm(P, dim=1, keepdim=True).clamp_min(1e-300)
                parts.append(P / nP)
                aparts.append(AP / nP)
        S = t.cat(parts, 0)
        AS = t.cat(aparts, 0)
        G = (S @ S.T).cpu().numpy()
        H = (S @ AS.T).cpu().numpy()
        H = 0.5 * (H + H.T)
        gv, gV = np.linalg.eigh(0.5 * (G + G.T))
        keep = gv > 1e-13 * gv[-1]
        T = gV[:, keep] / np.sqrt(gv[keep])
        if T.shape[1] < b:
            raise RuntimeError("LOBPCG: the basis lost rank")
        ev, Y = np.linalg.eigh(T.T @ H @ T)
        C = T @ Y[:, :b]
        Ct = t.as_tensor(C, device="cuda")
        Xn = Ct.T @ S
        AXn = Ct.T @ AS
        if len(parts) > 1:
            P = Ct[b:].T @ S[b:]
            AP = Ct[b:].T @ AS[b:]
        X, AX = Xn.contiguous(), AXn.contiguous()
        theta = t.as_tensor(ev[:b], device="cuda")
    raise RuntimeError("LOBPCG: no convergence in %d iterations" % maxit)
