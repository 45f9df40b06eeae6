"""FP64 CPU oracle for the AD-LBR hot path.

TEST INFRASTRUCTURE, NOT PRODUCT.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import this package.
It shares no code with the CUDA library (``paper_1301_3925_gb300``) and never
imports it.

Contents (each function cites the passage of Fehrenbach & Mirebeau, "Sparse
Non-Negative Stencils for Anisotropic Diffusion", that it follows):

* ``build2d`` / ``build3d``  -- stencils and weights, Sec. 2 (C code in
  ``adlbr_oracle.c``).
* ``apply`` -- A u = (1/2) grad E_h(u), Eq. def:E*, h = 1, Neumann rule of
  Sec. 1 or periodic wrap.
* ``step_explicit`` -- explicit Euler, Sec. 4.4 (CED), u <- u - dt A u.
* ``cg`` / ``fcg`` -- (I + dt A) x = b by conjugate gradients, Sec. 4.2
  (Eq. elliptic, solved "using Conjugate Gradient").
* ``ced`` (module) -- the coherence-enhancing diffusion tensor, Sec. 4.4.
* ``unet`` (module) -- the learned preconditioner's network (not in the paper).
* ``ann`` (module) -- the A-NN comparison scheme, Sec. 4.1, Remark rem:WG.

All floating point is FP64.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lp = ctypes.POINTER(ctypes.c_long)
        L.or_exact_sign.argtypes = [ctypes.c_int, dp, lp]
        L.or_exact_sign.restype = ctypes.c_int
        L.or_exact_value.argtypes = [ctypes.c_int, dp, lp]
        L.or_exact_value.restype = ctypes.c_double
        L.or_build2d.argtypes = [ctypes.c_int64, dp, dp, dp, i32p, dp, i32p, i32p]
        L.or_build2d.restype = ctypes.c_int
        L.or_build3d.argtypes = [ctypes.c_int64, dp, i32p, dp, i32p, i32p]
        L.or_build3d.restype = ctypes.c_int
        L.or_apply.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, i32p, dp, dp, dp]
        L.or_apply.restype = ctypes.c_int
        L.or_diag.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, i32p, dp, dp]
        L.or_diag.restype = ctypes.c_int
        L.or_energy.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, i32p, dp, dp]
        L.or_energy.restype = ctypes.c_double
        _LIB = L
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


NEUMANN, PERIODIC = 0, 1
STATUS = {0: "ok", 3: "not SPD", 4: "non-finite", 5: "not converged", 8: "range", 9: "internal"}


def exact_sign(x, n):
    """Exact sign of sum_k n[k] * x[k] (integers n, doubles x)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.int64).astype(np.dtype("l"))
    return lib().or_exact_sign(len(x), _p(x, ctypes.c_double), _p(n, ctypes.c_long))


def exact_value(x, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = np.ascontiguousarray(n, dtype=np.int64).astype(np.dtype("l"))
    return lib().or_exact_value(len(x), _p(x, ctypes.c_double), _p(n, ctypes.c_long))


def build2d(Dxx, Dxy, Dyy):
    """2D AD-LBR stencils, Sec. 2 (Eq. GaussAlgo, Corollary
    ObtuseSuperBaseFromReducedBasis2, Eqs. def:Vz and def:GammaZ).

    Inputs: three arrays of the same shape (the entries of D = [[a,b],[b,c]]).
    Returns (offs int32 [N,3,2] canonical half-stencil, w float64 [N,3],
    status int32 [N], iters int32 [N])."""
    a = np.ascontiguousarray(np.ravel(Dxx), dtype=np.float64)
    b = np.ascontiguousarray(np.ravel(Dxy), dtype=np.float64)
    c = np.ascontiguousarray(np.ravel(Dyy), dtype=np.float64)
    n = a.size
    offs = np.zeros((n, 3, 2), np.int32)
    w = np.zeros((n, 3), np.float64)
    st = np.zeros(n, np.int32)
    it = np.zeros(n, np.int32)
    lib().or_build2d(n, _p(a, ctypes.c_double), _p(b, ctypes.c_double), _p(c, ctypes.c_double),
                     _p(offs, ctypes.c_int32), _p(w, ctypes.c_double), _p(st, ctypes.c_int32),
                     _p(it, ctypes.c_int32))
    return offs, w, st, it


def build3d(D6):
    """3D AD-LBR stencils, Sec. 2 (Def. ReducedBasis, Prop. MakeObtuse,
    Lemma Selling).  D6: array [6, ...] with planes (xx, yy, zz, xy, xz, yz).
    Returns (offs int32 [N,6,3], w float64 [N,6], status, iters)."""
    D6 = np.asarray(D6, dtype=np.float64)
    D = np.ascontiguousarray(D6.reshape(6, -1))
    n = D.shape[1]
    offs = np.zeros((n, 6, 3), np.int32)
    w = np.zeros((n, 6), np.float64)
    st = np.zeros(n, np.int32)
    it = np.zeros(n, np.int32)
    lib().or_build3d(n, _p(D, ctypes.c_double), _p(offs, ctypes.c_int32), _p(w, ctypes.c_double),
                     _p(st, ctypes.c_int32), _p(it, ctypes.c_int32))
    return offs, w, st, it


def _grid(shape):
    """numpy shape (ny, nx) or (nz, ny, nx) -> (dim, int64[3] (nx, ny, nz))."""
    dim = len(shape)
    nn = np.ones(3, np.int64)
    nn[:dim] = shape[::-1]
    return dim, nn


def apply(shape, bc, offs, w, u):
    """A u with A = (1/2) grad E_h, Eq. def:E* (h = 1); the Neumann rule of
    Sec. 1 drops pairs leaving the grid, bc = PERIODIC wraps them."""
    dim, nn = _grid(shape)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    K = w.shape[-1]
    Au = np.zeros(u.size, np.float64)
    lib().or_apply(dim, _p(nn, ctypes.c_int64), bc, K, _p(offs, ctypes.c_int32),
                   _p(w, ctypes.c_double), _p(u, ctypes.c_double), _p(Au, ctypes.c_double))
    return Au.reshape(shape)


def diag(shape, bc, offs, w):
    """Diagonal of A (sum of the weights of every in-grid pair at z)."""
    dim, nn = _grid(shape)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    K = w.shape[-1]
    d = np.zeros(int(np.prod(shape)), np.float64)
    lib().or_diag(dim, _p(nn, ctypes.c_int64), bc, K, _p(offs, ctypes.c_int32),
                  _p(w, ctypes.c_double), _p(d, ctypes.c_double))
    return d.reshape(shape)


def energy(shape, bc, offs, w, u):
    """E_h(u), Eq. def:E* with h = 1."""
    dim, nn = _grid(shape)
    offs = np.ascontiguousarray(offs, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    K = w.shape[-1]
    return lib().or_energy(dim, _p(nn, ctypes.c_int64), bc, K, _p(offs, ctypes.c_int32),
                           _p(w, ctypes.c_double), _p(u, ctypes.c_double))


def dt_limit(shape, bc, offs, w):
    """Explicit time step dt = 1 / max_z A_zz (the monotone limit; it is
    below 2 / lambda_max(A) by Gershgorin, cf. Table 3's caption)."""
    return 1.0 / float(np.max(diag(shape, bc, offs, w)))


def step_explicit(shape, bc, offs, w, u, dt, nsteps=1):
    """Explicit Euler of Sec. 4.4: (u^{n+1} - u^n)/dt = div(D grad u^n),
    i.e. u^{n+1} = u^n - dt A u^n."""
    u = np.array(u, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        u = u - dt * apply(shape, bc, offs, w, u)
    return u


def cg(shape, bc, offs, w, b, x0, dt, rtol=1e-6, maxit=10000):
    """Plain conjugate gradients for (I + dt A) x = b (Eq. elliptic with
    lambda = dt, solved by CG as in Sec. 4.2).  Stops when the recursively
    updated residual satisfies |r| <= rtol |b|; returns (x, iters, true
    relative residual)."""
    def op(v):
        return v + dt * apply(shape, bc, offs, w, v)

    b = np.asarray(b, np.float64)
    x = np.array(x0, np.float64, copy=True)
    r = b - op(x)
    p = r.copy()
    rr = float(np.vdot(r, r))
    bn = float(np.sqrt(np.vdot(b, b)))
    it = 0
    while np.sqrt(rr) > rtol * bn and it < maxit:
        Ap = op(p)
        alpha = rr / float(np.vdot(p, Ap))
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(np.vdot(r, r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    true_res = float(np.linalg.norm(b - op(x)) / bn)
    return x, it, true_res


def fcg(shape, bc, offs, w, b, x0, dt, precond, rtol=1e-6, maxit=10000):
    """Flexible preconditioned CG (Polak-Ribiere beta) for (I + dt A) x = b
    with a possibly nonlinear preconditioner z = precond(r)."""
    def op(v):
        return v + dt * apply(shape, bc, offs, w, v)

    b = np.asarray(b, np.float64)
    x = np.array(x0, np.float64, copy=True)
    r = b - op(x)
    z = precond(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    bn = float(np.sqrt(np.vdot(b, b)))
    it = 0
    while np.linalg.norm(r) > rtol * bn and it < maxit:
        Ap = op(p)
        alpha = rz / float(np.vdot(p, Ap))
        x += alpha * p
        r_old = r.copy()
        r -= alpha * Ap
        z_new = precond(r)
        rz_new = float(np.vdot(r, z_new))
        beta = float(np.vdot(r - r_old, z_new)) / rz
        p = z_new + beta * p
        rz = rz_new
        it += 1
    true_res = float(np.linalg.norm(b - op(x)) / bn)
    return x, it, true_res
