"""Thin ctypes binding of libadlbr.so (include/adlbr.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, converts torch tensors (or raw integer addresses) to device
pointers and the stream to a cudaStream_t, and raises AdlbrError on a non-OK
status.  All computation happens in the library's CUDA kernels; there is no
fallback, and importing the module fails loudly if the library is missing.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# ADLBR_BOUNDS_CHECK=1 selects the bounds-checked build of the library
CHECKED = os.environ.get("ADLBR_BOUNDS_CHECK", "") == "1"
LIB_PATH = os.path.join(_HERE, "libadlbr_checked.so" if CHECKED else "libadlbr.so")

F64, F32, F16, BF16 = 0, 1, 2, 3
NEUMANN, PERIODIC = 0, 1
OP_AUTO, OP_SCATTER, OP_GATHER = 0, 1, 2
SCHEME_ADLBR, SCHEME_ANN = 0, 1

STATUS = {0: "OK", 1: "E_ARG", 2: "E_SHAPE", 3: "E_NOT_SPD", 4: "E_NONFINITE",
          5: "E_NOT_CONVERGED", 6: "E_TIMEOUT", 7: "E_CUDA", 8: "E_RANGE", 9: "E_INTERNAL"}


class AdlbrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(status, "?"), status, msg))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("bc", ctypes.c_int32), ("n", ctypes.c_int64 * 3)]


def grid(shape, bc=NEUMANN):
    """numpy/torch shape (ny, nx) or (nz, ny, nx) -> adlbr_grid (x fastest)."""
    g = Grid()
    g.dim = len(shape)
    g.bc = bc
    ext = list(shape)[::-1] + [1] * (3 - len(shape))
    for k in range(3):
        g.n[k] = int(ext[k])
    return g


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built (run paper_1301_3925_gb300.build%s)"
                              % (os.path.basename(LIB_PATH), " --checked" if CHECKED else ""))
        L = ctypes.CDLL(LIB_PATH)
        sigs = {
            "adlbr_version": (ctypes.c_char_p, []),
            "adlbr_last_error": (ctypes.c_char_p, []),
            "adlbr_build_stencils": (_i32, [ctypes.POINTER(Grid), _vp, _i32, _i32,
                                            ctypes.POINTER(_vp), _vp]),
            "adlbr_stencils_check": (_i32, [_vp, _vp]),
            "adlbr_build_stencils_scheme": (_i32, [ctypes.POINTER(Grid), _vp, _i32, _i32, _i32,
                                                   ctypes.POINTER(_vp), _vp]),
            "adlbr_stencils_scheme": (_i32, [_vp, ctypes.POINTER(_i32)]),
            "adlbr_stencils_grid": (_i32, [_vp, ctypes.POINTER(Grid)]),
            "adlbr_stencils_export": (_i32, [_vp, _vp, _vp, _vp]),
            "adlbr_stencils_destroy": (_i32, [_vp]),
            "adlbr_apply": (_i32, [_vp, _vp, _vp, _i32, _vp]),
            "adlbr_build_step_explicit": (_i32, [ctypes.POINTER(Grid), _vp, _i32, _i32, ctypes.POINTER(_vp), _vp,
                                                 _vp, ctypes.c_double, _vp]),
            "adlbr_stencils_set_operator": (_i32, [_vp, _i32]),
            "adlbr_stencils_get_operator": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
            "adlbr_step_scratch_bytes": (ctypes.c_size_t, [_vp, _i32]),
            "adlbr_step_explicit": (_i32, [_vp, _vp, _vp, _i32, ctypes.c_double, _i32, _vp]),
            "adlbr_step_explicit_noalloc": (_i32, [_vp, _vp, _i32, ctypes.c_double, _i32, _vp]),
            "adlbr_step_implicit": (_i32, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, _i32,
                                           _i32, _vp, ctypes.POINTER(_i32),
                                           ctypes.POINTER(ctypes.c_double), _vp]),
            "adlbr_last_fallback": (_i32, []),
            "adlbr_last_residual_met": (_i32, []),
            "adlbr_unet_set_tensor_cores": (_i32, [_vp, _i32]),
            "adlbr_batch_create": (_i32, [_i32, _vp, _vp, _vp, _i32, ctypes.POINTER(_vp), _vp]),
            "adlbr_batch_step": (_i32, [_vp, _i32, _vp]),
            "adlbr_batch_config": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_i32)]),
            "adlbr_batch_destroy": (_i32, [_vp]),
            "adlbr_unet_create": (_i32, [_i32, _i32, _i32, _i32, _i32, _i32, _i32,
                                         ctypes.POINTER(_vp)]),
            "adlbr_unet_destroy": (_i32, [_vp]),
            "adlbr_unet_num_params": (ctypes.c_int64, [_vp]),
            "adlbr_unet_forward": (_i32, [_vp, _vp, _vp, _vp, _vp]),
            "adlbr_unet_backward": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
            "adlbr_adam_step": (_i32, [_vp, _vp, _vp, _vp, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double, _i32, _vp]),
            "adlbr_nn_training_pairs": (_i32, [_vp, _vp, ctypes.c_double, ctypes.c_double, _i32,
                                               _i32, _i32, _vp, _vp, _vp, _vp,
                                               ctypes.POINTER(_i32), _vp]),
            "adlbr_stencils_max_diag": (_i32, [_vp, ctypes.POINTER(ctypes.c_double), _vp]),
            "adlbr_nn_precondition": (_i32, [_vp, _vp, ctypes.c_double, _vp, _vp, _vp]),
            "adlbr_mse_grad": (_i32, [_vp, _vp, ctypes.c_int64, _vp,
                                      ctypes.POINTER(ctypes.c_double), _vp]),
            "adlbr_block_dot": (_i32, [_vp, _i32, _vp, _i32, ctypes.c_int64, _vp, _vp]),
            "adlbr_block_combine": (_i32, [_vp, _i32, _i32, _vp, ctypes.c_int64, _vp, _vp]),
            "adlbr_block_residual": (_i32, [_vp, _vp, _vp, _i32, ctypes.c_int64, _vp, _vp, _vp]),
            "adlbr_ced_scratch_bytes": (ctypes.c_size_t, [ctypes.POINTER(Grid)]),
            "adlbr_ced_tensor": (_i32, [ctypes.POINTER(Grid), _vp, _vp, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double, _vp, _vp]),
            "adlbr_eed_tensor": (_i32, [ctypes.POINTER(Grid), _vp, _vp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, _vp, _vp]),
            "adlbr_ced_stencils": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(Grid), _vp, _vp,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, _i32, _vp]),
            "adlbr_ced_step": (_i32, [ctypes.POINTER(_vp), ctypes.POINTER(Grid), _vp, _vp,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, _i32, _i32, _vp]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st):
    if st != 0:
        raise AdlbrError(st, lib().adlbr_last_error().decode(errors="replace"))


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(t):
    """torch dtype -> adlbr_dtype."""
    import torch
    return {torch.float64: F64, torch.float32: F32, torch.float16: F16, torch.bfloat16: BF16}[t]


def adlbr_version():
    return lib().adlbr_version().decode()


def adlbr_last_error():
    return lib().adlbr_last_error().decode(errors="replace")


def adlbr_build_stencils(g, D, D_t, w_t, out=None, stream=None):
    """Returns the stencil handle (an int address); reuses ``out`` if given."""
    h = _vp(out)
    _check(lib().adlbr_build_stencils(ctypes.byref(g), _ptr(D), D_t, w_t, ctypes.byref(h),
                                      _stream(stream)))
    return h.value


def adlbr_build_stencils_scheme(g, D, D_t, w_t, scheme, out=None, stream=None):
    """adlbr_build_stencils for scheme SCHEME_ADLBR or SCHEME_ANN; returns the handle."""
    h = _vp(out)
    _check(lib().adlbr_build_stencils_scheme(ctypes.byref(g), _ptr(D), D_t, w_t, int(scheme), ctypes.byref(h),
                                             _stream(stream)))
    return h.value


def adlbr_stencils_scheme(h):
    v = _i32(0)
    _check(lib().adlbr_stencils_scheme(h, ctypes.byref(v)))
    return v.value


def adlbr_stencils_check(h, stream=None):
    _check(lib().adlbr_stencils_check(h, _stream(stream)))


def adlbr_stencils_grid(h):
    g = Grid()
    _check(lib().adlbr_stencils_grid(h, ctypes.byref(g)))
    return g


def adlbr_stencils_export(h, offs, w, stream=None):
    _check(lib().adlbr_stencils_export(h, _ptr(offs), _ptr(w), _stream(stream)))


def adlbr_stencils_destroy(h):
    _check(lib().adlbr_stencils_destroy(h))


def adlbr_apply(h, u, Au, u_t, stream=None):
    _check(lib().adlbr_apply(h, _ptr(u), _ptr(Au), u_t, _stream(stream)))


def adlbr_stencils_set_operator(h, form):
    """form: OP_AUTO, OP_SCATTER or OP_GATHER."""
    _check(lib().adlbr_stencils_set_operator(h, int(form)))


def adlbr_stencils_get_operator(h):
    """(form setting, 1 if the gather table matches the current stencils)."""
    f, r = _i32(0), _i32(0)
    _check(lib().adlbr_stencils_get_operator(h, ctypes.byref(f), ctypes.byref(r)))
    return f.value, r.value


def adlbr_step_scratch_bytes(h, u_t):
    return int(lib().adlbr_step_scratch_bytes(h, u_t))


def adlbr_step_explicit(h, u, scratch, u_t, dt, nsteps, stream=None):
    _check(lib().adlbr_step_explicit(h, _ptr(u), _ptr(scratch), u_t, float(dt), int(nsteps),
                                     _stream(stream)))


def adlbr_step_explicit_noalloc(h, u, u_t, dt, nsteps, stream=None):
    """The explicit step with the library's fixed scratch array (no allocation)."""
    _check(lib().adlbr_step_explicit_noalloc(h, _ptr(u), u_t, float(dt), int(nsteps),
                                             _stream(stream)))


def adlbr_unet_create(cin, c1, c2, c3, batch, H, W):
    h = _vp()
    _check(lib().adlbr_unet_create(cin, c1, c2, c3, batch, H, W, ctypes.byref(h)))
    return h.value


def adlbr_unet_destroy(n):
    _check(lib().adlbr_unet_destroy(n))


def adlbr_unet_num_params(n):
    return int(lib().adlbr_unet_num_params(n))


def adlbr_unet_forward(n, params, x, y, stream=None):
    _check(lib().adlbr_unet_forward(n, _ptr(params), _ptr(x), _ptr(y), _stream(stream)))


def adlbr_unet_backward(n, params, gy, gparams, gx=None, stream=None):
    _check(lib().adlbr_unet_backward(n, _ptr(params), _ptr(gy), _ptr(gparams), _ptr(gx),
                                     _stream(stream)))


def adlbr_adam_step(params, grads, m, v, n, lr, beta1, beta2, eps, t, stream=None):
    _check(lib().adlbr_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), int(n), float(lr),
                                 float(beta1), float(beta2), float(eps), int(t), _stream(stream)))


class NNPrecond(ctypes.Structure):
    """adlbr_nn_precond: network handle and its device parameter vector."""
    _fields_ = [("net", _vp), ("params", _vp)]


def nn_precond(net, params):
    return NNPrecond(net, _ptr(params))


def adlbr_nn_training_pairs(h, rhs, dt, rtol, maxit, every, max_pairs, nn, feats, targets, xbuf,
                            stream=None):
    """Returns the number of pairs written (nn: NNPrecond or None for CG)."""
    n = ctypes.c_int(0)
    nnp = ctypes.cast(ctypes.pointer(nn), ctypes.c_void_p).value if nn is not None else None
    _check(lib().adlbr_nn_training_pairs(h, _ptr(rhs), float(dt), float(rtol), int(maxit),
                                         int(every), int(max_pairs), nnp, _ptr(feats),
                                         _ptr(targets), _ptr(xbuf), ctypes.byref(n),
                                         _stream(stream)))
    return n.value


def adlbr_nn_precondition(h, nn, dt, r, z, stream=None):
    nnp = ctypes.cast(ctypes.pointer(nn), ctypes.c_void_p).value
    _check(lib().adlbr_nn_precondition(h, nnp, float(dt), _ptr(r), _ptr(z), _stream(stream)))


def adlbr_stencils_max_diag(h, stream=None):
    v = ctypes.c_double(0.0)
    _check(lib().adlbr_stencils_max_diag(h, ctypes.byref(v), _stream(stream)))
    return v.value


def adlbr_mse_grad(y, t, n, gy, want_loss=True, stream=None):
    v = ctypes.c_double(0.0)
    _check(lib().adlbr_mse_grad(_ptr(y), _ptr(t), int(n), _ptr(gy),
                                ctypes.byref(v) if want_loss else None, _stream(stream)))
    return v.value if want_loss else None


def adlbr_block_dot(A, B, G, stream=None):
    """G = A B^T for device FP64 blocks A (ma x n), B (mb x n), G (ma x mb)."""
    ma, n = A.shape
    mb = B.shape[0]
    _check(lib().adlbr_block_dot(_ptr(A), int(ma), _ptr(B), int(mb), int(n), _ptr(G), _stream(stream)))


def adlbr_block_combine(C, S, out, stream=None):
    """out = C^T S for device FP64 C (m x k), S (m x n), out (k x n)."""
    m, k = C.shape
    _check(lib().adlbr_block_combine(_ptr(C), int(m), int(k), _ptr(S), int(S.shape[1]), _ptr(out),
                                     _stream(stream)))


def adlbr_block_residual(AX, X, theta, R, rnorm, stream=None):
    """R = AX - theta X row by row and rnorm = the rows' 2-norms (device FP64)."""
    m, n = X.shape
    _check(lib().adlbr_block_residual(_ptr(AX), _ptr(X), _ptr(theta), int(m), int(n), _ptr(R), _ptr(rnorm),
                                      _stream(stream)))


def adlbr_ced_scratch_bytes(g):
    return int(lib().adlbr_ced_scratch_bytes(ctypes.byref(g)))


def adlbr_ced_tensor(g, u, D, sigma, rho, alpha, C, scratch, stream=None):
    _check(lib().adlbr_ced_tensor(ctypes.byref(g), _ptr(u), _ptr(D), float(sigma), float(rho),
                                  float(alpha), float(C), _ptr(scratch), _stream(stream)))


def adlbr_eed_tensor(g, u, D, sigma, rho, C, scratch, stream=None):
    _check(lib().adlbr_eed_tensor(ctypes.byref(g), _ptr(u), _ptr(D), float(sigma), float(rho), float(C),
                                  _ptr(scratch), _stream(stream)))


def adlbr_ced_step(h, g, u, scratch, sigma, rho, alpha, C, dt, nsteps, w_t, stream=None):
    """Returns the (possibly newly allocated) stencil handle."""
    hh = _vp(h)
    _check(lib().adlbr_ced_step(ctypes.byref(hh), ctypes.byref(g), _ptr(u), _ptr(scratch),
                                float(sigma), float(rho), float(alpha), float(C), float(dt),
                                int(nsteps), w_t, _stream(stream)))
    return hh.value


def adlbr_build_step_explicit(g, D, D_t, w_t, h, u, scratch, dt, stream=None):
    """Stencils of D into h (None allocates) and one explicit step of the FP32
    vector u; returns the handle."""
    hh = _vp(h)
    _check(lib().adlbr_build_step_explicit(ctypes.byref(g), _ptr(D), D_t, w_t, ctypes.byref(hh), _ptr(u),
                                           _ptr(scratch), float(dt), _stream(stream)))
    return hh.value


def adlbr_ced_stencils(h, g, u, scratch, sigma, rho, alpha, C, w_t, stream=None):
    """Returns the (possibly newly allocated) stencil handle."""
    hh = _vp(h)
    _check(lib().adlbr_ced_stencils(ctypes.byref(hh), ctypes.byref(g), _ptr(u), _ptr(scratch),
                                    float(sigma), float(rho), float(alpha), float(C), w_t,
                                    _stream(stream)))
    return hh.value


def adlbr_step_implicit(h, rhs, x, dt, rtol, maxit, precond=0, nn=None, stream=None):
    """Returns (iterations, true relative residual)."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    if isinstance(nn, NNPrecond):
        nnp = ctypes.cast(ctypes.pointer(nn), ctypes.c_void_p).value
    else:
        nnp = _ptr(nn)
    _check(lib().adlbr_step_implicit(h, _ptr(rhs), _ptr(x), float(dt), float(rtol), int(maxit),
                                     int(precond), nnp, ctypes.byref(it), ctypes.byref(rr),
                                     _stream(stream)))
    return it.value, rr.value


def adlbr_last_residual_met():
    """1 if the last implicit solve of this thread ended at or below rtol (true residual)."""
    return int(lib().adlbr_last_residual_met())


def adlbr_last_fallback():
    """1 if the last preconditioned implicit solve of this thread fell back to plain CG."""
    return int(lib().adlbr_last_fallback())


def adlbr_batch_create(handles, us, dts, autotune=True, stream=None):
    """Batch of explicit steps over items (handle, FP32 u tensor, dt); returns the batch address."""
    n = len(handles)
    H = (ctypes.c_void_p * n)(*handles)
    U = (ctypes.c_void_p * n)(*[_ptr(x) for x in us])
    T = (ctypes.c_double * n)(*[float(d) for d in dts])
    out = ctypes.c_void_p()
    _check(lib().adlbr_batch_create(n, ctypes.cast(H, ctypes.c_void_p), ctypes.cast(U, ctypes.c_void_p),
                                    ctypes.cast(T, ctypes.c_void_p), 1 if autotune else 0,
                                    ctypes.byref(out), _stream(stream)))
    return out.value


def adlbr_batch_step(b, nsteps, stream=None):
    _check(lib().adlbr_batch_step(b, int(nsteps), _stream(stream)))


def adlbr_batch_config(b):
    """(shape (tw, th, bx, by, bz), tuned ms, points, tiles)."""
    sh = (_i32 * 5)()
    ms = ctypes.c_double(0.0)
    pts = ctypes.c_int64(0)
    nt = _i32(0)
    _check(lib().adlbr_batch_config(b, sh, ctypes.byref(ms), ctypes.byref(pts), ctypes.byref(nt)))
    return tuple(sh), ms.value, pts.value, nt.value


def adlbr_batch_destroy(b):
    _check(lib().adlbr_batch_destroy(b))


def adlbr_unet_set_tensor_cores(net, on=True):
    _check(lib().adlbr_unet_set_tensor_cores(net, 1 if on else 0))
