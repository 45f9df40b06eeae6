"""Helpers for the GPU parity tests: run the CUDA path through the C-ABI and
bring results back as numpy arrays."""
import numpy as np

from paper_1301_3925_gb300 import adlbr as ab


def torch():
    import torch as _t
    return _t


def dev(a, dtype):
    t = torch()
    return t.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def build(D_planes, shape, D_dtype, w_t, bc=ab.NEUMANN):
    """D_planes: numpy (3|6, *shape) FP64.  Returns (handle, the exact D values
    the GPU saw as FP64 numpy)."""
    t = torch()
    Dd = dev(D_planes.reshape(D_planes.shape[0], -1), D_dtype)
    g = ab.grid(shape, bc)
    h = ab.adlbr_build_stencils(g, Dd, ab.dtype_code(D_dtype), w_t)
    seen = Dd.double().cpu().numpy().reshape(D_planes.shape)
    return h, seen, Dd


def export(h, shape, w_t):
    t = torch()
    dim = len(shape)
    N = int(np.prod(shape))
    K = 3 if dim == 2 else 6
    offs = t.zeros((N, K, dim), dtype=t.int16, device="cuda")
    w = t.zeros((N, K), dtype=t.float64 if w_t == ab.F64 else t.float32, device="cuda")
    ab.adlbr_stencils_export(h, offs, w)
    t.cuda.synchronize()
    return offs.cpu().numpy().astype(np.int32), w.double().cpu().numpy()


def weight_tol(w_ref, w_t, Dscale):
    """Per-entry tolerance of stored weights against the FP64 oracle."""
    wmax = np.max(w_ref, axis=-1, keepdims=True)
    if w_t == ab.F64:
        return 1e-13 * wmax + 1e-300
    if w_t == ab.F32:
        return 2.0 ** -22 * np.abs(w_ref) + 2.0 ** -40 * Dscale
    return 2.0 ** -11 * np.abs(w_ref) + 2.0 ** -23 * wmax
