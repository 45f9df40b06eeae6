"""Parity of the gather ("pull") form of the operator with the FP64 oracle and
with the scatter form, on the fields the path meets: CED stencils (kappa up
to 100, edges beyond the window halo), smooth fields, random tensors (many
edges without a reciprocal), periodic and ragged grids, FP32 / F16 / BF16
vectors.  The gather form exists for F16 weights; F32 handles keep the
scatter form."""
import numpy as np
import pytest

import oracle
import synth
from oracle import ced
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, dev, export, torch

pytestmark = pytest.mark.gpu


def _apply(h, u, form, out_dtype=None):
    t = torch()
    ab.adlbr_stencils_set_operator(h, form)
    Au = t.empty(u.numel(), dtype=out_dtype or t.float32, device="cuda")
    ab.adlbr_apply(h, u, Au, ab.dtype_code(u.dtype))
    t.cuda.synchronize()
    return Au


def _ced_field(shape, seed):
    img = synth.fingerprint(max(shape), seed)[:shape[0], :shape[1]]
    return np.stack(ced.ced_tensor(img, 1.0, 4.0, 1e-4, 1e-5))


FIELDS = {
    "ced": lambda shape: _ced_field(shape, 11),
    "smooth": lambda shape: synth.smooth_field2d(*shape, seed=3, kappa_min=1, kappa_max=50, lattice=8),
    "random": lambda shape: synth.random_spd2(shape[0] * shape[1], 5, 100.0).reshape(3, *shape),
}


@pytest.mark.parametrize("field", sorted(FIELDS))
@pytest.mark.parametrize("shape", [(96, 160), (77, 131)])
@pytest.mark.parametrize("bc", [ab.NEUMANN, ab.PERIODIC])
def test_gather_matches_oracle(field, shape, bc):
    """FP32 u: the gather form against the oracle's A u on the stored
    weights, relative L-inf <= 1e-5; equal to the scatter form to FP32
    rounding; ragged shapes leave partial tiles and row segments."""
    t = torch()
    w_t = ab.F16
    D = FIELDS[field](shape)
    h, seen, _ = build(D, shape, t.float32, w_t, bc)
    try:
        ab.adlbr_stencils_check(h)
        oo, ow = export(h, shape, w_t)
        u0 = synth.u_uniform(shape, 2)
        u = dev(u0.ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        Ag = _apply(h, u, ab.OP_GATHER)
        assert ab.adlbr_stencils_get_operator(h)[1] == 1, "gather table not built"
        As = _apply(h, u, ab.OP_SCATTER)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, bc, oo, ow, useen).ravel()
    scale = np.abs(ref).max()
    g = Ag.double().cpu().numpy()
    s = As.double().cpu().numpy()
    assert np.abs(g - ref).max() <= 1e-5 * scale
    assert np.abs(g - s).max() <= 2e-6 * scale


def test_gather_is_deterministic_and_conserves():
    """Two gather applications give the same bits; sum(A u) = 0 (A 1 = 0 and
    A symmetric, Neumann rule) to FP32 rounding."""
    t = torch()
    shape = (128, 192)
    h, _, _ = build(FIELDS["ced"](shape), shape, t.float32, ab.F16)
    try:
        u = dev(synth.u_uniform(shape, 4).ravel(), t.float32)
        a = _apply(h, u, ab.OP_GATHER)
        b = _apply(h, u, ab.OP_GATHER)
        one = _apply(h, t.ones_like(u), ab.OP_GATHER)
    finally:
        ab.adlbr_stencils_destroy(h)
    assert t.equal(a, b)
    assert float(one.abs().max()) == 0.0
    assert abs(float(a.double().sum())) <= 1e-5 * float(a.double().abs().sum())


@pytest.mark.parametrize("u_name,tol", [("float16", 4e-3), ("bfloat16", 2e-2)])
def test_gather_half_vectors(u_name, tol):
    """F16 / BF16 u (F16 weights): A u against the oracle fed the rounded u,
    and one explicit step per-step error as for the scatter form."""
    t = torch()
    shape = (96, 128)
    D = synth.smooth_field2d(*shape, seed=8, kappa_min=1, kappa_max=100, lattice=8)
    h, _, _ = build(D, shape, t.float32, ab.F16)
    ud = getattr(t, u_name)
    try:
        oo, ow = export(h, shape, ab.F16)
        u = dev(synth.u_uniform(shape, 3).ravel(), ud)
        useen = u.double().cpu().numpy().reshape(shape)
        Ag = _apply(h, u, ab.OP_GATHER).double().cpu().numpy().reshape(shape)
        dt = oracle.dt_limit(shape, oracle.NEUMANN, oo, ow)
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.dtype_code(ud)), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.dtype_code(ud), dt, 1)
        t.cuda.synchronize()
        ug = u.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, oracle.NEUMANN, oo, ow, useen)
    assert np.abs(Ag - ref).max() <= 1e-5 * np.abs(ref).max()
    step = oracle.step_explicit(shape, oracle.NEUMANN, oo, ow, useen, dt, 1)
    assert np.abs(ug - step).max() <= tol * np.abs(step).max()


@pytest.mark.parametrize("nsteps", [3, 4])
def test_gather_explicit_steps(nsteps):
    """nsteps explicit steps in the gather form (odd counts end in the
    scratch buffer and are copied back) against the oracle; maximum
    principle and mass conservation."""
    t = torch()
    shape = (100, 140)
    D = synth.smooth_field2d(*shape, seed=9, kappa_min=1, kappa_max=60, lattice=8)
    h, _, _ = build(D, shape, t.float32, ab.F16)
    try:
        oo, ow = export(h, shape, ab.F16)
        dt = oracle.dt_limit(shape, oracle.NEUMANN, oo, ow)
        u0 = synth.u_uniform(shape, 5)
        u = dev(u0.ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        ab.adlbr_stencils_set_operator(h, ab.OP_GATHER)
        scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
        ab.adlbr_step_explicit(h, u, scratch, ab.F32, dt, nsteps)
        t.cuda.synchronize()
        assert ab.adlbr_stencils_get_operator(h)[1] == 1
        ug = u.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.step_explicit(shape, oracle.NEUMANN, oo, ow, useen, dt, nsteps)
    assert np.abs(ug - ref).max() <= 1e-5 * np.abs(ref).max()
    assert ug.min() >= useen.min() - 1e-6 and ug.max() <= useen.max() + 1e-6
    assert abs(ug.sum() - useen.sum()) <= 1e-6 * useen.size


def test_f32_weights_keep_the_scatter_form():
    """F32 weights: no gather table is built (the form is F16-only) and the
    operator is the scatter one."""
    t = torch()
    shape = (64, 96)
    h, _, _ = build(FIELDS["smooth"](shape), shape, t.float32, ab.F32)
    try:
        oo, ow = export(h, shape, ab.F32)
        u = dev(synth.u_uniform(shape, 3).ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        Ag = _apply(h, u, ab.OP_GATHER).double().cpu().numpy()
        assert ab.adlbr_stencils_get_operator(h)[1] == 0
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, oracle.NEUMANN, oo, ow, useen).ravel()
    assert np.abs(Ag - ref).max() <= 1e-5 * np.abs(ref).max()


def test_gather_table_follows_in_place_rebuild():
    """The default form is the scatter (no table); asking for the gather form
    builds the table; rebuilding the stencils in place invalidates it, and the
    next gather applications use the new stencils."""
    t = torch()
    shape = (80, 96)
    DA = FIELDS["smooth"](shape)
    DB = FIELDS["ced"](shape)
    h, _, _ = build(DA, shape, t.float32, ab.F16)
    try:
        u = dev(synth.u_uniform(shape, 6).ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        assert ab.adlbr_stencils_get_operator(h) == (ab.OP_AUTO, 0)
        for _ in range(3):
            _apply(h, u, ab.OP_AUTO)
        assert ab.adlbr_stencils_get_operator(h)[1] == 0   # default: scatter, no table
        _apply(h, u, ab.OP_GATHER)
        assert ab.adlbr_stencils_get_operator(h)[1] == 1
        DBd = dev(DB.reshape(3, -1), t.float32)
        ab.adlbr_build_stencils(ab.grid(shape), DBd, ab.F32, ab.F16, out=h)
        assert ab.adlbr_stencils_get_operator(h)[1] == 0
        oo, ow = export(h, shape, ab.F16)
        Ab = [_apply(h, u, ab.OP_GATHER).double().cpu().numpy() for _ in range(2)]
        assert ab.adlbr_stencils_get_operator(h)[1] == 1
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, oracle.NEUMANN, oo, ow, useen).ravel()
    for a in Ab:
        assert np.abs(a - ref).max() <= 1e-5 * np.abs(ref).max()
    assert np.array_equal(Ab[0], Ab[1])


def test_gather_falls_back_beyond_int8_offsets():
    """Offsets beyond +-127 do not fit the table's int8 records: the table is
    marked unusable and the scatter form runs (same result)."""
    t = torch()
    shape = (48, 300)
    th = np.full(shape, np.arctan2(1.0, 150.0))
    D = synth.D_from_angle(th, 400.0)
    h, _, _ = build(D, shape, t.float64, ab.F16)
    try:
        oo, ow = export(h, shape, ab.F16)
        assert np.abs(oo).max() > 127
        u = dev(synth.u_uniform(shape, 7).ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        Ag = _apply(h, u, ab.OP_GATHER).double().cpu().numpy()
        assert ab.adlbr_stencils_get_operator(h)[1] == 0
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, oracle.NEUMANN, oo, ow, useen).ravel()
    assert np.abs(Ag - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("shape", [(3, 5), (4, 4), (1, 37)])
def test_gather_tiny_periodic(shape):
    """Periodic grids smaller than the offsets: several directions wrap onto
    the same neighbour, or onto the point itself."""
    t = torch()
    D = synth.random_spd2(shape[0] * shape[1], 12, 30.0).reshape(3, *shape)
    h, _, _ = build(D, shape, t.float64, ab.F16, ab.PERIODIC)
    try:
        oo, ow = export(h, shape, ab.F16)
        u = dev(synth.u_uniform(shape, 8).ravel(), t.float32)
        useen = u.double().cpu().numpy().reshape(shape)
        Ag = _apply(h, u, ab.OP_GATHER).double().cpu().numpy()
    finally:
        ab.adlbr_stencils_destroy(h)
    ref = oracle.apply(shape, oracle.PERIODIC, oo, ow, useen).ravel()
    assert np.abs(Ag - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-30


def test_gather_full_size_ced_4096():
    """The benchmark's launch: 4096^2 CED stencils (kappa <= 100), F16
    weights, FP32 u.  Gather == scatter over the whole grid (FP32 rounding),
    and 100,000 sampled points against the oracle's row sums computed from the
    exported stencils."""
    t = torch()
    n = 4096
    g = ab.grid((n, n))
    img = synth.fingerprint(n, 1).astype(np.float32)
    u = t.from_numpy(img.ravel()).cuda()
    scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
    h = ab.adlbr_ced_stencils(None, g, u, scratch, 1.0, 4.0, 1e-4, 1e-5, ab.F16)
    try:
        ab.adlbr_stencils_check(h)
        Ag = _apply(h, u, ab.OP_GATHER)
        As = _apply(h, u, ab.OP_SCATTER)
        oo, ow = export(h, (n, n), ab.F16)
    finally:
        ab.adlbr_stencils_destroy(h)
    g_ = Ag.double().cpu().numpy()
    s_ = As.double().cpu().numpy()
    scale = np.abs(s_).max()
    assert np.abs(g_ - s_).max() <= 2e-6 * scale
    # sampled rows: own edges plus every edge of the window that ends at z
    uu = img.astype(np.float64).reshape(n, n)
    rng = np.random.default_rng(0)
    zs = rng.integers(0, n * n, 100000)
    ref = _rows(oo, ow, uu, zs, n)
    assert np.abs(g_[zs] - ref).max() <= 1e-5 * scale
    assert np.abs(s_[zs] - ref).max() <= 1e-5 * scale


def _rows(oo, ow, uu, zs, n):
    """(A u)(z) at the sampled points: own terms, then the incoming terms of
    every point y within the largest offset's reach whose stencil holds
    z - y (Eq. def:E*, Neumann rule)."""
    R = int(np.abs(oo).max())
    ys, xs = np.divmod(zs, n)
    out = np.zeros(len(zs))
    for k in range(3):
        for s in (1, -1):
            dx, dy = s * oo[zs, k, 0], s * oo[zs, k, 1]
            xn, yn = xs + dx, ys + dy
            ok = (xn >= 0) & (xn < n) & (yn >= 0) & (yn < n)
            v = np.where(ok, uu[np.clip(yn, 0, n - 1), np.clip(xn, 0, n - 1)], 0.0)
            out += np.where(ok, ow[zs, k] * (uu[ys, xs] - v), 0.0)
    # incoming: candidates y = z - e for every offset e of the whole field
    # would be slow; use the set of distinct offsets present
    offs = np.unique(np.concatenate([oo[:, k, :] for k in range(3)]), axis=0)
    offs = offs[np.any(offs != 0, axis=1)]
    for e in offs:
        for s in (1, -1):
            ex, ey = s * e[0], s * e[1]
            yx, yy = xs - ex, ys - ey     # source y with y + (ex, ey) = z
            ok = (yx >= 0) & (yx < n) & (yy >= 0) & (yy < n)
            yi = np.clip(yy, 0, n - 1) * n + np.clip(yx, 0, n - 1)
            for k in range(3):
                hit = ok & (((oo[yi, k, 0] == e[0]) & (oo[yi, k, 1] == e[1])))
                out += np.where(hit, ow[yi, k] * (uu[ys, xs] - uu[np.clip(yy, 0, n - 1), np.clip(yx, 0, n - 1)]),
                                0.0)
    assert R >= 1
    return out


def test_cg_with_gather_operator():
    """The implicit step (CG and Jacobi-PCG, Sec. 4.2) on a handle set to the
    gather form: converges to the stated residual and agrees with the scatter
    form's solution to the solver tolerance."""
    t = torch()
    n = 192
    D = synth.smooth_field2d(n, n, 3, 1.0, 50.0, 8)
    h, _, _ = build(D, (n, n), t.float32, ab.F16)
    try:
        dt = 200.0 / ab.adlbr_stencils_max_diag(h)
        b = dev(synth.u_uniform((n, n), 3).ravel(), t.float32)
        xs = {}
        for form in (ab.OP_SCATTER, ab.OP_GATHER):
            ab.adlbr_stencils_set_operator(h, form)
            for pc in (0, 2):
                x = b.clone()
                it, rel = ab.adlbr_step_implicit(h, b, x, dt, 1e-6, 2000, precond=pc)
                assert rel <= 2e-5, (form, pc, rel)
                xs[(form, pc)] = (x.double().cpu().numpy(), it)
        assert ab.adlbr_stencils_get_operator(h)[1] == 1
    finally:
        ab.adlbr_stencils_destroy(h)
    for pc in (0, 2):
        xsc, its = xs[(ab.OP_SCATTER, pc)]
        xg, itg = xs[(ab.OP_GATHER, pc)]
        assert abs(its - itg) <= 3
        assert np.abs(xsc - xg).max() <= 1e-4 * np.abs(xsc).max()


def test_gather_table_follows_rebuilds_inside_ced_steps():
    """adlbr_ced_step rebuilds the stencils at every step of one call: with the
    gather form asked for, every step must use a table of its own stencils.
    Four steps in one call equal four calls of one step each (each call
    builds the table afresh), bit for bit (the gather form is deterministic),
    and equal the scatter form's four steps to FP32 rounding."""
    t = torch()
    shape = (96, 160)
    g = ab.grid(shape)
    img = synth.fingerprint(160, 21)[:96, :160].astype(np.float32)
    P = (1.0, 4.0, 1e-4, 1e-5, 0.02)

    def run(form, calls, per_call):
        u = t.from_numpy(img.ravel().copy()).cuda()
        scratch = t.empty(ab.adlbr_ced_scratch_bytes(g), dtype=t.uint8, device="cuda")
        h = ab.adlbr_ced_stencils(None, g, u, scratch, *P[:4], ab.F16)
        try:
            ab.adlbr_stencils_set_operator(h, form)
            for _ in range(calls):
                h = ab.adlbr_ced_step(h, g, u, scratch, *P, per_call, ab.F16)
            t.cuda.synchronize()
        finally:
            ab.adlbr_stencils_destroy(h)
        return u.cpu().numpy()

    one_call = run(ab.OP_GATHER, 1, 4)
    four_calls = run(ab.OP_GATHER, 4, 1)
    scatter = run(ab.OP_SCATTER, 1, 4)
    assert np.array_equal(one_call, four_calls)
    assert np.abs(one_call - scatter).max() <= 1e-5 * np.abs(scatter).max()
