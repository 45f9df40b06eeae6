"""Batched explicit steps over uneven 2D and 3D items: parity with the
single-grid step and with the FP64 oracle, autotuned and fixed shapes."""
import numpy as np
import pytest

import oracle
import synth
from paper_1301_3925_gb300 import adlbr as ab

from gpu_helpers import build, dev, export, torch

pytestmark = pytest.mark.gpu

# (shape, boundary, weight type, field seed)
ITEMS = [((50, 70), ab.NEUMANN, ab.F16, 1), ((33, 129), ab.PERIODIC, ab.F32, 2),
         ((96, 64), ab.NEUMANN, ab.F64, 3), ((13, 17, 19), ab.NEUMANN, ab.F16, 4),
         ((8, 10, 12), ab.PERIODIC, ab.F32, 5), ((130, 257), ab.NEUMANN, ab.F16, 6)]


def _field(shape, seed):
    if len(shape) == 2:
        return synth.smooth_field2d(*shape, seed=seed, kappa_min=1, kappa_max=40, lattice=6)
    n = max(shape)
    return synth.needle_field3d(n, seed=seed, kappa=12.0)[:, :shape[0], :shape[1], :shape[2]]


def _setup():
    t = torch()
    hs, us, dts, seen = [], [], [], []
    for k, (shape, bc, wt, seed) in enumerate(ITEMS):
        h, D, _ = build(_field(shape, seed), shape, t.float32, wt, bc)
        hs.append(h)
        seen.append(D)
        dts.append(0.9 / ab.adlbr_stencils_max_diag(h))
        us.append(dev(synth.u_uniform(shape, 10 + k).ravel(), t.float32))
    return hs, us, dts, seen


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_matches_single_grid_steps(autotune):
    t = torch()
    hs, us, dts, _ = _setup()
    ref = [u.clone() for u in us]
    b = None
    try:
        for h, u, d in zip(hs, ref, dts):
            scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
            ab.adlbr_step_explicit(h, u, scratch, ab.F32, d, 5)
        b = ab.adlbr_batch_create(hs, us, dts, autotune=autotune)
        shape, ms, pts, ntiles = ab.adlbr_batch_config(b)
        assert pts == sum(int(np.prod(s)) for s, _, _, _ in ITEMS) and ntiles > 0
        assert (ms > 0) == autotune
        if not autotune:
            assert shape == (64, 32, 32, 8, 4)
        ab.adlbr_batch_step(b, 5)
        t.cuda.synchronize()
        for k, (u, r) in enumerate(zip(us, ref)):
            err = (u - r).abs().max().item() / r.abs().max().item()
            assert err <= 1e-6, (k, ITEMS[k], err)
    finally:
        if b:
            ab.adlbr_batch_destroy(b)
        for h in hs:
            ab.adlbr_stencils_destroy(h)


@pytest.mark.parametrize("kind", [2, 3])
def test_batch_of_one_kind(kind):
    """Images only or volumes only: the other accumulate kernel has no tiles
    and is not launched; every tuned shape still matches the single-grid
    step."""
    t = torch()
    hs, us, dts, _ = _setup()
    keep = [k for k, it in enumerate(ITEMS) if len(it[0]) == kind]
    for k in range(len(ITEMS)):
        if k not in keep:
            ab.adlbr_stencils_destroy(hs[k])
    hs, us, dts = [hs[k] for k in keep], [us[k] for k in keep], [dts[k] for k in keep]
    ref = [u.clone() for u in us]
    b = None
    try:
        for h, u, d in zip(hs, ref, dts):
            scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
            ab.adlbr_step_explicit(h, u, scratch, ab.F32, d, 4)
        b = ab.adlbr_batch_create(hs, us, dts, autotune=True)
        _, ms, pts, ntiles = ab.adlbr_batch_config(b)
        assert pts == sum(int(np.prod(ITEMS[k][0])) for k in keep) and ntiles > 0 and ms > 0
        ab.adlbr_batch_step(b, 4)
        t.cuda.synchronize()
        for k, (u, r) in enumerate(zip(us, ref)):
            err = (u - r).abs().max().item() / r.abs().max().item()
            assert err <= 1e-6, (keep[k], err)
    finally:
        if b:
            ab.adlbr_batch_destroy(b)
        for h in hs:
            ab.adlbr_stencils_destroy(h)


def test_batch_matches_oracle():
    t = torch()
    hs, us, dts, seen = _setup()
    u0 = [u.double().cpu().numpy() for u in us]
    b = None
    try:
        stencils = [export(h, shape, wt) for h, (shape, _, wt, _) in zip(hs, ITEMS)]
        b = ab.adlbr_batch_create(hs, us, dts)
        ab.adlbr_batch_step(b, 3)
        t.cuda.synchronize()
        out = [u.double().cpu().numpy() for u in us]
    finally:
        if b:
            ab.adlbr_batch_destroy(b)
        for h in hs:
            ab.adlbr_stencils_destroy(h)
    for k, ((shape, bc, wt, _), (oo, ow)) in enumerate(zip(ITEMS, stencils)):
        uo = oracle.step_explicit(shape, bc, oo, ow, u0[k].reshape(shape), dts[k], 3)
        err = np.abs(out[k].reshape(shape) - uo).max() / np.abs(uo).max()
        assert err <= 1e-5, (k, err)


def test_batch_rejects_bad_input():
    t = torch()
    with pytest.raises(ab.AdlbrError):
        ab.adlbr_batch_create([], [], [])
    hs, us, dts, _ = _setup()
    try:
        with pytest.raises(ab.AdlbrError):
            ab.adlbr_batch_create(hs[:1], us[:1], [-1.0])
    finally:
        for h in hs:
            ab.adlbr_stencils_destroy(h)


def test_batch_full_size_serving_workload():
    """The serving batch at its full size (64 images of sides 256-2048 and 8
    volumes of sides 64-192, 137 M points, F16 weights, FP32 u), in the launch
    configuration the bench times (autotuned shapes, graph launches): two
    batched steps equal the same steps issued item by item to 1e-6 on every
    item, and the smallest image and the smallest volume equal the oracle's
    steps on the GPU's own stencils to 1e-5."""
    t = torch()
    items = synth.batch_items()
    hs, us, dts, ref, shapes = [], [], [], [], []
    b = None
    try:
        for it in items:
            shape = it["shape"]
            if it["dim"] == 2:
                D = synth.smooth_field2d_torch(*shape, it["seed"], 1.0, it["kappa"], 16).reshape(3, -1)
            else:
                D = t.from_numpy(synth.needle_field3d(shape[0], it["seed"], kappa=it["kappa"],
                                                      dtype=np.float32).reshape(6, -1)).cuda()
            h = ab.adlbr_build_stencils(ab.grid(shape), D, ab.F32, ab.F16)
            hs.append(h)
            del D
            dts.append(1.0 / ab.adlbr_stencils_max_diag(h))
            us.append(t.rand(int(np.prod(shape)), device="cuda",
                             generator=t.Generator(device="cuda").manual_seed(it["seed"])))
            ref.append(us[-1].clone())
            shapes.append(shape)
        small2 = min((k for k, s in enumerate(shapes) if len(s) == 2), key=lambda k: np.prod(shapes[k]))
        small3 = min((k for k, s in enumerate(shapes) if len(s) == 3), key=lambda k: np.prod(shapes[k]))
        u0 = {k: us[k].double().cpu().numpy() for k in (small2, small3)}
        for h, u, d in zip(hs, ref, dts):
            scratch = t.empty(ab.adlbr_step_scratch_bytes(h, ab.F32), dtype=t.uint8, device="cuda")
            ab.adlbr_step_explicit(h, u, scratch, ab.F32, d, 2)
        b = ab.adlbr_batch_create(hs, us, dts, autotune=True)
        assert ab.adlbr_batch_config(b)[2] == sum(int(np.prod(s)) for s in shapes)
        ab.adlbr_batch_step(b, 2)
        t.cuda.synchronize()
        for k, (u, r) in enumerate(zip(us, ref)):
            err = (u - r).abs().max().item() / r.abs().max().item()
            assert err <= 1e-6, (k, shapes[k], err)
        for k in (small2, small3):
            oo, ow = export(hs[k], shapes[k], ab.F16)
            uo = oracle.step_explicit(shapes[k], ab.NEUMANN, oo, ow, u0[k].reshape(shapes[k]), dts[k], 2)
            out = us[k].double().cpu().numpy().reshape(shapes[k])
            err = np.abs(out - uo).max() / np.abs(uo).max()
            assert err <= 1e-5, (k, shapes[k], err)
    finally:
        if b:
            ab.adlbr_batch_destroy(b)
        for h in hs:
            ab.adlbr_stencils_destroy(h)
