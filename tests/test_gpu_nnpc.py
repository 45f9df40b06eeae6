"""The learned preconditioner (not in the paper): M(r) against the FP64
oracle, solver-generated training pairs, flexible PCG with the Galerkin step
length, the plain-CG fallback, and the gain of the trained network over the
solver without it."""
import numpy as np
import pytest

import oracle
import synth
from oracle import unet as ou
from paper_1301_3925_gb300 import adlbr as ab
from paper_1301_3925_gb300 import nn

from gpu_helpers import build, dev, torch

pytestmark = pytest.mark.gpu


def _problem(shape, seed, kmax=50.0):
    t = torch()
    D = synth.smooth_field2d(*shape, seed=seed, kappa_min=1, kappa_max=kmax, lattice=8)
    h, seen, _ = build(D, shape, t.float32, ab.F32)
    oo, ow, st, _ = oracle.build2d(*seen.reshape(3, -1))
    assert np.all(st == 0)
    dmax = ab.adlbr_stencils_max_diag(h)
    diag = oracle.diag(shape, oracle.NEUMANN, oo, ow)
    assert abs(dmax - diag.max()) <= 1e-5 * diag.max()
    dt = 200.0 / diag.max()
    return h, oo, ow, diag, dt


def _params(seed, scale_out=1.0):
    P = ou.n_params(nn.NF)
    th = ou.init_params(nn.NF, seed) + 0.02 * np.random.default_rng(seed).normal(size=P)
    th[-17:] *= scale_out   # output layer (16 weights + bias)
    return th


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_precondition_matches_oracle(tensor_cores):
    t = torch()
    shape = (64, 96)
    h, oo, ow, diag, dt = _problem(shape, 5)
    theta = _params(1)
    pc = nn.Preconditioner(dev(theta, t.float32), shape[1], shape[0], tensor_cores=tensor_cores)
    try:
        r = synth.u_uniform(shape, 6) - 0.5
        rd = dev(r.ravel(), t.float32)
        z = t.empty_like(rd)
        ab.adlbr_nn_precondition(h, pc.desc, dt, rd, z)
        zg = z.double().cpu().numpy().reshape(shape)
    finally:
        pc.close()
        ab.adlbr_stencils_destroy(h)
    th32 = theta.astype(np.float32).astype(np.float64)
    r32 = r.astype(np.float32).astype(np.float64)
    zo = ou.precondition(th32, oo, ow, dt, diag, r32)
    if not tensor_cores:
        assert np.abs(zg - zo).max() <= 2e-4 * np.abs(zo).max()
        return
    # BF16 network: the Jacobi part r / d stays FP32; the error is bounded by
    # the forward's tolerance on the network's own term s P(y)
    net_part = zo - r32 / (1.0 + dt * diag)
    assert np.abs(zg - zo).max() <= 3e-2 * np.abs(net_part).max() + 2e-4 * np.abs(zo).max()


def test_training_pairs_match_oracle_features():
    t = torch()
    shape = (64, 64)
    h, oo, ow, diag, dt = _problem(shape, 7)
    try:
        b = dev(synth.u_uniform(shape, 8).ravel(), t.float32)
        feats, targets = nn.generate_pairs(h, b, dt, every=4, max_pairs=6)
        assert feats.shape[0] == 6
        bs = b.double().cpu().numpy().reshape(shape)
    finally:
        ab.adlbr_stencils_destroy(h)
    # pair 0 is the initial residual r0 = b - (I + dt A) b = -dt A b
    r0 = -dt * oracle.apply(shape, oracle.NEUMANN, oo, ow, bs)
    fo, s = ou.coarse_features(oo, ow, dt, r0)
    fg = feats[0].double().cpu().numpy()
    assert np.abs(fg - fo).max() <= 1e-4 * max(1.0, np.abs(fo).max())
    xs, _, _ = oracle.cg(shape, oracle.NEUMANN, oo, ow, bs, bs, dt, rtol=1e-10)
    to = ou.training_target(oo, ow, dt, diag, r0, xs - bs)
    tg = targets[0].double().cpu().numpy()
    assert np.abs(tg - to).max() <= 1e-2 * np.abs(to).max() + 1e-6


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_fcg_converges_to_cg_solution(tensor_cores):
    t = torch()
    shape = (96, 112)
    h, oo, ow, diag, dt = _problem(shape, 3)
    theta = _params(2, scale_out=0.001)
    pc = nn.Preconditioner(dev(theta, t.float32), shape[1], shape[0], tensor_cores=tensor_cores)
    try:
        b = dev(synth.u_uniform(shape, 3).ravel(), t.float32)
        x1 = b.clone()
        it_cg, rel_cg = ab.adlbr_step_implicit(h, b, x1, dt, 1e-6, 4000)
        x2 = b.clone()
        it_nn, rel_nn = ab.adlbr_step_implicit(h, b, x2, dt, 1e-6, 4000, precond=1, nn=pc.desc)
        d = (x1 - x2).abs().max().item()
    finally:
        pc.close()
        ab.adlbr_stencils_destroy(h)
    # both stop by the same rule (refinement rounds from the FP64 true
    # residual): the same bound as CG's, at the FP32 floor of x
    assert rel_cg <= 2e-5 and rel_nn <= 2e-5, (rel_cg, rel_nn)
    assert rel_nn <= 4.0 * rel_cg + 1e-6, (rel_cg, rel_nn)
    assert d <= 2e-4, d


def test_trained_preconditioner_report():
    """Trains the network on the solver's own (residual, error) pairs, then
    solves a held-out right-hand side three ways: plain CG, flexible PCG with
    the Jacobi part alone (output layer zeroed) and flexible PCG with the
    trained network (its correction taken with the Galerkin step length).
    Asserted: the training loss falls, every solve reaches the CG solution,
    and the trained network needs fewer iterations than the same solver
    without it (its gain over the method without it)."""
    t = torch()
    shape = (192, 192)
    h, oo, ow, diag, dt = _problem(shape, 11)
    try:
        b = dev(synth.u_uniform(shape, 12).ravel(), t.float32)
        # training problems: other right-hand sides on the same stencils;
        # pairs from CG, then from the preconditioned solver itself
        rhs = [dev(synth.u_uniform(shape, 100 + k).ravel(), t.float32) for k in range(3)]
        params, log = nn.fit(h, rhs, dt, rounds=3, steps=(1500, 700, 700), crop=48)
        for r in log:
            print("round", r["round"], "pairs", r["pairs"], "loss", r["loss"][0], r["loss"][-1])
        assert log[0]["loss"][-1][1] < 0.25 * log[0]["loss"][0][1], log[0]
        jac = params.clone()
        jac[-17:] = 0.0                       # output layer (16 weights + bias): M(r) = r / d
        x1 = b.clone()
        it_cg, _ = ab.adlbr_step_implicit(h, b, x1, dt, 1e-6, 4000)
        its = {}
        for name, th in (("jacobi", jac), ("trained", params)):
            pc = nn.Preconditioner(th, shape[1], shape[0])
            try:
                x2 = b.clone()
                its[name] = ab.adlbr_step_implicit(h, b, x2, dt, 1e-6, 4000, precond=1,
                                                   nn=pc.desc)
            finally:
                pc.close()
            its[name] += ((x1 - x2).abs().max().item(),)
    finally:
        ab.adlbr_stencils_destroy(h)
    print("iterations: CG %d, Jacobi FCG %d, trained-network FCG %d"
          % (it_cg, its["jacobi"][0], its["trained"][0]))
    for name, (it, rel, d) in its.items():
        assert rel <= 2e-5 and d <= 2e-4, (name, it, rel, d)
    assert its["trained"][0] < its["jacobi"][0], its


def test_badly_scaled_network_stays_near_jacobi():
    """An untrained network with an output layer 50 times too large: the
    Galerkin step length shrinks its correction, so the solve converges in
    about the iterations of Jacobi-preconditioned FCG, without the fallback."""
    t = torch()
    shape = (96, 112)
    h, oo, ow, diag, dt = _problem(shape, 3)
    pcs = []
    try:
        b = dev(synth.u_uniform(shape, 3).ravel(), t.float32)
        x1 = b.clone()
        it_cg, _ = ab.adlbr_step_implicit(h, b, x1, dt, 1e-6, 4000)
        its = {}
        for name, scale in (("jacobi", 0.0), ("bad", 50.0)):
            pcs.append(nn.Preconditioner(dev(_params(4, scale_out=scale), t.float32), shape[1], shape[0]))
            x2 = b.clone()
            its[name] = ab.adlbr_step_implicit(h, b, x2, dt, 1e-6, 4000, precond=1, nn=pcs[-1].desc)
            assert ab.adlbr_last_fallback() == 0
            assert (x1 - x2).abs().max().item() <= 2e-4
    finally:
        for pc in pcs:
            pc.close()
        ab.adlbr_stencils_destroy(h)
    print("CG %d, Jacobi FCG %d, bad-network FCG %d" % (it_cg, its["jacobi"][0], its["bad"][0]))
    assert its["bad"][0] <= 1.25 * its["jacobi"][0] + 5, its
    assert its["bad"][1] <= 2e-5


def test_non_finite_network_falls_back_to_cg():
    """A network whose output is not finite (a NaN output bias, made on the
    host) spoils the flexible solve; the solver detects it and finishes with
    plain CG at the same residual (iterations then count both phases)."""
    t = torch()
    shape = (96, 112)
    h, oo, ow, diag, dt = _problem(shape, 3)
    theta = _params(4)
    theta[-1] = np.nan
    pc = nn.Preconditioner(dev(theta, t.float32), shape[1], shape[0])
    try:
        b = dev(synth.u_uniform(shape, 3).ravel(), t.float32)
        x1 = b.clone()
        it_cg, _ = ab.adlbr_step_implicit(h, b, x1, dt, 1e-6, 4000)
        x2 = b.clone()
        it_nn, rel = ab.adlbr_step_implicit(h, b, x2, dt, 1e-6, 4000, precond=1, nn=pc.desc)
        fb = ab.adlbr_last_fallback()
        d = (x1 - x2).abs().max().item()
    finally:
        pc.close()
        ab.adlbr_stencils_destroy(h)
    print("CG %d, non-finite network solve %d (fallback %d)" % (it_cg, it_nn, fb))
    assert fb == 1
    assert it_nn >= it_cg
    assert rel <= 1e-5 and d <= 2e-4, (rel, d)
