"""Training of the learned preconditioner (not in the paper).

The network and its training run in the library's CUDA kernels (forward,
backward, Adam, MSE gradient); this module only orchestrates calls through
the C ABI and picks the random crops of a minibatch (a data copy).

Data: (residual, error) pairs that the implicit solver generates
(adlbr_nn_training_pairs): the coarse features of the CG residual r_k and the
target R((x* - x_k - r_k / d) / rms(r_k)) that the network should output.
"""
import numpy as np

from . import adlbr as ab

NF = 25        # input channels (16 residual values per 4x4 block + 9 stencil means)
RF = 4         # restriction factor of the preconditioner


def generate_pairs(h, rhs, dt, rtol=1e-6, maxit=4000, every=4, max_pairs=48, precond=None):
    """Solver-generated pairs for the stencils h: returns (feats [n,NF,Hc,Wc],
    targets [n,Hc,Wc]) as CUDA tensors.  precond (a Preconditioner) makes the
    recording solve the preconditioned one, so the pairs follow its residuals."""
    import torch

    g = ab.adlbr_stencils_grid(h)
    nx, ny = int(g.n[0]), int(g.n[1])
    Hc, Wc = ny // RF, nx // RF
    feats = torch.empty((max_pairs, NF, Hc, Wc), dtype=torch.float32, device="cuda")
    targets = torch.empty((max_pairs, Hc, Wc), dtype=torch.float32, device="cuda")
    xbuf = torch.empty(nx * ny, dtype=torch.float32, device="cuda")
    n = ab.adlbr_nn_training_pairs(h, rhs, dt, rtol, maxit, every, max_pairs,
                                   precond.desc if precond is not None else None, feats, targets,
                                   xbuf)
    return feats[:n], targets[:n]


def fit(h, rhs_list, dt, rounds=3, steps=(1500, 600, 600), every=3, max_pairs=40, batch=8,
        crop=64, lr=2e-3, seed=0, c=(16, 32, 64)):
    """Train on pairs from CG, then (rounds - 1 times) add pairs recorded along
    the preconditioned solver with the current network and keep training.
    Returns (params, log)."""
    import torch

    g = ab.adlbr_stencils_grid(h)
    nx, ny = int(g.n[0]), int(g.n[1])
    F, T = [], []
    for rhs in rhs_list:
        f, t = generate_pairs(h, rhs, dt, every=every, max_pairs=max_pairs)
        F.append(f)
        T.append(t)
    params, log = None, []
    for rd in range(rounds):
        feats, targets = torch.cat(F), torch.cat(T)
        params, losses = train(feats, targets, steps=steps[min(rd, len(steps) - 1)], batch=batch,
                               crop=crop, lr=lr, seed=seed + rd, c=c, params=params)
        log.append({"round": rd, "pairs": int(feats.shape[0]), "loss": losses})
        if rd == rounds - 1:
            break
        pc = Preconditioner(params, nx, ny, c)
        try:
            for rhs in rhs_list:
                f, t = generate_pairs(h, rhs, dt, every=every, max_pairs=max_pairs, precond=pc)
                F.append(f)
                T.append(t)
        finally:
            pc.close()
    return params, log


def init_params(n_params, layer_shapes, seed):
    """He-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    out = np.zeros(n_params, np.float32)
    o = 0
    for co, ci, k in layer_shapes:
        nw = co * ci * k * k
        out[o:o + nw] = rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), nw)
        o += nw + co
    assert o == n_params
    return out


def layer_shapes(cin=NF, c1=16, c2=32, c3=64):
    return [(c1, cin, 3), (c1, c1, 3), (c2, c1, 3), (c2, c2, 3), (c3, c2, 3), (c3, c3, 3),
            (c2, c3 + c2, 3), (c2, c2, 3), (c1, c2 + c1, 3), (c1, c1, 3), (1, c1, 1)]


def train(feats, targets, steps=400, batch=8, crop=64, lr=2e-3, seed=0, c=(16, 32, 64), log_every=50,
          params=None):
    """Adam on random crops of the pairs (continuing from params if given);
    returns (params, losses)."""
    import torch

    n, _, Hc, Wc = feats.shape
    crop = min(crop, Hc, Wc) // 4 * 4
    net = ab.adlbr_unet_create(NF, c[0], c[1], c[2], batch, crop, crop)
    try:
        P = ab.adlbr_unet_num_params(net)
        if params is None:
            params = torch.from_numpy(init_params(P, layer_shapes(NF, *c), seed)).cuda()
        else:
            params = params.clone()
        grads = torch.zeros_like(params)
        m = torch.zeros_like(params)
        v = torch.zeros_like(params)
        xb = torch.empty((batch, NF, crop, crop), dtype=torch.float32, device="cuda")
        tb = torch.empty((batch, crop, crop), dtype=torch.float32, device="cuda")
        yb = torch.empty((batch, crop, crop), dtype=torch.float32, device="cuda")
        gy = torch.empty_like(yb)
        rng = np.random.default_rng(seed + 1)
        losses = []
        for t in range(1, steps + 1):
            idx = rng.integers(0, n, batch)
            oy = rng.integers(0, Hc - crop + 1, batch)
            ox = rng.integers(0, Wc - crop + 1, batch)
            for b in range(batch):
                xb[b].copy_(feats[idx[b], :, oy[b]:oy[b] + crop, ox[b]:ox[b] + crop])
                tb[b].copy_(targets[idx[b], oy[b]:oy[b] + crop, ox[b]:ox[b] + crop])
            ab.adlbr_unet_forward(net, params, xb, yb)
            want = (t % log_every == 0) or t == 1 or t == steps
            loss = ab.adlbr_mse_grad(yb, tb, yb.numel(), gy, want_loss=want)
            if want:
                losses.append((t, loss))
            ab.adlbr_unet_backward(net, params, gy, grads)
            ab.adlbr_adam_step(params, grads, m, v, P, lr, 0.9, 0.999, 1e-8, t)
        return params, losses
    finally:
        ab.adlbr_unet_destroy(net)


class Preconditioner:
    """The trained network instantiated for a full-size grid (batch 1); its
    forward convolutions run on the tensor cores unless tensor_cores=False
    (BF16 operands, FP32 accumulation; 0.245 ms against 0.97 ms for the FP32
    kernels at 512^2)."""

    def __init__(self, params, nx, ny, c=(16, 32, 64), tensor_cores=True):
        self.net = ab.adlbr_unet_create(NF, c[0], c[1], c[2], 1, ny // RF, nx // RF)
        if tensor_cores:
            ab.adlbr_unet_set_tensor_cores(self.net, True)
        self.params = params
        self.desc = ab.nn_precond(self.net, params)

    def close(self):
        if self.net:
            ab.adlbr_unet_destroy(self.net)
            self.net = None
