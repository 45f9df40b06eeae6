"""Long coherence-enhancing-diffusion runs with checkpoints (Sec. 4.4, Eq.
parabolique: tensor stage, AD-LBR stencils, one explicit step, repeated).

The paper's CED loop keeps no state besides u: every step rebuilds D(u) and
the stencils from the current image.  So a checkpoint is the image and the
number of steps done; a run started with an existing checkpoint resumes from
it and rebuilds the stencils from u, exactly as an uninterrupted run does at
that step.

    h = run(u, steps=500, checkpoint="ced.npz", every=50)

Every step runs in the library (adlbr_ced_step); this module only moves u
between the device and the checkpoint file.  The file is written to a
temporary name and renamed, so an interrupted write leaves the previous
checkpoint intact.
"""
import os

import numpy as np

from . import adlbr as ab

PARAMS = ("sigma", "rho", "alpha", "C", "dt")


def _save(path, u_host, done, params):
    tmp = path + ".tmp.npz"
    np.savez(tmp, u=u_host, step=np.int64(done), **{k: np.float64(v) for k, v in params.items()})
    os.replace(tmp, path)


def load(path):
    """(u as a numpy array, steps done, the run's parameters) of a checkpoint."""
    with np.load(path) as z:
        return z["u"].copy(), int(z["step"]), {k: float(z[k]) for k in PARAMS}


def run(u, steps, sigma=1.0, rho=4.0, alpha=1e-4, C=1e-5, dt=0.02, w_t=ab.F16, checkpoint=None,
        every=0, stepper=None, stream=None):
    """Advances u (a CUDA float32 tensor of shape (ny, nx) or (nz, ny, nx), in
    place) to `steps` CED steps in total.

    checkpoint: path of an .npz file.  If it exists, u, the steps done and the
    parameters are taken from it (its parameters must equal these, and its
    image must have u's shape), and the run continues from there.  Every
    `every` steps (0: only at the end) and at the end the current u and the
    step count are written to it.
    stepper: None for the library's adlbr_ced_step; a test may pass a
    function (u, nsteps) -> None instead.
    Returns the number of steps done (= steps)."""
    import torch
    params = dict(sigma=sigma, rho=rho, alpha=alpha, C=C, dt=dt)
    done = 0
    if checkpoint and os.path.exists(checkpoint):
        u0, done, p0 = load(checkpoint)
        if tuple(u0.shape) != tuple(u.shape):
            raise ValueError("checkpoint image %s does not match u %s" % (u0.shape, tuple(u.shape)))
        if any(abs(p0[k] - params[k]) > 0 for k in PARAMS):
            raise ValueError("checkpoint parameters %s differ from %s" % (p0, params))
        if done > steps:
            raise ValueError("checkpoint is at step %d, beyond the %d asked for" % (done, steps))
        u.copy_(torch.from_numpy(u0.astype(np.float32)))
    h = None
    scratch = None
    if stepper is None:
        g = ab.grid(tuple(u.shape))
        scratch = torch.empty(ab.adlbr_ced_scratch_bytes(g), dtype=torch.uint8, device=u.device)

        def stepper(v, n):
            nonlocal h
            h = ab.adlbr_ced_step(h, g, v, scratch, sigma, rho, alpha, C, dt, n, w_t, stream)
    try:
        chunk = every if every > 0 else max(steps - done, 1)
        while done < steps:
            n = min(chunk, steps - done)
            stepper(u, n)
            done += n
            if checkpoint and (every > 0 or done == steps):
                _save(checkpoint, u.detach().cpu().numpy(), done, params)
    finally:
        if h is not None:
            ab.adlbr_stencils_destroy(h)
    return done
