"""Checkpoint and resume of long CED runs (paper_1301_3925_gb300.ced_run):
the host logic on the CPU with a stand-in stepper, and on the GPU a run
interrupted and resumed against one run straight through."""
import os

import numpy as np
import pytest

import synth


def _counter_stepper(fail_at=None):
    """u <- u + 1 per step (on a CPU tensor); raises before step fail_at."""
    state = {"done": 0}

    def step(u, n):
        for _ in range(n):
            if fail_at is not None and state["done"] + 1 == fail_at:
                raise RuntimeError("interrupted")
            u.add_(1.0)
            state["done"] += 1
    return step


def test_resume_after_interruption(tmp_path):
    import torch
    from paper_1301_3925_gb300 import ced_run
    path = str(tmp_path / "run.npz")
    u = torch.zeros((4, 6), dtype=torch.float32)
    with pytest.raises(RuntimeError):
        ced_run.run(u, 10, checkpoint=path, every=3, stepper=_counter_stepper(fail_at=8))
    u_saved, done, _ = ced_run.load(path)
    assert done == 6 and np.all(u_saved == 6.0)       # the last full chunk before the failure
    v = torch.full((4, 6), -5.0)                       # overwritten by the checkpoint
    assert ced_run.run(v, 10, checkpoint=path, every=3, stepper=_counter_stepper()) == 10
    assert torch.all(v == 10.0)
    assert ced_run.load(path)[1] == 10
    assert not os.path.exists(path + ".tmp.npz")


def test_checkpoint_refuses_other_runs(tmp_path):
    import torch
    from paper_1301_3925_gb300 import ced_run
    path = str(tmp_path / "run.npz")
    u = torch.zeros((3, 3))
    ced_run.run(u, 2, checkpoint=path, stepper=_counter_stepper())
    with pytest.raises(ValueError):
        ced_run.run(torch.zeros((3, 4)), 4, checkpoint=path, stepper=_counter_stepper())
    with pytest.raises(ValueError):
        ced_run.run(torch.zeros((3, 3)), 4, checkpoint=path, dt=0.01, stepper=_counter_stepper())
    with pytest.raises(ValueError):
        ced_run.run(torch.zeros((3, 3)), 1, checkpoint=path, stepper=_counter_stepper())


@pytest.mark.gpu
def test_gpu_run_resumed_equals_straight_run(tmp_path):
    """Six CED steps on a 256^2 crop of the fingerprint image, straight and as
    3 + 3 with a checkpoint in between: equal to FP32 rounding (the operator's
    atomic additions may change the last bits from run to run)."""
    import torch
    from paper_1301_3925_gb300 import ced_run
    img = synth.fingerprint(512, 3)[:256, :256].astype(np.float32)
    a = torch.from_numpy(img).cuda()
    ced_run.run(a, 6)
    path = str(tmp_path / "ced.npz")
    b = torch.from_numpy(img).cuda()
    ced_run.run(b, 3, checkpoint=path)
    c = torch.zeros_like(b)
    ced_run.run(c, 6, checkpoint=path)
    torch.cuda.synchronize()
    err = (a - c).abs().max().item() / a.abs().max().item()
    assert err <= 1e-5, err
    assert ced_run.load(path)[1] == 6
