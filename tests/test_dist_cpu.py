"""The multi-rank path of bench.py on CPU: two gloo ranks launched the way
torchrun launches them (RANK / WORLD_SIZE / MASTER_* in the environment).
Checks the per-rank sharding (distinct images), the barrier, the max over
ranks of the step time and the whole-job throughput."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import bench
ws, rank, local = bench.init_dist("gloo")
seed = bench.rank_seed(rank)
import synth
img = synth.fingerprint(64, seed)
bench.barrier(ws)
ms = 10.0 + 5.0 * rank          # a slower rank 1
mx = bench.allmax(ws, ms)
val = bench.job_value(ws, 4096 * 4096, mx)
print(json.dumps({"rank": rank, "ws": ws, "seed": seed, "sum": float(img.sum()), "max_ms": mx, "value": val}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    script = tmp_path / "worker.py"
    script.write_text(WORKER)
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT="29517")
        procs.append(subprocess.Popen([sys.executable, str(script), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=180)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    a, b = sorted(outs, key=lambda d: d["rank"])
    assert a["ws"] == b["ws"] == 2
    assert a["seed"] != b["seed"] and a["sum"] != b["sum"]          # independent units
    assert a["max_ms"] == b["max_ms"] == 15.0                       # the slowest rank
    assert abs(a["value"] - 2 * 4096 * 4096 / 15e-3 / 1e9) < 1e-9    # all ranks' points
