"""The bounds-checked build of the library (libadlbr_checked.so) runs the
GPU parity suites of the stencil builds, the operator in both forms, the
A-NN scheme, the CED pipeline (2D, and 3D with both tensors), the spectral
study's block kernels and the batched step with every guard on:
each of those tests compares with the oracle as in the normal build, and
any failed index or stencil-radius check would surface as ADLBR_E_INTERNAL
from adlbr_stencils_check or adlbr_stencils_destroy (the tests destroy every
handle they make)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_gpu_stencils.py", "tests/test_gpu_apply.py", "tests/test_gpu_gather.py",
          "tests/test_gpu_ann.py", "tests/test_gpu_ced.py", "tests/test_gpu_batch.py",
          "tests/test_gpu_ced3d.py", "tests/test_gpu_spectral.py"]


@pytest.mark.gpu
def test_parity_suites_under_bounds_checked_build():
    from paper_1301_3925_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, ADLBR_BOUNDS_CHECK="1")
    v = subprocess.run([sys.executable, "-c", "from paper_1301_3925_gb300 import adlbr; print(adlbr.adlbr_version())"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert v.returncode == 0, v.stderr
    assert "bounds-checked" in v.stdout
    # the full-size cases repeat the small ones' code paths at the bench's sizes;
    # they are left to the normal build
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "-k", "not full_size"] + SUITES,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
