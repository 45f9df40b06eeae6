"""The bounds-checked build (-DADLBR_BOUNDS_CHECK) compiles, and every
compute entry point and stage of the library opens an NVTX range (no GPU
needed).  The checked library itself runs the GPU parity suites in
test_gpu_checked_build.py."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1301_3925_gb300", "csrc")


@pytest.mark.parametrize("tu", ["build2d.cu", "pull.cu"])
def test_checked_translation_unit_compiles(tu):
    """The two units whose checks differ most from the normal build: the 2D
    build (stencil-radius check) and the gather operator (table indices)."""
    from paper_1301_3925_gb300 import build
    with tempfile.TemporaryDirectory() as d:
        cmd = [build._nvcc()] + build._flags(checked=True) + ["-c", os.path.join(CSRC, tu), "-o",
                                                              os.path.join(d, "t.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]


def _ranges(fn):
    return set(re.findall(r'ADLBR_NVTX\("([^"]+)"\)', open(os.path.join(CSRC, fn)).read()))


def test_nvtx_ranges_cover_entry_points_and_stages():
    api = _ranges("api.cu")
    for name in ["adlbr_build_stencils_scheme", "adlbr_apply", "adlbr_step_explicit", "adlbr_step_implicit",
                 "adlbr_ced_tensor", "adlbr_ced_stencils", "adlbr_ced_step", "adlbr_nn_precondition"]:
        assert name in api, name
    assert "adlbr_batch_step" in _ranges("batch.cu")
    assert {"adlbr_unet_forward", "adlbr_unet_backward"} <= _ranges("unet.cu")
    # stages: tensor (2D and 3D), build (2D, 3D, A-NN), operator (scatter and gather)
    assert "tensor" in _ranges("ced.cu") and "tensor" in _ranges("ced3d.cu")
    assert all("build" in _ranges(f) for f in ["build2d.cu", "build3d.cu", "ann.cu"])
    assert "operator" in _ranges("apply.cu") and "operator" in _ranges("pull.cu")


def test_binding_selects_checked_library():
    r = subprocess.run(["python", "-c", "from paper_1301_3925_gb300 import adlbr; print(adlbr.LIB_PATH)"],
                       cwd=ROOT, capture_output=True, text=True,
                       env=dict(os.environ, ADLBR_BOUNDS_CHECK="1"))
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip().endswith("libadlbr_checked.so")
