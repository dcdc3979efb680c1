"""The bounds-checked debug variant of the tensor-core sweep compiles (no GPU):
nvcc for sm_103a with -DSSV_BOUNDS_CHECK on the sweep's translation unit."""
import os
import shutil
import subprocess

import pytest

from paper_1708_06290_gb300 import build


def test_bounds_checked_sweep_compiles(tmp_path):
    nvcc = build._nvcc()
    if shutil.which(nvcc) is None and not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(build.SRC_DIR, "solve_tc.cu")
    cmd = [nvcc] + build.ARCH + build.NVCC_FLAGS + build.CHECK_FLAGS + [
        "-c", src, "-o", str(tmp_path / "solve_tc_check.o")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
