"""The packed FP32 routines (two events per thread, csrc/fx2.cuh) equal the scalar
routines of csrc/helas.cuh lane by lane.  Builds tests/packed_algebra_check.cu for the
host with nvcc (no GPU involved) and runs it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2312_02898_b300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="nvcc not available")
def test_packed_routines_equal_scalar_routines_lane_by_lane(tmp_path):
    exe = tmp_path / "packed_algebra_check"
    subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "packed_algebra_check.cu"),
                           "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
