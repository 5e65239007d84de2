"""The double-float arithmetic of the FP64-emulating mode (csrc/dfloat.cuh) against
exact quadruple-precision results: builds tests/dfloat_check.cu for the host with nvcc
(no GPU involved) and runs it."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2312_02898_b300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="nvcc not available")
def test_double_float_operations_within_their_published_bounds(tmp_path):
    exe = tmp_path / "dfloat_check"
    subprocess.check_call([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O2", "-I", CSRC,
                           os.path.join(HERE, "dfloat_check.cu"), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
