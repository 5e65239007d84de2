"""The generated code of the two-jet channels with one light-quark line, of the
four-quark channels and of g g > t t~ g g (its FP64 default variant, with pending
colour sums), run on the host:
nvcc compiles tests/generated_host_check.cu for the host around one generated process
header (its precompute, jamps and colour_sum in FP64, the computation the kernels perform
per event) and the result must equal the FP64 oracle within 1e-12, with and without the
top width and with the zero-width t-channel option.  The headers come from the product's
generator (gen/), written to a temporary directory; no GPU is involved."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2312_02898_b300", "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
# (process, tag, jamps variant): g g > t t~ g g in its FP64 default variant (twelve pending
# colour sums)
CASES = [("u u~ > t t~ g g", "qqttgg", 0), ("g u > t t~ u g", "gqttqg", 0), ("g g > t t~ u u~", "ggttqqx", 0),
         ("u d~ > t t~ u d~", "udxttudx", 0), ("u~ u > t t~ u u~", "uxuttuux", 0), ("g g > t t~ g g", "ggttgg", 9)]


@pytest.mark.skipif(not (os.path.exists(NVCC) or shutil.which("nvcc")), reason="nvcc not available")
@pytest.mark.parametrize("process,tag,variant", CASES)
def test_generated_code_on_the_host(oracle_mod, tmp_path, process, tag, variant):
    from paper_2312_02898_b300.gen import emit
    gen = tmp_path / "generated"
    emit.generate_all(str(gen), processes=[process])
    # the header includes "../helas.cuh": place it beside a copy of the routines
    shutil.copy(os.path.join(CSRC, "helas.cuh"), tmp_path / "helas.cuh")
    exe = tmp_path / "check"
    subprocess.check_call([NVCC, "-x", "cu", "-std=c++17", "-O1", f"-DPROC_HEADER=\"{gen}/proc_{tag}.cuh\"",
                           f"-DPROC=proc_{tag}", f"-DVARIANT={variant}", os.path.join(HERE, "generated_host_check.cu"), "-o", str(exe)])
    n = 40
    mom, _, _, _ = ps.make_batch(process, n, seed=21)
    for wt, zwt in ((0.0, 0), (1.4915, 0), (1.4915, 1)):
        r = subprocess.run([str(exe), str(n), repr(wt), str(zwt), "0.118"], input=np.ascontiguousarray(mom).tobytes(),
                           capture_output=True, timeout=300)
        assert r.returncode == 0, r.stderr
        got = np.array([float(x) for x in r.stdout.split()])
        ref = oracle_mod.me(process, mom, params=oracle_mod.Params(wt=wt, zero_width_tchan=zwt))["me"]
        rel = np.abs(got / ref - 1)
        print(f"{process} wt={wt} zwt={zwt}: max rel {rel.max():.2e}")
        assert rel.max() <= 1e-12
