"""me_compute_noalloc: the no-allocation entry point for callers that cannot let the
library allocate device memory (a framework that owns all device memory through its own
pool, or a caller under a hard memory cap or latency budget).

It must give what me_compute gives, on two calls in a row (the fixed scratch keeps the
previous call's contents, which must not leak into the next result), and it must turn
away a batch whose scratch would not fit the fixed array with a clear error.  This file
is collected last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-5}


def _entry(m):
    f = m.lib.me_compute_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 8
    f.restype = ctypes.c_int
    return f


def _dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


@pytest.mark.parametrize("process,nevt,precision", [("g g > t t~ g g", 3000, "fp64"),
                                                    ("g g > t t~ g g", 5000, "mixed"),
                                                    ("g g > t t~ g", 20000, "fp32")])
def test_noalloc_matches_me_compute_on_two_calls(process, nevt, precision):
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement(process, precision=precision)
    f = _entry(m)
    stream = torch.cuda.current_stream()
    for seed in (31, 32):
        mom, a, rh, rc = _dev(*ps.make_batch(process, nevt, seed=seed, alphas="uniform"))
        me_ref, sh_ref, sc_ref = m.compute(mom, a, rh, rc, stream=stream)
        me = torch.full((nevt,), float("nan"), dtype=torch.float64, device="cuda")
        sh = torch.full((nevt,), -1, dtype=torch.int32, device="cuda")
        sc = torch.full((nevt,), -1, dtype=torch.int32, device="cuda")
        rc_ = f(m.handle, nevt, mom.data_ptr(), a.data_ptr(), rh.data_ptr(), rc.data_ptr(), me.data_ptr(),
                sh.data_ptr(), sc.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc_ == 0, m.lib.me_last_error(m.handle)
        torch.cuda.synchronize()
        rel = (me / me_ref - 1).abs().max().item()
        assert rel <= TOL[precision], (seed, rel)
        assert torch.equal(sh, sh_ref) and torch.equal(sc, sc_ref)


def test_noalloc_rejects_batches_beyond_the_fixed_scratch():
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement("g g > t t~ g g", precision="fp64")
    f = _entry(m)
    nevt = 200000
    mom, a, rh, rc = _dev(*ps.make_batch("g g > t t~ g g", nevt, seed=33, alphas="uniform"))
    me = torch.empty(nevt, dtype=torch.float64, device="cuda")
    sh = torch.empty(nevt, dtype=torch.int32, device="cuda")
    sc = torch.empty(nevt, dtype=torch.int32, device="cuda")
    rc_ = f(m.handle, nevt, mom.data_ptr(), a.data_ptr(), rh.data_ptr(), rc.data_ptr(), me.data_ptr(),
            sh.data_ptr(), sc.data_ptr(), None)
    assert rc_ == -1
    msg = m.lib.me_last_error(m.handle).decode()
    assert "fixed" in msg and "scratch" in msg and "33554432" in msg
    # the limit it states is exact: that many events are accepted, one more is not
    limit = int(msg.split("at most ")[1].split()[0])
    assert 0 < limit < nevt
    for n, want in ((limit, 0), (limit + 1, -1)):
        rc_ = f(m.handle, n, mom.data_ptr(), a.data_ptr(), rh.data_ptr(), rc.data_ptr(), me.data_ptr(),
                sh.data_ptr(), sc.data_ptr(), None)
        assert rc_ == want, (n, m.lib.me_last_error(m.handle))
    torch.cuda.synchronize()
