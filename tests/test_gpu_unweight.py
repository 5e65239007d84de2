"""GPU-assisted batch unweighting against the oracle's plain hit-or-miss.  The
unweighting step takes the matrix elements as its input, so both sides get the same
GPU matrix elements and every output must agree exactly: the weight is one correctly
rounded product, the maximum and the decisions compare the same doubles."""
import numpy as np
import pytest

from paper_2312_02898_b300.phasespace import make_batch, uniforms
from oracle.unweight import unweight as oracle_unweight

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _gpu(m, me, wgt, rnd):
    import torch
    w, acc, wmax, nacc = m.unweight(_dev(me), _dev(wgt), None if rnd is None else _dev(rnd))
    torch.cuda.synchronize()
    return (w.cpu().numpy(), None if acc is None else acc.cpu().numpy(), float(wmax.item()),
            None if nacc is None else int(nacc.item()))


@pytest.fixture(scope="module")
def handle():
    from paper_2312_02898_b300.binding import MatrixElement
    return MatrixElement("g g > t t~ g g", precision="mixed")


@pytest.mark.parametrize("nevt", [1, 255, 257, 40000])
def test_matches_oracle_on_matrix_elements(handle, nevt):
    import torch
    mom, a, rh, rc = make_batch("g g > t t~ g g", nevt, seed=3, alphas="uniform")
    me_d, _, _ = handle.compute(_dev(mom), _dev(a))
    torch.cuda.synchronize()
    me = me_d.cpu().numpy()
    ev = np.arange(nevt, dtype=np.uint64)
    u = uniforms(11, ev, 0, 2)          # stand-in Jacobian x PDF factor and the hit-or-miss numbers
    wgt = 1e3 * u[:, 0] ** 3
    rnd = u[:, 1]
    w, acc, wmax, nacc = _gpu(handle, me, wgt, rnd)
    ow, oacc, owmax, onacc = oracle_unweight(me, wgt, rnd)
    np.testing.assert_array_equal(w, ow)
    assert wmax == owmax
    np.testing.assert_array_equal(acc, oacc)
    assert nacc == onacc


def test_invalid_weights_and_degenerate_batches(handle):
    me = np.array([2.0, 1.0, 4.0, 3.0, np.nan, 5.0, 1.0, 7.0])
    wgt = np.array([1.0, 3.0, 0.5, -1.0, 1.0, np.inf, 0.0, -0.0])
    rnd = np.array([0.9, 0.7, 0.4, 0.0, 0.0, 0.0, 0.0, 0.0])
    w, acc, wmax, nacc = _gpu(handle, me, wgt, rnd)
    ow, oacc, owmax, onacc = oracle_unweight(me, wgt, rnd)
    np.testing.assert_array_equal(w, ow)
    assert (wmax, nacc) == (owmax, onacc) == (3.0, 2)
    np.testing.assert_array_equal(acc, oacc)
    w, acc, wmax, nacc = _gpu(handle, np.zeros(1000), np.ones(1000), np.full(1000, 0.5))
    assert wmax == 0.0 and nacc == 0 and not acc.any()
    # the maximum alone (no random numbers)
    w, acc, wmax, nacc = _gpu(handle, np.arange(1000.0), np.full(1000, 2.0), None)
    assert wmax == 1998.0 and acc is None and nacc is None


def test_empty_batch_leaves_outputs_untouched(handle):
    import ctypes
    import torch
    x = torch.empty(0, dtype=torch.float64, device="cuda")
    wmax = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
    rc = handle.lib.me_unweight(handle.handle, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                None, None, None, ctypes.c_void_p(wmax.data_ptr()), None,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == 0 and wmax.item() == -7.0


def test_full_batch_sampled(handle):
    """one million events: the maximum and the count against the oracle on the same
    inputs (the oracle's loop takes a few seconds at this size)"""
    rng = np.random.default_rng(4)
    n = 1 << 20
    me = rng.exponential(size=n) * 1e-3
    wgt = rng.uniform(0.1, 10.0, size=n)
    rnd = rng.uniform(size=n)
    w, acc, wmax, nacc = _gpu(handle, me, wgt, rnd)
    ow, oacc, owmax, onacc = oracle_unweight(me, wgt, rnd)
    assert wmax == owmax and nacc == onacc
    np.testing.assert_array_equal(acc, oacc)


@pytest.mark.parametrize("process,precision,kappa", [("g g > t t~ g", "fp64", None), ("g g > t t~ g", "fp32", 1e-300),
                                                     ("g g > t t~ g", "fp32", None), ("g g > t t~ g g", "mixed", None),
                                                     ("e+ e- > mu+ mu-", "fp64", None)])
def test_fused_unweighting_equals_compute_then_unweight(process, precision, kappa):
    """me_compute_unweight forms the weights and the batch maximum in the matrix-element
    kernel's epilogue; its outputs equal me_compute followed by me_unweight bit for bit,
    also when the FP32 rescue pass re-evaluates every event (kappa below every event's)."""
    import torch
    from paper_2312_02898_b300 import phasespace as ps
    from paper_2312_02898_b300.binding import MatrixElement
    n = 3001 if process != "g g > t t~ g g" else 1501
    mom, a, rh, rc = ps.make_batch(process, n, seed=61, alphas="uniform")
    u = ps.uniforms(62, np.arange(n, dtype=np.uint64), 0, 2)
    wgt, rnd = u[:, 0] * 1e3, u[:, 1]
    d = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (mom, a, rh, rc, wgt, rnd)]
    kw = {} if kappa is None else {"rescue_kappa": kappa}
    m = MatrixElement(process, precision=precision, **kw)
    me, sh, sc, w, acc, wmax, nacc = m.compute_unweight(*d)
    me2, sh2, sc2 = m.compute(*d[:4])
    w2, acc2, wmax2, nacc2 = m.unweight(me2, d[4], d[5])
    torch.cuda.synchronize()
    for x, y in ((me, me2), (sh, sh2), (sc, sc2), (w, w2), (acc, acc2), (wmax, wmax2), (nacc, nacc2)):
        assert torch.equal(x, y)
    assert wmax.item() > 0 and 0 < nacc.item() < n
