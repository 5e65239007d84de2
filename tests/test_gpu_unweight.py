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
