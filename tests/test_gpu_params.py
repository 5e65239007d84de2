"""Standard-model parameters and options through the C ABI against the oracle: the
t-channel zero-width option, non-default masses and widths, the default alpha_s used
when no per-event array is given, and the per-call event limit."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps

pytestmark = pytest.mark.gpu

PROCS = ["g g > t t~", "g g > t t~ g", "g g > t t~ g g"]


def _run(m, mom, a=None):
    import torch
    me = m.compute(torch.from_numpy(mom).cuda(), None if a is None else torch.from_numpy(a).cuda())[0]
    torch.cuda.synchronize()
    return me.cpu().numpy()


@pytest.mark.parametrize("process", PROCS)
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_zero_width_tchannel_option(process, precision, bound):
    """zero_width_tchan = 1 drops the top width from the propagators that separate the
    two incoming gluons (the option of Section 3, Tables 1-2); the s-channel ones keep it"""
    from paper_2312_02898_b300.binding import MatrixElement
    mom, a, _, _ = ps.make_batch(process, 400, seed=41, alphas="uniform")
    ref_zw = oracle.me(process, mom, alphas=a, params=oracle.Params(zero_width_tchan=1))["me"]
    ref_w = oracle.me(process, mom, alphas=a)["me"]
    got = _run(MatrixElement(process, precision=precision, zero_width_tchan=1), mom, a)
    assert np.max(np.abs(got / ref_zw - 1)) <= bound
    assert np.max(np.abs(ref_zw / ref_w - 1)) > 1e-8  # the option changes the result


@pytest.mark.parametrize("process", PROCS)
def test_non_default_masses_widths_and_default_alphas(process):
    from paper_2312_02898_b300.binding import MatrixElement
    mt, wt, alphas = 172.5, 1.32, 0.1185
    mom = ps.rambo(1500.0, ps.PROCESS_FINAL_MASSES[process](mt), 43, 300)
    ref = oracle.me(process, mom, params=oracle.Params(mt=mt, wt=wt, alphas=alphas))["me"]
    got = _run(MatrixElement(process, precision="fp64", mt=mt, wt=wt, alphas=alphas), mom)
    assert np.max(np.abs(got / ref - 1)) <= 1e-12


def test_eemumu_with_other_electroweak_inputs():
    from paper_2312_02898_b300.binding import MatrixElement
    process = "e+ e- > mu+ mu-"
    p = dict(mZ=91.1876, wZ=2.4952, aEWM1=127.9)
    mom = ps.rambo(250.0, (0.0, 0.0), 44, 500)
    ref = oracle.me(process, mom, params=oracle.Params(**p))["me"]
    got = _run(MatrixElement(process, precision="fp64", **p), mom)
    assert np.max(np.abs(got / ref - 1)) <= 1e-12


def test_per_call_event_limit_is_enforced_before_any_work():
    import torch
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement("g g > t t~", precision="fp64")
    x = torch.empty(16, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = m.lib.me_compute(m.handle, 2 ** 31, ctypes.c_void_p(x.data_ptr()), None, None, None,
                          ctypes.c_void_p(x.data_ptr()), None, None, s)
    assert rc == -1 and b"2^31" in m.lib.me_last_error(m.handle)
