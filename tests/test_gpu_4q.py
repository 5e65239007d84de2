"""GPU parity of the four-quark channels of p p -> t tbar + 2 jets against the FP64 oracle:
two light flavours (u u~ > t t~ d d~ in both beam orders, u d > t t~ u d, u d~ > t t~ u d~,
u~ d~ > t t~ u~ d~) and one light flavour (u u > t t~ u u, u~ u~ > t t~ u~ u~,
u u~ > t t~ u u~ in both beam orders, both pairings of the light quarks).  FP64 within
1e-12 on every event, FP32 within 1e-5; selections equal except at running-sum
boundaries."""
import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps
from tests.test_gpu_quark_2jet import boundary_ok, collinear_events, mk, run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FOURQ = ("u u~ > t t~ d d~", "u~ u > t t~ d d~", "u d > t t~ u d", "u d~ > t t~ u d~", "u~ d~ > t t~ u~ d~")
SAME = ("u u > t t~ u u", "u~ u~ > t t~ u~ u~", "u u~ > t t~ u u~", "u~ u > t t~ u u~")


@pytest.mark.parametrize("process", FOURQ + SAME)
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_parity(process, precision, bound):
    n = 555
    mom, a, rh, rc = ps.make_batch(process, n, seed=81, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a, rnd_hel=rh, rnd_col=rc, want_hel=True, want_colw=True)
    me, sh, sc = run(mk(process, precision), mom, a, rh, rc)
    rel = np.abs(me / ref["me"] - 1)
    print(f"{process} {precision}: max rel {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= bound
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, tol)
    assert boundary_ok(sc, ref["sel_col"], ref["colw"], rc, tol)


@pytest.mark.parametrize("process", FOURQ + SAME)
def test_info_and_helicity_filter(process):
    m = mk(process)
    assert (m.npar, m.ncomb, m.ncol, m.ndiag) == (6, 64, 6, 14 if process in SAME else 7)
    # massless quark lines keep their helicity: 4 light patterns per pairing, and the two
    # pairings of identical quarks share the 2 where all four agree (6 x 4 top helicities)
    assert m.ngood == (24 if process in SAME else 16)
    mom, _, _, _ = ps.make_batch(process, 12, seed=97)
    ref = oracle.me(process, mom, want_hel=True)
    contributing = set(np.nonzero((ref["me_hel"] != 0).any(axis=0))[0].tolist())
    assert contributing <= set(m.good_helicities())


def test_zero_width_tchannel():
    process = "u d > t t~ u d"
    mom, a, rh, rc = ps.make_batch(process, 300, seed=82, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a, params=oracle.Params(zero_width_tchan=1))["me"]
    me = run(mk(process, "fp64", zero_width_tchan=1), mom, a, rh, rc)[0]
    assert np.max(np.abs(me / ref - 1)) <= 1e-12


@pytest.mark.parametrize("process,slot", [("u d > t t~ u d", 4), ("u d~ > t t~ u d~", 4), ("u u > t t~ u u", 4)])
def test_nearly_collinear_quark(process, slot):
    """the final quark 1-10 mrad from the beam of its own flavour (a nearly on-shell
    t-channel gluon): FP64 within 1e-12, FP32 rescued to the FP64 bits"""
    n = 48
    mom = collinear_events(n, seed=83, slot=slot)
    rng = np.random.default_rng(84)
    rh, rc = rng.random(n), rng.random(n)
    ref = oracle.me(process, mom, rnd_hel=rh, rnd_col=rc)["me"]
    r64 = run(mk(process, "fp64"), mom, None, rh, rc)
    rel = np.abs(r64[0] / ref - 1)
    print(f"{process} collinear: FP64 max rel {rel.max():.3e}")
    assert rel.max() <= 1e-12
    r32 = run(mk(process, "fp32"), mom, None, rh, rc)
    assert np.array_equal(r32[0], r64[0]) and np.array_equal(r32[1], r64[1])
