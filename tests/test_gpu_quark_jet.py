"""GPU parity of the one-jet quark channels of p p -> t tbar + jet (q qbar -> t tbar g,
q g -> t tbar q, qbar g -> t tbar qbar, both beam orders) against the FP64 oracle, and
the per-event dispatch of a p p -> t tbar + jet batch over all seven channels (with
g g -> t tbar g).

Bars as for the other processes: FP64 within 1e-12 of the oracle on every event, FP32
within 1e-5 (with the FP64 rescue of ill-conditioned events), double-float within its
own stated 1e-10; selections equal except
where r * total lies within 1e-10 of a running-sum boundary."""
import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps
from tests.collinear import top_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JET = ("u u~ > t t~ g", "u~ u > t t~ g", "u g > t t~ u", "g u > t t~ u", "u~ g > t t~ u~", "g u~ > t t~ u~")
PP_TTJ = ("g g > t t~ g",) + JET


def mk(process, precision="fp64", **kw):
    from paper_2312_02898_b300.binding import MatrixElement
    return MatrixElement(process, precision=precision, **kw)


def dev(*arrs):
    return [None if a is None else torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def run(m, mom, a, rh, rc):
    me, sh, sc = m.compute(*dev(mom, a, rh, rc))
    torch.cuda.synchronize()
    return me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()


def boundary_ok(sel_gpu, sel_ref, weights, r, rel):
    for e in np.nonzero(sel_gpu != sel_ref)[0]:
        c = np.cumsum(weights[e])
        if np.min(np.abs(c - r[e] * c[-1])) > rel * c[-1]:
            return False
    return True


@pytest.mark.parametrize("process", JET)
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5), ("dfloat", 1e-10)])
def test_parity(process, precision, bound):
    n = 777
    mom, a, rh, rc = ps.make_batch(process, n, seed=61, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a, rnd_hel=rh, rnd_col=rc, want_hel=True, want_colw=True)
    me, sh, sc = run(mk(process, precision), mom, a, rh, rc)
    rel = np.abs(me / ref["me"] - 1)
    print(f"{process} {precision}: max rel {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= bound
    tol = 1e-10 if precision in ("fp64", "dfloat") else 1e-5
    assert boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, tol)
    assert boundary_ok(sc, ref["sel_col"], ref["colw"], rc, tol)


@pytest.mark.parametrize("process", JET)
def test_info_and_helicity_filter(process):
    m = mk(process)
    assert (m.npar, m.ncomb, m.ncol, m.ndiag) == (5, 32, 4, 5)
    # massless light quarks keep only the helicity-conserving half
    assert m.ngood == 16
    mom, _, _, _ = ps.make_batch(process, 20, seed=99)
    ref = oracle.me(process, mom, want_hel=True)
    contributing = set(np.nonzero((ref["me_hel"] != 0).any(axis=0))[0].tolist())
    assert contributing <= set(m.good_helicities())


@pytest.mark.parametrize("process", ["u g > t t~ u", "g u~ > t t~ u~"])
def test_zero_width_tchannel(process):
    # both top propagators of the q g crossings are t-channel
    n = 300
    mom, a, rh, rc = ps.make_batch(process, n, seed=62, alphas="uniform")
    par = oracle.Params(zero_width_tchan=1)
    ref = oracle.me(process, mom, alphas=a, params=par)["me"]
    me = run(mk(process, "fp64", zero_width_tchan=1), mom, a, rh, rc)[0]
    assert np.max(np.abs(me / ref - 1)) <= 1e-12
    with_w = oracle.me(process, mom, alphas=a)["me"]
    assert np.max(np.abs(with_w / ref - 1)) > 1e-6


def collinear_jet_events(n, seed, theta=(1e-3, 1e-2), sqrt_s=1500.0, mt=173.0):
    """the jet (particle 4) a small angle theta from the first beam: the propagator
    between them (a light quark or a gluon, by channel) is nearly on shell"""
    rng = np.random.default_rng(seed)
    h = sqrt_s / 2
    p1, p2 = np.array([h, 0, 0, h]), np.array([h, 0, 0, -h])
    mom = np.zeros((n, 5, 4))
    for e in range(n):
        th, phi, en = rng.uniform(*theta), rng.uniform(0, 2 * np.pi), rng.uniform(100.0, 300.0)
        j = en * np.array([1.0, np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
        mom[e] = [p1, p2] + top_pair(p1 + p2 - j, mt, rng) + [j]
    return mom


@pytest.mark.parametrize("process", JET)
def test_nearly_collinear_jet(process):
    """FP64 stays within 1e-12 of the oracle where the propagator between the jet and the
    first beam cancels four to six digits (error-free invariants); FP32 flags every such
    event for its FP64 rescue and returns the FP64 bits."""
    n = 64
    mom = collinear_jet_events(n, seed=63)
    rng = np.random.default_rng(64)
    rh, rc = rng.random(n), rng.random(n)
    ref = oracle.me(process, mom, rnd_hel=rh, rnd_col=rc)["me"]
    r64 = run(mk(process, "fp64"), mom, None, rh, rc)
    rel = np.abs(r64[0] / ref - 1)
    print(f"{process} collinear jet: FP64 max rel {rel.max():.3e}")
    assert rel.max() <= 1e-12
    r32 = run(mk(process, "fp32"), mom, None, rh, rc)
    assert np.array_equal(r32[0], r64[0]) and np.array_equal(r32[1], r64[1])


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_pp_ttbar_jet_dispatch(precision, bound):
    """One batch of p p -> t tbar + jet events routed per event over the seven channels:
    every event gets its channel's single-call bits and the oracle's value."""
    from paper_2312_02898_b300.binding import compute_channels
    n = 4099
    mom, a, rh, rc = ps.make_batch(PP_TTJ[0], n, seed=65, alphas="uniform")
    w = np.array([0.55, 0.1, 0.1, 0.07, 0.07, 0.055, 0.055])
    ch = np.random.default_rng(66).choice(len(PP_TTJ), size=n, p=w / w.sum()).astype(np.int32)
    hs = [mk(p, precision) for p in PP_TTJ]
    d = dev(mom, a, rh, rc)
    me, sh, sc = compute_channels(hs, dev(ch)[0], *d)
    torch.cuda.synchronize()
    me, sh, sc = me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()
    for c, p in enumerate(PP_TTJ):
        sel = ch == c
        r = [x.cpu().numpy() for x in hs[c].compute(*d)]
        assert np.array_equal(me[sel], r[0][sel]) and np.array_equal(sh[sel], r[1][sel])
        assert np.array_equal(sc[sel], r[2][sel])
        ref = oracle.me(p, mom[sel], alphas=a[sel])["me"]
        rel = np.abs(me[sel] / ref - 1)
        print(f"{p} {precision}: {sel.sum()} events, max rel {rel.max():.3e}")
        assert rel.max() <= bound
