"""GPU parity of the two-jet channels with one light-quark line (q qbar -> t tbar g g,
q g -> t tbar q g, qbar g -> t tbar qbar g in both beam orders, g g -> t tbar q qbar)
against the FP64 oracle, and the per-event dispatch of a p p -> t tbar + 2 jets batch over
these channels, g g -> t tbar g g and the four-quark channels.

Bars as for the other processes: FP64 within 1e-12 of the oracle on every event, FP32
within 1e-5 (with the FP64 rescue of ill-conditioned events); selections equal except
where r * total lies within 1e-10 (FP64) of a running-sum boundary."""
import numpy as np
import pytest

import oracle
from paper_2312_02898_b300 import phasespace as ps
from tests.collinear import top_pair

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JET2 = ("u u~ > t t~ g g", "u~ u > t t~ g g", "u g > t t~ u g", "g u > t t~ u g", "u~ g > t t~ u~ g",
        "g u~ > t t~ u~ g", "g g > t t~ u u~")
FOURQ = ("u u~ > t t~ d d~", "u~ u > t t~ d d~", "u d > t t~ u d", "u d~ > t t~ u d~", "u~ d~ > t t~ u~ d~")
SAME = ("u u > t t~ u u", "u~ u~ > t t~ u~ u~", "u u~ > t t~ u u~", "u~ u > t t~ u u~")
PP_TT2J = ("g g > t t~ g g",) + JET2 + FOURQ + SAME


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


@pytest.mark.parametrize("process", JET2)
@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_parity(process, precision, bound):
    n = 333
    mom, a, rh, rc = ps.make_batch(process, n, seed=71, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a, rnd_hel=rh, rnd_col=rc, want_hel=True, want_colw=True)
    me, sh, sc = run(mk(process, precision), mom, a, rh, rc)
    rel = np.abs(me / ref["me"] - 1)
    print(f"{process} {precision}: max rel {rel.max():.3e}, median {np.median(rel):.3e}")
    assert rel.max() <= bound
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert boundary_ok(sh, ref["sel_hel"], ref["me_hel"], rh, tol)
    assert boundary_ok(sc, ref["sel_col"], ref["colw"], rc, tol)


@pytest.mark.parametrize("process", JET2)
def test_info_and_helicity_filter(process):
    m = mk(process)
    assert (m.npar, m.ncomb, m.ncol, m.ndiag) == (6, 64, 13, 36)
    assert m.ngood == 32
    mom, _, _, _ = ps.make_batch(process, 12, seed=98)
    ref = oracle.me(process, mom, want_hel=True)
    contributing = set(np.nonzero((ref["me_hel"] != 0).any(axis=0))[0].tolist())
    assert contributing <= set(m.good_helicities())


@pytest.mark.parametrize("process", ["u g > t t~ u g", "g g > t t~ u u~"])
def test_zero_width_tchannel(process):
    n = 200
    mom, a, rh, rc = ps.make_batch(process, n, seed=72, alphas="uniform")
    ref = oracle.me(process, mom, alphas=a, params=oracle.Params(zero_width_tchan=1))["me"]
    me = run(mk(process, "fp64", zero_width_tchan=1), mom, a, rh, rc)[0]
    assert np.max(np.abs(me / ref - 1)) <= 1e-12


def collinear_events(n, seed, slot, theta=(1e-3, 1e-2), sqrt_s=1500.0, mt=173.0):
    """the final light parton in slot (4 or 5) a small angle theta from the first beam:
    the propagator between them is 1e4 to 1e6 times smaller than the squared energies.
    Other propagators of such events can lie near their poles too, where an invariant
    formed from the complementary particle set would differ by the inputs' rounding-level
    momentum imbalance; both sides form each invariant from the set its momentum is
    routed from."""
    rng = np.random.default_rng(seed)
    h = sqrt_s / 2
    p1, p2 = np.array([h, 0, 0, h]), np.array([h, 0, 0, -h])
    mom = np.zeros((n, 6, 4))
    for e in range(n):
        th, phi, en = rng.uniform(*theta), rng.uniform(0, 2 * np.pi), rng.uniform(100.0, 250.0)
        j = en * np.array([1.0, np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        o = rng.uniform(100.0, 250.0) * np.concatenate([[1.0], u])
        tops = top_pair(p1 + p2 - j - o, mt, rng)
        row = [p1, p2] + tops + [None, None]
        row[slot], row[9 - slot] = j, o
        mom[e] = row
    return mom


@pytest.mark.parametrize("process,slot", [("u u~ > t t~ g g", 5), ("u g > t t~ u g", 4), ("g g > t t~ u u~", 4)])
def test_nearly_collinear_parton(process, slot):
    """FP64 within 1e-12 of the oracle where the propagator between a final light parton
    and the first beam cancels four to six digits; FP32 rescues every such event to the
    FP64 bits"""
    n = 48
    mom = collinear_events(n, seed=73, slot=slot)
    rng = np.random.default_rng(74)
    rh, rc = rng.random(n), rng.random(n)
    ref = oracle.me(process, mom, rnd_hel=rh, rnd_col=rc)["me"]
    r64 = run(mk(process, "fp64"), mom, None, rh, rc)
    rel = np.abs(r64[0] / ref - 1)
    print(f"{process} collinear: FP64 max rel {rel.max():.3e}")
    assert rel.max() <= 1e-12
    r32 = run(mk(process, "fp32"), mom, None, rh, rc)
    assert np.array_equal(r32[0], r64[0]) and np.array_equal(r32[1], r64[1])


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_pp_ttbar_2jet_dispatch(precision, bound):
    """one batch of p p -> t tbar + 2 jets events over all 17 channels (g g -> t tbar g g,
    seven with one light-quark line, five four-quark channels with two light flavours and
    four with one): every event gets its channel's single-call bits and the oracle's
    value"""
    from paper_2312_02898_b300.binding import compute_channels
    n = 2053
    mom, a, rh, rc = ps.make_batch(PP_TT2J[0], n, seed=75, alphas="uniform")
    w = np.array([0.36, 0.06, 0.06, 0.06, 0.06, 0.05, 0.05, 0.05, 0.04, 0.03, 0.04, 0.03, 0.03, 0.02, 0.02, 0.02, 0.02])
    ch = np.random.default_rng(76).choice(len(PP_TT2J), size=n, p=w / w.sum()).astype(np.int32)
    hs = [mk(p, precision) for p in PP_TT2J]
    d = dev(mom, a, rh, rc)
    me, sh, sc = compute_channels(hs, dev(ch)[0], *d)
    torch.cuda.synchronize()
    me, sh, sc = me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()
    for c, p in enumerate(PP_TT2J):
        sel = ch == c
        r = [x.cpu().numpy() for x in hs[c].compute(*d)]
        assert np.array_equal(me[sel], r[0][sel]) and np.array_equal(sh[sel], r[1][sel])
        assert np.array_equal(sc[sel], r[2][sel])
        idx = np.nonzero(sel)[0][:150]
        ref = oracle.me(p, mom[idx], alphas=a[idx])["me"]
        rel = np.abs(me[idx] / ref - 1)
        print(f"{p} {precision}: {sel.sum()} events, max rel {rel.max():.3e} over {len(idx)}")
        assert rel.max() <= bound
