"""Pins of the oracle's one-jet quark channels of p p -> t tbar + jet: q qbar -> t tbar g
and its crossings q g -> t tbar q and qbar g -> t tbar qbar (either beam order), written
as five Feynman diagrams with explicit colour indices.

Nothing here re-types the oracle's diagrams; each pin is a theorem about the full
amplitude:

* Gauge invariance.  With a zero top width, replacing the gluon's polarisation by its
  momentum makes every colour-flow amplitude of every helicity vanish: this fixes the
  relative sign, colour factor and momentum routing of the three-gluon diagram against
  the four diagrams with the gluon on a quark line.
* Soft-gluon factorisation (the eikonal limit): for a gluon of momentum k -> 0,
      <|M(q qbar -> t tbar g)|^2> -> -g_s^2 sum_{i,j} (p_i.p_j)/((p_i.k)(p_j.k))
                                       <T_i.T_j> <|M(q qbar -> t tbar)|^2>
  with the colour correlators of the Born colour tensor computed here from explicit
  Gell-Mann matrices (an independent brute force); the Born itself is pinned to its
  closed form elsewhere.  This fixes the absolute normalisation and the colour
  interference between emissions off the light and the top line.
* Initial-state collinear factorisation: a final parton of momentum fraction 1 - x
  emitted collinear to a beam of momentum p leaves the spin- and colour-averaged
      <|M_{n+1}|^2> -> g_s^2 P(x) / (x p.p_5) <|M_n(x p)|^2>
  (azimuthally averaged where the parton entering the hard process is a gluon), with the
  Altarelli-Parisi splitting functions P_qq = C_F (1 + x^2)/(1 - x),
  P_gq = C_F (1 + (1 - x)^2)/x and P_qg = T_R (x^2 + (1 - x)^2).  The reduced processes
  (q qbar -> t tbar, g g -> t tbar) carry their own closed-form pins, so each limit pins
  a crossing's normalisation, its initial-state averaging (IDEN) and its external
  wavefunctions.
* The zero-width t-channel reading: in q g -> t tbar q both top propagators separate the
  beams; with the physical width there the gluon-collinear limit fails by a 1/theta^2
  term (the width breaks the gauge cancellation), with the option set it converges.
* Charge conjugation (qbar g -> t tbar qbar equals q g -> t tbar q with the top and
  antitop momenta exchanged), beam order, Lorentz invariance, and the colour matrix of
  the four flows against an explicit sum.
"""
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

QQG = "u u~ > t t~ g"
QXQG = "u~ u > t t~ g"
QG = "u g > t t~ u"
GQ = "g u > t t~ u"
QXG = "u~ g > t t~ u~"
GQX = "g u~ > t t~ u~"
ALL = (QQG, QXQG, QG, GQ, QXG, GQX)
GLUON = {QQG: 4, QXQG: 4, QG: 1, GQ: 0, QXG: 1, GQX: 0}
MT = 173.0
E = 750.0
PA = np.array([E, 0.0, 0.0, E])
PB = np.array([E, 0.0, 0.0, -E])
NSTAR = np.array([math.sin(1.1) * math.cos(0.4), math.sin(1.1) * math.sin(0.4), math.cos(1.1)])
CF, TR = 4.0 / 3.0, 0.5

# Gell-Mann matrices T^a = lambda^a / 2 (the test's own)
T = np.zeros((8, 3, 3), complex)
T[0][0, 1] = T[0][1, 0] = 0.5
T[1][0, 1], T[1][1, 0] = -0.5j, 0.5j
T[2][0, 0], T[2][1, 1] = 0.5, -0.5
T[3][0, 2] = T[3][2, 0] = 0.5
T[4][0, 2], T[4][2, 0] = -0.5j, 0.5j
T[5][1, 2] = T[5][2, 1] = 0.5
T[6][1, 2], T[6][2, 1] = -0.5j, 0.5j
T[7][0, 0] = T[7][1, 1] = 0.5 / math.sqrt(3.0)
T[7][2, 2] = -1.0 / math.sqrt(3.0)


def mdot(a, b):
    return a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]


def boost_from_rest(Q, v):
    M = math.sqrt(mdot(Q, Q))
    b = Q[1:] / Q[0]
    g = Q[0] / M
    bv, b2 = b @ v[1:], b @ b
    pv = v[1:] + ((g - 1.0) * bv / b2 if b2 > 0 else 0.0) * b + g * v[0] * b
    return np.concatenate([[g * (v[0] + bv)], pv])


def two_body(Q, n):
    """t and tbar from a system Q, the top along n in the rest frame of Q"""
    M = math.sqrt(mdot(Q, Q))
    pz = math.sqrt(M * M / 4 - MT * MT)
    t = np.concatenate([[M / 2], pz * n])
    tb = np.concatenate([[M / 2], -pz * n])
    return boost_from_rest(Q, t), boost_from_rest(Q, tb)


def me1(oracle_mod, proc, moms, par):
    return oracle_mod.me(proc, np.asarray(moms)[None], params=par)["me"][0]


def random_lorentz(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    eta = rng.uniform(-1.5, 1.5)
    L = np.eye(4)
    L[0, 0] = math.cosh(eta)
    L[0, 1:] = L[1:, 0] = math.sinh(eta) * n
    L[1:, 1:] = np.eye(3) + (math.cosh(eta) - 1.0) * np.outer(n, n)
    Rot = np.eye(4)
    Rot[1:, 1:] = R
    return L @ Rot


# ---------------------------------------------------------------------------
def test_colour_matrix_of_the_four_flows(oracle_mod):
    # flows over the colours (B, K, t, tbar, a) of the light row end, light column end,
    # top, antitop and gluon: T^a_{B tbar} d_{t K}, T^a_{t K} d_{B tbar}, T^a_{B K} d_{t tbar},
    # T^a_{t tbar} d_{B K}
    d = np.eye(3)
    flows = [np.einsum("aBy,tK->BKtya", T, d), np.einsum("atK,By->BKtya", T, d),
             np.einsum("aBK,ty->BKtya", T, d), np.einsum("aty,BK->BKtya", T, d)]
    G = np.array([[np.vdot(f, g) for g in flows] for f in flows])
    assert np.abs(G.imag).max() < 1e-12
    for proc in ALL:
        num, den = oracle_mod.colour_matrix(proc)
        np.testing.assert_allclose(num / den, G.real, atol=1e-12)


@pytest.mark.parametrize("proc", ALL)
def test_flows_rebuild_every_helicity(oracle_mod, proc):
    # the flow amplitudes J (projections onto the basis) give back the explicit colour sum:
    # |M_h|^2 = J^dagger C J for every helicity, so the four flows span the colour space
    mom, _, _, _ = ps.make_batch(proc, 6, seed=11)
    r = oracle_mod.me(proc, mom, want_hel=True, want_jamp=True)
    num, den = oracle_mod.colour_matrix(proc)
    C = num / den
    J = r["jamp"]
    rebuilt = np.einsum("ehi,ij,ehj->eh", J.conj(), C, J).real
    np.testing.assert_allclose(rebuilt, r["me_hel"], rtol=1e-12, atol=1e-14 * r["me_hel"].max())
    # massless light quarks: only helicity-conserving configurations contribute
    nz = np.count_nonzero(r["me_hel"].max(axis=0) > 1e-20 * r["me_hel"].max())
    assert nz == 16


@pytest.mark.parametrize("proc", ALL)
def test_gauge_invariance(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, 12, seed=6)
    par = oracle_mod.Params(wt=0.0)
    phys = oracle_mod.me(proc, mom, params=par, want_jamp=True)["jamp"]
    gauge = oracle_mod.me(proc, mom, params=par, want_jamp=True, gauge_leg=GLUON[proc])["jamp"]
    scale = np.abs(phys).max(axis=(1, 2))
    assert np.all(np.abs(gauge).max(axis=(1, 2)) <= 1e-10 * scale)


def test_gauge_check_is_sensitive(oracle_mod):
    # with the physical top width the Ward identity is broken at O(m w / (q^2 - m^2))
    mom, _, _, _ = ps.make_batch(QQG, 5, seed=6)
    phys = oracle_mod.me(QQG, mom, want_jamp=True)["jamp"]
    gauge = oracle_mod.me(QQG, mom, want_jamp=True, gauge_leg=4)["jamp"]
    assert np.abs(gauge).max() > 1e-6 * np.abs(phys).max()


@pytest.mark.parametrize("proc", ALL)
def test_lorentz_invariance(oracle_mod, proc):
    rng = np.random.default_rng(5)
    mom, _, _, _ = ps.make_batch(proc, 40, seed=7)
    par = oracle_mod.Params(wt=0.0)
    ref = oracle_mod.me(proc, mom, params=par)["me"]
    got = oracle_mod.me(proc, np.einsum("ij,epj->epi", random_lorentz(rng), mom), params=par)["me"]
    assert np.max(np.abs(got / ref - 1)) < 1e-11


@pytest.mark.parametrize("a,b", [(QQG, QXQG), (QG, GQ), (QXG, GQX)])
def test_beam_order(oracle_mod, a, b):
    mom, _, _, _ = ps.make_batch(a, 40, seed=9)
    swapped = mom.copy()
    swapped[:, [0, 1]] = mom[:, [1, 0]]
    ra = oracle_mod.me(a, mom)["me"]
    rb = oracle_mod.me(b, swapped)["me"]
    np.testing.assert_allclose(rb, ra, rtol=1e-12)


@pytest.mark.parametrize("a,b", [(QG, QXG), (GQ, GQX), (QQG, QXQG)])
def test_charge_conjugation(oracle_mod, a, b):
    # C maps q g -> t(p3) tbar(p4) q(p5) to qbar g -> tbar(p3) t(p4) qbar(p5), and
    # u(p1) u~(p2) -> t(p3) t~(p4) g to u~(p1) u(p2) -> t~(p3) t(p4) g; process b lists the
    # top before the antitop, so its momenta take p3 and p4 exchanged
    mom, _, _, _ = ps.make_batch(a, 40, seed=10)
    conj = mom.copy()
    conj[:, [2, 3]] = mom[:, [3, 2]]
    np.testing.assert_allclose(oracle_mod.me(b, conj)["me"], oracle_mod.me(a, mom)["me"], rtol=1e-12)


# ---------------------------------------------------------------------------
def _born_colour_correlators(order):
    """<c|T_i.T_j|c> / <c|c> for the Born tensor c_{ijkl} = sum_b T^b_{j i} T^b_{k l} of
    q(i) qbar(j) -> t(k) tbar(l), particles in 'order'.  Row indices (incoming antiquark,
    outgoing quark) carry +T^a, column indices (incoming quark, outgoing antiquark) -T^a
    transposed, which makes sum_i T_i c = 0 (checked)."""
    c = np.einsum("bji,bkl->ijkl", T, T)
    slot = {"q": 0, "qb": 1, "t": 2, "tb": 3}
    c = np.transpose(c, [slot[r] for r in order])
    row = {"q": False, "qb": True, "t": True, "tb": False}

    def charge(s, a):
        if row[order[s]]:
            return np.moveaxis(np.tensordot(T[a], c, axes=([1], [s])), 0, s)
        return -np.moveaxis(np.tensordot(T[a], c, axes=([0], [s])), 0, s)

    TC = [[charge(s, a) for a in range(8)] for s in range(4)]
    for a in range(8):
        assert np.abs(sum(TC[s][a] for s in range(4))).max() < 1e-14
    C = np.array([[sum(np.vdot(TC[i][a], TC[j][a]) for a in range(8)).real for j in range(4)] for i in range(4)])
    np.testing.assert_allclose(np.diag(C) / np.vdot(c, c).real, CF)
    return C / np.vdot(c, c).real


@pytest.mark.parametrize("proc,born,order", [(QQG, "u u~ > t t~", ["q", "qb", "t", "tb"]),
                                             (QXQG, "u~ u > t t~", ["qb", "q", "t", "tb"])])
def test_soft_gluon_limit(oracle_mod, proc, born, order):
    par = oracle_mod.Params(wt=0.0)
    C = _born_colour_correlators(order)
    t0, tb0 = two_body(PA + PB, NSTAR)
    red = me1(oracle_mod, born, [PA, PB, t0, tb0], par)
    nk = np.array([math.sin(0.7) * math.cos(2.0), math.sin(0.7) * math.sin(2.0), math.cos(0.7)])
    gs2 = 4 * math.pi * par.alphas
    dev = {}
    for lam in (1e-3, 1e-4):
        k = lam * E * np.concatenate([[1.0], nk])
        t, tb = two_body(PA + PB - k, NSTAR)
        full = me1(oracle_mod, proc, [PA, PB, t, tb, k], par)
        p = [PA, PB, t, tb]
        eik = -sum(C[i, j] * mdot(p[i], p[j]) / (mdot(p[i], k) * mdot(p[j], k)) for i in range(4) for j in range(4))
        dev[lam] = abs(full / (gs2 * eik * red) - 1)
    # next-to-soft corrections fall linearly with the gluon energy
    assert dev[1e-3] < 1e-4 and dev[1e-4] < 1e-5, dev
    # without the initial-final colour interference the limit is off at O(1)
    Cd = np.diag(np.diag(C))
    k = 1e-4 * E * np.concatenate([[1.0], nk])
    t, tb = two_body(PA + PB - k, NSTAR)
    p = [PA, PB, t, tb]
    eik_d = -sum(Cd[i, j] * mdot(p[i], p[j]) / (mdot(p[i], k) * mdot(p[j], k)) for i in range(4) for j in range(4))
    assert abs(me1(oracle_mod, proc, [PA, PB, t, tb, k], par) / (gs2 * eik_d * red) - 1) > 0.05


def _collinear_ratio(oracle_mod, proc, born, beam, split, par, theta, x=0.6):
    """<|M_{n+1}|^2> over its collinear approximation, averaged over four azimuths (which
    removes the cos 2 phi spin correlation of a gluon entering the hard process)"""
    P = {"qq": CF * (1 + x * x) / (1 - x), "gq": CF * (1 + (1 - x) ** 2) / x,
         "qg": TR * (x * x + (1 - x) ** 2)}[split]
    gs2 = 4 * math.pi * par.alphas
    pbeam = PA if beam == 0 else PB
    sgn = 1.0 if beam == 0 else -1.0
    pa2, pb2 = (x * PA, PB) if beam == 0 else (PA, x * PB)
    t0, tb0 = two_body(pa2 + pb2, NSTAR)
    red = me1(oracle_mod, born, [pa2, pb2, t0, tb0], par)
    rs = []
    for phi in 0.3 + np.arange(4) * math.pi / 2:
        p5 = (1 - x) * E * np.array([1.0, math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
                                     sgn * math.cos(theta)])
        t, tb = two_body(PA + PB - p5, NSTAR)
        full = me1(oracle_mod, proc, [PA, PB, t, tb, p5], par)
        rs.append(full / (gs2 * P / (x * mdot(pbeam, p5)) * red))
    return float(np.mean(rs))


@pytest.mark.parametrize("proc,born,beam,split", [
    (QQG, "u u~ > t t~", 0, "qq"), (QQG, "u u~ > t t~", 1, "qq"),
    (QXQG, "u~ u > t t~", 0, "qq"),
    (QG, "g g > t t~", 0, "gq"), (QG, "u u~ > t t~", 1, "qg"),
    (GQ, "g g > t t~", 1, "gq"), (GQ, "u~ u > t t~", 0, "qg"),
    (QXG, "g g > t t~", 0, "gq"), (QXG, "u~ u > t t~", 1, "qg"),
    (GQX, "u u~ > t t~", 0, "qg"),
])
def test_initial_state_collinear_limit(oracle_mod, proc, born, beam, split):
    par = oracle_mod.Params(wt=0.0)
    d2 = abs(_collinear_ratio(oracle_mod, proc, born, beam, split, par, 1e-2) - 1)
    d3 = abs(_collinear_ratio(oracle_mod, proc, born, beam, split, par, 1e-3) - 1)
    # corrections fall as theta^2
    assert d3 < 1e-5 and d3 < 0.05 * d2 + 1e-9, (d2, d3)


def test_zero_width_tchannel_in_the_qg_crossing(oracle_mod):
    # both top propagators of q g -> t tbar q separate the beams: with the physical width
    # kept there, the gluon-collinear limit picks up a 1/theta^2 term; the zero-width
    # t-channel option removes it
    with_w = oracle_mod.Params()
    zwt = oracle_mod.Params(zero_width_tchan=1)
    bad = abs(_collinear_ratio(oracle_mod, QG, "g g > t t~", 0, "gq", with_w, 1e-4) - 1)
    good = abs(_collinear_ratio(oracle_mod, QG, "g g > t t~", 0, "gq", zwt, 1e-4) - 1)
    assert bad > 1.0 and good < 1e-6, (bad, good)
