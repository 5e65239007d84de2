"""Pins of the oracle's two-jet quark channels of p p -> t tbar + 2 jets with one light-quark
line: q qbar -> t tbar g g, q g -> t tbar q g, qbar g -> t tbar qbar g (either beam
order) and g g -> t tbar q qbar, written as 36 Feynman diagrams (38 terms) with explicit
colour indices.

As for the one-jet channels, each pin is a theorem about the full amplitude, not a
re-typing of the diagrams:

* gauge invariance in each gluon separately (zero top width), which fixes the relative
  signs, colours and momentum routing of the diagrams with three- and four-gluon
  vertices against those with the gluons on the quark lines;
* the soft limit of either final gluon of q qbar -> t tbar g g onto q qbar -> t tbar g,
  with the colour correlators <M|T_i.T_j|M> of the one-jet amplitude built here from its
  flow amplitudes and the test's own Gell-Mann matrices (five coloured partons, the
  gluon's charge -i f);
* initial-state collinear limits with the Altarelli-Parisi splitting functions P_qq,
  P_qg, P_gq and P_gg (azimuthally averaged where a gluon enters the hard process) onto
  the pinned one-jet channels and g g -> t tbar g;
* Bose symmetry of the two gluons, charge conjugation, beam order, Lorentz invariance,
  and the 13-flow colour basis (with its Gram matrix) against an explicit sum.
"""
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps
from tests.test_oracle_qq_jet import CF, E, NSTAR, PA, PB, T, TR, mdot, random_lorentz, two_body

QQGG = "u u~ > t t~ g g"
QXQGG = "u~ u > t t~ g g"
QGQG = "u g > t t~ u g"
GQQG = "g u > t t~ u g"
QXGQXG = "u~ g > t t~ u~ g"
GQXQXG = "g u~ > t t~ u~ g"
GGQQ = "g g > t t~ u u~"
ALL = (QQGG, QXQGG, QGQG, GQQG, QXGQXG, GQXQXG, GGQQ)
GLUONS = {QQGG: (4, 5), QXQGG: (4, 5), QGQG: (1, 5), GQQG: (0, 5), QXGQXG: (1, 5), GQXQXG: (0, 5), GGQQ: (0, 1)}
CA = 3.0
F = np.real(-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T)))
KO = 0.25 * E * np.array([1.0, math.sin(1.3) * math.cos(0.3), math.sin(1.3) * math.sin(0.3), math.cos(1.3)])


def flows13():
    """the 13 flow tensors over (B, K, t, y, a, b): light row end, light column end, top,
    antitop, first and second gluon"""
    d, d8, E_ = np.eye(3), np.eye(8), np.einsum
    return [E_("aBm,bmy,tK->BKtyab", T, T, d), E_("bBm,amy,tK->BKtyab", T, T, d),
            E_("aBy,btK->BKtyab", T, T), E_("bBy,atK->BKtyab", T, T),
            E_("By,atm,bmK->BKtyab", d, T, T), E_("By,btm,amK->BKtyab", d, T, T),
            E_("aBm,bmK,ty->BKtyab", T, T, d), E_("bBm,amK,ty->BKtyab", T, T, d),
            E_("aBK,bty->BKtyab", T, T), E_("bBK,aty->BKtyab", T, T),
            E_("BK,atm,bmy->BKtyab", d, T, T), E_("BK,btm,amy->BKtyab", d, T, T),
            E_("ab,By,tK->BKtyab", d8, d, d)]


def test_thirteen_flows_are_a_basis(oracle_mod):
    fl = flows13()
    Fm = np.stack([f.ravel() for f in fl], axis=1)
    assert np.linalg.matrix_rank(Fm) == 13
    # the second trace tensor d^{ab} d_{BK} d_{ty} is the combination the Fierz identity
    # gives, so the 13 span the 14 natural string products
    extra = np.einsum("ab,BK,ty->BKtyab", np.eye(8), np.eye(3), np.eye(3)).ravel()
    c = np.linalg.lstsq(Fm, extra, rcond=None)[0]
    assert np.abs(Fm @ c - extra).max() < 1e-12
    G = Fm.conj().T @ Fm
    assert np.abs(G.imag).max() < 1e-12
    for proc in ALL:
        num, den = oracle_mod.colour_matrix(proc)
        np.testing.assert_allclose(num / den, G.real, atol=1e-12)


@pytest.mark.parametrize("proc", ALL)
def test_flows_rebuild_every_helicity(oracle_mod, proc):
    # every term's colour lies in the span of the flows: J^dagger C J gives back the
    # explicit colour sum for every helicity
    mom, _, _, _ = ps.make_batch(proc, 3, seed=12)
    r = oracle_mod.me(proc, mom, want_hel=True, want_jamp=True)
    num, den = oracle_mod.colour_matrix(proc)
    J = r["jamp"]
    rebuilt = np.einsum("ehi,ij,ehj->eh", J.conj(), num / den, J).real
    np.testing.assert_allclose(rebuilt, r["me_hel"], rtol=1e-11, atol=1e-13 * r["me_hel"].max())
    assert np.count_nonzero(r["me_hel"].max(axis=0) > 1e-20 * r["me_hel"].max()) == 32


@pytest.mark.parametrize("proc", ALL)
def test_gauge_invariance_in_each_gluon(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, 6, seed=6)
    par = oracle_mod.Params(wt=0.0)
    phys = oracle_mod.me(proc, mom, params=par, want_jamp=True)["jamp"]
    scale = np.abs(phys).max(axis=(1, 2))
    for leg in GLUONS[proc]:
        gauge = oracle_mod.me(proc, mom, params=par, want_jamp=True, gauge_leg=leg)["jamp"]
        assert np.all(np.abs(gauge).max(axis=(1, 2)) <= 1e-10 * scale), leg


def test_gauge_check_is_sensitive(oracle_mod):
    mom, _, _, _ = ps.make_batch(QQGG, 3, seed=6)
    phys = oracle_mod.me(QQGG, mom, want_jamp=True)["jamp"]
    gauge = oracle_mod.me(QQGG, mom, want_jamp=True, gauge_leg=5)["jamp"]
    assert np.abs(gauge).max() > 1e-6 * np.abs(phys).max()


@pytest.mark.parametrize("proc", ALL)
def test_lorentz_invariance(oracle_mod, proc):
    rng = np.random.default_rng(15)
    mom, _, _, _ = ps.make_batch(proc, 10, seed=17)
    par = oracle_mod.Params(wt=0.0)
    ref = oracle_mod.me(proc, mom, params=par)["me"]
    got = oracle_mod.me(proc, np.einsum("ij,epj->epi", random_lorentz(rng), mom), params=par)["me"]
    assert np.max(np.abs(got / ref - 1)) < 1e-10


@pytest.mark.parametrize("proc,perm", [(QQGG, [0, 1, 2, 3, 5, 4]), (GGQQ, [1, 0, 2, 3, 4, 5])])
def test_bose_symmetry(oracle_mod, proc, perm):
    mom, _, _, _ = ps.make_batch(proc, 10, seed=18)
    np.testing.assert_allclose(oracle_mod.me(proc, mom[:, perm])["me"], oracle_mod.me(proc, mom)["me"], rtol=1e-12)


@pytest.mark.parametrize("a,b", [(QQGG, QXQGG), (QGQG, GQQG), (QXGQXG, GQXQXG)])
def test_beam_order(oracle_mod, a, b):
    mom, _, _, _ = ps.make_batch(a, 10, seed=19)
    swapped = mom.copy()
    swapped[:, [0, 1]] = mom[:, [1, 0]]
    np.testing.assert_allclose(oracle_mod.me(b, swapped)["me"], oracle_mod.me(a, mom)["me"], rtol=1e-12)


@pytest.mark.parametrize("a,b,perm", [(QGQG, QXGQXG, [0, 1, 3, 2, 4, 5]), (QQGG, QXQGG, [0, 1, 3, 2, 4, 5]),
                                      (GGQQ, GGQQ, [0, 1, 3, 2, 5, 4])])
def test_charge_conjugation(oracle_mod, a, b, perm):
    mom, _, _, _ = ps.make_batch(a, 10, seed=20)
    np.testing.assert_allclose(oracle_mod.me(b, mom[:, perm])["me"], oracle_mod.me(a, mom)["me"], rtol=1e-12)


# ---------------------------------------------------------------------------
def _charge(M, slot, kind, c):
    """colour charge T^c of one parton acting on the amplitude tensor M: +T^c on a row
    index, -T^c transposed on a column index, -i f^{c..} on an adjoint index"""
    if kind == "row":
        return np.moveaxis(np.tensordot(T[c], M, axes=([1], [slot])), 0, slot)
    if kind == "col":
        return -np.moveaxis(np.tensordot(T[c], M, axes=([0], [slot])), 0, slot)
    return np.moveaxis(np.tensordot(-1j * F[c], M, axes=([1], [slot])), 0, slot)


@pytest.mark.parametrize("soft", [4, 5])
def test_soft_gluon_limit(oracle_mod, soft):
    """either final gluon of u u~ -> t t~ g g soft: sum |M|^2 -> -g^2 sum_ij
    (p_i.p_j)/((p_i.k)(p_j.k)) sum_h <M_h|T_i.T_j|M_h> of u u~ -> t t~ g, with the
    one-jet colour vectors M_h = sum_n J_hn c_n from the oracle's flow amplitudes"""
    par = oracle_mod.Params(wt=0.0)
    d = np.eye(3)
    flows3 = np.array([np.einsum("aBy,tK->BKtya", T, d), np.einsum("atK,By->BKtya", T, d),
                       np.einsum("aBK,ty->BKtya", T, d), np.einsum("aty,BK->BKtya", T, d)])
    t0, tb0 = two_body(PA + PB - KO, NSTAR)
    born = oracle_mod.me("u u~ > t t~ g", np.array([[PA, PB, t0, tb0, KO]]), params=par, want_jamp=True)
    Mh = np.einsum("hn,nBKtya->hBKtya", born["jamp"][0], flows3)
    # partons of the Born: quark (column K), antiquark (row B), top (row), antitop (column), gluon
    parts = [(PA, 2, "col"), (PB, 1, "row"), (t0, 3, "row"), (tb0, 4, "col"), (KO, 5, "adj")]
    TM = [[_charge(Mh, s, kd, c) for c in range(8)] for (_, s, kd) in parts]
    for c in range(8):
        assert np.abs(sum(TM[i][c] for i in range(5))).max() < 1e-14 * np.abs(Mh).max()
    corr = np.array([[sum(np.vdot(TM[i][c], TM[j][c]) for c in range(8)).real for j in range(5)] for i in range(5)])
    total = np.vdot(Mh, Mh).real
    np.testing.assert_allclose(total, 36 * born["me"][0], rtol=1e-12)
    nk = np.array([math.sin(0.7) * math.cos(2.0), math.sin(0.7) * math.sin(2.0), math.cos(0.7)])
    gs2 = 4 * math.pi * par.alphas
    dev = {}
    for lam in (1e-3, 1e-4):
        k = lam * E * np.concatenate([[1.0], nk])
        t, tb = two_body(PA + PB - KO - k, NSTAR)
        mom = [PA, PB, t, tb, None, None]
        mom[soft], mom[9 - soft] = k, KO
        full = 72 * oracle_mod.me(QQGG, np.array([mom]), params=par)["me"][0]
        p = [x for x, _, _ in parts]
        eik = -sum(corr[i, j] * mdot(p[i], p[j]) / (mdot(p[i], k) * mdot(p[j], k)) for i in range(5) for j in range(5))
        dev[lam] = abs(full / (gs2 * eik) - 1)
    assert dev[1e-3] < 1e-2 and dev[1e-4] < 1e-3 and dev[1e-4] < 0.2 * dev[1e-3], dev


def _collinear_ratio(oracle_mod, proc, born, beam, split, emit, par, theta, x=0.6, ident=1.0):
    """the final parton in slot emit collinear to beam (fraction 1 - x), the other final
    light parton at KO; averaged over four azimuths"""
    P = {"qq": CF * (1 + x * x) / (1 - x), "gq": CF * (1 + (1 - x) ** 2) / x, "qg": TR * (x * x + (1 - x) ** 2),
         "gg": 2 * CA * (x / (1 - x) + (1 - x) / x + x * (1 - x))}[split]
    gs2 = 4 * math.pi * par.alphas
    pbeam, sgn = (PA, 1.0) if beam == 0 else (PB, -1.0)
    pa2, pb2 = (x * PA, PB) if beam == 0 else (PA, x * PB)
    t0, tb0 = two_body(pa2 + pb2 - KO, NSTAR)
    red = oracle_mod.me(born, np.array([[pa2, pb2, t0, tb0, KO]]), params=par)["me"][0]
    rs = []
    for phi in 0.3 + np.arange(4) * math.pi / 2:
        p5 = (1 - x) * E * np.array([1.0, math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
                                     sgn * math.cos(theta)])
        t, tb = two_body(PA + PB - KO - p5, NSTAR)
        mom = [PA, PB, t, tb, None, None]
        mom[emit], mom[9 - emit] = p5, KO
        full = ident * oracle_mod.me(proc, np.array([mom]), params=par)["me"][0]
        rs.append(full / (gs2 * P / (x * mdot(pbeam, p5)) * red))
    return float(np.mean(rs))


@pytest.mark.parametrize("proc,born,beam,split,emit,ident", [
    (QQGG, "u u~ > t t~ g", 0, "qq", 5, 2.0), (QQGG, "u u~ > t t~ g", 1, "qq", 5, 2.0),
    (GGQQ, "u~ g > t t~ u~", 0, "qg", 4, 1.0), (GGQQ, "u g > t t~ u", 0, "qg", 5, 1.0),
    (QGQG, "u g > t t~ u", 1, "gg", 5, 1.0), (QGQG, "u g > t t~ u", 0, "qq", 5, 1.0),
    (QGQG, "g g > t t~ g", 0, "gq", 4, 1.0), (QGQG, "u u~ > t t~ g", 1, "qg", 4, 1.0),
    (QXGQXG, "u~ g > t t~ u~", 1, "gg", 5, 1.0),
])
def test_initial_state_collinear_limit(oracle_mod, proc, born, beam, split, emit, ident):
    # ident = 2 where the two final gluons are identical (IDEN 72 against 36)
    par = oracle_mod.Params(wt=0.0, zero_width_tchan=1)
    d2 = abs(_collinear_ratio(oracle_mod, proc, born, beam, split, emit, par, 1e-2, ident=ident) - 1)
    d3 = abs(_collinear_ratio(oracle_mod, proc, born, beam, split, emit, par, 1e-3, ident=ident) - 1)
    assert d3 < 2e-5 and d3 < 0.05 * d2 + 1e-9, (d2, d3)
