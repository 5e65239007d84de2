"""Pins of the oracle's four-quark channels of p p -> t tbar + 2 jets with two light quarks of
different flavours (u u~ > t t~ d d~ in both beam orders, u d > t t~ u d, u d~ > t t~ u d~,
u~ d~ > t t~ u~ d~): three fermion lines joined by gluons, 7 Feynman diagrams with
explicit colour indices.

* The final-state collinear limit of the d d~ pair of u u~ -> t t~ d d~ onto
  u u~ -> t t~ g with the splitting function T_R (z^2 + (1 - z)^2) (azimuthally averaged;
  the parent is a gluon).
* Initial-state collinear limits where a light quark keeps going into the final state and
  a spacelike gluon enters the hard process (P_gq, azimuthally averaged) onto the pinned
  one-jet channels g u > t t~ u, u g > t t~ u and g u~ > t t~ u~.
* Lorentz invariance, beam order, charge conjugation, the flows rebuilding every helicity
  and their colour matrix against an explicit sum.

One light flavour (u u > t t~ u u, u~ u~ > t t~ u~ u~, u u~ > t t~ u u~ in both beam
orders) adds the second pairing of the light quarks with the sign -1 of exchanging
identical fermions.  That sign is pinned by Pauli antisymmetry: with two identical final
quarks of equal momentum and helicity the amplitude is antisymmetric in their colours
(and the one-pairing amplitude of the distinct-flavour channel at the same point is not).
The q qbar channel uses the same rule (the second pairing exchanges the two light
column ends); its two pairings are pinned separately by their collinear limits.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps
from tests.test_oracle_qq_jet import CF, E, NSTAR, PA, PB, TR, mdot, random_lorentz, two_body

UUDD = "u u~ > t t~ d d~"
UXUDD = "u~ u > t t~ d d~"
UDUD = "u d > t t~ u d"
UDXUDX = "u d~ > t t~ u d~"
UXDX = "u~ d~ > t t~ u~ d~"
ALL = (UUDD, UXUDD, UDUD, UDXUDX, UXDX)
KO = 0.25 * E * np.array([1.0, math.sin(1.3) * math.cos(0.3), math.sin(1.3) * math.sin(0.3), math.cos(1.3)])


def test_colour_matrix_of_the_six_flows(oracle_mod):
    # flows over (B0, K0, B1, K1, t, y): d_{B0 K_s0} d_{B1 K_s1} d_{t K_s2} for the
    # permutations s of the column ends in lexicographic order
    d = np.eye(3)
    flows = []
    for s in itertools.permutations(range(3)):
        f = np.zeros((3,) * 6)
        for B0, K0, B1, K1, t, y in itertools.product(range(3), repeat=6):
            K = (K0, K1, y)
            f[B0, K0, B1, K1, t, y] = d[B0, K[s[0]]] * d[B1, K[s[1]]] * d[t, K[s[2]]]
        flows.append(f.ravel())
    F = np.array(flows)
    assert np.linalg.matrix_rank(F) == 6
    for proc in ALL:
        num, den = oracle_mod.colour_matrix(proc)
        np.testing.assert_allclose(num / den, F @ F.T)


@pytest.mark.parametrize("proc", ALL)
def test_flows_rebuild_every_helicity(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, 4, seed=13)
    r = oracle_mod.me(proc, mom, want_hel=True, want_jamp=True)
    num, den = oracle_mod.colour_matrix(proc)
    J = r["jamp"]
    rebuilt = np.einsum("ehi,ij,ehj->eh", J.conj(), num / den, J).real
    np.testing.assert_allclose(rebuilt, r["me_hel"], rtol=1e-11, atol=1e-13 * r["me_hel"].max())
    # two massless light lines: a quarter of the helicities survive
    assert np.count_nonzero(r["me_hel"].max(axis=0) > 1e-20 * r["me_hel"].max()) == 16


@pytest.mark.parametrize("proc", ALL)
def test_lorentz_invariance(oracle_mod, proc):
    rng = np.random.default_rng(25)
    mom, _, _, _ = ps.make_batch(proc, 20, seed=27)
    par = oracle_mod.Params(wt=0.0)
    ref = oracle_mod.me(proc, mom, params=par)["me"]
    got = oracle_mod.me(proc, np.einsum("ij,epj->epi", random_lorentz(rng), mom), params=par)["me"]
    assert np.max(np.abs(got / ref - 1)) < 1e-11


def test_beam_order(oracle_mod):
    mom, _, _, _ = ps.make_batch(UUDD, 20, seed=29)
    swapped = mom.copy()
    swapped[:, [0, 1]] = mom[:, [1, 0]]
    np.testing.assert_allclose(oracle_mod.me(UXUDD, swapped)["me"], oracle_mod.me(UUDD, mom)["me"], rtol=1e-12)


def test_charge_conjugation(oracle_mod):
    # C maps u d -> t(p3) t~(p4) u d to u~ d~ -> t~(p3) t(p4) u~ d~
    mom, _, _, _ = ps.make_batch(UDUD, 20, seed=30)
    np.testing.assert_allclose(oracle_mod.me(UXDX, mom[:, [0, 1, 3, 2, 4, 5]])["me"],
                               oracle_mod.me(UDUD, mom)["me"], rtol=1e-12)


def test_final_state_g_to_quark_pair(oracle_mod):
    """d d~ collinear in u u~ -> t t~ d d~: sum |M|^2 -> (8 pi alpha_s / s_dd) T_R
    (z^2 + (1 - z)^2) sum |M(u u~ -> t t~ g)|^2 (same initial-state averaging)"""
    par = oracle_mod.Params(wt=0.0)
    gs2 = 4 * math.pi * par.alphas
    n = np.array([math.sin(1.3) * math.cos(0.3), math.sin(1.3) * math.sin(0.3), math.cos(1.3)])
    u = np.cross(n, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    Eg, z = 300.0, 0.35
    pg = Eg * np.concatenate([[1.0], n])
    t0, tb0 = two_body(PA + PB - pg, NSTAR)
    red = oracle_mod.me("u u~ > t t~ g", np.array([[PA, PB, t0, tb0, pg]]), params=par)["me"][0]
    P = TR * (z * z + (1 - z) ** 2)
    dev = []
    for th in (1e-2, 1e-3):
        rs = []
        for phi in 0.2 + np.arange(4) * math.pi / 2:
            nd = math.cos(th) * n + math.sin(th) * (math.cos(phi) * u + math.sin(phi) * v)
            pd, pdb = z * pg, (1 - z) * Eg * np.concatenate([[1.0], nd])
            t, tb = two_body(PA + PB - pd - pdb, NSTAR)
            full = oracle_mod.me(UUDD, np.array([[PA, PB, t, tb, pd, pdb]]), params=par)["me"][0]
            rs.append(full / (gs2 * P / mdot(pd, pdb) * red))
        dev.append(abs(np.mean(rs) - 1))
    assert dev[1] < 2e-5 and dev[1] < 0.05 * dev[0], dev


@pytest.mark.parametrize("proc,born,beam,emit", [(UDUD, "g u > t t~ u", 0, 4), (UDUD, "u g > t t~ u", 1, 5),
                                                 (UDXUDX, "u g > t t~ u", 1, 5), (UDXUDX, "g u~ > t t~ u~", 0, 4),
                                                 (UXDX, "g u~ > t t~ u~", 0, 4)])
def test_initial_state_collinear_limit(oracle_mod, proc, born, beam, emit):
    """the final quark in slot emit collinear to the beam of its own flavour (fraction
    1 - x): P_gq onto the one-jet channel with a gluon of momentum x p in that beam"""
    par = oracle_mod.Params(wt=0.0, zero_width_tchan=1)
    gs2 = 4 * math.pi * par.alphas
    x = 0.6
    P = CF * (1 + (1 - x) ** 2) / x
    pbeam, sgn = (PA, 1.0) if beam == 0 else (PB, -1.0)
    pa2, pb2 = (x * PA, PB) if beam == 0 else (PA, x * PB)
    t0, tb0 = two_body(pa2 + pb2 - KO, NSTAR)
    red = oracle_mod.me(born, np.array([[pa2, pb2, t0, tb0, KO]]), params=par)["me"][0]
    dev = []
    for th in (1e-2, 1e-3):
        rs = []
        for phi in 0.3 + np.arange(4) * math.pi / 2:
            p5 = (1 - x) * E * np.array([1.0, math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi),
                                         sgn * math.cos(th)])
            t, tb = two_body(PA + PB - KO - p5, NSTAR)
            mom = [PA, PB, t, tb, None, None]
            mom[emit], mom[9 - emit] = p5, KO
            full = oracle_mod.me(proc, np.array([mom]), params=par)["me"][0]
            rs.append(full / (gs2 * P / (x * mdot(pbeam, p5)) * red))
        dev.append(abs(np.mean(rs) - 1))
    assert dev[1] < 1e-5 and dev[1] < 0.05 * dev[0], dev


# ---------------------------------------------------------------------------
# one light flavour: both pairings of the light quarks, the second with the sign -1
UUUU = "u u > t t~ u u"
UXUXUX = "u~ u~ > t t~ u~ u~"
UUXUUX = "u u~ > t t~ u u~"
UXUUUX = "u~ u > t t~ u u~"
SAME = (UUUU, UXUXUX, UUXUUX, UXUUUX)


def _flow_tensors():
    d = np.eye(3)
    out = []
    for s in itertools.permutations(range(3)):
        f = np.zeros((3,) * 6)
        for B0, K0, B1, K1, t, y in itertools.product(range(3), repeat=6):
            K = (K0, K1, y)
            f[B0, K0, B1, K1, t, y] = d[B0, K[s[0]]] * d[B1, K[s[1]]] * d[t, K[s[2]]]
        out.append(f)
    return np.array(out)


@pytest.mark.parametrize("proc,slots,axes", [(UUUU, (4, 5), (0, 2)), (UXUXUX, (4, 5), (1, 3))])
def test_pauli_antisymmetry(oracle_mod, proc, slots, axes):
    """two identical final quarks with the same momentum: for equal helicities the
    amplitude is antisymmetric under exchange of their colours (the two row ends B0, B1
    for quarks, the two column ends K0, K1 for antiquarks), which fixes the relative sign
    of the two pairings; the distinct-flavour amplitude at the same point (one pairing)
    is not antisymmetric"""
    from tests.collinear import top_pair
    rng = np.random.default_rng(31)
    F = _flow_tensors()
    for _ in range(3):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        q = rng.uniform(100.0, 250.0) * np.concatenate([[1.0], u])
        mom = np.array([[PA, PB] + top_pair(PA + PB - 2 * q, 173.0, rng) + [q, q]])
        for p, expect_anti in ((proc, True), (UDUD if proc == UUUU else UXDX, False)):
            J = oracle_mod.me(p, mom, want_jamp=True)["jamp"][0]
            worst = norm = 0.0
            for hel in range(64):
                if ((hel >> (5 - slots[0])) & 1) != ((hel >> (5 - slots[1])) & 1):
                    continue
                M = np.einsum("n,nabcdef->abcdef", J[hel], F)
                worst = max(worst, np.abs(M + np.swapaxes(M, *axes)).max())
                norm = max(norm, np.abs(M).max())
            assert norm > 0
            if expect_anti:
                assert worst <= 1e-13 * norm, (p, worst / norm)
            else:
                assert worst > 1e-3 * norm, (p, worst / norm)


@pytest.mark.parametrize("proc", SAME)
def test_same_flavour_flows_and_lorentz(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, 6, seed=32)
    r = oracle_mod.me(proc, mom, want_hel=True, want_jamp=True)
    num, den = oracle_mod.colour_matrix(proc)
    J = r["jamp"]
    np.testing.assert_allclose(np.einsum("ehi,ij,ehj->eh", J.conj(), num / den, J).real, r["me_hel"],
                               rtol=1e-11, atol=1e-13 * r["me_hel"].max())
    par = oracle_mod.Params(wt=0.0)
    ref = oracle_mod.me(proc, mom, params=par)["me"]
    got = oracle_mod.me(proc, np.einsum("ij,epj->epi", random_lorentz(np.random.default_rng(33)), mom), params=par)["me"]
    assert np.max(np.abs(got / ref - 1)) < 1e-11


@pytest.mark.parametrize("proc,perm", [(UUUU, [0, 1, 2, 3, 5, 4]), (UUUU, [1, 0, 2, 3, 4, 5]),
                                       (UXUXUX, [0, 1, 2, 3, 5, 4])])
def test_same_flavour_bose_fermi_relabelling(oracle_mod, proc, perm):
    # the summed |M|^2 is symmetric under exchange of identical particles
    mom, _, _, _ = ps.make_batch(proc, 12, seed=34)
    np.testing.assert_allclose(oracle_mod.me(proc, mom[:, perm])["me"], oracle_mod.me(proc, mom)["me"], rtol=1e-12)


def test_same_flavour_beam_order_and_charge_conjugation(oracle_mod):
    mom, _, _, _ = ps.make_batch(UUXUUX, 12, seed=35)
    sw = mom.copy()
    sw[:, [0, 1]] = mom[:, [1, 0]]
    np.testing.assert_allclose(oracle_mod.me(UXUUUX, sw)["me"], oracle_mod.me(UUXUUX, mom)["me"], rtol=1e-12)
    mom, _, _, _ = ps.make_batch(UUUU, 12, seed=36)
    np.testing.assert_allclose(oracle_mod.me(UXUXUX, mom[:, [0, 1, 3, 2, 4, 5]])["me"], oracle_mod.me(UUUU, mom)["me"],
                               rtol=1e-12)


@pytest.mark.parametrize("proc,born,beam,emit,ident", [(UUUU, "g u > t t~ u", 0, 4, 2.0),
                                                       (UUXUUX, "g u~ > t t~ u~", 0, 4, 1.0),
                                                       (UUXUUX, "u g > t t~ u", 1, 5, 1.0)])
def test_same_flavour_initial_state_collinear_limit(oracle_mod, proc, born, beam, emit, ident):
    """one pairing singular: P_gq onto the one-jet channel (ident = 2 where the two final
    quarks are identical, IDEN 72 against 36)"""
    par = oracle_mod.Params(wt=0.0, zero_width_tchan=1)
    gs2 = 4 * math.pi * par.alphas
    x = 0.6
    P = CF * (1 + (1 - x) ** 2) / x
    pbeam, sgn = (PA, 1.0) if beam == 0 else (PB, -1.0)
    pa2, pb2 = (x * PA, PB) if beam == 0 else (PA, x * PB)
    t0, tb0 = two_body(pa2 + pb2 - KO, NSTAR)
    red = oracle_mod.me(born, np.array([[pa2, pb2, t0, tb0, KO]]), params=par)["me"][0]
    dev = []
    for th in (1e-2, 1e-3):
        rs = []
        for phi in 0.3 + np.arange(4) * math.pi / 2:
            p5 = (1 - x) * E * np.array([1.0, math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi),
                                         sgn * math.cos(th)])
            t, tb = two_body(PA + PB - KO - p5, NSTAR)
            mom = [PA, PB, t, tb, None, None]
            mom[emit], mom[9 - emit] = p5, KO
            full = ident * oracle_mod.me(proc, np.array([mom]), params=par)["me"][0]
            rs.append(full / (gs2 * P / (x * mdot(pbeam, p5)) * red))
        dev.append(abs(np.mean(rs) - 1))
    assert dev[1] < 1e-5 and dev[1] < 0.05 * dev[0], dev


def test_same_flavour_final_state_g_to_quark_pair(oracle_mod):
    """u u~ final pair collinear in u u~ -> t t~ u u~: the annihilation pairing onto
    u u~ -> t t~ g"""
    par = oracle_mod.Params(wt=0.0)
    gs2 = 4 * math.pi * par.alphas
    n = np.array([math.sin(1.3) * math.cos(0.3), math.sin(1.3) * math.sin(0.3), math.cos(1.3)])
    u = np.cross(n, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    v = np.cross(n, u)
    Eg, z = 300.0, 0.35
    pg = Eg * np.concatenate([[1.0], n])
    t0, tb0 = two_body(PA + PB - pg, NSTAR)
    red = oracle_mod.me("u u~ > t t~ g", np.array([[PA, PB, t0, tb0, pg]]), params=par)["me"][0]
    P = TR * (z * z + (1 - z) ** 2)
    dev = []
    for th in (1e-2, 1e-3):
        rs = []
        for phi in 0.2 + np.arange(4) * math.pi / 2:
            nd = math.cos(th) * n + math.sin(th) * (math.cos(phi) * u + math.sin(phi) * v)
            pq, pqb = z * pg, (1 - z) * Eg * np.concatenate([[1.0], nd])
            t, tb = two_body(PA + PB - pq - pqb, NSTAR)
            full = oracle_mod.me(UUXUUX, np.array([[PA, PB, t, tb, pq, pqb]]), params=par)["me"][0]
            rs.append(full / (gs2 * P / mdot(pq, pqb) * red))
        dev.append(abs(np.mean(rs) - 1))
    assert dev[1] < 2e-5 and dev[1] < 0.05 * dev[0], dev
