"""Pins of the oracle's quark-initiated channel q qbar -> t tbar (the second channel of
p p -> t tbar), written with explicit colour indices.

* The spin- and colour-averaged |M|^2 equals the closed form of Combridge (Nucl. Phys.
  B151 (1979) 429; Ellis, Stirling, Webber, QCD and Collider Physics, eq. 10.12):
      <|M|^2> = (4/9) g_s^4 (tau1^2 + tau2^2 + rho / 2),
  tau1 = 2 p1.p3 / s, tau2 = 2 p2.p3 / s, rho = 4 mt^2 / s, which reduces to the
  textbook q qbar -> q' qbar' entry (4/9)(t^2 + u^2)/s^2 for mt -> 0.
* The colour matrix of the two flows equals the explicit sum over colour indices of the
  flow tensors, and the flow amplitudes rebuild |M|^2 through it.
* Swapping the beams ("u~ u > t t~" with the momenta of the first two particles
  exchanged) gives the same |M|^2; massless quarks keep only the helicity-conserving
  configurations (8 of 16); Lorentz invariance under a random boost.
"""
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

P = "u u~ > t t~"
PR = "u~ u > t t~"


def combridge(mom, mt, alphas):
    p1, p2, p3 = mom[:, 0], mom[:, 1], mom[:, 2]
    dot = lambda a, b: a[:, 0] * b[:, 0] - np.sum(a[:, 1:] * b[:, 1:], axis=1)
    s = dot(p1 + p2, p1 + p2)
    t1, t2, rho = 2 * dot(p1, p3) / s, 2 * dot(p2, p3) / s, 4 * mt * mt / s
    g4 = (4 * math.pi * alphas) ** 2
    return g4 * 4.0 / 9.0 * (t1 ** 2 + t2 ** 2 + rho / 2)


@pytest.mark.parametrize("mt", [173.0, 1e-3])
def test_qqbar_tt_matches_combridge(oracle_mod, mt):
    mom, _, _, _ = ps.make_batch(P, 200, seed=3, mt=mt)
    par = oracle_mod.Params(mt=mt, wt=0.0)
    got = oracle_mod.me(P, mom, params=par)["me"]
    ref = combridge(mom, mt, 0.118)
    assert np.max(np.abs(got / ref - 1)) < 1e-12


def test_qqbar_colour_flows_rebuild_the_matrix_element(oracle_mod):
    num, den = oracle_mod.colour_matrix(P)
    assert np.array_equal(num, [[9, 3], [3, 9]]) and np.all(den == 1)
    mom, _, rh, rc = ps.make_batch(P, 20, seed=4)
    out = oracle_mod.me(P, mom, rnd_hel=rh, rnd_col=rc, want_hel=True, want_jamp=True, want_colw=True)
    J = out["jamp"]  # [nevt][ncomb][2]
    m2 = np.einsum("ehi,ij,ehj->eh", J.conj(), num / den, J).real
    np.testing.assert_allclose(m2, out["me_hel"], rtol=1e-12, atol=1e-300)
    # the colour factor T^a_{ji} T^a_{kl} = (c_0 - c_1 / 3) / 2: flow 1 is -1/3 of flow 0
    nz = np.abs(J[..., 0]) > 0
    np.testing.assert_allclose(J[..., 1][nz] / J[..., 0][nz], -1.0 / 3.0, rtol=1e-12)
    # helicity conservation on the massless line: 8 of the 16 configurations contribute
    assert np.sum(np.any(out["me_hel"] != 0, axis=0)) == 8


def test_beam_swap_and_lorentz_invariance(oracle_mod):
    mom, _, _, _ = ps.make_batch(P, 50, seed=5)
    a = oracle_mod.me(P, mom)["me"]
    sw = mom.copy()
    sw[:, [0, 1]] = mom[:, [1, 0]]
    b = oracle_mod.me(PR, sw)["me"]
    np.testing.assert_allclose(a, b, rtol=1e-13)
    # boost along a random direction (rapidity 0.7): Lorentz invariant (no width here)
    rng = np.random.default_rng(6)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    eta = 0.7
    ch, sh = np.cosh(eta), np.sinh(eta)
    E, pv = mom[..., 0], mom[..., 1:]
    pn = pv @ n
    boosted = np.empty_like(mom)
    boosted[..., 0] = ch * E + sh * pn
    boosted[..., 1:] = pv + ((ch - 1) * pn + sh * E)[..., None] * n
    par = oracle_mod.Params(wt=0.0)
    np.testing.assert_allclose(oracle_mod.me(P, boosted, params=par)["me"], oracle_mod.me(P, mom, params=par)["me"],
                               rtol=1e-11)
