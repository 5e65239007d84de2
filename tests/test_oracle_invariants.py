"""Invariance pins of the oracle on every process.

* Lorentz invariance of the helicity-summed |M|^2 under a random rotation and boost
  (zero top width: with a fixed width the Ward identity fails at O(width/mass), so the
  sum over the two physical, frame-dependent gluon polarisations is not exactly frame
  independent; the residual with the physical width is checked separately).
* Gauge invariance: with one gluon's polarisation replaced by its momentum (k/E) and
  every other leg physical, each colour-ordered amplitude vanishes (zero top width,
  since a fixed width breaks the Ward identity).
* Bose symmetry under exchange of two identical gluons (initial or final).
* alpha_s scaling: pure-QCD |M|^2 is proportional to alpha_s^(npar-2).
* Positivity of every |M_h|^2 and of the sum; helicity count 2^npar.
"""
import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

ALL = ["e+ e- > mu+ mu-", "g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"]
QCD = ALL[1:]
NEV = {"e+ e- > mu+ mu-": 200, "g g > t t~": 200, "g g > t t~ g": 100, "g g > t t~ g g": 40,
       "g g > t t~ g g g": 6}


def random_lorentz(rng):
    # rotation from a random unit quaternion, then a boost with |eta| <= 2 along a random axis
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    R = np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                  [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                  [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    eta = rng.uniform(-2, 2)
    ch, sh = np.cosh(eta), np.sinh(eta)
    L = np.eye(4)
    L[1:, 1:] = R
    B = np.eye(4)
    B[0, 0] = ch
    B[0, 1:] = B[1:, 0] = sh * n
    B[1:, 1:] = np.eye(3) + (ch - 1) * np.outer(n, n)
    return B @ L


@pytest.mark.parametrize("proc", ALL)
def test_lorentz_invariance(oracle_mod, proc):
    rng = np.random.default_rng(1)
    mom, _, _, _ = ps.make_batch(proc, NEV[proc], seed=4)
    par = oracle_mod.Params(wt=0.0)
    ref = oracle_mod.me(proc, mom, params=par)["me"]
    for _ in range(2):
        L = random_lorentz(rng)
        mom2 = np.einsum("ij,epj->epi", L, mom)
        got = oracle_mod.me(proc, mom2, params=par)["me"]
        assert np.max(np.abs(got / ref - 1)) < 1e-11


def test_lorentz_residual_with_width(oracle_mod):
    # with the physical top width the frame dependence stays far below the width effect
    rng = np.random.default_rng(2)
    mom, _, _, _ = ps.make_batch("g g > t t~ g", 50, seed=4)
    ref = oracle_mod.me("g g > t t~ g", mom)["me"]
    got = oracle_mod.me("g g > t t~ g", np.einsum("ij,epj->epi", random_lorentz(rng), mom))["me"]
    assert np.max(np.abs(got / ref - 1)) < 1e-5


@pytest.mark.parametrize("proc", QCD)
def test_gauge_invariance(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, min(NEV[proc], 20), seed=6)
    par = oracle_mod.Params(wt=0.0)
    phys = oracle_mod.me(proc, mom, params=par, want_jamp=True)["jamp"]
    npar = mom.shape[1]
    gluons = [0, 1] + list(range(4, npar))
    for leg in gluons:
        gauge = oracle_mod.me(proc, mom, params=par, want_jamp=True, gauge_leg=leg)["jamp"]
        # per event: every colour-ordered amplitude of every helicity vanishes
        scale = np.abs(phys).max(axis=(1, 2))
        assert np.all(np.abs(gauge).max(axis=(1, 2)) <= 1e-10 * scale), leg


def test_gauge_check_is_sensitive(oracle_mod):
    # the same check fails when the Ward identity is broken (a fixed top width), so it
    # is not vacuous
    mom, _, _, _ = ps.make_batch("g g > t t~ g", 5, seed=6)
    phys = oracle_mod.me("g g > t t~ g", mom, want_jamp=True)["jamp"]
    gauge = oracle_mod.me("g g > t t~ g", mom, want_jamp=True, gauge_leg=4)["jamp"]
    assert np.abs(gauge).max() > 1e-6 * np.abs(phys).max()


@pytest.mark.parametrize("proc", QCD)
def test_bose_symmetry(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, NEV[proc], seed=8)
    ref = oracle_mod.me(proc, mom)["me"]
    npar = mom.shape[1]
    swaps = [(0, 1)] + [(i, j) for i in range(4, npar) for j in range(i + 1, npar)]
    for i, j in swaps:
        m2 = mom.copy()
        m2[:, [i, j]] = m2[:, [j, i]]
        if (i, j) == (0, 1):
            # swapping the beams is a reflection z -> -z; undo it with a rotation about x
            m2[:, :, 2] *= -1
            m2[:, :, 3] *= -1
        got = oracle_mod.me(proc, m2)["me"]
        assert np.max(np.abs(got / ref - 1)) < 1e-12, (i, j)


@pytest.mark.parametrize("proc", QCD)
def test_alphas_scaling(oracle_mod, proc):
    mom, _, _, _ = ps.make_batch(proc, NEV[proc] // 2, seed=10)
    npar = mom.shape[1]
    a1, a2 = 0.118, 0.1
    m1 = oracle_mod.me(proc, mom, alphas=a1)["me"]
    m2 = oracle_mod.me(proc, mom, alphas=a2)["me"]
    assert np.max(np.abs(m1 / m2 / (a1 / a2) ** (npar - 2) - 1)) < 1e-13


@pytest.mark.parametrize("proc", ALL)
def test_positivity_and_helicity_table(oracle_mod, proc):
    mom, _, rh, rc = ps.make_batch(proc, 10, seed=12)
    out = oracle_mod.me(proc, mom, rnd_hel=rh, rnd_col=rc, want_hel=True, want_colw=True)
    npar, ncomb, ncol, iden = oracle_mod.info(proc)
    assert ncomb == 2 ** npar
    assert out["me_hel"].shape == (10, ncomb)
    assert np.all(out["me_hel"] >= 0)
    assert np.allclose(out["me_hel"].sum(1) / iden, out["me"], rtol=1e-14)
    assert np.all(out["me"] > 0)
    # the selected helicity and colour carry non-zero weight
    assert np.all(out["me_hel"][np.arange(10), out["sel_hel"]] > 0)
    assert np.all(out["colw"][np.arange(10), out["sel_col"]] > 0)


def test_selection_rule_definition(oracle_mod):
    # first index whose running sum exceeds r * total, checked by hand on one event
    proc = "g g > t t~ g"
    mom, _, _, _ = ps.make_batch(proc, 1, seed=13)
    for r in (1e-9, 0.3, 0.5, 0.999999):
        out = oracle_mod.me(proc, mom, rnd_hel=[r], rnd_col=[r], want_hel=True, want_colw=True)
        w = out["me_hel"][0]
        c = np.cumsum(w)
        assert out["sel_hel"][0] == int(np.argmax(c > r * w.sum()))
        wc = out["colw"][0]
        assert out["sel_col"][0] == int(np.argmax(np.cumsum(wc) > r * wc.sum()))
