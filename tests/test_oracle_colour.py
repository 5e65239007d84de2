"""Pins of the oracle's colour algebra and of its colour-ordered recursion.

* The Fierz-evaluated colour matrix C_st = Tr(T^s (T^t)^dagger) equals the same trace
  summed over explicit Gell-Mann matrices (brute force) entry by entry for two to five
  gluons, is symmetric positive semi-definite, and has the closed-form diagonal C_F^n N.
* The full spin- and colour-summed |M|^2 for g g -> t t~ and g g -> t t~ g equals an
  explicit-colour Feynman-rule computation (tests/explicit_colour.py) that uses no
  colour decomposition at all.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps
from tests import explicit_colour as ec

QCD = ["g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g"]


def brute_colour_matrix(n):
    perms = list(itertools.permutations(range(n)))
    C = np.zeros((len(perms), len(perms)))
    for a in itertools.product(range(8), repeat=n):
        prods = []
        for p in perms:
            m = np.eye(3, dtype=complex)
            for j in p:
                m = m @ ec.T[a[j]]
            prods.append(m)
        for s, ms in enumerate(prods):
            for t, mt in enumerate(prods):
                C[s, t] += np.real(np.trace(ms @ mt.conj().T))
    return C


def brute_colour_matrix_batched(n, chunk=4096):
    """The same explicit sum over all 8^n colour assignments, vectorised: for a chunk of
    assignments, the string products of every ordering are formed as batched 3x3
    products and C += Re(X X^dagger) over the flattened (assignment, i, j) axis."""
    perms = list(itertools.permutations(range(n)))
    assign = np.array(list(itertools.product(range(8), repeat=n)), dtype=np.int64)
    C = np.zeros((len(perms), len(perms)))
    for a0 in range(0, len(assign), chunk):
        a = assign[a0:a0 + chunk]
        X = np.empty((len(perms), len(a), 9), dtype=complex)
        for s, p in enumerate(perms):
            m = ec.T[a[:, p[0]]]
            for j in p[1:]:
                m = m @ ec.T[a[:, j]]
            X[s] = m.reshape(len(a), 9)
        X = X.reshape(len(perms), -1)
        C += np.real(X @ X.conj().T)
    return C


def test_ggtt_colour_matrix_exact(oracle_mod):
    num, den = oracle_mod.colour_matrix("g g > t t~")
    assert np.array_equal(num * (3 // den), np.array([[16, -2], [-2, 16]]))


@pytest.mark.parametrize("n,proc", [(2, "g g > t t~"), (3, "g g > t t~ g")])
def test_colour_matrix_matches_explicit_sum(oracle_mod, n, proc):
    num, den = oracle_mod.colour_matrix(proc)
    assert np.allclose(num / den, brute_colour_matrix(n), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("n,proc", [(2, "g g > t t~"), (3, "g g > t t~ g"), (4, "g g > t t~ g g"),
                                    (5, "g g > t t~ g g g")])
def test_colour_matrix_matches_explicit_sum_every_entry(oracle_mod, n, proc):
    """Entry by entry against the explicit Gell-Mann sum for 24 and 120 flows too, so
    that a wrong power of 1/N in an off-diagonal entry cannot hide behind permutation
    covariance.  The sum runs in FP64 over 8^n terms of size O(1); every exact entry
    is a rational with denominator dividing 324."""
    num, den = oracle_mod.colour_matrix(proc)
    B = brute_colour_matrix_batched(n)
    assert B.shape == num.shape
    assert np.max(np.abs(num / den - B)) < 1e-10
    # the brute force resolves every distinct entry: rounding it to the oracle's
    # denominators gives back the oracle's numerators exactly
    assert np.array_equal(np.rint(B * den).astype(np.int64), num)


@pytest.mark.parametrize("proc", QCD)
def test_colour_matrix_structure(oracle_mod, proc):
    num, den = oracle_mod.colour_matrix(proc)
    C = num / den
    n = {2: 2, 6: 3, 24: 4, 120: 5}[C.shape[0]]
    assert np.array_equal(num * den.T, num.T * den)  # exact symmetry
    # diagonal: Tr(T^a1..T^an T^an..T^a1) = C_F^n N
    assert np.allclose(np.diag(C), (4.0 / 3.0) ** n * 3)
    w = np.linalg.eigvalsh(C)
    assert w.min() > -1e-12 * w.max()
    # colour sum of the all-gluon string against itself summed over orderings:
    # sum_{s,t} C_st = Tr(S S^dagger) with S = sum_s T^s; checked against the explicit sum
    if n <= 3:
        assert abs(C.sum() - brute_colour_matrix(n).sum()) < 1e-10


@pytest.mark.parametrize("proc,roles", [
    ("g g > t t~", ["gin", "gin", "t", "tb"]),
    ("g g > t t~ g", ["gin", "gin", "t", "tb", "gout"]),
])
def test_explicit_colour_brute_force(oracle_mod, proc, roles):
    mom, _, _, _ = ps.make_batch(proc, 3, seed=21)
    par = oracle_mod.Params(wt=0.0)
    out = oracle_mod.me(proc, mom, params=par)
    npar, ncomb, ncol, iden = oracle_mod.info(proc)
    gs = math.sqrt(4 * math.pi * 0.118)
    for e in range(mom.shape[0]):
        ref = ec.summed_me2(mom[e], 173.0, gs, roles) / iden
        assert abs(out["me"][e] / ref - 1) < 1e-12, (e, out["me"][e], ref)


@pytest.mark.parametrize("zwt", [0, 1])
def test_explicit_colour_top_width_and_zero_width_tchannel(oracle_mod, zwt):
    """g g > t t~ g at the physical top width: the oracle's width per top propagator,
    in every one (zwt = 0) or only where the propagator is not in the t channel
    (zwt = 1), equals the explicit-colour computation with its own per-propagator
    width rule.  On these events the width moves |M|^2 far above the tolerance, in the
    s-channel propagators (top + final gluon) as well as in the t-channel ones, so a
    rule that dropped the width from the wrong propagators would fail."""
    proc, roles = "g g > t t~ g", ["gin", "gin", "t", "tb", "gout"]
    cand, _, _, _ = ps.make_batch(proc, 64, seed=23)
    # the event of this seeded batch whose s-channel top propagator (top or antitop plus
    # the final gluon) is nearest its pole, where the width matters most
    dots = lambda a, b: a[..., 0] * b[..., 0] - np.sum(a[..., 1:] * b[..., 1:], axis=-1)
    near = np.minimum(dots(cand[:, 2], cand[:, 4]), dots(cand[:, 3], cand[:, 4]))
    mom = cand[np.argsort(near)[:1]]
    wt = 1.4915
    gs = math.sqrt(4 * math.pi * 0.118)
    _, _, _, iden = oracle_mod.info(proc)
    out = oracle_mod.me(proc, mom, params=oracle_mod.Params(wt=wt, zero_width_tchan=zwt))["me"]
    for e in range(mom.shape[0]):
        ref = ec.summed_me2(mom[e], 173.0, gs, roles, wt=wt, zero_width_tchan=bool(zwt)) / iden
        assert abs(out[e] / ref - 1) < 1e-12, (e, out[e], ref)
        # the other rules differ by far more than the tolerance
        for other in ({"wt": 0.0}, {"wt": wt, "zero_width_tchan": not zwt}):
            alt = ec.summed_me2(mom[e], 173.0, gs, roles, **other) / iden
            assert abs(alt / ref - 1) > 1e-8, (e, other, abs(alt / ref - 1))
