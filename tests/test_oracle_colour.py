"""Pins of the oracle's colour algebra and of its colour-ordered recursion.

* The Fierz-evaluated colour matrix C_st = Tr(T^s (T^t)^dagger) equals the same trace
  summed over explicit Gell-Mann matrices (brute force) for two and three gluons, is
  symmetric positive semi-definite, and has the closed-form diagonal C_F^n N.
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


def test_ggtt_colour_matrix_exact(oracle_mod):
    num, den = oracle_mod.colour_matrix("g g > t t~")
    assert np.array_equal(num * (3 // den), np.array([[16, -2], [-2, 16]]))


@pytest.mark.parametrize("n,proc", [(2, "g g > t t~"), (3, "g g > t t~ g")])
def test_colour_matrix_matches_explicit_sum(oracle_mod, n, proc):
    num, den = oracle_mod.colour_matrix(proc)
    assert np.allclose(num / den, brute_colour_matrix(n), rtol=1e-13, atol=1e-13)


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
