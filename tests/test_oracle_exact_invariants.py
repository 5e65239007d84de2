"""Pin of the oracle's propagator invariants against exact rational arithmetic.

The recursion of the oracle takes every gluon invariant K^2 and every top-line
denominator q^2 - mt^2 from a per-event table formed in quadruple precision.  Here each
entry is compared with the exact value of the same expression on the same FP64 inputs,
computed with Python fractions.  The events include nearly collinear gluons whose
invariant is 1e4 to 1e6 times smaller than the square of the summed energies, where a
plain FP64 square loses 1e-12 or more; the oracle's entries must still be the exact
value rounded once (within 2^-52 relative).
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps
from tests.collinear import COLLINEAR_TERMS, GGTTG, GGTTGG, collinear_events

ROLES = {"g g > t t~": "ggtb", "g g > t t~ g": "ggtbg", "g g > t t~ g g": "ggtbgg",
         "g g > t t~ g g g": "ggtbggg"}
MT = 173.0


def exact_tables(process, mom_e):
    """{mask: exact K^2} and {mask: exact q^2 - mt^2} for every non-empty gluon subset"""
    npar = mom_e.shape[0]
    gluons = [i for i in range(npar) if i not in (2, 3)]
    kin = {i: [Fraction(x) * (1 if i < 2 else -1) for x in mom_e[i]] for i in gluons}
    pt = [Fraction(x) for x in mom_e[2]]
    gsq, tden = {}, {}
    for mask in range(1, 1 << npar):
        members = [i for i in range(npar) if mask >> i & 1]
        if any(i not in gluons for i in members):
            continue
        K = [sum(kin[i][m] for i in members) for m in range(4)]
        q = [pt[m] - K[m] for m in range(4)]
        gsq[mask] = K[0] ** 2 - K[1] ** 2 - K[2] ** 2 - K[3] ** 2
        tden[mask] = q[0] ** 2 - q[1] ** 2 - q[2] ** 2 - q[3] ** 2 - Fraction(MT) ** 2
    return gsq, tden


def check_event(g_row, t_row, gsq, tden):
    worst = 0.0
    for mask, ex in gsq.items():
        # (a single gluon's entry is the exact p^2 of its rounded momentum, near 0)
        if ex == 0:
            assert g_row[mask] == 0.0
            continue
        rel = abs(Fraction(g_row[mask]) / ex - 1)
        worst = max(worst, float(rel))
    for mask, ex in tden.items():
        rel = abs(Fraction(t_row[mask]) / ex - 1)
        worst = max(worst, float(rel))
    return worst


@pytest.mark.parametrize("process", [GGTTG, GGTTGG])
def test_invariants_exact_on_nearly_collinear_events(oracle_mod, process):
    mom = collinear_events(process, 24, seed=31)
    # the inputs are as ill-conditioned as intended: the plain FP64 square of the
    # collinear pair misses its exact value by more than 1e-12 in the median
    terms = COLLINEAR_TERMS[process]
    k = sum(sg * mom[:, i] for sg, i in terms)
    plain = k[:, 0] ** 2 - k[:, 1] ** 2 - k[:, 2] ** 2 - k[:, 3] ** 2
    mask = sum(1 << i for _, i in terms if i >= 4) | (1 if process == GGTTG else 0)
    gsq_o, tden_o = oracle_mod.invariants(process, mom)
    exact = []
    worst = 0.0
    for e in range(mom.shape[0]):
        gsq, tden = exact_tables(process, mom[e])
        exact.append(float(gsq[mask]))
        worst = max(worst, check_event(gsq_o[e], tden_o[e], gsq, tden))
    exact = np.array(exact)
    assert np.median(np.abs(plain / exact - 1)) > 1e-12
    esum = sum(mom[:, i, 0] for _, i in terms)
    assert (esum ** 2 / np.abs(exact)).min() > 1e4  # conditioning of the collinear invariant
    assert worst <= 2.0 ** -52, worst


@pytest.mark.parametrize("process", list(ROLES))
def test_invariants_exact_on_rambo_events(oracle_mod, process):
    mom, _, _, _ = ps.make_batch(process, 6, seed=5)
    gsq_o, tden_o = oracle_mod.invariants(process, mom)
    for e in range(mom.shape[0]):
        gsq, tden = exact_tables(process, mom[e])
        assert check_event(gsq_o[e], tden_o[e], gsq, tden) <= 2.0 ** -52
        # masks holding a top or antitop have no entry
        assert gsq_o[e][1 << 2] == 0.0 and tden_o[e][(1 << 3) | 1] == 0.0
