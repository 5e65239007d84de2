"""Absolute pin of the oracle's colour-ordered amplitudes for any number of gluons:
the Parke-Taylor formula for maximally-helicity-violating (MHV) amplitudes.

With massless quarks, the tree-level colour-ordered amplitude of an antiquark, a quark
and n_g gluons in the all-outgoing convention, cyclic order (q, g_s1, ..., g_sn, qbar),
has a closed form when exactly two particles have negative helicity (one of them a
quark): its modulus squared is

    |A|^2 = |s_{-j}|^3 |s_{+j}| / prod_{cyclic neighbours (a, b)} |s_ab|,   s_ab = 2 p_a.p_b

with j the negative-helicity gluon, '-' ('+') the quark of negative (positive) helicity
(Parke & Taylor, Phys. Rev. Lett. 56 (1986) 2459; Mangano & Parke, Phys. Rep. 200
(1991) 301, with generators normalised to Tr(T^a T^b) = delta^ab).  The parity image
(exactly two positive helicities) is the same with the signs exchanged.  The oracle
decomposes in generators with Tr(T^a T^b) = delta^ab / 2 and keeps the coupling in its
flow amplitudes, so its J of flow (T^{a_s1} ... T^{a_sn})_{i_t j_tbar} must be
(sqrt(2) g_s)^{n_g} times that amplitude:  |J|^2 = (2 g_s^2)^{n_g} |A|^2 -- for every
ordering, every MHV helicity, every phase-space point and every n_g.  Helicity
amplitudes with equal quark helicities or with fewer than two negative (or positive)
helicities vanish.

This checks the Berends-Giele recursion of the oracle for 2 to 5 gluons in absolute
normalisation, independently of the closed forms for gg -> ttbar: a dropped current,
a wrong vertex sign, a mis-ordered flow or a wrong coupling power breaks the ratio.
The physical top mass only enters the massive spinors and propagator denominators
pinned elsewhere (closed forms, gauge invariance); here the tops are made massless.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2312_02898_b300.phasespace import make_batch

PROCS = ("g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g")
ALPHAS = 0.118
T, TBAR = 2, 3  # particle positions of t and t~


def _mdot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def _classify(hout):
    """("mhv"|"mhvbar", quark of the cubed invariant, the other quark, gluon j); "zero"
    for a helicity amplitude that vanishes; None where no one-line closed form exists"""
    n = len(hout)
    if hout[T] == hout[TBAR]:
        return "zero"
    neg = [i for i in range(n) if hout[i] < 0]
    pos = [i for i in range(n) if hout[i] > 0]
    if len(neg) < 2 or len(pos) < 2:
        return "zero"
    if len(neg) == 2:  # MHV: one quark and one gluon negative
        q = T if hout[T] < 0 else TBAR
        j = next(i for i in neg if i not in (T, TBAR))
        return ("mhv", q, TBAR if q == T else T, j)
    if len(pos) == 2:  # parity image
        q = T if hout[T] > 0 else TBAR
        j = next(i for i in pos if i not in (T, TBAR))
        return ("mhvbar", q, TBAR if q == T else T, j)
    return None  # NMHV and beyond: no one-line closed form


@pytest.mark.parametrize("process", PROCS)
def test_flow_amplitudes_are_parke_taylor_times_coupling(process):
    npar, ncomb, ncol, _ = oracle.info(process)
    ng = npar - 2
    mom = make_batch(process, 3, seed=21, mt=0.0)[0]
    out = oracle.me(process, mom, params=oracle.Params(mt=0.0, wt=0.0, alphas=ALPHAS), want_jamp=True)
    J = out["jamp"]
    gluons = [0, 1] + list(range(4, npar))
    flows = list(itertools.permutations(gluons))  # lexicographic: the flow index
    assert len(flows) == ncol
    want = (2.0 * 4.0 * np.pi * ALPHAS) ** ng
    n_mhv = 0
    for e in range(mom.shape[0]):
        p = mom[e] * np.array([-1, -1] + [1] * (npar - 2))[:, None]  # all outgoing
        s = lambda a, b: abs(2.0 * _mdot(p[a], p[b]))
        typical = np.sqrt(np.mean(np.abs(J[e]) ** 2))
        for h in range(ncomb):
            hel = [1 if (h >> (npar - 1 - i)) & 1 else -1 for i in range(npar)]
            hout = [-hel[i] if i < 2 else hel[i] for i in range(npar)]  # crossing flips incoming helicities
            kind = _classify(hout)
            if kind == "zero":
                assert np.max(np.abs(J[e, h])) < 1e-12 * typical, (process, h)
                continue
            if kind is None:
                continue
            _, q3, q1, j = kind
            num = s(q3, j) ** 3 * s(q1, j)
            for k, perm in enumerate(flows):
                cyc = [T] + list(perm) + [TBAR]
                den = np.prod([s(cyc[a], cyc[(a + 1) % len(cyc)]) for a in range(len(cyc))])
                ratio = abs(J[e, h, k]) ** 2 / (num / den)
                assert ratio == pytest.approx(want, rel=1e-10), (process, e, h, perm)
                n_mhv += 1
    # every MHV and MHV-bar helicity of every flow was checked (with two gluons the two
    # classes coincide): 2 quark helicities x ng choices of j, per class
    per_event = (2 * ng if ng == 2 else 4 * ng) * ncol
    assert n_mhv == mom.shape[0] * per_event

