"""Pins of the oracle against closed-form spin- and colour-summed results.

e+ e- -> mu+ mu- via photon and Z (standard electroweak textbook result): with
c = cos(angle between e- and mu-) and A_XY = Q_e Q_mu / s + g_X^e g_Y^mu / (s - mZ^2 + i mZ wZ),
    <|M|^2> = (e^4 s^2 / 4) [ (|A_LL|^2 + |A_RR|^2)(1+c)^2 + (|A_LR|^2 + |A_RL|^2)(1-c)^2 ]
which reduces to e^4 (1 + c^2) without the Z.

g g -> Q Qbar (Combridge 1979; Ellis, Stirling, Webber eq. 10.12), averaged over
initial spins and colours, with tau_{1,2} = 2 p_{1,2}.p_Q / s and rho = 4 m^2 / s:
    <|M|^2> = g^4 (1/(6 tau1 tau2) - 3/8) (tau1^2 + tau2^2 + rho - rho^2/(4 tau1 tau2)).
It holds for a zero top width, which these tests set.
"""
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import phasespace as ps

ALPHA = 1.0 / 132.5
MZ, WZ, GF = 91.188, 2.4414, 1.16639e-5


def _sw2():
    # derived independently here: mW^2 = mZ^2/2 + sqrt(mZ^4/4 - pi alpha mZ^2/(sqrt2 GF))
    mw2 = MZ ** 2 / 2 + math.sqrt(MZ ** 4 / 4 - math.pi * ALPHA * MZ ** 2 / (math.sqrt(2) * GF))
    return 1 - mw2 / MZ ** 2


def eemumu_closed(s, c, with_z=True):
    e2 = 4 * math.pi * ALPHA
    sw2 = _sw2()
    sw, cw = math.sqrt(sw2), math.sqrt(1 - sw2)
    gl = (-0.5 + sw2) / (sw * cw)
    gr = sw2 / (sw * cw)
    z = 1.0 / complex(s - MZ ** 2, MZ * WZ) if with_z else 0.0
    A = {(x, y): 1.0 / s + gx * gy * z for x, gx in (("L", gl), ("R", gr)) for y, gy in (("L", gl), ("R", gr))}
    return (e2 ** 2 * s ** 2 / 4) * ((abs(A["L", "L"]) ** 2 + abs(A["R", "R"]) ** 2) * (1 + c) ** 2
                                     + (abs(A["L", "R"]) ** 2 + abs(A["R", "L"]) ** 2) * (1 - c) ** 2)


def _cos_e_mu(mom):
    pe, pm = mom[:, 1, 1:], mom[:, 3, 1:]
    return (pe * pm).sum(-1) / np.linalg.norm(pe, axis=1) / np.linalg.norm(pm, axis=1)


def test_sw2_value():
    # G_F scheme with alpha = 1/132.5: sin^2(theta_W) close to 0.2223
    assert abs(_sw2() - 0.22226) < 1e-4


def test_eemumu_rambo_events(oracle_mod):
    mom, _, _, _ = ps.make_batch("e+ e- > mu+ mu-", 500, seed=0)
    out = oracle_mod.me("e+ e- > mu+ mu-", mom)
    s = 1500.0 ** 2
    ref = np.array([eemumu_closed(s, c) for c in _cos_e_mu(mom)])
    assert np.max(np.abs(out["me"] / ref - 1)) < 1e-12


@pytest.mark.parametrize("c", [0.0, 0.5, -0.3, 0.97, -0.999])
def test_eemumu_fixed_angles(oracle_mod, c):
    E = 750.0
    st = math.sqrt(1 - c * c)
    # mu- along the e- direction (-z) rotated by theta: cos(e-, mu-) = c
    mom = np.array([[[E, 0, 0, E], [E, 0, 0, -E], [E, E * st, 0, E * c], [E, -E * st, 0, -E * c]]])
    out = oracle_mod.me("e+ e- > mu+ mu-", mom, want_hel=True)
    assert abs(out["me"][0] / eemumu_closed(E * E * 4, c) - 1) < 1e-12
    # exactly four of the sixteen helicity combinations are non-zero (massless chirality)
    assert int((out["me_hel"][0] != 0).sum()) == 4


def test_eemumu_qed_limit(oracle_mod):
    # Z decoupled by a huge width (its propagator vanishes): e^4 (1 + c^2)
    p = oracle_mod.Params(wZ=1e30)
    mom, _, _, _ = ps.make_batch("e+ e- > mu+ mu-", 50, seed=5)
    out = oracle_mod.me("e+ e- > mu+ mu-", mom, params=p)
    c = _cos_e_mu(mom)
    e2 = 4 * math.pi * ALPHA
    assert np.max(np.abs(out["me"] / (e2 ** 2 * (1 + c ** 2)) - 1)) < 1e-9


def ggqq_closed(p1, p2, p3, m, gs):
    s = 2 * _dot(p1, p2)
    t1 = 2 * _dot(p1, p3) / s
    t2 = 2 * _dot(p2, p3) / s
    rho = 4 * m * m / s
    return gs ** 4 * (1 / (6 * t1 * t2) - 3 / 8) * (t1 ** 2 + t2 ** 2 + rho - rho ** 2 / (4 * t1 * t2))


def _dot(a, b):
    return a[..., 0] * b[..., 0] - (a[..., 1:] * b[..., 1:]).sum(-1)


@pytest.mark.parametrize("ct", [0.0, 0.5, -0.8, 0.99])
def test_ggtt_fixed_angles(oracle_mod, ct):
    mt, E = 173.0, 750.0
    pz = math.sqrt(E * E - mt * mt)
    st = math.sqrt(1 - ct * ct)
    mom = np.array([[[E, 0, 0, E], [E, 0, 0, -E], [E, pz * st, 0, pz * ct], [E, -pz * st, 0, -pz * ct]]])
    par = oracle_mod.Params(wt=0.0)
    out = oracle_mod.me("g g > t t~", mom, params=par)
    gs = math.sqrt(4 * math.pi * 0.118)
    ref = ggqq_closed(mom[0, 0], mom[0, 1], mom[0, 2], mt, gs)
    assert abs(out["me"][0] / ref - 1) < 1e-12


def test_ggtt_rambo_events_and_width(oracle_mod):
    mom, _, _, _ = ps.make_batch("g g > t t~", 400, seed=2)
    gs = math.sqrt(4 * math.pi * 0.118)
    ref = ggqq_closed(mom[:, 0], mom[:, 1], mom[:, 2], 173.0, gs)
    out0 = oracle_mod.me("g g > t t~", mom, params=oracle_mod.Params(wt=0.0))
    assert np.max(np.abs(out0["me"] / ref - 1)) < 1e-12
    # with the physical width the t-channel propagators shift only slightly
    out1 = oracle_mod.me("g g > t t~", mom)
    dev = np.abs(out1["me"] / ref - 1)
    assert dev.max() < 1e-4 and dev.max() > 0
    # zero-width t-channel mode: for gg -> ttbar every top propagator is t-channel
    out2 = oracle_mod.me("g g > t t~", mom, params=oracle_mod.Params(zero_width_tchan=1))
    assert np.max(np.abs(out2["me"] / ref - 1)) < 1e-12


def test_ggqq_massless_limit(oracle_mod):
    # rho -> 0: (t^2+u^2)/(6tu) - 3(t^2+u^2)/(8 s^2), the textbook gg -> q qbar entry
    mom, _, _, _ = ps.make_batch("e+ e- > mu+ mu-", 50, seed=9)  # massless 2 -> 2 kinematics
    par = oracle_mod.Params(mt=0.0, wt=0.0)
    out = oracle_mod.me("g g > t t~", mom, params=par)
    s = 1500.0 ** 2
    t = -2 * _dot(mom[:, 0], mom[:, 2])
    u = -2 * _dot(mom[:, 1], mom[:, 2])
    gs = math.sqrt(4 * math.pi * 0.118)
    ref = gs ** 4 * ((t * t + u * u) / (6 * t * u) - 3 * (t * t + u * u) / (8 * s * s))
    assert np.max(np.abs(out["me"] / ref - 1)) < 1e-11
