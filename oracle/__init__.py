"""Plain FP64 CPU oracle for tree-level matrix elements (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The product path (``paper_2312_02898_b300``) never does;
the two share no code.  The C source ``me_oracle.c`` states the physics, the
conventions and the published methods it follows.

Pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` against closed
forms (e+e- -> mu+mu-, gg -> ttbar), an explicit-colour brute force (also at the
physical top width, with and without width in t-channel propagators), exact colour
algebra checked entry by entry against explicit Gell-Mann sums for 2 to 5 gluons, the
propagator invariants checked against exact rational arithmetic on nearly collinear
events, the Lorentz / gauge / Bose / alpha_s-scaling invariants, and the Parke-Taylor
formula: with massless quarks every MHV colour-ordered amplitude for 2 to
5 gluons equals (sqrt(2) g_s)^n_g times its closed form, which fixes the absolute
normalisation of the recursion for gg -> ttbar gg and gg -> ttbar ggg.  What the
massless limit leaves open there (the massive spinors and top propagators at 4-5
gluons) is pinned by the same code being exact for gg -> ttbar against its closed
form, and by gauge invariance and Bose symmetry at the physical top mass.

The one-jet quark channels of p p -> t tbar + jet (q qbar -> t tbar g, q g -> t tbar q,
qbar g -> t tbar qbar, in either beam order) are pinned by gauge invariance, the
soft-gluon limit with colour correlators from an explicit Gell-Mann sum, the
initial-state collinear limits with the Altarelli-Parisi splitting functions (onto the
closed-form-pinned q qbar -> t tbar and g g -> t tbar), charge conjugation, beam order,
Lorentz invariance and their flow colour matrix.  The two-jet channels with one light
line (q qbar -> t tbar g g, q g -> t tbar q g and its antiquark and beam-order crossings,
g g -> t tbar q qbar) are pinned the same way: gauge invariance in each gluon, the soft
limit onto q qbar -> t tbar g with colour correlators built from its flow amplitudes,
initial-state collinear limits (P_qq, P_qg, P_gq, P_gg) onto the one-jet channels and
g g -> t tbar g, Bose symmetry, charge conjugation, beam order and the 13-flow basis.
The four-quark channels with two light flavours (u u~ -> t t~ d d~, u d -> t t~ u d,
u d~ -> t t~ u d~, u~ d~ -> t t~ u~ d~) are pinned by the final-state g -> d d~ and the
initial-state collinear limits onto the one-jet channels, Lorentz invariance, beam order,
charge conjugation and their six-flow colour basis; the same-flavour channels
(u u -> t t~ u u, u~ u~ -> t t~ u~ u~, u u~ -> t t~ u u~) add Pauli antisymmetry at equal
final momenta, which fixes the sign of the exchange pairing, and Bose/Fermi relabelling.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "me_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libme_oracle.so")

PROCESSES = (
    "e+ e- > mu+ mu-",
    "g g > t t~",
    "g g > t t~ g",
    "g g > t t~ g g",
    "g g > t t~ g g g",
    "u u~ > t t~",
    "u~ u > t t~",
    "u u~ > t t~ g",
    "u~ u > t t~ g",
    "u g > t t~ u",
    "g u > t t~ u",
    "u~ g > t t~ u~",
    "g u~ > t t~ u~",
    "u u~ > t t~ g g",
    "u~ u > t t~ g g",
    "u g > t t~ u g",
    "g u > t t~ u g",
    "u~ g > t t~ u~ g",
    "g u~ > t t~ u~ g",
    "g g > t t~ u u~",
    "u u~ > t t~ d d~",
    "u~ u > t t~ d d~",
    "u d > t t~ u d",
    "u d~ > t t~ u d~",
    "u~ d~ > t t~ u~ d~",
    "u u > t t~ u u",
    "u~ u~ > t t~ u~ u~",
    "u u~ > t t~ u u~",
    "u~ u > t t~ u u~",
)


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("mZ", ctypes.c_double), ("wZ", ctypes.c_double),
        ("mt", ctypes.c_double), ("wt", ctypes.c_double),
        ("aEWM1", ctypes.c_double), ("Gf", ctypes.c_double),
        ("alphas", ctypes.c_double), ("zero_width_tchan", ctypes.c_int),
    ]


@dataclass
class Params:
    mZ: float = 91.188
    wZ: float = 2.4414
    mt: float = 173.0
    wt: float = 1.4915
    aEWM1: float = 132.5
    Gf: float = 1.16639e-5
    alphas: float = 0.118
    zero_width_tchan: int = 0

    def c(self) -> OracleParams:
        return OracleParams(self.mZ, self.wZ, self.mt, self.wt, self.aEWM1, self.Gf,
                            self.alphas, int(self.zero_width_tchan))


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP over events)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        i64 = ctypes.POINTER(ctypes.c_int64)
        _lib.oracle_me.argtypes = [ctypes.c_int, ctypes.POINTER(OracleParams), ctypes.c_int64, d, d, d, d,
                                   d, d, d, d, i32, i32, ctypes.c_int]
        _lib.oracle_me.restype = ctypes.c_int
        _lib.oracle_info.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4
        _lib.oracle_colour_matrix_exact.argtypes = [ctypes.c_int, i64, i64]
        _lib.oracle_process_id.argtypes = [ctypes.c_char_p]
        _lib.oracle_sm_derived.argtypes = [ctypes.POINTER(OracleParams), d]
        _lib.oracle_invariants.argtypes = [ctypes.c_int, ctypes.POINTER(OracleParams), ctypes.c_int64, d, d, d]
        _lib.oracle_invariants.restype = ctypes.c_int
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def process_id(process: str) -> int:
    pid = lib().oracle_process_id(process.encode())
    if pid < 0:
        raise ValueError(f"unknown process {process!r}")
    return pid


def info(process: str):
    """(npar, ncomb, ncol, iden) of a process."""
    v = [ctypes.c_int() for _ in range(4)]
    lib().oracle_info(process_id(process), *[ctypes.byref(x) for x in v])
    return tuple(x.value for x in v)


def colour_matrix(process: str):
    """Exact colour matrix as (numerator, denominator) int64 arrays [ncol][ncol]."""
    _, _, ncol, _ = info(process)
    num = np.zeros((ncol, ncol), dtype=np.int64)
    den = np.zeros((ncol, ncol), dtype=np.int64)
    lib().oracle_colour_matrix_exact(process_id(process), _ptr(num, ctypes.c_int64), _ptr(den, ctypes.c_int64))
    return num, den


def sm_derived(params: Params | None = None):
    """(e, sw2, mW, gZ_L, gZ_R) derived from (alpha, G_F, mZ)."""
    out = np.zeros(5)
    p = (params or Params()).c()
    lib().oracle_sm_derived(ctypes.byref(p), _ptr(out))
    return tuple(out)


def invariants(process: str, momenta, params: Params | None = None):
    """The propagator invariants the oracle's recursion uses, per event and particle
    mask (bit i = particle i): (gsq, tden), each [nevt][2^npar].  gsq[mask] is K^2 of
    the gluons in the mask (incoming +p, outgoing -p); tden[mask] is q^2 - mt^2 of the
    top-line propagator q = p_t - K(mask).  Formed in quadruple precision and rounded
    once to FP64."""
    npar, ncomb, _, _ = info(process)
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    nevt = mom.shape[0]
    assert mom.shape == (nevt, npar, 4)
    gsq, tden = np.zeros((nevt, ncomb)), np.zeros((nevt, ncomb))
    p = (params or Params()).c()
    if lib().oracle_invariants(process_id(process), ctypes.byref(p), nevt, _ptr(mom), _ptr(gsq), _ptr(tden)) != 0:
        raise ValueError(f"no invariant table for {process!r}")
    return gsq, tden


def me(process: str, momenta, alphas=None, rnd_hel=None, rnd_col=None, params: Params | None = None,
       want_hel=False, want_jamp=False, want_colw=False, gauge_leg=-1):
    """Evaluate the oracle on a batch.  Returns a dict of numpy arrays."""
    npar, ncomb, ncol, _ = info(process)
    mom = np.ascontiguousarray(momenta, dtype=np.float64)
    nevt = mom.shape[0]
    assert mom.shape == (nevt, npar, 4)
    a = None if alphas is None else np.ascontiguousarray(np.broadcast_to(alphas, (nevt,)), dtype=np.float64)
    rh = None if rnd_hel is None else np.ascontiguousarray(rnd_hel, dtype=np.float64)
    rc = None if rnd_col is None else np.ascontiguousarray(rnd_col, dtype=np.float64)
    out = {"me": np.zeros(nevt)}
    if want_hel:
        out["me_hel"] = np.zeros((nevt, ncomb))
    if want_jamp:
        out["jamp"] = np.zeros((nevt, ncomb, ncol, 2))
    if want_colw:
        out["colw"] = np.zeros((nevt, ncol))
    if rh is not None:
        out["sel_hel"] = np.zeros(nevt, dtype=np.int32)
    if rc is not None:
        out["sel_col"] = np.zeros(nevt, dtype=np.int32)
    p = (params or Params()).c()
    rc_ = lib().oracle_me(process_id(process), ctypes.byref(p), nevt, _ptr(mom), _ptr(a), _ptr(rh), _ptr(rc),
                          _ptr(out["me"]), _ptr(out.get("me_hel")), _ptr(out.get("jamp")), _ptr(out.get("colw")),
                          _ptr(out.get("sel_hel"), ctypes.c_int32), _ptr(out.get("sel_col"), ctypes.c_int32),
                          int(gauge_leg))
    if rc_ != 0:
        raise RuntimeError(f"oracle_me failed with {rc_}")
    if "jamp" in out:
        out["jamp"] = out["jamp"][..., 0] + 1j * out["jamp"][..., 1]
    return out
