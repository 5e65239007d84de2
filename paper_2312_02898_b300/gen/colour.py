"""Colour matrix C_st = sum over colours of (T^s)_ij (T^t)*_ij for the colour-flow basis.

Build-time generator code.  Evaluated by explicitly summing over every assignment of
adjoint indices with the Gell-Mann matrices T^a = lambda^a / 2, then recovered exactly:
every entry is an integer multiple of 1/(2^n N^n) (n Fierz steps, each a factor 1/2
and at most one 1/N), so C * 2^n N^n is rounded to integers and reduced by the common
gcd.  Returned as an integer matrix plus one common denominator.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def gell_mann_T():
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1], l[1][1, 0] = -1j, 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2], l[4][2, 0] = -1j, 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2], l[6][2, 1] = -1j, 1j
    l[7] = np.diag([1.0, 1.0, -2.0]) / math.sqrt(3.0)
    return l / 2.0


def colour_matrix(n: int):
    """(CF integer [n!][n!], denominator) for strings of n gluons in lexicographic
    permutation order."""
    if n == 0:
        return np.ones((1, 1), dtype=np.int64), 1
    T = gell_mann_T()
    perms = list(itertools.permutations(range(n)))
    assigns = np.array(list(itertools.product(range(8), repeat=n)), dtype=np.int64)
    C = np.zeros((len(perms), len(perms)))
    chunk = 4096
    for c0 in range(0, len(assigns), chunk):
        a = assigns[c0:c0 + chunk]
        mats = np.empty((len(perms), len(a), 9), dtype=np.complex128)
        for ip, p in enumerate(perms):
            m = T[a[:, p[0]]]
            for j in p[1:]:
                m = m @ T[a[:, j]]
            mats[ip] = m.reshape(len(a), 9)
        flat = mats.reshape(len(perms), -1)
        C += np.real(flat @ flat.conj().T)
    scale = (2 ** n) * (3 ** n)
    X = C * scale
    Xi = np.rint(X).astype(np.int64)
    if np.max(np.abs(X - Xi)) > 1e-6 * max(1.0, np.max(np.abs(X))):
        raise RuntimeError("colour matrix is not a multiple of 1/(2^n 3^n)")
    g = scale
    for v in np.unique(np.abs(Xi)):
        g = math.gcd(g, int(v))
    return Xi // g, scale // g


def quark_jet_colour():
    """Colour of the five Feynman diagrams of q qbar -> t tbar g (and its crossings) on the
    four flow tensors.

    Index order (B, K, t, tb, a): the colours of the light line's row end B (an incoming
    antiquark or an outgoing quark), its column end K (an incoming quark or an outgoing
    antiquark), the top, the antitop and the gluon.  Diagram colour tensors:
      D1 (T^b T^a)_{BK} T^b_{t tb},  D2 (T^a T^b)_{BK} T^b_{t tb},
      D3 T^b_{BK} (T^a T^b)_{t tb},  D4 T^b_{BK} (T^b T^a)_{t tb},
      D5 f^{bca} T^b_{BK} T^c_{t tb},  f^{abc} = -2i Tr([T^a, T^b] T^c);
    flows c0 = T^a_{B tb} d_{tK}, c1 = T^a_{tK} d_{B tb}, c2 = T^a_{BK} d_{t tb},
    c3 = T^a_{t tb} d_{BK}.  Each diagram is solved for its flow coefficients over all 648
    assignments; the coefficients are multiples of 1/6 (one Fierz step with its 1/N) and
    are returned times 6 as Gaussian integers, with the integer Gram matrix of the flows.
    """
    T = gell_mann_T()
    f = np.real(-2j * (np.einsum("aij,bjk,cki->abc", T, T, T) - np.einsum("bij,ajk,cki->abc", T, T, T)))
    d = np.eye(3)
    diagrams = [np.einsum("bBm,amK,bty->BKtya", T, T, T), np.einsum("aBm,bmK,bty->BKtya", T, T, T),
                np.einsum("bBK,atm,bmy->BKtya", T, T, T), np.einsum("bBK,btm,amy->BKtya", T, T, T),
                np.einsum("bca,bBK,cty->BKtya", f, T, T)]
    flows = [np.einsum("aBy,tK->BKtya", T, d), np.einsum("atK,By->BKtya", T, d),
             np.einsum("aBK,ty->BKtya", T, d), np.einsum("aty,BK->BKtya", T, d)]
    F = np.stack([x.ravel() for x in flows], axis=1)
    coef = []
    for x in diagrams:
        c = np.linalg.lstsq(F, x.ravel(), rcond=None)[0]
        if np.abs(F @ c - x.ravel()).max() > 1e-12:
            raise RuntimeError("a diagram's colour is not in the span of the flows")
        c6 = 6.0 * c
        ci = np.rint(c6.real) + 1j * np.rint(c6.imag)
        if np.abs(c6 - ci).max() > 1e-9:
            raise RuntimeError("flow coefficient not a multiple of 1/6")
        coef.append([complex(int(z.real), int(z.imag)) for z in ci])
    G = F.conj().T @ F
    Gi = np.rint(G.real).astype(np.int64)
    if np.abs(G - Gi).max() > 1e-9:
        raise RuntimeError("flow Gram matrix is not integer")
    return coef, Gi
