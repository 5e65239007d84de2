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
