"""Batch unweighting, written out plainly (TEST INFRASTRUCTURE ONLY).

Section 3 of the paper (with Table 2): the full weight of an event is its matrix
element times the rest of its weight (Jacobian, PDFs); with the largest weight of the
whole batch known, each event is kept by hit-or-miss against it.  The rule written out
here is the textbook acceptance-rejection method (von Neumann 1951): keep event i when
w_i > r_i * w_max with r_i uniform in [0, 1), so that an event is kept with
probability w_i / w_max.  Weights that are not finite or are negative take no part.
Only tests, the smoke check and the benchmark's baseline leg use this module.
"""
from __future__ import annotations

import math

import numpy as np


def unweight(me, wgt, rnd):
    """(w, accept, w_max, n_accept) for one batch, one event at a time"""
    me = np.asarray(me, dtype=np.float64)
    wgt = np.asarray(wgt, dtype=np.float64)
    rnd = np.asarray(rnd, dtype=np.float64)
    n = me.shape[0]
    w = np.empty(n)
    w_max = 0.0
    for i in range(n):
        w[i] = me[i] * wgt[i]
        if math.isfinite(w[i]) and w[i] >= 0.0 and w[i] > w_max:
            w_max = w[i]
    accept = np.zeros(n, dtype=np.uint8)
    for i in range(n):
        if math.isfinite(w[i]) and w[i] >= 0.0 and w[i] > rnd[i] * w_max:
            accept[i] = 1
    return w, accept, w_max, int(accept.sum())
