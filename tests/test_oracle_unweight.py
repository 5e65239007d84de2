"""Pins of the batch-unweighting oracle: a hand-worked batch, the acceptance
probability w_i / w_max of hit-or-miss, and the weighted distribution of what is kept."""
import numpy as np
import pytest

from oracle.unweight import unweight


def test_hand_worked_batch():
    me = np.array([2.0, 1.0, 4.0, 3.0, np.nan, 5.0, 1.0])
    wgt = np.array([1.0, 3.0, 0.5, -1.0, 1.0, np.inf, 0.0])
    rnd = np.array([0.9, 0.7, 0.4, 0.0, 0.0, 0.0, 0.0])
    w, acc, wmax, nacc = unweight(me, wgt, rnd)
    # weights 2, 3, 2, -3 (negative), nan, inf, 0: only the finite non-negative ones count
    np.testing.assert_array_equal(w[:4], [2.0, 3.0, 2.0, -3.0])
    assert wmax == 3.0
    # 2 > 0.9*3? no;  3 > 0.7*3 yes;  2 > 0.4*3 yes;  negative, nan, inf never;  0 > 0? no
    np.testing.assert_array_equal(acc, [0, 1, 1, 0, 0, 0, 0])
    assert nacc == 2


def test_degenerate_batches():
    assert unweight([], [], [])[2:] == (0.0, 0)
    w, acc, wmax, nacc = unweight([0.0, 0.0], [1.0, 2.0], [0.5, 0.0])
    assert wmax == 0.0 and nacc == 0          # no positive weight: nothing is kept
    w, acc, wmax, nacc = unweight([1.0], [1.0], [0.999999])
    assert wmax == 1.0 and nacc == 1          # the largest weight is always kept (r < 1)


def test_acceptance_probability_is_weight_over_max():
    """hit-or-miss keeps event i with probability w_i / w_max: over many events the
    kept count is sum w / w_max within its binomial spread"""
    rng = np.random.default_rng(5)
    n = 200000
    me = rng.exponential(size=n)
    wgt = rng.uniform(0.5, 1.5, size=n)
    rnd = rng.uniform(size=n)
    w, acc, wmax, nacc = unweight(me, wgt, rnd)
    p = w / wmax
    mean = p.sum()
    sd = np.sqrt((p * (1 - p)).sum())
    assert abs(nacc - mean) < 5 * sd


def test_kept_events_follow_the_weighted_distribution():
    """unweighted events are distributed like the weighted sample: a histogram of an
    observable over kept events matches the w-weighted histogram (chi-square)"""
    rng = np.random.default_rng(9)
    n = 400000
    x = rng.uniform(size=n)                   # an observable
    me = 1.0 + 3.0 * x ** 2                   # weight depends on it
    w, acc, wmax, nacc = unweight(me, np.ones(n), rng.uniform(size=n))
    bins = np.linspace(0, 1, 11)
    kept, _ = np.histogram(x[acc == 1], bins)
    weighted, _ = np.histogram(x, bins, weights=w)
    expect = weighted / weighted.sum() * nacc
    chi2 = ((kept - expect) ** 2 / expect).sum()
    assert chi2 < 30.0                        # 9 degrees of freedom; p ~ 4e-4
