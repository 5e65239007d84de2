"""Host-side logic of the serving loop: buckets, padding, admission, percentiles, the
request stream and the scheduling policies (no GPU)."""
import collections
import math

import numpy as np
import pytest

from paper_2312_02898_b300 import serving


def test_bucket_is_smallest_power_of_two_or_one_and_a_half_times_one_holding_the_batch():
    assert serving.bucket_for(1) == 256
    assert serving.bucket_for(256) == 256
    assert serving.bucket_for(257) == 384
    assert serving.bucket_for(385) == 512
    assert serving.bucket_for(8193) == 12288
    assert serving.bucket_for(65536) == 65536
    with pytest.raises(ValueError):
        serving.bucket_for(65537)
    # padding never adds more than half of a batch
    for n in range(256, 65537, 97):
        assert serving.bucket_for(n) <= 1.5 * n


def test_padding_repeats_the_last_event_and_keeps_the_rest():
    x = np.arange(3 * 2 * 4, dtype=float).reshape(3, 2, 4)
    y = serving.pad_to(x, 5)
    assert y.shape == (5, 2, 4)
    np.testing.assert_array_equal(y[:3], x)
    np.testing.assert_array_equal(y[3], x[2])
    np.testing.assert_array_equal(y[4], x[2])
    assert serving.pad_to(x, 3) is x


def test_percentile_matches_numpy_linear_interpolation():
    rng = np.random.default_rng(3)
    v = rng.exponential(size=257).tolist()
    for q in (0, 50, 90, 99, 100):
        assert serving.percentile(v, q) == pytest.approx(np.percentile(v, q), rel=1e-12)
    assert math.isnan(serving.percentile([], 50))


def test_admission_blocks_beyond_budget_but_never_starves_an_empty_device():
    a = serving.MemoryAdmission(100)
    assert a.try_take(60)
    assert not a.try_take(60)       # would exceed the budget while 60 are held
    assert a.try_take(40)
    a.give(60)
    a.give(40)
    assert a.used == 0
    assert a.try_take(500)          # alone on the device a request always starts
    assert not a.try_take(1)
    a.give(500)
    # the reserved workspaces count against the budget
    r = serving.MemoryAdmission(100, reserved=70)
    assert r.try_take(20)
    assert not r.try_take(20)
    assert r.try_take(10) and r.used == 30


def test_request_stream_follows_weights_sizes_and_poisson_arrivals():
    n = 20000
    reqs = serving.request_stream(n, rate_hz=1000.0, seed=7)
    t = np.array([r[0] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential inter-arrival times: mean 1/rate, coefficient of variation 1
    assert gaps.mean() == pytest.approx(1e-3, rel=0.05)
    assert gaps.std() / gaps.mean() == pytest.approx(1.0, rel=0.05)
    names = [r[1] for r in reqs]
    for p, w in serving.STREAM_PROCESSES:
        assert names.count(p) / n == pytest.approx(w, abs=0.015)
    sizes = np.array([r[2] for r in reqs])
    assert sizes.min() >= 256 and sizes.max() <= 65536
    # log-uniform: log2 of the size is uniform on [8, 16]
    u = (np.log2(sizes) - 8) / 8
    assert u.mean() == pytest.approx(0.5, abs=0.01)
    assert np.mean(u < 0.25) == pytest.approx(0.25, abs=0.015)
    assert [r[3] for r in reqs] == list(range(n))


def test_request_stream_weights_are_the_process_class_weights():
    w = dict(serving.STREAM_PROCESSES)
    assert w["e+ e- > mu+ mu-"] == pytest.approx(0.1)
    assert w["g g > t t~"] + w["g g > t t~ g"] == pytest.approx(0.3)
    assert w["g g > t t~ g g"] == pytest.approx(0.4)
    assert w["g g > t t~ g g g"] == pytest.approx(0.2)


def _req(n, cost, done=0):
    r = serving.Request("p", np.zeros((n, 4, 4)), None, np.zeros(n), np.zeros(n))
    r.cost, r.next_event = cost, done
    return r


def test_fifo_takes_the_oldest_request():
    q = [_req(60000, 1e7), _req(300, 1e4), _req(5000, 1e5)]
    assert serving.pick_next(q, "fifo") is q[0]


def test_srpt_takes_the_least_remaining_work():
    big, small, mid = _req(60000, 1e7), _req(300, 1e4), _req(5000, 1e5)
    q = [big, small, mid]
    assert serving.pick_next(q, "srpt") is small
    # remaining work counts only undispatched events: a nearly finished large request
    # goes before a fresh medium one
    big.next_event = 59990
    assert serving.pick_next([mid, big], "srpt") is big
    # equal work: the older request
    a, b = _req(1000, 1e5), _req(1000, 1e5)
    assert serving.pick_next([a, b], "srpt") is a


def test_requests_compare_by_identity():
    a, b = _req(10, 1.0), _req(10, 1.0)
    assert a != b and a == a
    q = collections.deque([a, b])
    q.remove(b)
    assert list(q) == [a]
