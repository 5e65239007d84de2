"""Serving loop on the GPU: every request's result is the same alone and in a mix of
overlapping requests of all processes and many sizes."""
import numpy as np
import pytest

from paper_2312_02898_b300.phasespace import make_batch

pytestmark = pytest.mark.gpu

PROCS = ("e+ e- > mu+ mu-", "g g > t t~", "g g > t t~ g", "g g > t t~ g g", "g g > t t~ g g g")


def _alone(server, process, mom, alphas, rh, rc):
    """the request evaluated by itself, unpadded, through the plain device entry point"""
    import torch
    m = server.handles[process]
    dev = server.device
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    me, sh, sc = m.compute(t(mom), t(alphas), t(rh), t(rc))
    torch.cuda.synchronize()
    return me.cpu().numpy(), sh.cpu().numpy(), sc.cpu().numpy()


@pytest.mark.parametrize("use_graphs", [True, False])
def test_results_are_the_same_alone_and_in_the_mix(use_graphs):
    from paper_2312_02898_b300 import serving
    server = serving.Server(PROCS, precision="mixed", n_slots=4, use_graphs=use_graphs)
    try:
        rng = np.random.default_rng(11)
        reqs = []
        for k in range(24):
            proc = PROCS[k % len(PROCS)]
            hi = 3000 if proc == "g g > t t~ g g g" else 9000
            n = int(rng.integers(1, hi))
            mom, a, rh, rc = make_batch(proc, n, seed=100 + k, alphas="uniform")
            reqs.append((proc, mom, a, rh, rc))
        futs = [server.submit(p, mom, a, rh, rc) for p, mom, a, rh, rc in reqs]
        mixed = [f.result(timeout=300) for f in futs]
        st = server.stats()
        assert st["requests"] == len(reqs)
        assert st["events"] == sum(r[1].shape[0] for r in reqs)
        for (proc, mom, a, rh, rc), (me, sh, sc) in zip(reqs, mixed):
            me0, sh0, sc0 = _alone(server, proc, mom, a, rh, rc)
            assert np.all(np.isfinite(me)) and np.all(me > 0)
            # the same kernels on the same events: identical bits, not just within tolerance
            np.testing.assert_array_equal(me, me0, err_msg=proc)
            np.testing.assert_array_equal(sh, sh0, err_msg=proc)
            np.testing.assert_array_equal(sc, sc0, err_msg=proc)
    finally:
        server.close()


def test_overlapping_requests_are_admitted_while_others_run():
    """with several slots, requests are on the GPU at the same time (continuous batching),
    and a tight memory budget still lets every request through one at a time"""
    from paper_2312_02898_b300 import serving
    server = serving.Server(("g g > t t~ g g",), precision="mixed", n_slots=3, mem_budget_bytes=1)
    try:
        futs = []
        for k in range(6):
            mom, a, rh, rc = make_batch("g g > t t~ g g", 4000 + 100 * k, seed=k, alphas="uniform")
            futs.append(server.submit("g g > t t~ g g", mom, a, rh, rc))
        out = [f.result(timeout=300) for f in futs]
        assert all(np.all(np.isfinite(o[0])) for o in out)
        assert server.admission.used == 0
        assert server.max_running == 1  # the 1-byte budget admits one request at a time
    finally:
        server.close()
    server = serving.Server(("g g > t t~ g g",), precision="mixed", n_slots=3)
    try:
        for b in (4096, 8192):
            server.warm("g g > t t~ g g", b)
        batch = [make_batch("g g > t t~ g g", 8000, seed=k, alphas="uniform") for k in range(9)]
        futs = [server.submit("g g > t t~ g g", *x) for x in batch]  # a burst: all queued at once
        [f.result(timeout=300) for f in futs]
        assert server.max_running >= 2
    finally:
        server.close()


def test_large_requests_run_in_chunks_with_the_same_results():
    """A request larger than the chunk size is split; its result equals the request
    evaluated alone, and requests beyond the largest bucket are served too."""
    from paper_2312_02898_b300 import serving
    server = serving.Server(("g g > t t~ g", "g g > t t~ g g"), precision="mixed", n_slots=3, chunk_events=4096)
    try:
        reqs = [("g g > t t~ g g", 10000, 5), ("g g > t t~ g", 70000, 6), ("g g > t t~ g g", 4096, 7)]
        batches = [(p,) + make_batch(p, n, seed=s, alphas="uniform") for p, n, s in reqs]
        futs = [server.submit(*b) for b in batches]
        for (p, mom, a, rh, rc), f in zip(batches, futs):
            me, sh, sc = f.result(timeout=300)
            me0, sh0, sc0 = _alone(server, p, mom, a, rh, rc)
            np.testing.assert_array_equal(me, me0)
            np.testing.assert_array_equal(sh, sh0)
            np.testing.assert_array_equal(sc, sc0)
    finally:
        server.close()


def test_srpt_lets_small_requests_pass_a_large_one():
    """With the least-remaining-work policy, small requests submitted just after a large
    one finish before it; with first-come scheduling they wait behind it."""
    from paper_2312_02898_b300 import serving
    big = ("g g > t t~ g g g",) + make_batch("g g > t t~ g g g", 24000, seed=1, alphas="uniform")
    small = [("g g > t t~",) + make_batch("g g > t t~", 2000, seed=10 + k, alphas="uniform") for k in range(3)]
    order = {}
    for policy in ("srpt", "fifo"):
        server = serving.Server(("g g > t t~", "g g > t t~ g g g"), precision="mixed", n_slots=1,
                                chunk_events=4096, policy=policy)
        try:
            server.warm("g g > t t~", 2048)
            server.warm("g g > t t~ g g g", 4096)
            futs = [server.submit(*big, tag="big")] + [server.submit(*s, tag=f"s{k}") for k, s in enumerate(small)]
            [f.result(timeout=600) for f in futs]
            order[policy] = [x[4] for x in sorted(server.done, key=lambda x: x[3])]
        finally:
            server.close()
    assert order["srpt"][-1] == "big"
    assert order["fifo"][0] == "big"
