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
