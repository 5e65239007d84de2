"""The N-rank benchmark path on CPU (gloo, world size 2): every rank evaluates its own
disjoint slice of events, the slices together are exactly one large batch (the
generator is counter-based), and the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nevt, q):
    import torch.distributed as dist
    from paper_2312_02898_b300.phasespace import make_batch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first = bench.shard_events(rank, nevt)
        mom, a, rh, rc = make_batch("g g > t t~ g", nevt, seed=0, first_event=first, alphas="uniform")
        slow = bench.max_over_ranks(1.0 + rank, dist)  # rank 1 is the slower one
        dist.barrier()
        q.put((rank, first, mom, a, rh, rc, slow))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_events_and_take_the_max_time():
    world, nevt = 2, 96
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nevt, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted([q.get(timeout=120) for _ in range(world)], key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2312_02898_b300.phasespace import make_batch
    whole = make_batch("g g > t t~ g", world * nevt, seed=0, alphas="uniform")
    for rank, first, mom, a, rh, rc, slow in got:
        assert first == rank * nevt
        sl = slice(first, first + nevt)
        for part, full in zip((mom, a, rh, rc), whole):
            np.testing.assert_array_equal(part, full[sl])
        assert slow == 2.0


def test_max_over_ranks_without_a_group_is_the_identity():
    assert bench.max_over_ranks(3.5) == 3.5
