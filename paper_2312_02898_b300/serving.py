"""Continuous-batching request loop over the C ABI (one GPU).

Requests -- (process, momenta, alphas, rnd_hel, rnd_col) batches of uneven size, as they
come from many integration channels (the multi-event interface of the paper's
Section 3) -- are queued on the host and admitted onto the GPU as soon as a stream slot
and device memory are free, so work from many requests overlaps on the device.

* Every process keeps one handle (helicity list, couplings, colour matrix resident).
* A chunk is padded to a size bucket (powers of two and 1.5 times powers of two, from
  256 events up to the chunk size, so padding adds at most half) by repeating its last
  event; events are independent, so padding does not
  change any result, and a request's results are the same alone and in any mix.
* Each (slot, process, bucket) owns pinned host staging, device buffers and, once used,
  a captured CUDA graph of [copy in -> me_compute -> copy out] that is replayed.
* A request larger than the chunk size (16384 events by default) runs as several
  chunks.  When a slot frees up, the scheduler takes the next chunk either of the oldest
  request ("fifo") or of the request with the least remaining work, events times the
  process's flops per event ("srpt"), so that small requests need not wait behind a
  large one.
* Admission: a chunk starts when a slot is idle and the device bytes of all running
  chunks plus its own, on top of the per-stream workspaces the handles hold for the
  largest chunk, stay within the budget: by default 80% of the device memory that is
  free once those workspaces exist.
* Latency is measured from submit() to the moment all of a request's results are on
  the host.

Only host bookkeeping lives here; every evaluation runs in libme_b300.so.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np

from .phasespace import make_batch

# 256, 384, 512, 768, ..., 49152, 65536: a chunk is padded by at most half of itself
BUCKETS = tuple(sorted({2 ** k for k in range(8, 17)} | {3 * 2 ** (k - 1) for k in range(8, 16)}))


def bucket_for(n: int, buckets=BUCKETS) -> int:
    """smallest bucket holding n events (n <= largest bucket): a power of two or 1.5
    times one"""
    for b in buckets:
        if n <= b:
            return b
    raise ValueError(f"request of {n} events exceeds the largest bucket {buckets[-1]}")


def pad_to(x: np.ndarray, n: int) -> np.ndarray:
    """pad along axis 0 to n rows by repeating the last row"""
    if x.shape[0] == n:
        return x
    reps = np.repeat(x[-1:], n - x.shape[0], axis=0)
    return np.concatenate([x, reps], axis=0)


def percentile(values, q):
    v = sorted(values)
    if not v:
        return float("nan")
    k = (len(v) - 1) * q / 100.0
    f, c = math.floor(k), math.ceil(k)
    return v[f] if f == c else v[f] + (v[c] - v[f]) * (k - f)


def pick_next(queue, policy):
    """the request whose next chunk goes out: the oldest with events left ("fifo"), or
    the one with the least remaining work, undispatched events times flops per event
    ("srpt"; ties go to the older request)"""
    if policy == "fifo":
        return queue[0]
    return min(queue, key=lambda q: (q.nevt - q.next_event) * q.cost)


class MemoryAdmission:
    """Device-byte budget shared by running requests (host-side accounting).

    ``reserved`` is what the server holds whatever runs (the handles' per-stream
    workspaces); a chunk is admitted while reserved + running chunks + itself fit the
    budget, except that a chunk alone on the device always starts."""

    def __init__(self, budget_bytes: int, reserved: int = 0):
        self.budget = budget_bytes
        self.reserved = reserved
        self.used = 0

    def try_take(self, nbytes: int) -> bool:
        if self.reserved + self.used + nbytes > self.budget and self.used > 0:
            return False
        self.used += nbytes
        return True

    def give(self, nbytes: int):
        self.used -= nbytes
        assert self.used >= 0


@dataclass(eq=False)  # requests compare by identity (the scheduler removes them from its queue)
class Request:
    process: str
    momenta: np.ndarray
    alphas: np.ndarray | None
    rnd_hel: np.ndarray
    rnd_col: np.ndarray
    t_submit: float = 0.0
    future: Future = field(default_factory=Future)
    tag: object = None
    cost: float = 1.0        # flops per event of the process (scheduling weight)
    next_event: int = 0      # first event not yet dispatched
    outstanding: int = 0     # chunks on the GPU
    out: tuple = None        # (me, sel_hel, sel_col) filled chunk by chunk

    @property
    def nevt(self):
        return self.momenta.shape[0]


class _Buffers:
    """pinned staging, device buffers and the captured graph of one (slot, process, bucket)"""

    def __init__(self, torch, npar, nb, device):
        pin = dict(dtype=torch.float64, pin_memory=True)
        self.h_mom = torch.empty((nb, npar, 4), **pin)
        self.h_as = torch.empty(nb, **pin)
        self.h_rh = torch.empty(nb, **pin)
        self.h_rc = torch.empty(nb, **pin)
        self.h_me = torch.empty(nb, **pin)
        self.h_sh = torch.empty(nb, dtype=torch.int32, pin_memory=True)
        self.h_sc = torch.empty(nb, dtype=torch.int32, pin_memory=True)
        d = dict(dtype=torch.float64, device=device)
        self.d_mom = torch.empty((nb, npar, 4), **d)
        self.d_as = torch.empty(nb, **d)
        self.d_rh = torch.empty(nb, **d)
        self.d_rc = torch.empty(nb, **d)
        self.d_me = torch.empty(nb, **d)
        self.d_sh = torch.empty(nb, dtype=torch.int32, device=device)
        self.d_sc = torch.empty(nb, dtype=torch.int32, device=device)
        self.graph = None
        self.nbytes = sum(t.numel() * t.element_size() for t in
                          (self.d_mom, self.d_as, self.d_rh, self.d_rc, self.d_me, self.d_sh, self.d_sc))


class Server:
    def __init__(self, processes, precision="mixed", n_slots=4, mem_budget_bytes=None, use_graphs=True,
                 device=0, params=None, policy="srpt", chunk_events=16384):
        if policy not in ("fifo", "srpt"):
            raise ValueError(f"unknown scheduling policy {policy!r}")
        self.policy = policy
        self.chunk = bucket_for(chunk_events)
        import torch
        from paper_2312_02898_b300.binding import MatrixElement, MEError
        self.torch = torch
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.handles = {}
        self.precision = {}
        for p in processes:
            try:
                self.handles[p] = MatrixElement(p, precision=precision, **(params or {}))
                self.precision[p] = precision
            except MEError as e:
                if e.code != -2:
                    raise
                # no tensor-core path for this process: FP32 amplitudes and colour sum
                self.handles[p] = MatrixElement(p, precision="fp32", **(params or {}))
                self.precision[p] = "fp32"
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_slots)]
        # size every (process, stream) workspace for the largest chunk up front, so no
        # later call moves a workspace that a captured graph points into
        # (every bucket up to the chunk: a call's workspace need not grow with its size,
        # e.g. a smaller batch may spread each event over more threads)
        self.workspace_bytes = 0
        sizes = [b for b in BUCKETS if b <= self.chunk]
        for m in self.handles.values():
            for s in self.streams:
                for b in sizes:
                    m.reserve(b, s)
                self.workspace_bytes += max(m.plan(b)[1] for b in sizes)
        torch.cuda.synchronize()
        free, _ = torch.cuda.mem_get_info(self.device)
        room = int(0.8 * free) if mem_budget_bytes is None else min(int(mem_budget_bytes), int(0.8 * free))
        self.mem_budget = self.workspace_bytes + room
        self.slot_busy = [None] * n_slots           # (request, buffers, event, nbytes)
        self.buffers = {}                           # (slot, process, bucket) -> _Buffers
        self._warmed = set()                        # processes whose kernels have run once
        self.admission = MemoryAdmission(self.mem_budget, reserved=self.workspace_bytes)
        self.use_graphs = use_graphs
        self.queue = collections.deque()
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.stop = False
        self.done = []                              # (process, nevt, latency s, finish time, tag)
        self.max_running = 0                        # most requests on the GPU at once
        self.error = None                           # what stopped the loop, if anything
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    # ------------------------------------------------------------------ API
    def submit(self, process, momenta, alphas=None, rnd_hel=None, rnd_col=None, tag=None) -> Future:
        n = momenta.shape[0]
        if n < 1:
            raise ValueError("a request needs at least one event")
        if process not in self.handles:
            raise KeyError(f"process {process!r} is not served here")
        rh = rnd_hel if rnd_hel is not None else np.full(n, 0.5)
        rc = rnd_col if rnd_col is not None else np.full(n, 0.5)
        r = Request(process, np.ascontiguousarray(momenta, dtype=np.float64),
                    None if alphas is None else np.ascontiguousarray(alphas, dtype=np.float64),
                    np.ascontiguousarray(rh, dtype=np.float64), np.ascontiguousarray(rc, dtype=np.float64), tag=tag)
        r.cost = float(self.handles[process].flops_per_event())
        r.out = (np.empty(n), np.empty(n, dtype=np.int32), np.empty(n, dtype=np.int32))
        r.t_submit = time.perf_counter()
        if self.error is not None:
            raise RuntimeError("the serving loop has stopped") from self.error
        with self.cv:
            self.queue.append(r)
            self.cv.notify()
        return r.future

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify()
        self.thread.join()

    def warm(self, process, bucket, slots=None):
        """allocate buffers, grow workspaces and capture graphs ahead of traffic (buckets
        above the chunk size are never used)"""
        if bucket > self.chunk:
            return
        for s in (slots if slots is not None else range(len(self.streams))):
            self._prepare(s, process, bucket)

    # ------------------------------------------------------------------ internals
    def _prepare(self, slot, process, bucket):
        key = (slot, process, bucket)
        b = self.buffers.get(key)
        if b is not None:
            return b
        torch = self.torch
        m = self.handles[process]
        b = _Buffers(torch, m.npar, bucket, self.device)
        s = self.streams[slot]
        mom1 = make_batch(process, 1, seed=0)[0]  # one physical event for the warm-up call
        b.d_mom.copy_(torch.from_numpy(np.repeat(mom1, bucket, axis=0)))
        b.d_as.fill_(0.118)
        b.d_rh.fill_(0.5)
        b.d_rc.fill_(0.5)
        torch.cuda.synchronize()
        # one uncaptured call per process loads its kernels before the first capture (the
        # workspaces were reserved for the largest chunk when the server started)
        if process not in self._warmed:
            self._run(m, b, s, bucket)
            s.synchronize()
            self._warmed.add(process)
        if self.use_graphs:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
                self._copy_in(b, s, bucket)
                self._run(m, b, s, bucket)
                self._copy_out(b, s, bucket)
            b.graph = g
        self.buffers[key] = b
        return b

    def _copy_in(self, b, s, n):
        with self.torch.cuda.stream(s):
            b.d_mom[:n].copy_(b.h_mom[:n], non_blocking=True)
            b.d_as[:n].copy_(b.h_as[:n], non_blocking=True)
            b.d_rh[:n].copy_(b.h_rh[:n], non_blocking=True)
            b.d_rc[:n].copy_(b.h_rc[:n], non_blocking=True)

    def _copy_out(self, b, s, n):
        with self.torch.cuda.stream(s):
            b.h_me[:n].copy_(b.d_me[:n], non_blocking=True)
            b.h_sh[:n].copy_(b.d_sh[:n], non_blocking=True)
            b.h_sc[:n].copy_(b.d_sc[:n], non_blocking=True)

    def _run(self, m, b, s, n):
        m.compute_raw(n, b.d_mom.data_ptr(), b.d_as.data_ptr(), b.d_rh.data_ptr(), b.d_rc.data_ptr(),
                      b.d_me.data_ptr(), b.d_sh.data_ptr(), b.d_sc.data_ptr(), s.cuda_stream)

    def _launch(self, slot, r: Request):
        """dispatch the next chunk of r on 'slot'; False when memory admission refuses"""
        lo = r.next_event
        n = min(self.chunk, r.nevt - lo)
        nb = bucket_for(n)
        b = self._prepare(slot, r.process, nb)
        if not self.admission.try_take(b.nbytes):
            return False
        sl = slice(lo, lo + n)
        a = r.alphas[sl] if r.alphas is not None else np.full(n, self.handles[r.process].params.alphas_default)
        b.h_mom.numpy()[:] = pad_to(r.momenta[sl], nb)
        b.h_as.numpy()[:] = pad_to(a, nb)
        b.h_rh.numpy()[:] = pad_to(r.rnd_hel[sl], nb)
        b.h_rc.numpy()[:] = pad_to(r.rnd_col[sl], nb)
        r.next_event = lo + n
        r.outstanding += 1
        s = self.streams[slot]
        if b.graph is not None:
            with self.torch.cuda.stream(s):
                b.graph.replay()
        else:
            self._copy_in(b, s, nb)
            self._run(self.handles[r.process], b, s, nb)
            self._copy_out(b, s, nb)
        ev = self.torch.cuda.Event()
        ev.record(s)
        self.slot_busy[slot] = (r, b, ev, b.nbytes, lo, n)
        self.max_running = max(self.max_running, sum(x is not None for x in self.slot_busy))
        return True

    def _complete(self, slot):
        r, b, ev, nbytes, lo, n = self.slot_busy[slot]
        r.out[0][lo:lo + n] = b.h_me.numpy()[:n]
        r.out[1][lo:lo + n] = b.h_sh.numpy()[:n]
        r.out[2][lo:lo + n] = b.h_sc.numpy()[:n]
        self.slot_busy[slot] = None
        self.admission.give(nbytes)
        r.outstanding -= 1
        if r.outstanding == 0 and r.next_event == r.nevt:
            now = time.perf_counter()
            self.done.append((r.process, r.nevt, now - r.t_submit, now, r.tag))
            r.future.set_result(r.out)

    def _pick(self):
        return pick_next(self.queue, self.policy)

    def _loop(self):
        try:
            self._serve()
        except BaseException as e:  # fail every pending request instead of leaving it hanging
            self.error = e
            with self.lock:
                pending = list(self.queue) + [b[0] for b in self.slot_busy if b is not None]
                self.queue.clear()
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(e)

    def _serve(self):
        while True:
            with self.cv:
                if self.stop and not self.queue and all(x is None for x in self.slot_busy):
                    return
                if not self.queue and all(x is None for x in self.slot_busy):
                    self.cv.wait(0.01)
            progressed = False
            for slot, busy in enumerate(self.slot_busy):
                if busy is not None and busy[2].query():
                    self._complete(slot)
                    progressed = True
            with self.lock:
                for slot in range(len(self.slot_busy)):
                    if not self.queue:
                        break
                    if self.slot_busy[slot] is None:
                        r = self._pick()
                        if self._launch(slot, r):
                            if r.next_event == r.nevt:
                                self.queue.remove(r)
                            progressed = True
            if not progressed:
                time.sleep(20e-6)

    # ------------------------------------------------------------------ reporting
    def stats(self):
        lat = [x[2] * 1e3 for x in self.done]
        return {"requests": len(self.done), "events": int(sum(x[1] for x in self.done)),
                "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
                "mean_ms": float(np.mean(lat)) if lat else float("nan")}


# ---------------------------------------------------------------------------
# the request stream of the serving workload
# ---------------------------------------------------------------------------
STREAM_PROCESSES = (("e+ e- > mu+ mu-", 0.10), ("g g > t t~", 0.15), ("g g > t t~ g", 0.15),
                    ("g g > t t~ g g", 0.40), ("g g > t t~ g g g", 0.20))


def request_stream(nreq, rate_hz, seed=0, lo=256, hi=65536, first=0):
    """(arrival time, process, nevt, request seed) for nreq Poisson arrivals at rate_hz;
    process drawn with the stream weights, size log-uniform in [lo, hi]; request k uses
    seed k for its own inputs."""
    rng = np.random.default_rng(seed)
    names = [p for p, _ in STREAM_PROCESSES]
    w = np.array([x for _, x in STREAM_PROCESSES])
    t = 0.0
    out = []
    for k in range(first, first + nreq):
        t += rng.exponential(1.0 / rate_hz)
        proc = names[rng.choice(len(names), p=w / w.sum())]
        n = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append((t, proc, min(max(n, lo), hi), k))
    return out


def make_requests(stream, alphas="uniform"):
    """momenta and random numbers of each request of a stream (request k from seed k)"""
    out = []
    for t, proc, n, seed in stream:
        mom, a, rh, rc = make_batch(proc, n, seed=seed, alphas=alphas)
        out.append((t, proc, mom, a, rh, rc))
    return out


def run_saturated(server, reqs):
    """submit every request at once; sustained ME/s = events / makespan"""
    server.done.clear()
    t0 = time.perf_counter()
    futs = [server.submit(p, mom, a, rh, rc) for _, p, mom, a, rh, rc in reqs]
    for f in futs:
        f.result()
    dt = time.perf_counter() - t0
    return sum(r[2].shape[0] for r in reqs) / dt


def run_open_loop(server, reqs, rate_scale=1.0, warmup=0):
    """replay the arrival times (divided by rate_scale) in real time.  Latency statistics
    cover the requests after the first `warmup`; ME/s is their events over the time from
    the first of them being submitted to the last of them finishing."""
    server.done.clear()
    t0 = time.perf_counter()
    futs = []
    t_first = None
    for k, (t, p, mom, a, rh, rc) in enumerate(reqs):
        wait = t0 + t / rate_scale - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        if k == warmup:
            t_first = time.perf_counter()
        futs.append(server.submit(p, mom, a, rh, rc, tag=k))
    for f in futs:
        f.result()
    t_last = max(x[3] for x in server.done if x[4] >= warmup)
    kept = [x for x in server.done if x[4] >= warmup]
    lat = [x[2] * 1e3 for x in kept]
    ev = sum(x[1] for x in kept)
    per_process = {}
    for proc in sorted({x[0] for x in kept}):
        lp = [x[2] * 1e3 for x in kept if x[0] == proc]
        per_process[proc] = {"requests": len(lp), "p50_ms": percentile(lp, 50), "p99_ms": percentile(lp, 99)}
    return {"requests": len(kept), "events": int(ev), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
            "mean_ms": float(np.mean(lat)), "me_per_s": ev / (t_last - t_first), "per_process": per_process}
