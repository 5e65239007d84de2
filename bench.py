"""Throughput benchmark: tree-level matrix elements per second on one B300 (or N, as
independent shards of events).

Workload (one "step"): g g -> t t~ g g, 1048576 RAMBO events at sqrt(s) = 1500 GeV with
per-event alpha_s ~ U[0.10, 0.13] and both selection outputs -- every row of the hot
path (momentum load, couplings, wavefunctions, currents, diagram closings, colour sum,
helicity sum, selections).  Inputs (226 MB) are larger than the 126 MB L2, so no L2
flush is needed between steps.  Each precision mode is timed separately; the headline
``value`` is the mode named by --mode (default: fp64, the mode that matches the FP64
oracle at 1e-12).  The default single-GPU run also carries the rest of the metric in the
same JSON line: every process at its own workload size in each precision mode
(``processes``) and a short serving stream in mixed precision and in FP64 with p50/p99
latency (``serving``); --no-extra leaves them out.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--mode fp64|fp32|mixed]
    python bench.py --impl reference      # the FP64 CPU oracle on the host cores
    python bench.py --serving             # the request stream: p50/p99 latency, sustained ME/s
    python bench.py --processes           # ME/s of every process and precision

Multi-GPU: every rank evaluates its own batch (disjoint event indices); the timed
region is bracketed by barriers and the maximum over ranks is taken.  No data-path
collective exists: events are independent ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PROCESS = "g g > t t~ g g"
NEVT = 1048576
METRIC = "ME evals/s per process, FP64 vs mixed at stated rel. err; serving p50/p99 ms"
UNIT = "ME evals/s"
FLOP_DTYPE = {"fp64": "f64", "fp32": "f32", "mixed": "f32+bf16", "dfloat": "f32 pairs (double-float)"}
ERR_BOUND = {"fp64": 1e-12, "fp32": 1e-5, "mixed": 1e-5, "dfloat": 1e-10}
# DRAM bytes per event of each mode's default main-pass kernel of g g > t t~ g g, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of a 655360-event launch;
# the traffic grows with the events processed.  Keyed by the kernel's layout, so a
# changed default reports no traffic; an entry is removed when its kernel's code changes
# and comes back with a new capture.
DRAM_BYTES_PER_EVENT = {
    ("fp64", "Layout<9, 64, 1, 1, 1, 2, 2, 3, 1>"): (6.136e10 + 8.949e10) / 655360,
    ("fp32", "Layout<10, 64, 1, 0, 1, 1, 2, 3, 1>"): (1.482e8 + 9.32e7) / 655360,
}
DEFAULT_LAYOUT = {"fp64": "Layout<9, 64, 1, 1, 1, 2, 2, 3, 1>", "fp32": "Layout<10, 64, 1, 0, 1, 1, 2, 3, 1>",
                  "mixed": "pipelined Layout<7, 128, 1, 0, 1, 2, 2, 3, 1>"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_events(rank: int, nevt_per_rank: int):
    """first event index of this rank's batch (disjoint, batch-independent RNG)"""
    return rank * nevt_per_rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """the maximum of x over all ranks (x itself without a process group)"""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region"""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples go to ME_B300_CLOCKS_DIR (default: the system temporary directory)
        out_dir = os.environ.get("ME_B300_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"me_b300_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append((float(f[1]), float(f[2]), f[4:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["active_mask", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(1, 5) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(process, nevt_sample, first_event, alphas="uniform"):
    """the FP64 CPU oracle (as it stands) on a bounded sample: (ME/s, cores, seconds)"""
    import oracle
    from paper_2312_02898_b300 import phasespace as ps
    oracle.build()
    mom, a, rh, rc = ps.make_batch(process, nevt_sample, seed=0, first_event=first_event, alphas=alphas)
    t0 = time.perf_counter()
    oracle.me(process, mom, alphas=a, rnd_hel=rh, rnd_col=rc)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return nevt_sample / dt, cores, dt


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sample = args.ref_sample
    for _ in range(args.warmup):
        oracle_rate(PROCESS, max(64, sample // 8), 0)
    times = []
    for k in range(args.steps):
        rate, cores, dt = oracle_rate(PROCESS, sample, k * sample)
        times.append(dt)
    value = sample * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (RAMBO, Philox4x32-10 seed 0)",
            "config": {"workload": f"{PROCESS}, sqrt(s)=1500 GeV, alpha_s~U[0.10,0.13], both selections",
                       "events_per_gpu": NEVT, "global_batch": NEVT, "precision": "fp64",
                       "parallelism": "host cores (OpenMP over events), rank 0 only",
                       "events_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{sample} events of the {NEVT}-event workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_mode(mode, dev_inputs, host_inputs, steps, warmup, dist, process=None, e2e=True):
    """device-resident timing and end-to-end timing of one precision mode"""
    import torch
    from paper_2312_02898_b300.binding import MatrixElement
    m = MatrixElement(process or PROCESS, precision=mode)
    mom, a, rh, rc = dev_inputs
    nevt = mom.shape[0]
    out = (torch.empty(nevt, dtype=torch.float64, device=mom.device),
           torch.empty(nevt, dtype=torch.int32, device=mom.device),
           torch.empty(nevt, dtype=torch.int32, device=mom.device))
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        m.compute(mom, a, rh, rc, out=out, stream=stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rank = dist.get_rank() if dist else 0
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        e0.record(stream)
        for _ in range(steps):
            m.compute(mom, a, rh, rc, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dist, mom.device)
    launches, ws_bytes = m.plan(nevt)
    res = {"ms": ms, "launches": launches, "workspace_bytes": ws_bytes, "clocks": clk.summary(),
           "flops_per_event": m.flops_per_event(), "ngood": m.ngood, "me": out[0], "sel": (out[1], out[2])}
    if not e2e:
        return res
    # end to end through the host entry point: pinned host inputs, copies inside
    hmom, ha, hrh, hrc = host_inputs
    hout = (torch.empty(nevt, dtype=torch.float64).pin_memory(), torch.empty(nevt, dtype=torch.int32).pin_memory(),
            torch.empty(nevt, dtype=torch.int32).pin_memory())
    for _ in range(max(1, warmup // 2)):
        m.compute_host(hmom, ha, hrh, hrc, out=hout, stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        m.compute_host(hmom, ha, hrh, hrc, out=hout, stream=stream)
    res["e2e_ms"] = max_over_ranks((time.perf_counter() - t0) * 1e3 / steps, dist, mom.device)
    return res


def time_testbed(mode, steps, warmup):
    """The standalone testbed flow (Section 2, Fig. 1b) on the device: every step
    generates the batch (RAMBO momenta, alpha_s, the two selection numbers) with the
    counter-based generator on the GPU and evaluates it, with no host round trip."""
    import ctypes
    import torch
    from paper_2312_02898_b300.binding import MatrixElement, _ptr
    m = MatrixElement(PROCESS, precision=mode)
    dev = torch.device("cuda", torch.cuda.current_device())
    mom = torch.empty((NEVT, m.npar, 4), dtype=torch.float64, device=dev)
    a, rh, rc = (torch.empty(NEVT, dtype=torch.float64, device=dev) for _ in range(3))
    out = (torch.empty(NEVT, dtype=torch.float64, device=dev), torch.empty(NEVT, dtype=torch.int32, device=dev),
           torch.empty(NEVT, dtype=torch.int32, device=dev))
    s = torch.cuda.current_stream()
    sp = ctypes.c_void_p(s.cuda_stream)

    def step(k):
        first = k * NEVT
        m._check(m.lib.me_rambo(m.handle, NEVT, 0, first, 1500.0, _ptr(mom), sp))
        for t, (stream_id, off, sc) in zip((a, rh, rc), ((1, 0.10, 0.03), (2, 0.0, 1.0), (3, 0.0, 1.0))):
            m._check(m.lib.me_uniforms(NEVT, 0, first, stream_id, off, sc, _ptr(t), sp))
        m.compute(mom, a, rh, rc, out=out, stream=s)

    for k in range(warmup):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for k in range(steps):
        step(warmup + k)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    e0.record(s)
    for k in range(steps):
        m._check(m.lib.me_rambo(m.handle, NEVT, 0, k * NEVT, 1500.0, _ptr(mom), sp))
    e1.record(s)
    torch.cuda.synchronize()
    gen_ms = e0.elapsed_time(e1) / steps
    launches = 4 + m.plan(NEVT)[0]  # RAMBO, three uniform streams, the compute call
    m.close()
    return {"value": NEVT / (ms * 1e-3), "unit": UNIT, "mode": mode, "ms_per_step": ms,
            "rambo_ms_per_batch": gen_ms, "launches_per_step": launches,
            "note": "device RAMBO + alpha_s + selection numbers + me_compute per step, no host transfer"}


def time_unweight(me, warmup, reps):
    """GPU-assisted batch unweighting of the step's matrix elements: the whole batch and
    the 16384-event batches madevent uses (Section 3, Table 2); time per call on the
    device and the achieved bandwidth of the 33 algorithmic bytes per event (read me,
    weight, random number; write weight and decision)"""
    import torch
    from paper_2312_02898_b300.binding import MatrixElement
    from paper_2312_02898_b300.phasespace import uniforms
    m = MatrixElement(PROCESS, precision="fp64")
    n = me.shape[0]
    u = torch.from_numpy(uniforms(7, np.arange(n, dtype=np.uint64), 0, 2)).cuda()
    wgt, rnd = u[:, 0].contiguous(), u[:, 1].contiguous()
    out = {}
    for size in (n, 16384):
        args = (me[:size], wgt[:size], rnd[:size])
        for _ in range(warmup):
            m.unweight(*args)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            r = m.unweight(*args)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        out[str(size)] = {"us_per_call": us, "gb_per_s": 33 * size / (us * 1e-6) / 1e9,
                          "accepted": int(r[3].item()), "launches_per_call": 2}
    m.close()
    out["note"] = "inputs resident (L2-sized); bound by launch latency at madevent's batch size"
    out["fused"] = time_fused_unweight(warmup, reps)
    return out


def time_fused_unweight(warmup, reps, n=16384):
    """me_compute_unweight (weights and batch maximum in the matrix-element kernel's
    epilogue, then one accept pass) against me_compute followed by me_unweight, per call
    of a madevent-sized batch, for a cheap and an expensive process (FP64)"""
    import torch
    from paper_2312_02898_b300 import phasespace as ps
    from paper_2312_02898_b300.binding import MatrixElement
    from paper_2312_02898_b300.phasespace import uniforms
    res = {}
    for process in ("e+ e- > mu+ mu-", PROCESS):
        m = MatrixElement(process, precision="fp64")
        mom, a, rh, rc = ps.make_batch(process, n, seed=3, alphas="uniform")
        u = uniforms(7, np.arange(n, dtype=np.uint64), 0, 2)
        d = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (mom, a, rh, rc, u[:, 0], u[:, 1])]

        def fused():
            return m.compute_unweight(*d)

        def separate():
            me, _, _ = m.compute(*d[:4])
            return m.unweight(me, d[4], d[5])

        times = {}
        for name, fn in (("fused", fused), ("separate", separate)):
            for _ in range(warmup):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) * 1e3 / reps
        res[process] = {"events": n, "us_per_call_fused": times["fused"], "us_per_call_separate": times["separate"]}
        m.close()
    return res


def accuracy_sample(mode_out, host_inputs, n=4096, process=None):
    """max / median relative error of a mode against the FP64 oracle on sampled events"""
    import oracle
    hmom, ha, hrh, hrc = (x.numpy() for x in host_inputs)
    nevt = hmom.shape[0]
    idx = np.unique(np.linspace(0, nevt - 1, n).astype(np.int64))
    ref = oracle.me(process or PROCESS, hmom[idx], alphas=ha[idx])["me"]
    got = mode_out.cpu().numpy()[idx]
    rel = np.abs(got / ref - 1)
    return float(rel.max()), float(np.median(rel)), len(idx)


def process_row(process, nevt, alphas, modes, peaks, steps, err_n, budget_s=10.0):
    """ME/s of one process at nevt events for each precision mode, with the achieved
    fraction of the measured FMA peak and the error against the FP64 oracle on err_n
    sampled events; steps adapt so that each mode's timed work stays near budget_s"""
    import torch
    from paper_2312_02898_b300 import binding
    from paper_2312_02898_b300 import phasespace as ps
    mom, a, rh, rc = ps.make_batch(process, nevt, seed=0, alphas=alphas)
    if a is None:
        a = np.full(nevt, 0.118)
    host = [torch.from_numpy(x).pin_memory() for x in (mom, a, rh, rc)]
    dev = [x.cuda(non_blocking=True) for x in host]
    torch.cuda.synchronize()
    row = {"events": nevt, "input_mb": round(sum(x.numel() * x.element_size() for x in host) / 1e6, 1)}
    for mode in modes:
        # one untimed probe call sizes the steps (and allocates the workspace)
        try:
            probe = time_mode(mode, dev, host, 1, 0, None, process=process, e2e=False)
        except binding.MEError as e:
            row[mode] = {"unavailable": str(e)}
            continue
        k = int(max(2, min(steps, budget_s / max(probe["ms"] * 1e-3, 1e-6))))
        r = time_mode(mode, dev, host, k, 2 if probe["ms"] < 1000 else 0, None, process=process, e2e=False)
        mx, med, ns = accuracy_sample(r["me"], host, n=err_n, process=process)
        tf = r["flops_per_event"] * nevt / (r["ms"] * 1e-3) / 1e12
        # the double-float mode is rated against the FP64 peak it emulates
        pk = peaks["fp64" if mode in ("fp64", "dfloat") else "fp32"] / 1e12
        row[mode] = {"me_per_s": nevt / (r["ms"] * 1e-3), "ms_per_step": r["ms"], "steps": k, "tflops": tf,
                     "frac_of_measured_peak": tf / pk, "launches_per_step": r["launches"], "max_rel_err": mx,
                     "median_rel_err": med, "err_sample": ns, "bound": ERR_BOUND[mode], "clocks": r["clocks"]}
        del r, probe
    del dev, host
    torch.cuda.synchronize()
    return row


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    from paper_2312_02898_b300 import binding
    from paper_2312_02898_b300 import phasespace as ps
    first = shard_events(rank, NEVT)
    mom, a, rh, rc = ps.make_batch(PROCESS, NEVT, seed=0, first_event=first, alphas="uniform")
    host = [torch.from_numpy(x).pin_memory() for x in (mom, a, rh, rc)]
    dev = [x.cuda(non_blocking=True) for x in host]
    torch.cuda.synchronize()
    modes = [args.mode] + [m for m in ("fp64", "fp32", "mixed") if m != args.mode and not args.only]
    results = {}
    for mode in modes:
        try:
            results[mode] = time_mode(mode, dev, host, args.steps, args.warmup, dist)
        except binding.MEError as e:
            results[mode] = {"error": str(e)}
    head = results[args.mode]
    if "error" in head:
        raise SystemExit(f"headline mode {args.mode} failed: {head['error']}")
    value = world * NEVT / (head["ms"] * 1e-3)
    unw = time_unweight(head["me"], args.warmup, max(args.steps, 10))
    testbed = time_testbed(args.mode, min(args.steps, 3), 3)
    peaks = {p: binding.alu_peak(p, 0.3) for p in ("fp64", "fp32")}
    per_launch_ms = head["ms"] / head["launches"]
    events_per_launch = NEVT / head["launches"]
    peak_key = "fp64" if args.mode == "fp64" else "fp32"
    achieved = head["flops_per_event"] * events_per_launch / (per_launch_ms * 1e-3) / 1e12
    peak = peaks[peak_key] / 1e12
    line = None
    if rank == 0:
        acc = {}
        for mode, r in results.items():
            if "error" in r:
                acc[mode] = {"error": r["error"]}
                continue
            mx, med, ns = accuracy_sample(r["me"], host, n=args.err_sample)
            acc[mode] = {"value": NEVT * world / (r["ms"] * 1e-3), "ms_per_step": r["ms"],
                         "max_rel_err": mx, "median_rel_err": med, "err_sample": ns, "bound": ERR_BOUND[mode],
                         "gpu_launches_per_step": r["launches"], "clocks": r["clocks"]}
        try:
            ref_rate, cores, dt = oracle_rate(PROCESS, args.cpu_sample, 0)
            cpu = {"value": ref_rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"first {args.cpu_sample} events of the workload ({dt:.1f} s)"}
        except Exception as e:  # the oracle needs gcc; report rather than fail
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": f"failed: {e}"}
        h2d = sum(x.numel() * x.element_size() for x in host)
        d2h = NEVT * (8 + 4 + 4)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": FLOP_DTYPE[args.mode], "data": "synthetic (RAMBO, Philox4x32-10 seed 0)",
                "config": {"workload": f"{PROCESS}, sqrt(s)=1500 GeV, alpha_s~U[0.10,0.13], both selections",
                           "events_per_gpu": NEVT, "global_batch": NEVT * world, "precision": args.mode,
                           "parallelism": f"events sharded over {world} GPU(s), no collective",
                           "l2": f"inputs ({NEVT * 216 / 1e6:.0f} MB per GPU) "
                                 + ("larger than L2; no flush" if NEVT * 216 > 126e6 else "smaller than L2")},
                "clocks": head["clocks"],
                "gpu_launches": head["launches"] * args.steps,
                "e2e": {"value": world * NEVT / (head["e2e_ms"] * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h, "entry": "me_compute_host"},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak,
                             "traffic": (DRAM_BYTES_PER_EVENT.get((args.mode, DEFAULT_LAYOUT[args.mode]), 0) * NEVT
                                         / head["launches"] or None),
                             "traffic_source": "ncu dram__bytes of the default layout at 655360 events, scaled to "
                                               "one launch of this step",
                             "peak_source": f"measured {peak_key.upper()} FMA probe (me_probe_alu_peak) in this run",
                             "flops_per_event": head["flops_per_event"], "kernel": "me_kernel (amplitudes + colour sum)"},
                "modes": acc,
                "unweight": unw,
                "testbed": testbed,
                "cpu_baseline": cpu,
                "alu_peaks_tflops": {k: v / 1e12 for k, v in peaks.items()}}
        if world == 1 and not args.no_extra:
            # the rest of the metric: every process at its own workload size, and the
            # serving stream in mixed precision beside the same stream in FP64
            line["processes"] = processes_table(args, peaks, reuse={PROCESS: (results, acc)})
            line["dispatch"] = dispatch_table(args, DISPATCH_CHANNELS)
            line["dispatch_jet"] = dispatch_table(args, DISPATCH_JET_CHANNELS)
            line["dispatch_2jet"] = dispatch_table(args, DISPATCH_2JET_CHANNELS, nevt=262144)
            line["serving"] = serving_table(args, quick=True)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


# the per-process workloads: (process, events, alpha_s)
PROCESS_TABLE = (("e+ e- > mu+ mu-", 16384, None), ("g g > t t~", 524288, 0.118), ("g g > t t~ g", 524288, 0.118),
                 ("g g > t t~ g g", 1048576, "uniform"), ("g g > t t~ g g g", 262144, 0.118),
                 ("u u~ > t t~", 524288, 0.118), ("u u~ > t t~ g", 524288, 0.118), ("u g > t t~ u", 524288, 0.118),
                 ("u u~ > t t~ g g", 262144, 0.118), ("u g > t t~ u g", 262144, 0.118), ("g g > t t~ u u~", 262144, 0.118),
                 ("u u~ > t t~ d d~", 262144, 0.118), ("u d > t t~ u d", 262144, 0.118), ("u u > t t~ u u", 262144, 0.118))


DISPATCH_CHANNELS = (("g g > t t~", 0.90), ("u u~ > t t~", 0.05), ("u~ u > t t~", 0.05))
# p p -> t t~ + jet: g g -> t t~ g and the six quark channels (synthetic shares)
DISPATCH_JET_CHANNELS = (("g g > t t~ g", 0.55), ("u u~ > t t~ g", 0.10), ("u~ u > t t~ g", 0.10),
                         ("u g > t t~ u", 0.07), ("g u > t t~ u", 0.07), ("u~ g > t t~ u~", 0.055),
                         ("g u~ > t t~ u~", 0.055))
# p p -> t t~ + 2 jets: g g -> t t~ g g, the seven channels with one light-quark line and
# the nine four-quark channels (two light flavours, or one with both pairings); synthetic
# shares
DISPATCH_2JET_CHANNELS = (("g g > t t~ g g", 0.36), ("u u~ > t t~ g g", 0.06), ("u~ u > t t~ g g", 0.06),
                          ("u g > t t~ u g", 0.06), ("g u > t t~ u g", 0.06), ("u~ g > t t~ u~ g", 0.05),
                          ("g u~ > t t~ u~ g", 0.05), ("g g > t t~ u u~", 0.05), ("u u~ > t t~ d d~", 0.04),
                          ("u~ u > t t~ d d~", 0.03), ("u d > t t~ u d", 0.04), ("u d~ > t t~ u d~", 0.03),
                          ("u~ d~ > t t~ u~ d~", 0.03), ("u u > t t~ u u", 0.02), ("u~ u~ > t t~ u~ u~", 0.02),
                          ("u u~ > t t~ u u~", 0.02), ("u~ u > t t~ u u~", 0.02))


def dispatch_table(args, channels, nevt=524288):
    """p p -> t t~ (+ jet) with per-event channel dispatch (me_compute_channels): one
    batch of RAMBO events (massless beams and jet, massive tops: valid for every channel
    of the list), each event assigned a channel with the list's fractions (synthetic,
    close to the g g / q q~ / q g shares of top-pair production at the LHC); ME/s of the
    mixed batch beside the first (g g) channel alone, and the error of each channel
    against its oracle."""
    import torch
    import oracle
    from paper_2312_02898_b300 import phasespace as ps
    from paper_2312_02898_b300.binding import MatrixElement, compute_channels
    mom, a, rh, rc = (torch.from_numpy(x).cuda() for x in
                      ps.make_batch(channels[0][0], nevt, seed=0, alphas="uniform"))
    rng = np.random.default_rng(0)
    ch_np = rng.choice(len(channels), size=nevt, p=[f for _, f in channels]).astype(np.int32)
    ch = torch.from_numpy(ch_np).cuda()
    out = {"events": nevt, "channels": {p: float(f) for p, f in channels}}
    for prec in ("fp64", "fp32"):
        hs = [MatrixElement(p, precision=prec) for p, _ in channels]
        res = (torch.empty(nevt, dtype=torch.float64, device="cuda"), torch.empty(nevt, dtype=torch.int32, device="cuda"),
               torch.empty(nevt, dtype=torch.int32, device="cuda"))

        def timed(fn, steps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        ms = timed(lambda: compute_channels(hs, ch, mom, a, rh, rc, out=res), args.steps)
        ms_gg = timed(lambda: hs[0].compute(mom, a, rh, rc, out=res), args.steps)
        compute_channels(hs, ch, mom, a, rh, rc, out=res)
        torch.cuda.synchronize()
        got = res[0].cpu().numpy()
        errs = {}
        for c, (p, _) in enumerate(channels):
            idx = np.nonzero(ch_np == c)[0][:512]
            ref = oracle.me(p, mom[idx].cpu().numpy(), alphas=a[idx].cpu().numpy())["me"]
            errs[p] = float(np.max(np.abs(got[idx] / ref - 1)))
        out[prec] = {"me_per_s": nevt / (ms * 1e-3), "ms_per_step": ms, "gg_alone_me_per_s": nevt / (ms_gg * 1e-3),
                     "max_rel_err_per_channel": errs, "err_sample_per_channel": 512,
                     "launches_per_step": 2 + sum(h.plan(nevt)[0] for h in hs)}
        for h in hs:
            h.close()
    return out


def processes_table(args, peaks, reuse=None):
    """per-process rows (process_row) for every process of PROCESS_TABLE; a process whose
    modes were already timed at its workload size (the headline step) reuses them"""
    table = {}
    for process, nevt, alphas in PROCESS_TABLE:
        if args.only_process and args.only_process != process:
            continue
        if args.process_nevt:
            nevt = args.process_nevt
        if reuse and process in reuse and nevt == NEVT:
            results, acc = reuse[process]
            row = {"events": nevt, "reused": "the headline step of this run"}
            for mode, r in results.items():
                if "error" in r:
                    row[mode] = {"unavailable": r["error"]}
                    continue
                tf = r["flops_per_event"] * nevt / (r["ms"] * 1e-3) / 1e12
                pk = peaks["fp64" if mode == "fp64" else "fp32"] / 1e12
                row[mode] = {"me_per_s": nevt / (r["ms"] * 1e-3), "ms_per_step": r["ms"], "tflops": tf,
                             "frac_of_measured_peak": tf / pk, "launches_per_step": r["launches"],
                             "max_rel_err": acc[mode]["max_rel_err"], "median_rel_err": acc[mode]["median_rel_err"],
                             "err_sample": acc[mode]["err_sample"], "bound": ERR_BOUND[mode]}
            table[process] = row
            continue
        modes = [m for m in args.process_modes.split(",")]
        table[process] = process_row(process, nevt, alphas, modes, peaks, args.steps, args.process_err_sample)
    return table


def run_processes(args):
    """ME/s of every process and precision at its own workload size, with the achieved
    fraction of the measured FP64 / FP32 FMA peak and the error against the oracle on
    sampled events (one JSON line)."""
    import torch
    from paper_2312_02898_b300 import binding
    torch.cuda.set_device(0)
    peaks = {p: binding.alu_peak(p, 0.3) for p in ("fp64", "fp32")}
    table = processes_table(args, peaks)
    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "data": "synthetic (RAMBO, Philox4x32-10 seed 0)",
            "config": {"workload": "every process at its own batch size, inputs resident, both selections"},
            "alu_peaks_tflops": {k: v / 1e12 for k, v in peaks.items()}, "processes": table}
    print(json.dumps(line), flush=True)


def _gen_request(item):
    from paper_2312_02898_b300.phasespace import make_batch
    t, proc, n, seed = item
    mom, a, rh, rc = make_batch(proc, n, seed=seed, alphas="uniform")
    return t, proc, mom, a, rh, rc


def serving_table(args, quick=False):
    """The serving stream: Poisson arrivals of requests for all processes (weights
    0.1 / 0.15 / 0.15 / 0.4 / 0.2 for e+e- -> mu+mu-, gg -> tt~, gg -> tt~g, gg -> tt~gg,
    gg -> tt~ggg), sizes log-uniform in [256, 65536], request k from seed k.  For each
    precision: the sustained capacity with every request queued at once, then the
    open-loop stream at fractions of that capacity with p50/p99 latency (submit to
    results on the host), pooled and per process.  quick: the short form the default
    benchmark run carries (fewer requests, 70% load only, no first-come comparison)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_2312_02898_b300 import serving
    if quick:
        nmeas, nwarm, nother, loads_first, fifo = args.quick_serving_requests, 50, 100, [0.7], False
    else:
        nmeas, nwarm, nother, fifo = args.serving_requests, args.serving_warmup, args.serving_requests_other, True
        loads_first = [float(x) for x in args.serving_loads.split(",")]
    nother_warm = min(nwarm, 20) if quick else nwarm
    nreq = nmeas + nwarm
    stream = serving.request_stream(nreq, rate_hz=1.0, seed=0)
    with cf.ProcessPoolExecutor(max_workers=min(32, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as ex:
        reqs = list(ex.map(_gen_request, stream, chunksize=8))
    import torch
    mean_events = float(np.mean([r[2].shape[0] for r in reqs]))
    out = {}
    runs = [(prec, "srpt") for prec in args.serving_precisions.split(",")]
    if fifo:
        runs.insert(1, (runs[0][0], "fifo"))  # the same precision with first-come scheduling, for comparison
    for prec, policy in runs:
        server = serving.Server([p for p, _ in serving.STREAM_PROCESSES], precision=prec, n_slots=args.serving_slots,
                                policy=policy, chunk_events=args.serving_chunk)
        try:
            t0 = time.perf_counter()
            for p, _ in serving.STREAM_PROCESSES:
                for b in serving.BUCKETS:
                    server.warm(p, b)
            warm_s = time.perf_counter() - t0
            first = not out
            same_stream = first or policy == "fifo"   # fifo replays the whole stream beside srpt
            # the slower precisions replay a prefix of the same stream (their own warm-up)
            warm = nwarm if same_stream else nother_warm
            sub = reqs if same_stream else reqs[nwarm - warm: nwarm + nother]
            if policy == "fifo":
                cap = next(iter(out.values()))["capacity_me_per_s"]
            else:
                cap = serving.run_saturated(server, sub[: warm + (nmeas if same_stream else nother) // 4])
            res = {"capacity_me_per_s": cap, "graphs": len(server.buffers), "warm_s": warm_s, "policy": policy,
                   "chunk_events": server.chunk, "precision_per_process": server.precision,
                   "workspace_bytes": server.workspace_bytes, "mem_budget_bytes": server.mem_budget,
                   "requests_measured": len(sub) - warm, "requests_warmup": warm, "load": {}}
            loads = loads_first if first else [0.7]
            for frac in loads:
                rate = frac * cap / mean_events                   # requests per second
                st = serving.run_open_loop(server, sub, rate_scale=rate, warmup=warm)
                st["offered_requests_per_s"] = rate
                st["offered_me_per_s"] = frac * cap
                res["load"][f"{int(round(frac * 100))}%"] = st
            out[prec if policy == "srpt" else f"{prec}_fifo"] = res
        finally:
            server.close()
            del server
            torch.cuda.synchronize()
    return {"slots": args.serving_slots, "buckets": list(serving.BUCKETS), "mean_events_per_request": mean_events,
            "stream": "Poisson arrivals over the five processes, log-uniform 256-65536 events per request, "
                      "alpha_s~U[0.10,0.13], request k from seed k; latency = submit to results on the host",
            "precisions": out}


def run_serving(args):
    """the full serving study as its own JSON line (headline: p99 at 70% load)"""
    res = serving_table(args)
    head = next(iter(res["precisions"].values()))
    key = "70%" if "70%" in head["load"] else next(iter(head["load"]))
    line = {"metric": METRIC, "value": head["load"][key]["p99_ms"], "unit": "ms (p99 latency)",
            "higher_is_better": False, "n_gpus": 1, "steps": args.serving_requests, "warmup": args.serving_warmup,
            "data": "synthetic (RAMBO, Philox4x32-10, request k from seed k)",
            "config": {"workload": "serving stream: Poisson arrivals over the five processes, "
                                   "log-uniform 256-65536 events per request, alpha_s~U[0.10,0.13]",
                       "slots": args.serving_slots, "buckets": res["buckets"],
                       "mean_events_per_request": res["mean_events_per_request"], "headline_load": key},
            "serving": res["precisions"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--mode", default="fp64", choices=["fp64", "fp32", "mixed"])
    ap.add_argument("--only", action="store_true", help="time only the headline mode")
    ap.add_argument("--ref-sample", type=int, default=4096, help="oracle events per step of --impl reference")
    ap.add_argument("--cpu-sample", type=int, default=49152,
                    help="oracle events of the cpu_baseline leg (about 10 s on 16 host cores)")
    ap.add_argument("--serving", action="store_true", help="run the serving stream instead of the throughput step")
    ap.add_argument("--serving-requests", type=int, default=2000)
    ap.add_argument("--serving-warmup", type=int, default=200)
    ap.add_argument("--serving-requests-other", type=int, default=300,
                    help="requests of the stream replayed for the precisions after the first")
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--serving-chunk", type=int, default=16384, help="events per chunk of a large request")
    ap.add_argument("--serving-loads", default="0.5,0.7,0.9,1.1",
                    help="offered load as fractions of capacity (first precision; the others run at 0.7)")
    ap.add_argument("--serving-precisions", default="mixed,fp64")
    ap.add_argument("--nevt", type=int, default=NEVT,
                    help="events per GPU per step (a smaller case for profiling; the workload is 1048576)")
    ap.add_argument("--processes", action="store_true", help="per-process ME/s table instead of the step")
    ap.add_argument("--only-process", default="", help="with --processes: only this process")
    ap.add_argument("--process-nevt", type=int, default=0, help="with --processes: events instead of the workload's")
    ap.add_argument("--process-modes", default="fp64,fp32,mixed,dfloat", help="with --processes: precisions to time")
    ap.add_argument("--process-err-sample", type=int, default=256,
                    help="oracle events per process and mode for the error of the per-process table")
    ap.add_argument("--err-sample", type=int, default=4096,
                    help="oracle events for the max / median error of each mode of the step")
    ap.add_argument("--no-extra", action="store_true",
                    help="leave the per-process table and the serving stream out of the default run")
    ap.add_argument("--quick-serving-requests", type=int, default=300,
                    help="measured requests of the mixed stream in the default run (FP64: 100)")
    args = ap.parse_args()
    globals()["NEVT"] = args.nevt
    if args.serving:
        return run_serving(args)
    if args.processes:
        return run_processes(args)
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
