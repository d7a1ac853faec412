#!/usr/bin/env python
"""Benchmark: TPC timeframe reconstruction throughput on B300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload full_tpc]

A step is one pass of the whole hot path (decode + peak/cluster finder + CA +
merge + Kalman fit) over one synthetic timeframe.  `value` is clusters/s with
the ZS pages already resident in HBM (device-timed with CUDA events on the
library's stream, L2 flushed by a 256 MB write before every step); `e2e` is the
same metric through the C ABI with host buffers (pinned), host->device copy of
the pages and device->host copy of clusters, tracks and the cluster-to-track
map inside the timed region.  Under torchrun each rank reconstructs its own
timeframe (replicas, no collective); the slowest rank's time counts.

--impl reference times the CPU oracle (test infrastructure, never tuned) on a
bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tpcgen  # noqa: E402

METRIC = "TPC clusters/s & tracks/s per B300; timeframe p50/p99 latency, batched vs plain"
WORKLOADS = {
    "full_tpc": (lambda seed, bins=0: tpcgen.full_tpc(seed),
                 "full_tpc: 36 sectors x 152 rows (66-138 pads), 1000 time bins, 10,000 tracks "
                 "(5% loopers) from one vertex, Bz 0.5 T, Landau(60) Gaussian clouds, noise 1 ADC, ZS >= 3"),
    "single_sector": (lambda seed, bins=0: tpcgen.single_sector(seed),
                      "single_sector: 1 sector x 152 rows, 500 time bins, 150 tracks"),
    "continuous_50khz": (lambda seed, bins=0: tpcgen.continuous_tf(seed, n_time_bins=bins or 55000),
                         "continuous_50khz: 36 sectors x 152 rows, 55,000 time bins (11 ms at 5 MHz), "
                         "Poisson(550) Pb-Pb-like collisions at uniform start times, multiplicity "
                         "floor(15000 U^7.82) (mean ~1,700), 5% loopers, same charge/noise/ZS model"),
}
REF_SAMPLE_BYTES = 20 << 20
# The CPU baseline of our arm's line: about 320 MB of ZS pages (two whole
# sectors of the 55,000-bin timeframe, ~10-20 s of single-core oracle work),
# the reference arm's steps keep the smaller sample above.
CPU_SAMPLE_BYTES = 320 << 20
# ncu counters of one find stage (its kernels summed: k_decode_runs,
# k_unit_descs, k_find_units and k_compact_clusters; the unit-count scan, ~1 %
# of the stage, is left out): DRAM bytes read + written and warp instructions
# (smsp__inst_executed.sum), from a metrics-only capture of the current
# kernels, keyed by (workload, finder, finder threads), with the ZS bytes of the
# captured case.  The 55,000-bin continuous timeframe (5.7 GB of pages) is
# beyond a capture's size, so its figures are those of an 11,000-bin
# continuous timeframe of the same occupancy law (seed 1, 1.17 GB of pages)
# scaled by the ZS bytes (the stage's traffic and instructions grow with the
# pages and clusters).  Must be cleared whenever a finder kernel changes.
FINDER_COUNTERS = {
    ("full_tpc", "two_pass", 128): {"zs": 70336448, "dram": 210552320 + 37405440, "instr": 391738998},
    ("continuous_50khz", "two_pass", 128): {"zs": 1173460064, "dram": 3438739456 + 2626760192,
                                            "instr": 5978795343},
}
# Warp-instruction issue peak: 148 SMs x 4 schedulers x 1 instruction per cycle
# at the 2032 MHz maximum SM clock.
ISSUE_PEAK = 148 * 4 * 2.032e9
# FP32 peak from the unit counts: 148 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2032 MHz.
FP32_NOMINAL = 148 * 128 * 2 * 2.032e9
# Algorithmic FLOP of the step-8 fit per cluster on a track: ~400 per pass x 3 passes.
FIT_FLOP_PER_CLUSTER = 1200
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int, out_dir=None):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(), f"tpc_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return self
        # the timed region starts once the sampler is producing samples
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(v: float, op: str) -> float:
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(world, v: float) -> float:
    return v if world == 1 else _reduce(v, "max")


def sum_over_ranks(world, v: float) -> float:
    return v if world == 1 else _reduce(v, "sum")


def job_totals(world, n_cl: int, n_tr: int, steps: int, dev_s: float):
    """Whole-job totals of the replicas: every rank reconstructs its own
    timeframes, so the job's clusters and tracks are the sum over ranks and its
    time the slowest rank's.  Returns (clusters, tracks, seconds)."""
    return (sum_over_ranks(world, n_cl * steps), sum_over_ranks(world, n_tr * steps),
            max_over_ranks(world, dev_s))


def ref_sample_tf(tf, sample_bytes: float = REF_SAMPLE_BYTES):
    """The timeframe the oracle samples from: the whole one, or, where one
    sector holds more than sample_bytes of pages (long continuous timeframes),
    its first fragments, as many as keep one sector near sample_bytes."""
    per_sector = tf.pages.nbytes / max(tf.n_sectors, 1)
    if per_sector <= sample_bytes:
        return tf, ""
    k = max(1, int(tf.n_fragments * sample_bytes / per_sector))
    return tpcgen.time_prefix(tf, k), f"the first {min(tf.n_time_bins, 256 * k)} time bins of "


def ref_sample_sectors(tf, sample_bytes: float = REF_SAMPLE_BYTES) -> int:
    """Sectors in the oracle's sample: about sample_bytes of ZS pages (20 MB: a
    few seconds of single-core CPU work), at least one sector."""
    per_sector = tf.pages.nbytes / max(tf.n_sectors, 1)
    return int(max(1, min(tf.n_sectors, sample_bytes // max(per_sector, 1))))


def cpu_baseline(tf, steps=1, sample_bytes: float = REF_SAMPLE_BYTES):
    import oracle
    tf, what = ref_sample_tf(tf, sample_bytes)
    sub = tpcgen.sector_prefix(tf, ref_sample_sectors(tf, sample_bytes))
    times, ncl, ntr = [], 0, 0
    for _ in range(steps):
        t0 = time.perf_counter()
        r = oracle.reconstruct(sub)
        times.append(time.perf_counter() - t0)
        ncl, ntr = len(r.clusters), len(r.track_first)
    return {"times": times, "clusters": ncl, "tracks": ntr,
            "sample": f"{what}sectors 0-{sub.n_sectors - 1} of the same timeframe ({sub.n_sectors}/{tf.n_sectors}), "
                      f"{ncl} clusters, {ntr} tracks per step"}


def _oracle_sector_job(sub):
    """Worker of the all-cores oracle run: one single-sector timeframe."""
    import oracle
    r = oracle.reconstruct(sub)
    return len(r.clusters), len(r.track_first)


def _oracle_warm(_):
    import oracle
    oracle.build()
    return os.getpid()


class OraclePool:
    """A spawn pool of one oracle process per host core (spawned, never forked:
    the parent may already hold a CUDA context).  Sectors are independent
    through step 8, so the all-cores run gives each process whole sectors."""

    def __init__(self, procs: int | None = None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_warm, range(self.procs))   # imports and loads outside the timed region

    def run(self, tf, sample_bytes: float = REF_SAMPLE_BYTES, steps: int = 1):
        """Time `steps` passes over the first sectors, one task per sector: as
        many sectors as processes, but no more ZS bytes than sample_bytes per
        process (the work stays bounded on long timeframes), at least one."""
        tf, what = ref_sample_tf(tf, sample_bytes)
        per_sector = tf.pages.nbytes / max(tf.n_sectors, 1)
        n = int(min(tf.n_sectors, self.procs, max(1, self.procs * sample_bytes // max(per_sector, 1))))
        subs = [tpcgen.sector_slice(tf, s) for s in range(n)]
        times, ncl, ntr = [], 0, 0
        for _ in range(steps):
            t0 = time.perf_counter()
            res = self.pool.map(_oracle_sector_job, subs, chunksize=1)
            times.append(time.perf_counter() - t0)
            ncl, ntr = sum(r[0] for r in res), sum(r[1] for r in res)
        return {"times": times, "clusters": ncl, "tracks": ntr, "cores": min(self.procs, n),
                "sample": f"{what}sectors 0-{n - 1} of the same timeframe ({n}/{tf.n_sectors}), one oracle process "
                          f"per sector on a spawn pool of {self.procs}, {ncl} clusters, {ntr} tracks per step"}

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "serve":   # one Pb-Pb-like timeframe of the serving pool
        make, desc = (lambda seed: tpcgen.continuous_tf(7, n_time_bins=args.serve_bins),
                      f"serve pool: Pb-Pb-like continuous timeframe of {args.serve_bins} time bins")
    else:
        make, desc = WORKLOADS[args.workload]
    tf = tpcgen.generate(make(args.seed))
    # each step a bounded sample, smaller when many steps are asked for, so the
    # whole run stays around a minute of CPU time
    per_step = REF_SAMPLE_BYTES * min(1.0, 20.0 / max(args.steps + args.warmup, 1))
    # the oracle on all host cores, one process per sector (the single-core
    # figure is kept beside it)
    pool = OraclePool()
    try:
        pool.run(tf, per_step, args.warmup)
        cb = pool.run(tf, per_step, args.steps)
    finally:
        pool.close()
    one = cpu_baseline(tf, 1, per_step)
    t = sum(cb["times"])
    v = cb["clusters"] * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f64",
            "data": "synthetic", "config": {"workload": desc, "seed": args.seed},
            "tracks_per_s": cb["tracks"] * args.steps / t,
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": cb["cores"], "kind": "oracle",
                             "sample": cb["sample"]},
            "single_core": {"value": one["clusters"] / one["times"][0], "unit": "clusters/s", "cores": 1,
                            "sample": one["sample"]},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def pct(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def batched_vs_plain(tpc, torch, local, n_events=64, seed=1000, reps=3, tuning=None):
    """Uneven events on the full geometry (multiplicity log-uniform in
    [200, 20000], 1000 time bins each), device-resident: the whole set as ONE
    batched pipeline run, against one plain run per event (one slot, events in
    sequence) and against the served path (4 slots, every event submitted at
    once, admitted as slots free up).  Host wall time from the first submit to
    the last result resident on the device."""
    mult = tpcgen.batch_multiplicities(seed, n_events=n_events)
    tfs = [tpcgen.generate(tpcgen.full_tpc(seed + i, n_tracks=int(m), want_labels=False))
           for i, m in enumerate(mult)]
    dev = [(torch.from_numpy(tf.pages).cuda(), torch.from_numpy(tf.page_offsets.view(np.int64)).cuda())
           for tf in tfs]
    torch.cuda.synchronize()   # the uploads ran on torch's stream, the library uses its own
    T = tfs[0].n_time_bins
    tot = sum(tf.pages.nbytes for tf in tfs)
    free_b, _ = torch.cuda.mem_get_info()
    budget = int(min(free_b * 0.8, 16 * tot + (8 << 30)))

    def timed(fn):
        fn()                                   # warm-up (captures the graphs)
        torch.cuda.synchronize()
        best = []
        for _ in range(reps):
            t0 = time.perf_counter()
            out = fn()
            best.append(time.perf_counter() - t0)
        return statistics.median(best), out

    # one batched run
    with tpc.Reconstructor.for_timeframe(tfs[0], device=local, mem_budget=budget) as R:
        if tuning:
            tpc.tpc_set_tuning(R.ctx, **tuning)
        def batch():
            t, keep = tpc.tpc_submit_batch(R.ctx, dev, T)
            R.wait(t)
            c = tpc.tpc_get_counters(R.ctx, t)
            tpc.tpc_release(R.ctx, t)
            return c
        batch_s, ctr = timed(batch)
    n_cl, n_tr = ctr["clusters"], ctr["tracks"]

    # plain: one event after the other on one slot
    with tpc.Reconstructor.for_timeframe(tfs[0], device=local, mem_budget=budget) as R:
        if tuning:
            tpc.tpc_set_tuning(R.ctx, **tuning)
        def plain():
            lat, ncl = [], 0
            for p, o in dev:
                a = time.perf_counter()
                t = R.submit(p, o, T)
                R.wait(t)
                ncl += tpc.tpc_get_counters(R.ctx, t)["clusters"]
                tpc.tpc_release(R.ctx, t)
                lat.append(time.perf_counter() - a)
            return lat, ncl
        plain_s, (lat, ncl_plain) = timed(plain)

    # served: all submitted at once to 4 slots; each release admits the next
    with tpc.Reconstructor.for_timeframe(tfs[0], device=local, mem_budget=budget, n_slots=4) as R:
        if tuning:
            tpc.tpc_set_tuning(R.ctx, **tuning)
        def served():
            t0 = time.perf_counter()
            tickets = [R.submit(p, o, T) for p, o in dev]
            done, ncl = [], 0
            pending = list(tickets)
            while pending:
                # admission is in submission order: only the oldest 4 can be running
                progressed = False
                for t in pending[:4]:
                    if tpc.tpc_poll(R.ctx, t, 0) == tpc.TPC_STATE_DONE:
                        ncl += tpc.tpc_get_counters(R.ctx, t)["clusters"]
                        tpc.tpc_release(R.ctx, t)
                        pending.remove(t)
                        done.append(time.perf_counter() - t0)
                        progressed = True
                if not progressed:
                    time.sleep(20e-6)
            return done, ncl
        served_s, (done, ncl_served) = timed(served)
    assert ncl_plain == n_cl == ncl_served, (ncl_plain, n_cl, ncl_served)
    return {
        "workload": f"{n_events} events, full 36-sector geometry, 1000 time bins, multiplicity log-uniform "
                    f"[200, 20000] (seed {seed}: {int(mult.sum())} tracks, {tot / 1e9:.2f} GB ZS, "
                    f"{n_cl} clusters, {n_tr} tracks), device-resident inputs",
        "clusters_per_s": {"batched": n_cl / batch_s, "plain": n_cl / plain_s, "served_4_slots": n_cl / served_s},
        "tracks_per_s": {"batched": n_tr / batch_s, "plain": n_tr / plain_s, "served_4_slots": n_tr / served_s},
        "speedup_vs_plain": {"batched": plain_s / batch_s, "served_4_slots": plain_s / served_s},
        "latency_ms": {"plain_event_p50": 1e3 * pct(lat, 50), "plain_event_p99": 1e3 * pct(lat, 99),
                       "batched_whole_batch": 1e3 * batch_s,
                       "served_completion_p50": 1e3 * pct(done, 50), "served_completion_p99": 1e3 * pct(done, 99)},
        "timing": f"host wall clock, median of {reps} passes after one warm-up pass",
    }


def serve_pass(tpc, R, pool, arrivals, n_slots):
    """Feed requests (pool index per arrival time, seconds from the start) to a
    context: each is submitted when due; finished ones are released, which
    admits queued ones.  Admission is in arrival order, so only the oldest
    n_slots requests in flight can be running: only those are polled.  Returns
    per-request latency (s) and the makespan."""
    t0 = time.perf_counter()
    nxt, inflight, lat, ncl = 0, {}, [], 0
    while nxt < len(arrivals) or inflight:
        now = time.perf_counter() - t0
        while nxt < len(arrivals) and arrivals[nxt][0] <= now:
            tf, pages, offs = pool[arrivals[nxt][1]]
            inflight[R.submit(pages, offs, tf.n_time_bins)] = arrivals[nxt][0]
            nxt += 1
        progressed = False
        for t in list(inflight)[:n_slots]:
            if tpc.tpc_poll(R.ctx, t, 0) == tpc.TPC_STATE_DONE:
                ncl += tpc.tpc_get_counters(R.ctx, t)["clusters"]
                tpc.tpc_release(R.ctx, t)
                lat.append(time.perf_counter() - t0 - inflight.pop(t))
                progressed = True
        if not progressed:
            time.sleep(20e-6)
    return lat, time.perf_counter() - t0, ncl


def serve_measure(args, local):
    """Served vs plain sequential path under Poisson arrivals of timeframes
    mixing pp-like and Pb-Pb-like occupancy, inputs in pinned host memory
    (each request is copied in when it is admitted).  Returns the measurement
    as a dict (the serve workload's line, without the common keys)."""
    import torch
    from paper_2208_07412_b300 import tpc
    torch.cuda.set_device(local)
    # timeframe lengths uniform in [serve_bins / 5.5, serve_bins] (2-11 ms scaled by serve_bins / 55,000)
    rng_len = np.random.default_rng(77)
    bins = [int(b) for b in rng_len.integers(args.serve_bins * 2 // 11, args.serve_bins + 1, size=16)]
    cfgs = [tpcgen.pp_tf(7 + i, n_time_bins=bins[i]) for i in range(8)] + \
           [tpcgen.continuous_tf(7 + i, n_time_bins=bins[8 + i]) for i in range(8)]
    pool = []
    for c in cfgs:
        tf = tpcgen.generate(c)
        pool.append((tf, torch.from_numpy(tf.pages).pin_memory(),
                     torch.from_numpy(tf.page_offsets.view(np.int64)).pin_memory()))
    n_req = 3 * len(pool)
    rng = np.random.default_rng(7)
    order = rng.integers(0, len(pool), size=n_req)
    free_b, _ = torch.cuda.mem_get_info()
    biggest = max(tf.pages.nbytes for tf, _, _ in pool)
    budget = int(min(free_b * 0.8, 4 * 16 * biggest + (8 << 30)))
    points = []
    with tpc.Reconstructor.for_timeframe(pool[0][0], device=local, mem_budget=budget, n_slots=1) as Rp, \
            tpc.Reconstructor.for_timeframe(pool[0][0], device=local, mem_budget=budget, n_slots=4) as Rs:
        burst = [(0.0, int(i)) for i in order]
        serve_pass(tpc, Rp, pool, burst[:len(pool)], 1)     # warm-up: grow slots, capture graphs
        serve_pass(tpc, Rs, pool, burst[:len(pool)], 4)
        lat, span, ncl = serve_pass(tpc, Rp, pool, burst, 1)
        rate_plain = n_req / span                            # saturation throughput, plain
        for f in args.serve_load:
            lam = f * rate_plain
            gaps = rng.exponential(1.0 / lam, size=n_req)
            arr = [(float(a), int(i)) for a, i in zip(np.cumsum(gaps) - gaps[0], order)]
            row = {"offered_tf_per_s": lam, "load_vs_plain_saturation": f}
            for name, R, ns in (("plain", Rp, 1), ("served", Rs, 4)):
                lat, span, ncl = serve_pass(tpc, R, pool, arr, ns)
                row[name] = {"tf_per_s": n_req / span, "clusters_per_s": ncl / span,
                             "latency_ms_p50": 1e3 * pct(lat, 50), "latency_ms_p99": 1e3 * pct(lat, 99)}
            points.append(row)
        lat_p, span_p, ncl_p = serve_pass(tpc, Rp, pool, burst, 1)
        lat_s, span_s, ncl_s = serve_pass(tpc, Rs, pool, burst, 4)
    sizes = sorted(tf.pages.nbytes for tf, _, _ in pool)
    return {
        "n_req": n_req, "n_pool": len(pool), "span_s": span_s, "ncl_s": ncl_s,
        "config": {"workload": f"serve: pool of 8 pp-like (1 MHz, Poisson(30) tracks) + 8 Pb-Pb-like (50 kHz, "
                               f"floor(15000 U^7.82)) continuous timeframes of {min(bins)}-{max(bins)} time bins, "
                               f"{sizes[0] / 1e9:.2f}-{sizes[-1] / 1e9:.2f} GB ZS each, {n_req} requests drawn "
                               f"from the pool, pinned host inputs",
                   "served": "4 slots, queued requests admitted as slots and memory free up",
                   "plain": "1 slot, one timeframe at a time in arrival order"},
        "saturation": {"served_tf_per_s": n_req / span_s, "plain_tf_per_s": n_req / span_p,
                       "served_clusters_per_s": ncl_s / span_s, "plain_clusters_per_s": ncl_p / span_p,
                       "speedup": span_p / span_s,
                       "served_latency_ms_p50": 1e3 * pct(lat_s, 50), "served_latency_ms_p99": 1e3 * pct(lat_s, 99),
                       "plain_latency_ms_p50": 1e3 * pct(lat_p, 50), "plain_latency_ms_p99": 1e3 * pct(lat_p, 99)},
        "poisson_sweep": points,
        "h2d_bytes_per_request": int(np.mean([pool[i][0].pages.nbytes + pool[i][0].page_offsets.nbytes
                                              for i in order])),
    }


def run_serve(args, world, rank, local):
    """The serve workload's own line (C5)."""
    m = serve_measure(args, local)
    line = {
        "metric": METRIC, "value": m["ncl_s"] / m["span_s"], "unit": "clusters/s", "n_gpus": 1,
        "steps": m["n_req"], "warmup": m["n_pool"], "ms_per_step": 1e3 * m["span_s"] / m["n_req"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f32", "data": "synthetic",
        "config": m["config"], "saturation": m["saturation"], "poisson_sweep": m["poisson_sweep"],
        "e2e": {"value": m["ncl_s"] / m["span_s"], "unit": "clusters/s",
                "h2d_bytes_per_step": m["h2d_bytes_per_request"], "d2h_bytes_per_step": 256},
    }
    print(json.dumps(line), flush=True)


def cross_sector_timing(tpc, torch, R, pages_d, offs_d, tf, reps=5):
    """The optional step 9 (tpc_merge_sectors) on a finished timeframe: host
    wall time of the call (it runs on the slot's stream and waits for it)."""
    t = R.submit(pages_d, offs_d, tf.n_time_bins)
    R.wait(t)
    n_in = tpc.tpc_get_counters(R.ctx, t)["tracks"]
    tpc.tpc_merge_sectors(R.ctx, t)   # warm-up (allocates its work space)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        n_out = tpc.tpc_merge_sectors(R.ctx, t)
        times.append(time.perf_counter() - t0)
    tpc.tpc_release(R.ctx, t)
    return {"ms": 1e3 * statistics.median(times), "tracks_in": n_in, "tracks_out": n_out,
            "links": n_in - n_out, "timing": f"host wall clock of the call, median of {reps}"}


def compression_stats(tpc, R, pages_d, offs_d, tf, reps=5):
    """The optional step 10 (tpc_compress_clusters): time of the call and the
    size of the position information of the clusters on tracks, as the Shannon
    entropy of the residual codes against the 32 bits of the raw (pad_fp,
    time_fp) pair, and as the stream that step 10c (tpc_entropy_encode) codes."""
    t = R.submit(pages_d, offs_d, tf.n_time_bins)
    R.wait(t)
    n_cl = tpc.tpc_get_counters(R.ctx, t)["clusters"]
    tpc.tpc_compress_clusters(R.ctx, t)   # warm-up (allocates its work space)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        coded, escaped = tpc.tpc_compress_clusters(R.ctx, t)
        times.append(time.perf_counter() - t0)
    cy, cz, st = tpc.tpc_get_compressed(R.ctx, t, n_cl)
    # step 10c: the codes entropy-coded into a stream (canonical Huffman)
    tpc.tpc_entropy_encode(R.ctx, t)      # warm-up
    etimes = []
    for _ in range(reps):
        t0 = time.perf_counter()
        _, n_bits, _ = tpc.tpc_entropy_encode(R.ctx, t, fetch=False)
        etimes.append(time.perf_counter() - t0)
    tpc.tpc_release(R.ctx, t)

    def entropy(v):
        _, c = np.unique(v, return_counts=True)
        p = c / c.sum()
        return float(-(p * np.log2(p)).sum())
    ok = st == 1
    bits = entropy(cy[ok]) + entropy(cz[ok]) if ok.any() else 0.0
    return {"ms": 1e3 * statistics.median(times), "clusters": int(n_cl), "coded": coded, "escaped": escaped,
            "position_bits_per_coded_cluster": bits, "raw_position_bits": 32,
            "position_compression": 32.0 / bits if bits else None,
            "stream_bits_per_coded_cluster": n_bits / coded if coded else None,
            "stream_bytes": (n_bits + 7) // 8,
            "entropy_coding_ms": 1e3 * statistics.median(etimes),
            "timing": f"host wall clock of the call, median of {reps} (entropy_coding_ms: the stream left in device "
                      "memory)"}


def calibration_stats(tpc, R, pages_d, offs_d, tf, reps=5):
    """The optional step 11 (tpc_calibrate_drift): time of the call and the
    vertex time it finds (the workload's collision is at t0 = 250 bins with
    the nominal drift velocity, so eps_vd should be ~0)."""
    t = R.submit(pages_d, offs_d, tf.n_time_bins)
    R.wait(t)
    tpc.tpc_calibrate_drift(R.ctx, t, 250.0)   # warm-up (allocates its work space)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        tv, eps, t0v, n = tpc.tpc_calibrate_drift(R.ctx, t, 250.0)
        times.append(time.perf_counter() - t0)
    tpc.tpc_release(R.ctx, t)
    return {"ms": 1e3 * statistics.median(times), "t_vertex_bins": tv, "eps_vd": eps, "tracks_used": n,
            "timing": f"host wall clock of the call, median of {reps}"}


def finder_variants(tpc, torch, tf, pages_d, offs_d, flush, main_ms, reps=5):
    """The measured variants of steps 1-4 beside the default two-pass finder
    (pages decoded into 8-byte pad-run records in device memory, then each
    64-bin time chunk of a window expanded into a small shared plane and
    clustered there): the fused
    finder (each window's pages decoded straight into a shared plane of the
    whole window) and the dense-plane finder (a decode pass writes a dense
    (sector row, time bin, pad) ADC plane to device memory, a find pass reads it
    back).  Find-stage time from the library's stage events, L2 flushed before
    each step, each variant with its own autotuned launch shape."""
    stride = (int(tf.npads.max()) + 7) & ~7
    plane = tf.n_sectors * len(tf.npads) * tf.n_time_bins * stride * 2
    n_frag = (tf.n_time_bins + 255) // 256
    alloc = tf.n_sectors * len(tf.npads) * n_frag * 256 * stride * 2
    out = {"two_pass_find_ms": main_ms}
    for name, flag in (("fused", tpc.TPC_CTX_FUSED_FINDER), ("dense", tpc.TPC_CTX_DENSE_FINDER)):
        free_now, _ = torch.cuda.mem_get_info()
        times = []
        try:
            Rv = tpc.Reconstructor.for_timeframe(tf, device=torch.cuda.current_device(),
                                                 flags=tpc.TPC_CTX_STAGE_TIMING | flag, mem_budget=int(0.9 * free_now))
        except tpc.TpcError as e:
            out[f"{name}_skipped"] = str(e)
            continue
        try:
            tpc.tpc_autotune(Rv.ctx, pages_d, offs_d, tf.n_time_bins, reps=2)
            for i in range(reps + 2):
                flush.fill_(1)
                t = Rv.submit(pages_d, offs_d, tf.n_time_bins)
                Rv.wait(t)
                if i >= 2:
                    times.append(tpc.tpc_get_stage_times(Rv.ctx, t)["find"])
                tpc.tpc_release(Rv.ctx, t)
        except tpc.TpcError as e:   # the dense plane and a slot do not fit the free memory
            out[f"{name}_skipped"] = f"{alloc / 1e9:.1f} GB dense plane or slot does not fit: {e}"
            continue
        finally:
            Rv.close()
        out[f"{name}_find_ms"] = statistics.mean(times)
        out[f"{name}_over_two_pass"] = statistics.mean(times) / main_ms
    if "dense_find_ms" in out:
        # algorithmic bytes of the dense pair: the pages once, the plane written
        # once and read once (+6 halo rows per 256-bin window)
        dense_bytes = tf.pages.nbytes + plane + plane * (262 / 256)
        out["dense_plane_bytes"] = int(plane)
        out["dense_algorithmic_gbs"] = dense_bytes / (out["dense_find_ms"] * 1e-3) / 1e9
    out["timing"] = f"find stage (decode + find + scan + compaction), mean of {reps}, L2 flushed"
    return out


def noise_suppression_stats(tpc, torch, tf, pages_d, offs_d, tuning, flush, n_cl, fused_ms, dip=10, reps=5):
    """The optional step 2b (5x5 noise suppression, tpc_params.ns_min_dip):
    clusters and tracks it leaves, and the find-stage time with it on."""
    prm = tpc.tpc_params_default()
    prm.ns_min_dip = dip
    free_now, _ = torch.cuda.mem_get_info()
    Rn = tpc.Reconstructor.for_timeframe(tf, params=prm, device=torch.cuda.current_device(),
                                         flags=tpc.TPC_CTX_STAGE_TIMING, mem_budget=int(0.5 * free_now))
    tpc.tpc_set_tuning(Rn.ctx, **tuning)
    times = []
    for i in range(reps + 2):
        flush.fill_(1)
        t = Rn.submit(pages_d, offs_d, tf.n_time_bins)
        Rn.wait(t)
        ctr = tpc.tpc_get_counters(Rn.ctx, t)
        if i >= 2:
            times.append(tpc.tpc_get_stage_times(Rn.ctx, t)["find"])
        tpc.tpc_release(Rn.ctx, t)
    Rn.close()
    return {"ns_min_dip": dip, "clusters": ctr["clusters"], "tracks": ctr["tracks"],
            "clusters_removed_frac": 1.0 - ctr["clusters"] / n_cl, "find_ms": statistics.mean(times),
            "find_ms_without": fused_ms, "timing": f"find stage, mean of {reps}, L2 flushed"}


FINDER_KERNELS = {"two_pass": "find stage: k_decode_runs + k_unit_descs + k_find_units + k_scan + k_compact_clusters",
                  "fused": "find stage: k_find_classify + k_find_light + k_find_clusters + k_scan + k_compact_clusters",
                  "dense": "find stage: k_find_clusters (dense-plane decode and find passes) + k_scan + "
                           "k_compact_clusters"}


def finder_roofline(tf, n_cl, find_ms, find_threads, workload, seed, time_bins, finder, hbm, peak_kind):
    """HBM roofline of the find stage (algorithmic bytes: ZS pages + 8 B page
    offset per window + 16 B per cluster record, over the stage's CUDA-event
    time) and its issue roofline, with the ncu traffic of a capture of the
    current kernels where one exists (scaled by ZS bytes from the captured
    case), else null."""
    n_windows = len(tf.page_offsets)
    alg_bytes = tf.pages.nbytes + 8 * n_windows + 16 * n_cl
    if finder == "dense":   # + the dense plane written once and read once (with 6 halo rows per window)
        plane = tf.n_sectors * len(tf.npads) * tf.n_time_bins * ((int(tf.npads.max()) + 7) & ~7) * 2
        alg_bytes += plane + plane * 262 // 256
    achieved = alg_bytes / (find_ms * 1e-3) / 1e9
    cap = None
    if seed == 1 and (workload == "full_tpc" or (workload == "continuous_50khz" and not time_bins)):
        cap = FINDER_COUNTERS.get((workload, finder, int(find_threads)))
    scale = tf.pages.nbytes / cap["zs"] if cap else None
    kernel = FINDER_KERNELS[finder]
    roof = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": int(cap["dram"] * scale) if cap else None,
            "peak_kind": f"{peak_kind} hbm_gbs (copy)", "algorithmic_bytes_per_launch": int(alg_bytes)}
    issue = None
    if cap:
        ins = cap["instr"] * scale
        issue = {"kernel": kernel, "bound": "issue", "achieved": ins / (find_ms * 1e-3), "peak": ISSUE_PEAK,
                 "unit": "warp-instr/s", "frac": ins / (find_ms * 1e-3) / ISSUE_PEAK,
                 "instructions": "ncu smsp__inst_executed.sum of one launch" +
                                 (", scaled by ZS bytes from the captured case" if scale != 1.0 else ""),
                 "peak_kind": "148 SMs x 4 schedulers x 2032 MHz"}
    return roof, issue


def fit_roofline(n_cl_on_tracks, fit_ms, fma_peak):
    """ALU roofline of the step-8 fit: algorithmic FLOP (1,200 per cluster on a
    track) over the fit stage's CUDA-event time, against the measured FP32 FMA
    peak (and the nominal one from the unit counts)."""
    flops = FIT_FLOP_PER_CLUSTER * n_cl_on_tracks
    achieved = flops / (fit_ms * 1e-3) / 1e12
    peak = (fma_peak or FP32_NOMINAL) / 1e12
    return {"kernel": "k_fit", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "algorithmic_flop_per_launch": int(flops),
            "flop_per_cluster": FIT_FLOP_PER_CLUSTER, "nominal_peak": FP32_NOMINAL / 1e12,
            "peak_kind": "measured FP32 FMA probe (tpc_measure_fma_peak)" if fma_peak else
                         "nominal 148 SMs x 128 lanes x 2 x 2032 MHz"}


# ncu --set full counters of k_ca_neighbours (the CA stage's main kernel) on
# full_tpc, seed 1 (profiles/k_ca_neighbours_full_tpc.md): L2 throughput
# (lts__throughput, % of peak), L2 sector rate, warp efficiency (threads per
# warp instruction / 32), issue active.  Must be cleared whenever the kernel
# changes.
CA_COUNTERS = {"workload": "full_tpc seed 1", "l2_throughput_pct_of_peak": 8.57, "l2_sectors_per_ns": 59.1,
               "lts_hit_rate_pct": 53.5, "warp_efficiency": 19.13 / 32, "issue_active_pct": 53.2,
               "warps_active_pct": 44.9}


def ca_roofline(n_cl, ca_ms, hbm):
    """The CA stage (steps 5-6): irregular, latency-bound.  Algorithmic bytes
    ~32 per cluster (coordinates in, up / down / score and chain data out) over
    the stage's CUDA-event time, against the measured HBM rate for scale; with
    the L2 throughput and warp efficiency of an ncu capture of k_ca_neighbours."""
    alg = 32 * n_cl
    achieved = alg / (ca_ms * 1e-3) / 1e9
    return {"kernel": "CA stage: k_ca_neighbours + edge rows + links + chains", "bound": "latency",
            "achieved": achieved, "unit": "GB/s", "peak": hbm, "frac": achieved / hbm,
            "algorithmic_bytes_per_launch": int(alg), "ncu_k_ca_neighbours": CA_COUNTERS}


def extra_workload(tpc, torch, local, name, seed, steps, warmup, flush, hbm, peak_kind, fma_peak):
    """A second workload measured like the main one (device-resident pages, L2
    flushed before every step, CUDA events on the library's stream, the
    autotuner's configuration): clusters/s, tracks/s, latency, stages and
    rooflines."""
    make, desc = WORKLOADS[name]
    tf = tpcgen.generate(make(seed))
    stream = torch.cuda.Stream()
    free_b, _ = torch.cuda.mem_get_info()
    R = tpc.Reconstructor.for_timeframe(tf, device=local, stream=stream.cuda_stream, flags=tpc.TPC_CTX_STAGE_TIMING,
                                        mem_budget=int(min(free_b * 0.5, max(16 << 30, 40 * tf.pages.nbytes))))
    try:
        pages_d = torch.from_numpy(tf.pages).to("cuda")
        offs_d = torch.from_numpy(tf.page_offsets.view(np.int64)).to("cuda")
        torch.cuda.synchronize()
        tuning = tpc.tpc_autotune(R.ctx, pages_d, offs_d, tf.n_time_bins, reps=3)
        recs = []
        for i in range(warmup + steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            t = R.submit(pages_d, offs_d, tf.n_time_bins)
            e1.record(stream)
            R.wait(t)
            if i >= warmup:
                recs.append((e0, e1, tpc.tpc_get_counters(R.ctx, t), tpc.tpc_get_stage_times(R.ctx, t)))
            tpc.tpc_release(R.ctx, t)
    finally:
        R.close()
    step_ms = [a.elapsed_time(b) for a, b, _, _ in recs]
    ctr = recs[-1][2]
    stages = {k: statistics.mean(r[3][k] for r in recs) for k in tpc.STAGES}
    t_s = sum(step_ms) / 1e3
    roof, issue = finder_roofline(tf, ctr["clusters"], stages["find"], tuning["find_threads"], name, seed, 0,
                                  "two_pass", hbm, peak_kind)
    return {"workload": desc, "seed": seed, "zs_bytes": int(tf.pages.nbytes), "clusters_per_tf": ctr["clusters"],
            "tracks_per_tf": ctr["tracks"], "clusters_per_s": ctr["clusters"] * steps / t_s,
            "tracks_per_s": ctr["tracks"] * steps / t_s, "ms_per_step": 1e3 * t_s / steps,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "stages_ms": stages, "roofline": roof, "roofline_issue": issue,
            "roofline_fit": fit_roofline(ctr["clusters_on_tracks"], stages["fit"], fma_peak),
            "roofline_ca": ca_roofline(ctr["clusters"], stages["ca"], hbm),
            "tuning": tuning, "steps": steps, "warmup": warmup,
            "timing": "CUDA events on the library's stream, L2 flushed before every step"}


def run_ours(args, world, rank, local):
    import torch
    from paper_2208_07412_b300 import tpc
    torch.cuda.set_device(local)
    make, desc = WORKLOADS[args.workload]
    if args.workload == "continuous_50khz" and args.time_bins:
        desc = desc.replace("55,000 time bins (11 ms at 5 MHz)", f"{args.time_bins} time bins") + \
            ", Poisson(0.01 x bins) collisions"
        tf = tpcgen.generate(make(args.seed + rank, args.time_bins))
    else:
        tf = tpcgen.generate(make(args.seed + rank))
    # a dedicated stream: the library runs slot 0 on it and the CUDA events
    # below are recorded on it (the legacy default stream has handle 0, which
    # the library would replace by a stream of its own)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flags = tpc.TPC_CTX_STAGE_TIMING | (tpc.TPC_CTX_NO_GRAPHS if args.no_graphs else 0) | \
        (tpc.TPC_CTX_DENSE_FINDER if args.dense_finder else 0) | (tpc.TPC_CTX_FUSED_FINDER if args.fused_finder else 0)
    # device memory for one slot: the pages, ~150 B per cluster of capacity
    # (pages/20 clusters) and the rest; the budget is what the GPU has free
    free_b, _ = torch.cuda.mem_get_info()
    budget = int(min(free_b * 0.85, max(16 << 30, 40 * tf.pages.nbytes)))
    R = tpc.Reconstructor.for_timeframe(tf, device=local, stream=stream.cuda_stream,
                                        flags=flags, mem_budget=budget)
    pages_d = torch.from_numpy(tf.pages).to("cuda")
    offs_d = torch.from_numpy(tf.page_offsets.view(np.int64)).to("cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    # launch configuration: the autotuner's pick on this workload (untimed setup)
    if args.tuning:   # a fixed configuration, e.g. one the autotuner picked earlier
        tpc.tpc_set_tuning(R.ctx, **{k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))})
        tuning = tpc.tpc_get_tuning(R.ctx)
    elif args.no_autotune:
        tuning = tpc.tpc_get_tuning(R.ctx)
    else:
        tuning = tpc.tpc_autotune(R.ctx, pages_d, offs_d, tf.n_time_bins, reps=3)

    def dev_step():
        flush.fill_(1)  # evict the pages from L2 before the timed region of the step
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = R.submit(pages_d, offs_d, tf.n_time_bins)
        e1.record(stream)
        R.wait(t)
        ctr = tpc.tpc_get_counters(R.ctx, t)
        st = tpc.tpc_get_stage_times(R.ctx, t)
        tpc.tpc_release(R.ctx, t)
        return e0, e1, ctr, st

    for _ in range(args.warmup):
        dev_step()
    torch.cuda.synchronize()
    barrier(world)
    recs = []
    with ClockSampler(local, args.clocks_dir) as clk:
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            recs.append(dev_step())
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b, _, _ in recs]
    ctr = recs[-1][2]
    n_cl, n_tr = ctr["clusters"], ctr["tracks"]
    cl_all, tr_all, dev_s_max = job_totals(world, n_cl, n_tr, args.steps, sum(step_ms) / 1e3)
    stages = {k: statistics.mean(r[3][k] for r in recs) for k in tpc.STAGES}
    launches = sum(r[2]["kernel_launches"] for r in recs)
    # the optional steps on the device context's last timeframe, before its
    # memory goes to the end-to-end contexts below
    extras = {}
    if rank == 0 and world == 1 and args.workload in ("full_tpc", "continuous_50khz"):
        extras["cross_sector"] = cross_sector_timing(tpc, torch, R, pages_d, offs_d, tf)
        extras["compression"] = compression_stats(tpc, R, pages_d, offs_d, tf)
    if rank == 0 and world == 1 and args.workload == "full_tpc":   # one collision: its vertex time
        extras["calibration"] = calibration_stats(tpc, R, pages_d, offs_d, tf)
    R.close()

    # ---- end to end through the C ABI with host (pinned) buffers, on a
    # context of three slots with the memory left (at 55,000 bins a slot holds
    # ~95 GB: two fit, and the third submit queues)
    pages_h = torch.from_numpy(tf.pages).pin_memory()
    offs_h = torch.from_numpy(tf.page_offsets.view(np.int64)).pin_memory()
    # results land in pinned host memory, like the inputs
    cl_buf = torch.empty(max(n_cl, 1) * 16, dtype=torch.uint8).pin_memory()
    tr_buf = torch.empty(max(n_tr, 1) * 112, dtype=torch.uint8).pin_memory()
    map_buf = torch.empty(max(n_cl, 1), dtype=torch.int32).pin_memory()
    import ctypes
    L = tpc.load()
    n = ctypes.c_uint64()

    free_now, _ = torch.cuda.mem_get_info()
    depth = 3
    Rp = tpc.Reconstructor.for_timeframe(tf, device=local, flags=flags & ~tpc.TPC_CTX_STAGE_TIMING,
                                         mem_budget=int(free_now * 0.85), n_slots=depth)
    tpc.tpc_set_tuning(Rp.ctx, **tuning)

    def e2e_step():
        t = Rp.submit(pages_h, offs_h, tf.n_time_bins)
        Rp.wait(t)
        L.tpc_get_clusters(Rp.ctx, t, cl_buf.data_ptr(), max(n_cl, 1), ctypes.byref(n))
        L.tpc_get_tracks(Rp.ctx, t, tr_buf.data_ptr(), max(n_tr, 1), ctypes.byref(n), map_buf.data_ptr())
        tpc.tpc_release(Rp.ctx, t)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    e2e_t = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_seq_s_max = max_over_ranks(world, sum(e2e_t))

    # ---- end to end, pipelined: the next timeframes submitted before this one
    # is read back, so that their host->device copies and kernels overlap its
    # device->host read-back (slots that do not fit the budget queue)

    def fetch(t):
        Rp.wait(t)
        L.tpc_get_clusters(Rp.ctx, t, cl_buf.data_ptr(), max(n_cl, 1), ctypes.byref(n))
        L.tpc_get_tracks(Rp.ctx, t, tr_buf.data_ptr(), max(n_tr, 1), ctypes.byref(n), map_buf.data_ptr())
        tpc.tpc_release(Rp.ctx, t)

    def pipelined(k_steps):
        inflight = []
        for _ in range(k_steps):
            inflight.append(Rp.submit(pages_h, offs_h, tf.n_time_bins))
            if len(inflight) == depth:
                fetch(inflight.pop(0))
        for t in inflight:
            fetch(t)

    pipelined(max(3, args.warmup))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    pipelined(args.steps)
    e2e_s_max = max_over_ranks(world, time.perf_counter() - t0)
    Rp.close()
    h2d = tf.pages.nbytes + tf.page_offsets.nbytes
    d2h = n_cl * 16 + n_tr * 112 + n_cl * 4

    if rank == 0:
        peaks, peak_kind = load_peaks()
        hbm = float(peaks["hbm_gbs"])
        finder = "dense" if args.dense_finder else ("fused" if args.fused_finder else "two_pass")
        roof, issue = finder_roofline(tf, n_cl, stages["find"], tuning["find_threads"], args.workload, args.seed,
                                      args.time_bins, finder, hbm, peak_kind)
        fma_peak = None
        try:
            fma_peak = tpc.tpc_measure_fma_peak(local, 5)
        except tpc.TpcError:
            pass
        line = {
            "metric": METRIC, "value": cl_all / dev_s_max, "unit": "clusters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f32",
            "data": "synthetic",
            "config": {"workload": desc, "seed": args.seed, "zs_bytes": int(tf.pages.nbytes),
                       "digits": int(tf.n_digits), "clusters_per_tf": n_cl, "tracks_per_tf": n_tr,
                       "l2": "flushed before every step (256 MB write)", "parallelism": f"replicas x{world}",
                       "tuning": {"autotuned": not (args.no_autotune or args.tuning), **tuning},
                       "path": ("plain per-timeframe kernel launches" if args.no_graphs
                                else "per-timeframe pipeline replayed from a captured CUDA graph"),
                       "finder": ("dense-plane variant" if args.dense_finder else
                                  "fused variant" if args.fused_finder else "two-pass")},
            "tracks_per_s": tr_all / dev_s_max,
            "fp64_redos_per_tf": int(ctr["fp64_redos"]),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "stages_ms": stages,
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "roofline": roof,
            "roofline_issue": issue,
            "roofline_fit": fit_roofline(ctr["clusters_on_tracks"], stages["fit"], fma_peak),
            "roofline_ca": ca_roofline(n_cl, stages["ca"], hbm),
            "e2e": {"value": cl_all / e2e_s_max, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "path": "submit from pinned host pages, read clusters, tracks and map back into pinned "
                            "memory; a context of three slots within the memory left (slots that do not fit queue), "
                            "the next two timeframes submitted before this one is read back",
                    "sequential_value": cl_all / e2e_seq_s_max},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        line.update(extras)
        if world == 1 and not (args.no_variants or args.dense_finder or args.fused_finder) and \
                args.workload in ("full_tpc", "continuous_50khz"):
            line["finder_variants"] = finder_variants(tpc, torch, tf, pages_d, offs_d, flush, stages["find"])
        if world == 1 and not args.no_variants and args.workload == "full_tpc":
            line["noise_suppression"] = noise_suppression_stats(tpc, torch, tf, pages_d, offs_d, tuning, flush,
                                                                n_cl, stages["find"])
        if world == 1 and not args.no_extras and args.workload == "continuous_50khz" and not args.time_bins:
            # the full-TPC collision (one timeframe of 1000 bins) measured the same way
            line["full_tpc"] = extra_workload(tpc, torch, local, "full_tpc", 1, 20, 3, flush, hbm, peak_kind,
                                              fma_peak)
        if world == 1 and not args.no_batched and args.workload in ("full_tpc", "continuous_50khz"):
            line["batched"] = batched_vs_plain(tpc, torch, local,
                                               tuning=tuning if args.workload == "full_tpc"
                                               else line.get("full_tpc", {}).get("tuning"))
        if world == 1 and not args.no_serve and args.workload == "continuous_50khz" and not args.time_bins:
            # C5: served vs plain sequential under Poisson arrivals (the serve workload's figures)
            m = serve_measure(args, local)
            line["served"] = {k: m[k] for k in ("config", "saturation", "poisson_sweep")}
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(tf, 1, CPU_SAMPLE_BYTES)
            line["cpu_baseline"] = {"value": cb["clusters"] / cb["times"][0], "unit": "clusters/s", "cores": 1,
                                    "kind": "oracle", "sample": cb["sample"]}
            pool = OraclePool()
            try:
                pb = pool.run(tf, CPU_SAMPLE_BYTES, 1)
            finally:
                pool.close()
            line["cpu_baseline_all_cores"] = {"value": pb["clusters"] / pb["times"][0], "unit": "clusters/s",
                                              "cores": pb["cores"], "kind": "oracle", "sample": pb["sample"]}
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serve"], default="continuous_50khz")
    ap.add_argument("--serve-bins", type=int, default=5500,
                    help="longest served timeframe in time bins (1.1 ms; lengths uniform down to 2/11 of it)")
    ap.add_argument("--time-bins", type=int, default=0, help="continuous_50khz: time bins (default 55,000)")
    ap.add_argument("--serve-load", type=float, nargs="*", default=[0.5, 0.8, 1.0, 1.3],
                    help="offered load as fractions of the plain path's saturation rate")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written (default: the temp dir)")
    ap.add_argument("--no-graphs", action="store_true", help="enqueue every kernel instead of graph replay")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-plain comparison")
    ap.add_argument("--no-serve", action="store_true",
                    help="continuous_50khz: skip the served-vs-plain measurement under Poisson arrivals")
    ap.add_argument("--no-extras", action="store_true",
                    help="continuous_50khz: skip the extra full_tpc measurement")
    ap.add_argument("--no-variants", action="store_true", help="skip the fused-vs-dense finder comparison")
    ap.add_argument("--dense-finder", action="store_true",
                    help="time the dense-plane finder variant instead of the fused finder")
    ap.add_argument("--fused-finder", action="store_true",
                    help="time the fused finder variant instead of the two-pass finder")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch configuration")
    ap.add_argument("--tuning", default="", help="fixed launch configuration, e.g. find_threads=384,fit_threads=32")
    args = ap.parse_args()
    world, rank, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        elif args.workload == "serve":
            if rank == 0:
                run_serve(args, world, rank, local)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
