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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tpcgen  # noqa: E402

METRIC = "TPC clusters/s & tracks/s per B300; timeframe p50/p99 latency, batched vs plain"
WORKLOADS = {
    "full_tpc": (lambda seed: tpcgen.full_tpc(seed),
                 "full_tpc: 36 sectors x 152 rows (66-138 pads), 1000 time bins, 10,000 tracks "
                 "(5% loopers) from one vertex, Bz 0.5 T, Landau(60) Gaussian clouds, noise 1 ADC, ZS >= 3"),
    "single_sector": (lambda seed: tpcgen.single_sector(seed),
                      "single_sector: 1 sector x 152 rows, 500 time bins, 150 tracks"),
}
REF_SAMPLE_SECTORS = 9
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
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


def max_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def sample_tf(tf, n_sectors):
    """The first n_sectors sectors of a timeframe (their pages are a prefix)."""
    import copy
    s = copy.copy(tf)
    nwin = n_sectors * tf.n_rows * tf.n_fragments
    s.page_offsets = tf.page_offsets[:nwin].copy()
    end = int(tf.page_offsets[nwin]) if nwin < len(tf.page_offsets) else len(tf.pages)
    s.pages = tf.pages[:end]
    s.n_sectors = n_sectors
    return s


def cpu_baseline(tf, steps=1):
    import oracle
    sub = sample_tf(tf, min(REF_SAMPLE_SECTORS, tf.n_sectors))
    times, ncl, ntr = [], 0, 0
    for _ in range(steps):
        t0 = time.perf_counter()
        r = oracle.reconstruct(sub)
        times.append(time.perf_counter() - t0)
        ncl, ntr = len(r.clusters), len(r.track_first)
    return {"times": times, "clusters": ncl, "tracks": ntr,
            "sample": f"sectors 0-{sub.n_sectors - 1} of the same timeframe ({sub.n_sectors}/{tf.n_sectors}), "
                      f"{ncl} clusters, {ntr} tracks per step"}


def run_reference(args, world, rank):
    if rank != 0:
        return
    make, desc = WORKLOADS[args.workload]
    tf = tpcgen.generate(make(args.seed))
    for _ in range(args.warmup):
        cpu_baseline(tf, 1)
    cb = cpu_baseline(tf, args.steps)
    t = sum(cb["times"])
    v = cb["clusters"] * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f64",
            "data": "synthetic", "config": {"workload": desc, "seed": args.seed},
            "tracks_per_s": cb["tracks"] * args.steps / t,
            "cpu_baseline": {"value": v, "unit": "clusters/s", "cores": 1, "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_2208_07412_b300 import tpc
    torch.cuda.set_device(local)
    make, desc = WORKLOADS[args.workload]
    tf = tpcgen.generate(make(args.seed + rank))
    # a dedicated stream: the library runs slot 0 on it and the CUDA events
    # below are recorded on it (the legacy default stream has handle 0, which
    # the library would replace by a stream of its own)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    R = tpc.Reconstructor.for_timeframe(tf, device=local, stream=stream.cuda_stream,
                                        flags=tpc.TPC_CTX_STAGE_TIMING, mem_budget=16 << 30)
    pages_d = torch.from_numpy(tf.pages).to("cuda")
    offs_d = torch.from_numpy(tf.page_offsets.view(np.int64)).to("cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

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
    with ClockSampler(local) as clk:
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
    dev_s = sum(step_ms) / 1e3
    dev_s_max = max_over_ranks(world, dev_s)
    cl_all = sum_over_ranks(world, n_cl * args.steps)
    tr_all = sum_over_ranks(world, n_tr * args.steps)
    stages = {k: statistics.mean(r[3][k] for r in recs) for k in tpc.STAGES}
    launches = sum(r[2]["kernel_launches"] for r in recs)

    # ---- end to end through the C ABI with host (pinned) buffers
    pages_h = torch.from_numpy(tf.pages).pin_memory()
    offs_h = torch.from_numpy(tf.page_offsets.view(np.int64)).pin_memory()
    # results land in pinned host memory, like the inputs
    cl_buf = torch.empty(max(n_cl, 1) * 16, dtype=torch.uint8).pin_memory()
    tr_buf = torch.empty(max(n_tr, 1) * 112, dtype=torch.uint8).pin_memory()
    map_buf = torch.empty(max(n_cl, 1), dtype=torch.int32).pin_memory()
    import ctypes
    L = tpc.load()
    n = ctypes.c_uint64()

    def e2e_step():
        t = R.submit(pages_h, offs_h, tf.n_time_bins)
        R.wait(t)
        L.tpc_get_clusters(R.ctx, t, cl_buf.data_ptr(), max(n_cl, 1), ctypes.byref(n))
        L.tpc_get_tracks(R.ctx, t, tr_buf.data_ptr(), max(n_tr, 1), ctypes.byref(n), map_buf.data_ptr())
        tpc.tpc_release(R.ctx, t)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    e2e_t = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_s_max = max_over_ranks(world, sum(e2e_t))
    h2d = tf.pages.nbytes + tf.page_offsets.nbytes
    d2h = n_cl * 16 + n_tr * 112 + n_cl * 4

    if rank == 0:
        peaks, peak_kind = load_peaks()
        hbm = float(peaks["hbm_gbs"])
        n_windows = len(tf.page_offsets)
        alg_bytes = tf.pages.nbytes + 8 * n_windows + 16 * n_cl
        achieved = alg_bytes / (stages["find"] * 1e-3) / 1e9
        line = {
            "metric": METRIC, "value": cl_all / dev_s_max, "unit": "clusters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i64+f32",
            "data": "synthetic",
            "config": {"workload": desc, "seed": args.seed, "zs_bytes": int(tf.pages.nbytes),
                       "digits": int(tf.n_digits), "clusters_per_tf": n_cl, "tracks_per_tf": n_tr,
                       "l2": "flushed before every step (256 MB write)", "parallelism": f"replicas x{world}",
                       "path": "plain per-timeframe launches"},
            "tracks_per_s": tr_all / dev_s_max,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "stages_ms": stages,
            "wall_ms_per_step": 1e3 * wall / args.steps,
            "roofline": {"kernel": "k_find_clusters", "bound": "hbm", "achieved": achieved, "peak": hbm,
                         "unit": "GB/s", "frac": achieved / hbm, "traffic": None,
                         "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                         "algorithmic_bytes_per_launch": int(alg_bytes)},
            "e2e": {"value": cl_all / e2e_s_max, "unit": "clusters/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "clocks": clk.summary(),
            "gpu_launches": int(launches),
        }
        if world == 1 and not args.no_cpu_baseline:
            cb = cpu_baseline(tf, 1)
            line["cpu_baseline"] = {"value": cb["clusters"] / cb["times"][0], "unit": "clusters/s", "cores": 1,
                                    "kind": "oracle", "sample": cb["sample"]}
        print(json.dumps(line), flush=True)
    R.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="full_tpc")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            run_reference(args, world, rank)
        else:
            run_ours(args, world, rank, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
