"""The N>1 path of bench.py on CPU: world_size-2 `gloo` ranks.  Each rank is a
replica reconstructing its own timeframes (no data-path collective); only the
job totals cross ranks — clusters and tracks summed, time the slowest rank's —
and under torchrun the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup(world)
    assert (w, r) == (world, rank)
    # rank r: 1000 (r + 1) clusters and 10 (r + 1) tracks per step, 3 steps, r + 0.5 s
    cl, tr, sec = bench.job_totals(w, 1000 * (rank + 1), 10 * (rank + 1), 3, rank + 0.5)
    bench.barrier(w)
    out[rank] = (cl, tr, sec)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_job_totals_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()   # never fork: the process may hold a CUDA context
    out = mgr.dict()
    mp.spawn(_worker, args=(2, free_port(), out), nprocs=2, join=True)
    for r in range(2):
        assert out[r] == (3 * (1000 + 2000), 3 * (10 + 20), 1.5)


def test_reference_arm_under_torchrun_prints_one_line_from_rank_0():
    env = dict(os.environ, BENCH_BACKEND="gloo")
    p = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py",
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
                        "--workload", "single_sector"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
