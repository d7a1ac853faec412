"""Oracle runs on whole sectors in a spawn pool (test infrastructure).

Every step of the method stays inside a sector, so sector k of a timeframe
reconstructed whole equals that sector reconstructed alone.  The pool is
spawned, never forked: the test process may already hold a CUDA context."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np


def _reconstruct_sector(job):
    import oracle
    import tpcgen
    k, pages, offs, n_time_bins, npads, row_x = job
    tf = tpcgen.Timeframe(pages=pages, page_offsets=offs, n_time_bins=n_time_bins, n_sectors=1, npads=npads,
                          row_x=row_x, n_digits=0, digit_labels=None, tracks=np.zeros(0, tpcgen.TRACK_DTYPE),
                          hits=np.zeros(0, tpcgen.HIT_DTYPE), config=None)
    return k, oracle.reconstruct(tf)


def oracle_sectors(tf, sectors, procs: int | None = None):
    """Yields (k, OracleResult of sector k alone, as sector 0) for each k."""
    import tpcgen
    procs = min(len(sectors), procs or os.cpu_count() or 1)

    def jobs():
        for k in sectors:
            s = tpcgen.sector_slice(tf, k)
            yield k, s.pages, s.page_offsets, s.n_time_bins, s.npads, s.row_x

    with mp.get_context("spawn").Pool(procs) as pool:
        yield from pool.imap_unordered(_reconstruct_sector, jobs())


def sector_view(gpu: dict, k: int) -> dict:
    """The GPU results of sector k, indices rebased to the sector's first
    cluster and track and the sector field set to 0, as the oracle reports a
    sector reconstructed alone."""
    cl, tr = gpu["clusters"], gpu["tracks"]
    c0, c1 = (int(v) for v in np.searchsorted(cl["sector"], [k, k + 1]))
    t0, t1 = (int(v) for v in np.searchsorted(tr["sector"], [k, k + 1]))

    def rebase(a, off):
        a = a[c0:c1].astype(np.int64)
        return np.where(a >= 0, a - off, -1).astype(np.int32)
    sub = cl[c0:c1].copy()
    sub["sector"] = 0
    tracks = tr[t0:t1].copy()
    tracks["first_cluster"] -= c0
    return {"clusters": sub, "up": rebase(gpu["up"], c0), "down": rebase(gpu["down"], c0),
            "chain_of": rebase(gpu["chain_of"], c0), "cl2trk": rebase(gpu["cl2trk"], t0), "tracks": tracks,
            "counters": gpu["counters"]}
