"""Sector independence of the oracle, which the GPU parity tests of large
timeframes rely on: the oracle run on one sector alone (in a spawn pool) gives
that sector's part of the oracle run on the whole timeframe, indices rebased."""
import numpy as np

import oracle
import tpcgen
from oracle_pool import oracle_sectors, sector_view
from parity import compare_integer


def test_sector_alone_equals_sector_of_the_whole():
    tf = tpcgen.generate(tpcgen.full_tpc(3, n_tracks=2000))
    whole = oracle.reconstruct(tf)
    as_gpu = {"clusters": whole.clusters, "up": whole.up, "down": whole.down, "chain_of": whole.chain_of,
              "cl2trk": whole.cl2trk, "counters": {},
              "tracks": np.zeros(len(whole.track_first), dtype=[("first_cluster", "<i4"), ("n_clusters", "<i4"),
                                                                 ("sector", "<i2")])}
    as_gpu["tracks"]["first_cluster"] = whole.track_first
    as_gpu["tracks"]["n_clusters"] = whole.track_ncl
    as_gpu["tracks"]["sector"] = whole.clusters["sector"][whole.track_first]
    picked = [0, 17, 18, 35]
    seen = []
    for k, alone in oracle_sectors(tf, picked, procs=4):
        view = sector_view(as_gpu, k)
        compare_integer(view, alone)
        t0 = int(np.searchsorted(as_gpu["tracks"]["sector"], k))
        n = len(alone.track_first)
        assert np.array_equal(alone.fits["par"], whole.fits["par"][t0:t0 + n])
        assert np.array_equal(alone.fits["cov"], whole.fits["cov"][t0:t0 + n])
        seen.append(k)
    assert sorted(seen) == picked
