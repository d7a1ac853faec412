"""The input-side helpers the CPU baselines sample with: a sector of a
timeframe as a timeframe of its own, and the first fragments of a long
timeframe.  Their clusters equal those of the whole timeframe (away from the
cut in time)."""
import numpy as np

import oracle
import tpcgen


def test_sector_slice_equals_the_sector_in_the_whole_timeframe():
    tf = tpcgen.generate(tpcgen.full_tpc(1, n_tracks=500))
    full = oracle.find_clusters(tpcgen.sector_prefix(tf, 4))
    for s in (0, 3):
        a = oracle.find_clusters(tpcgen.sector_slice(tf, s))
        b = full[full["sector"] == s].copy()
        b["sector"] = 0
        assert len(a) > 0 and a.tobytes() == b.tobytes()


def test_time_prefix_equals_the_whole_timeframe_before_the_cut():
    tf = tpcgen.generate(tpcgen.continuous_tf(1, n_time_bins=2000))
    sub = tpcgen.time_prefix(tf, 3)
    assert sub.n_time_bins == 768 and sub.n_fragments == 3
    a = oracle.find_clusters(sub)
    b = oracle.find_clusters(tf)
    cut = 768 - 3          # the last 3 bins lose their next-fragment halo
    ka, kb = a[a["t_peak"] < cut], b[b["t_peak"] < cut]
    assert len(ka) > 1000 and ka.tobytes() == kb.tobytes()
    assert np.all(a["t_peak"] < 768)
