"""Batched events: several independent timeframes of uneven occupancy in one
pipeline run (tpc_submit_batch).  Each event's results must equal, bit for bit,
those of the same event submitted alone, and match the oracle."""
import copy

import numpy as np
import pytest

import oracle
import tpcgen
from parity import compare_fit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def alone(lib, tf):
    with lib.Reconstructor.for_timeframe(tf) as R:
        return R.run(tf)


def assert_same(ev, ref):
    assert ev["clusters"].tobytes() == ref["clusters"].tobytes()
    assert ev["tracks"].tobytes() == ref["tracks"].tobytes()
    assert np.array_equal(ev["cl2trk"], ref["cl2trk"])


def test_single_sector_batch_equals_alone_and_oracle(lib):
    mult = [150, 0, 1000, 40, 400, 2500]
    tfs = [tpcgen.generate(tpcgen.single_sector(30 + i, n_tracks=m)) for i, m in enumerate(mult)]
    with lib.Reconstructor.for_timeframe(tfs[0]) as R:
        batch = R.run_batch(tfs)
    for tf, ev in zip(tfs, batch):
        assert_same(ev, alone(lib, tf))
        orc = oracle.reconstruct(tf)
        assert ev["clusters"].tobytes() == orc.clusters.tobytes()
        assert np.array_equal(ev["cl2trk"], orc.cl2trk)
        assert np.array_equal(ev["tracks"]["first_cluster"], orc.track_first)
        compare_fit({"tracks": ev["tracks"]}, orc)


def test_full_tpc_uneven_batch_equals_alone(lib):
    """Full 36-sector events, multiplicities log-uniform in [200, 20000]."""
    mult = tpcgen.batch_multiplicities(1000, n_events=5)
    tfs = [tpcgen.generate(tpcgen.full_tpc(1000 + i, n_tracks=int(m))) for i, m in enumerate(mult)]
    with lib.Reconstructor.for_timeframe(tfs[0], mem_budget=32 << 30) as R:
        batch = R.run_batch(tfs)
        # the same slot replays its captured graph for a second batch of the same shape
        batch2 = R.run_batch(tfs[::-1])
    for tf, ev, ev2 in zip(tfs, batch, batch2[::-1]):
        ref = alone(lib, tf)
        assert_same(ev, ref)
        assert_same(ev2, ref)


def test_batch_info_and_device_input(lib):
    import torch
    tfs = [tpcgen.generate(tpcgen.single_sector(40 + i, n_tracks=100 * (i + 1))) for i in range(3)]
    dev = [(torch.from_numpy(tf.pages).cuda(), torch.from_numpy(tf.page_offsets.view(np.int64)).cuda())
           for tf in tfs]
    with lib.Reconstructor.for_timeframe(tfs[0]) as R:
        t, keep = lib.tpc_submit_batch(R.ctx, dev, tfs[0].n_time_bins)
        R.wait(t)
        cs, ts = lib.tpc_get_batch_info(R.ctx, t)
        allcl = lib.tpc_get_clusters(R.ctx, t)
        alltr, allmap = lib.tpc_get_tracks(R.ctx, t, len(allcl))
        per = [lib.tpc_get_event_clusters(R.ctx, t, e) for e in range(3)]
        with pytest.raises(lib.TpcError):
            lib.tpc_get_event_clusters(R.ctx, t, 3)
        lib.tpc_release(R.ctx, t)
    assert cs[0] == 0 and cs[-1] == len(allcl) and ts[-1] == len(alltr)
    for e, tf in enumerate(tfs):
        ref = alone(lib, tf)
        assert allcl[cs[e]:cs[e + 1]].tobytes() == ref["clusters"].tobytes() == per[e].tobytes()
        tr = alltr[ts[e]:ts[e + 1]].copy()
        tr["first_cluster"] -= int(cs[e])
        assert tr.tobytes() == ref["tracks"].tobytes()
        m = allmap[cs[e]:cs[e + 1]].copy()
        m[m >= 0] -= int(ts[e])
        assert np.array_equal(m, ref["cl2trk"])


def test_batch_rejects_mixed_time_ranges_and_reports_corruption(lib):
    a = tpcgen.generate(tpcgen.single_sector(50))
    b = tpcgen.generate(tpcgen.single_sector(51, n_time_bins=400))
    with lib.Reconstructor.for_timeframe(a) as R:
        with pytest.raises(lib.TpcError) as ei:
            lib.tpc_submit_batch(R.ctx, [(a.pages, a.page_offsets, 500), (b.pages, b.page_offsets, 400)], 500)
        assert ei.value.code == -1
        bad = copy.copy(a)
        bad.pages = a.pages.copy()
        bad.pages[int(a.page_offsets[7]) + 14] ^= 0xFF   # magic of one page
        t, keep = lib.tpc_submit_batch(R.ctx, [(a.pages, a.page_offsets), (bad.pages, bad.page_offsets)], 500)
        with pytest.raises(lib.TpcError) as ei:
            R.wait(t)
        assert ei.value.code == -5
        lib.tpc_release(R.ctx, t)
        # an offset pointing past its own event's pages is corrupt too
        offs = a.page_offsets.copy()
        offs[3] = a.pages.nbytes + 16
        t, keep = lib.tpc_submit_batch(R.ctx, [(a.pages, offs), (a.pages, a.page_offsets)], 500)
        with pytest.raises(lib.TpcError) as ei:
            R.wait(t)
        assert ei.value.code == -5
        lib.tpc_release(R.ctx, t)
        ok = R.run_batch([a, a])
    ref = alone(lib, a)
    for ev in ok:
        assert_same(ev, ref)
