"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs, plus the edge cases of the method."""
import copy

import numpy as np
import pytest

import oracle
import tpcgen
from parity import compare_fit, compare_integer

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def run_gpu(tpc, tf, **kw):
    with tpc.Reconstructor.for_timeframe(tf, **kw) as R:
        return R.run(tf)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_single_sector_parity(lib, seed):
    tf = tpcgen.generate(tpcgen.single_sector(seed))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    compare_fit(gpu, orc)
    assert gpu["counters"]["error_word"] == 0


def test_full_tpc_parity(lib):
    """36 sectors, 1000 time bins, 10,000 tracks: the benchmark workload."""
    tf = tpcgen.generate(tpcgen.full_tpc(1))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    rep = compare_fit(gpu, orc)
    print("full_tpc fit precision vs FP64 oracle:", rep)
    assert rep["n_tracks"] > 10000
    assert gpu["counters"]["merge_passes"] == orc.merge_passes


@pytest.mark.parametrize("n_time_bins", [1, 3, 255, 256, 257, 511, 700])
def test_ragged_time_ranges(lib, n_time_bins):
    """Partial last fragment, fragments shorter than the halo, a single bin."""
    tf = tpcgen.generate(tpcgen.single_sector(5, n_tracks=60, n_time_bins=n_time_bins,
                                              coll_t0=[n_time_bins - 500.0]))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    compare_fit(gpu, orc)


def test_maximum_time_range(lib):
    """The longest timeframe the ABI takes (65,535 bins: 256 fragments, the
    last one 255 bins long) on one sector, with collisions at its start, middle
    and end: the largest fragment index and zeta the records and the fit see."""
    n = 65535
    tf = tpcgen.generate(tpcgen.single_sector(9, n_time_bins=n, coll_t0=[0.0, 32000.0, n - 500.0],
                                              coll_ntracks=[60, 60, 60]))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    compare_fit(gpu, orc)
    assert int(gpu["clusters"]["t_peak"].max()) >= 65280 and len(gpu["tracks"]) > 30


def test_empty_and_noise_only(lib):
    tf = tpcgen.generate(tpcgen.single_sector(6, n_tracks=0))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    assert len(gpu["tracks"]) == 0
    # no digits at all: zero threshold above every ADC
    tf2 = tpcgen.generate(tpcgen.single_sector(6, n_tracks=0, zs_threshold=1024))
    gpu2 = run_gpu(lib, tf2)
    assert len(gpu2["clusters"]) == 0 and len(gpu2["tracks"]) == 0


def test_dense_occupancy(lib):
    """Heavy pile-up in one sector: many neighbouring peaks, excluded pixels."""
    tf = tpcgen.generate(tpcgen.single_sector(8, n_tracks=3000))
    orc = oracle.reconstruct(tf)
    gpu = run_gpu(lib, tf)
    compare_integer(gpu, orc)
    compare_fit(gpu, orc)


FINDER_FLAGS = [0, 8]   # the two-pass finder (default), the fused variant


@pytest.mark.parametrize("flags", FINDER_FLAGS)
def test_corrupt_page_reported(lib, flags):
    tf = tpcgen.generate(tpcgen.single_sector(1))
    bad = copy.copy(tf)
    bad.pages = tf.pages.copy()
    o = int(tf.page_offsets[40 * 2 + 1])
    bad.pages[o + 14] ^= 0xFF  # magic
    with lib.Reconstructor.for_timeframe(bad, flags=flags) as R:
        t = R.submit(bad.pages, bad.page_offsets, bad.n_time_bins)
        with pytest.raises(lib.TpcError) as ei:
            R.wait(t)
        assert ei.value.code == -5
        lib.tpc_release(R.ctx, t)
        # the context stays usable
        good = R.run(tf)
    orc = oracle.reconstruct(tf)
    compare_integer(good, orc)


def test_device_input_matches_host(lib):
    import torch
    tf = tpcgen.generate(tpcgen.single_sector(2))
    host = run_gpu(lib, tf)
    pages = torch.from_numpy(tf.pages).cuda()
    offs = torch.from_numpy(tf.page_offsets.view(np.int64)).cuda()
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(pages, offs, tf.n_time_bins)
        R.wait(t)
        cl = lib.tpc_get_clusters(R.ctx, t)
        tr, m = lib.tpc_get_tracks(R.ctx, t, len(cl))
        lib.tpc_release(R.ctx, t)
    assert cl.tobytes() == host["clusters"].tobytes()
    assert tr.tobytes() == host["tracks"].tobytes()
    assert np.array_equal(m, host["cl2trk"])


def test_slots_in_flight_give_identical_results(lib):
    """Several timeframes in flight on different slots/streams at once: each
    result equals the same timeframe run alone (bitwise, the kernels are
    deterministic)."""
    tfs = [tpcgen.generate(tpcgen.single_sector(s)) for s in (11, 12, 13)]
    alone = [run_gpu(lib, tf) for tf in tfs]
    with lib.Reconstructor.for_timeframe(tfs[0], n_slots=3) as R:
        tickets = [R.submit(tf.pages, tf.page_offsets, tf.n_time_bins) for tf in tfs]
        for tf, t, a in zip(tfs, tickets, alone):
            R.wait(t)
            cl = lib.tpc_get_clusters(R.ctx, t)
            tr, m = lib.tpc_get_tracks(R.ctx, t, len(cl))
            assert cl.tobytes() == a["clusters"].tobytes()
            assert tr.tobytes() == a["tracks"].tobytes()
            lib.tpc_release(R.ctx, t)


def test_stage_times_and_counters(lib):
    tf = tpcgen.generate(tpcgen.single_sector(3))
    with lib.Reconstructor.for_timeframe(tf, flags=lib.TPC_CTX_STAGE_TIMING) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        ms = lib.tpc_get_stage_times(R.ctx, t)
        ctr = lib.tpc_get_counters(R.ctx, t)
        lib.tpc_release(R.ctx, t)
    assert set(ms) == {"find", "ca", "merge", "fit"} and all(v >= 0 for v in ms.values())
    assert ctr["kernel_launches"] > 10 and ctr["runs"] == 1 and ctr["error_word"] == 0


def test_graph_replay_matches_plain_launches(lib):
    """The slot's captured CUDA graph, replayed for new inputs (host copies into
    the same buffers; device inputs at new addresses, which update the graph in
    place), gives bitwise the results of plain kernel launches."""
    import torch
    tfs = [tpcgen.generate(tpcgen.single_sector(s)) for s in (21, 22)]
    plain = [run_gpu(lib, tf, flags=lib.TPC_CTX_NO_GRAPHS) for tf in tfs]
    with lib.Reconstructor.for_timeframe(tfs[0]) as R:
        for rep in range(2):
            for tf, a in zip(tfs, plain):
                if rep == 0:
                    t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
                else:
                    pages = torch.from_numpy(tf.pages).cuda()
                    offs = torch.from_numpy(tf.page_offsets.view(np.int64)).cuda()
                    t = R.submit(pages, offs, tf.n_time_bins)
                R.wait(t)
                cl = lib.tpc_get_clusters(R.ctx, t)
                tr, m = lib.tpc_get_tracks(R.ctx, t, len(cl))
                lib.tpc_release(R.ctx, t)
                assert cl.tobytes() == a["clusters"].tobytes()
                assert tr.tobytes() == a["tracks"].tobytes()
                assert np.array_equal(m, a["cl2trk"])


def _hdr(pages, o):
    h = pages[o:o + 32].view(np.uint16)
    return {"n_tb": int(h[2]), "n_runs": int(h[3]), "n_dig": int(h[4]), "lo_dig": int(h[10]), "lo_runs": int(h[9]),
            "hi_dig": int(h[13]), "hi_runs": int(h[12])}


@pytest.mark.parametrize("flags", FINDER_FLAGS)
@pytest.mark.parametrize("where", ["run", "entry"])
def test_corrupt_light_window_reported(lib, where, flags):
    """A full-TPC timeframe (its sparse windows go to the one-warp path): a
    page body broken in such a window -- a run past the row's end, or time
    bins out of order -- is reported as corruption, and the context stays usable."""
    tf = tpcgen.generate(tpcgen.full_tpc(5, n_tracks=2000))
    nf = tf.n_fragments
    offs = tf.page_offsets.astype(np.int64)
    w = None
    for cand in range(1, len(offs) - 1):
        if cand % nf in (0, nf - 1):
            continue
        h, hp, hn = (_hdr(tf.pages, int(offs[cand + k])) for k in (0, -1, 1))
        total = h["n_dig"] + hp["n_dig"] - hp["hi_dig"] + hn["lo_dig"]
        if 4 <= h["n_tb"] and 0 < total <= 200:
            w = cand
            break
    assert w is not None
    o = int(offs[w])
    h = _hdr(tf.pages, o)
    bad = copy.copy(tf)
    bad.pages = tf.pages.copy()
    if where == "run":
        bad.pages[o + 32 + 2 * h["n_tb"] + 1] = 200          # run 0's length: past any row
    else:
        bad.pages[o + 32 + 2] = bad.pages[o + 32]             # entry 1 at entry 0's time bin
    with lib.Reconstructor.for_timeframe(bad, flags=flags) as R:
        t = R.submit(bad.pages, bad.page_offsets, bad.n_time_bins)
        with pytest.raises(lib.TpcError) as ei:
            R.wait(t)
        assert ei.value.code == -5
        lib.tpc_release(R.ctx, t)
        good = R.run(tf)
    assert good["clusters"].tobytes() == oracle.find_clusters(tf).tobytes()


def _break(pages, o, h, defect):
    """One defect of a page body or header (the oracle rejects each)."""
    ent, run = o + 32, o + 32 + 2 * h["n_tb"]
    if defect == "run_overlap":        # run 1 of entry 0 starts inside run 0
        pages[run + 2] = pages[run]
    elif defect == "zero_runs":        # entry 0 with no run
        pages[ent + 1] = 0
    elif defect == "zero_length":      # run 0 of length 0
        pages[run + 1] = 0
    elif defect == "digit_count":      # header digit count one short
        v = int(pages[o + 8]) | int(pages[o + 9]) << 8
        pages[o + 8:o + 10] = np.frombuffer(np.uint16(v - 1).tobytes(), np.uint8)
    elif defect == "run_count":        # header run count one more
        v = int(pages[o + 6]) | int(pages[o + 7]) << 8
        pages[o + 6:o + 8] = np.frombuffer(np.uint16(v + 1).tobytes(), np.uint8)
    elif defect == "row":              # header names another row
        pages[o + 11] ^= 1


@pytest.mark.parametrize("flags", FINDER_FLAGS)
@pytest.mark.parametrize("defect", ["run_overlap", "zero_runs", "zero_length", "digit_count", "run_count", "row"])
def test_page_defects_reported_like_the_oracle(lib, defect, flags):
    tf = tpcgen.generate(tpcgen.single_sector(1))
    offs = tf.page_offsets.astype(np.int64)
    # a page whose first entry has at least two runs
    w = next(k for k in range(len(offs)) if _hdr(tf.pages, int(offs[k]))["n_tb"] > 0 and
             tf.pages[int(offs[k]) + 33] >= 2)
    o = int(offs[w])
    bad = copy.copy(tf)
    bad.pages = tf.pages.copy()
    _break(bad.pages, o, _hdr(tf.pages, o), defect)
    with pytest.raises(oracle.CorruptPage):
        oracle.find_clusters(bad)
    with lib.Reconstructor.for_timeframe(bad, flags=flags) as R:
        t = R.submit(bad.pages, bad.page_offsets, bad.n_time_bins)
        with pytest.raises(lib.TpcError) as ei:
            R.wait(t)
        assert ei.value.code == -5
        lib.tpc_release(R.ctx, t)
