"""Serving: timeframes that arrive while others run are queued and admitted as
slots and device memory free up; their work overlaps on the device.  Every
result must be the same in the mix as alone, bit for bit."""
import numpy as np
import pytest

import tpcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


@pytest.fixture(scope="module")
def mix():
    """Uneven occupancies on one geometry: pp-like to central Pb-Pb-like."""
    mult = [300, 10000, 1200, 50, 6000, 2500, 10000, 800]
    return [tpcgen.generate(tpcgen.full_tpc(700 + i, n_tracks=m)) for i, m in enumerate(mult)]


def fetch(lib, ctx, t):
    cl = lib.tpc_get_clusters(ctx, t)
    tr, m = lib.tpc_get_tracks(ctx, t, len(cl))
    return cl, tr, m


def test_burst_is_admitted_by_slots_and_memory(lib, mix):
    alone = []
    for tf in mix:
        with lib.Reconstructor.for_timeframe(tf) as R:
            alone.append(R.run(tf))
    # 3 slots, and a budget that holds about two large timeframes at once
    with lib.Reconstructor.for_timeframe(mix[0], n_slots=3, mem_budget=2 << 30) as R:
        tickets = [R.submit(tf.pages, tf.page_offsets, tf.n_time_bins) for tf in mix]
        states = [lib.tpc_poll(R.ctx, t, 0) for t in tickets]
        assert states[0] != lib.TPC_STATE_QUEUED
        assert states[3:].count(lib.TPC_STATE_QUEUED) == len(mix) - 3   # only 3 slots
        # a non-waiting submit is refused while everything is busy
        with pytest.raises(lib.TpcError) as ei:
            R.submit(mix[0].pages, mix[0].page_offsets, mix[0].n_time_bins, flags=lib.TPC_TF_NOWAIT)
        assert ei.value.code == -3
        # consume in completion order; each release admits the oldest queued request
        left = dict(zip(tickets, range(len(mix))))
        while left:
            for t in list(left):
                if lib.tpc_poll(R.ctx, t, 0) == lib.TPC_STATE_DONE:
                    i = left.pop(t)
                    cl, tr, m = fetch(lib, R.ctx, t)
                    lib.tpc_release(R.ctx, t)
                    assert cl.tobytes() == alone[i]["clusters"].tobytes()
                    assert tr.tobytes() == alone[i]["tracks"].tobytes()
                    assert np.array_equal(m, alone[i]["cl2trk"])


def test_queued_request_can_be_cancelled(lib, mix):
    with lib.Reconstructor.for_timeframe(mix[0], n_slots=1) as R:
        t0 = R.submit(mix[1].pages, mix[1].page_offsets, mix[1].n_time_bins)
        t1 = R.submit(mix[2].pages, mix[2].page_offsets, mix[2].n_time_bins)
        t2 = R.submit(mix[3].pages, mix[3].page_offsets, mix[3].n_time_bins)
        assert lib.tpc_poll(R.ctx, t1, 0) == lib.TPC_STATE_QUEUED
        lib.tpc_release(R.ctx, t1)               # cancelled before it started
        with pytest.raises(lib.TpcError):
            lib.tpc_poll(R.ctx, t1, 0)
        R.wait(t0)
        lib.tpc_release(R.ctx, t0)               # admits t2
        R.wait(t2)
        cl = lib.tpc_get_clusters(R.ctx, t2)
        lib.tpc_release(R.ctx, t2)
    with lib.Reconstructor.for_timeframe(mix[3]) as R:
        ref = R.run(mix[3])
    assert cl.tobytes() == ref["clusters"].tobytes()


def test_request_larger_than_the_budget_fails_cleanly(lib, mix):
    with lib.Reconstructor.for_timeframe(mix[0], mem_budget=512 << 20) as R:
        with pytest.raises(lib.TpcError) as ei:
            R.submit(mix[1].pages, mix[1].page_offsets, mix[1].n_time_bins)
        assert ei.value.code == -2
        small = tpcgen.generate(tpcgen.full_tpc(9, n_tracks=20))
        out = R.run(small)
        assert out["counters"]["error_word"] == 0
