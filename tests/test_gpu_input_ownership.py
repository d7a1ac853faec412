"""Ownership of the input pages, and the cluster capacity bound.

A device-resident timeframe is read in place by every run of the pipeline,
including the re-run after a cluster-capacity overflow, so the library must not
report TPC_STATE_INPUT_RELEASED for it before it is done.  The test overwrites
the pages the moment that state would show and checks the results against an
undisturbed run from host memory.

The input is the densest pattern the page format allows: on every other time
bin a single run over the whole row whose ADCs alternate 100, 50, so that every
even pad of every even time bin is a peak.  That is 0.366 clusters per page
byte, above the 1/3 the cluster capacity was once capped at; the bound derived
from the format is 3/8 (every peak needs its own 10-bit ADC and, between two
peaks of one entry, either a digit or a new run)."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from parity import cluster_bytes
from synth import encode_planes

pytestmark = pytest.mark.gpu

N_ROWS, NPADS, N_FRAG = 3, 138, 40


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


@pytest.fixture(scope="module")
def dense_tf():
    T = 256 * N_FRAG
    planes = np.zeros((1, N_ROWS, T, NPADS), np.uint16)
    planes[0, :, 0::2, 0::2] = 100
    planes[0, :, 0::2, 1::2] = 50
    npads = np.full(N_ROWS, NPADS, np.int32)
    pages, offs = encode_planes(planes, T, npads)
    return SimpleNamespace(pages=pages, page_offsets=offs, n_time_bins=T, n_sectors=1, npads=npads,
                           row_x=np.array([1697, 1712, 1727], np.int32))


def test_worst_case_density_and_device_input_held_until_done(lib, dense_tf):
    import torch
    tf = dense_tf
    want_n = N_ROWS * N_FRAG * 128 * (NPADS // 2)
    assert want_n / tf.pages.nbytes > 1 / 3 and want_n <= tf.pages.nbytes * 3 // 8
    with lib.Reconstructor.for_timeframe(tf) as R:
        ref = R.run(tf)
    assert len(ref["clusters"]) == want_n
    assert ref["counters"]["runs"] >= 2, "the timeframe should overflow the initial capacity and re-run"
    orc = oracle.find_clusters(tf)
    assert cluster_bytes(ref["clusters"]).tobytes() == cluster_bytes(orc).tobytes()

    pages = torch.from_numpy(tf.pages).cuda()
    offs = torch.from_numpy(tf.page_offsets.view(np.int64)).cuda()
    torch.cuda.synchronize()
    released_seen = False
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(pages, offs, tf.n_time_bins)
        while True:
            st = lib.tpc_poll(R.ctx, t, 0)
            if st == lib.TPC_STATE_INPUT_RELEASED and not released_seen:
                released_seen = True
                pages.zero_()              # the caller reuses memory it was told is free
            if st == lib.TPC_STATE_DONE:
                break
            assert st in (lib.TPC_STATE_RUNNING, lib.TPC_STATE_INPUT_RELEASED)
        cl = lib.tpc_get_clusters(R.ctx, t)
        up, down, chain = lib.tpc_get_links(R.ctx, t, len(cl))
        tracks, m = lib.tpc_get_tracks(R.ctx, t, len(cl))
        runs = lib.tpc_get_counters(R.ctx, t)["runs"]
        lib.tpc_release(R.ctx, t)
    assert not released_seen, "device input must stay borrowed until the timeframe is done"
    assert runs >= 2
    assert cluster_bytes(cl).tobytes() == cluster_bytes(ref["clusters"]).tobytes()
    for k, v in (("up", up), ("down", down), ("chain_of", chain), ("cl2trk", m)):
        assert np.array_equal(v, ref[k]), k
    assert tracks.tobytes() == ref["tracks"].tobytes()
