"""The finder variants of steps 1-4 against the default two-pass finder
(pages decoded into pad-run records in device memory, then each 64-bin time
chunk of a window expanded into a small shared plane and clustered there): the fused variant (context
flag TPC_CTX_FUSED_FINDER: each window decoded straight into a shared plane of
the whole window) and the dense-plane variant (TPC_CTX_DENSE_FINDER: pages
decoded into a dense (sector row, time bin, pad) plane in device memory,
windows read back from it).  All must give, bit for bit, the same clusters,
tracks and cluster-to-track map, and so the oracle's."""
import numpy as np
import pytest

import oracle
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


def run(lib, tf, flags, **kw):
    with lib.Reconstructor.for_timeframe(tf, flags=flags, **kw) as R:
        return R.run(tf)


def assert_same(a, b):
    assert a["clusters"].tobytes() == b["clusters"].tobytes()
    assert a["tracks"].tobytes() == b["tracks"].tobytes()
    assert np.array_equal(a["cl2trk"], b["cl2trk"])


@pytest.mark.parametrize("n_time_bins", [1, 3, 257, 700])
def test_ragged_time_ranges_variants_equal(lib, n_time_bins):
    tf = tpcgen.generate(tpcgen.single_sector(5, n_tracks=60, n_time_bins=n_time_bins,
                                              coll_t0=[n_time_bins - 500.0]))
    dense = run(lib, tf, lib.TPC_CTX_DENSE_FINDER)
    two_pass = run(lib, tf, 0)
    assert_same(dense, two_pass)
    assert_same(run(lib, tf, lib.TPC_CTX_FUSED_FINDER), two_pass)
    assert dense["clusters"].tobytes() == oracle.reconstruct(tf).clusters.tobytes()


def test_dense_occupancy_variants_equal(lib):
    """3000 tracks in one sector: windows past the 4096-digit list walk the
    occupancy bitmap instead."""
    tf = tpcgen.generate(tpcgen.single_sector(8, n_tracks=3000))
    dense = run(lib, tf, lib.TPC_CTX_DENSE_FINDER)
    two_pass = run(lib, tf, 0)
    assert_same(dense, two_pass)
    assert_same(run(lib, tf, lib.TPC_CTX_FUSED_FINDER), two_pass)
    assert dense["clusters"].tobytes() == oracle.reconstruct(tf).clusters.tobytes()


def test_full_tpc_variants_equal(lib):
    tf = tpcgen.generate(tpcgen.full_tpc(1))
    dense = run(lib, tf, lib.TPC_CTX_DENSE_FINDER)
    two_pass = run(lib, tf, 0)
    assert_same(dense, two_pass)
    assert_same(run(lib, tf, lib.TPC_CTX_FUSED_FINDER), two_pass)
    orc = oracle.reconstruct(tf)
    assert dense["clusters"].tobytes() == orc.clusters.tobytes()
    assert np.array_equal(dense["cl2trk"], orc.cl2trk)


def test_batch_variants_equal(lib):
    tfs = [tpcgen.generate(tpcgen.full_tpc(70 + i, n_tracks=m)) for i, m in enumerate((500, 6000, 2000))]
    out = {}
    for flags in (0, lib.TPC_CTX_DENSE_FINDER, lib.TPC_CTX_FUSED_FINDER):
        with lib.Reconstructor.for_timeframe(tfs[0], flags=flags, mem_budget=16 << 30) as R:
            out[flags] = R.run_batch(tfs)
    for flags in (lib.TPC_CTX_DENSE_FINDER, lib.TPC_CTX_FUSED_FINDER):
        for a, b in zip(out[0], out[flags]):
            assert_same(b, a)
