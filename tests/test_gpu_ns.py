"""Parity of the optional 5x5 noise suppression (step 2b, tpc_params.ns_min_dip)
with the oracle: clusters bit for bit, then the tracks built on them, through
the fused finder and the dense-plane variant (the allocation-free entry point:
in the last-collected test file)."""
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


def params(lib, dip):
    p = lib.tpc_params_default()
    p.ns_min_dip = dip
    return p


def check(lib, tf, dip, flags=0):
    orc = oracle.reconstruct(tf, oracle.OracleParams(ns_min_dip=dip))
    with lib.Reconstructor.for_timeframe(tf, params=params(lib, dip), flags=flags) as R:
        g = R.run(tf)
    assert g["clusters"].tobytes() == orc.clusters.tobytes()
    assert np.array_equal(g["cl2trk"], orc.cl2trk)
    assert np.array_equal(g["tracks"]["first_cluster"], orc.track_first)
    return g


@pytest.mark.parametrize("dip", [1, 10, 1023])
def test_single_sector(lib, dip):
    tf = tpcgen.generate(tpcgen.single_sector(4, n_tracks=300))
    g = check(lib, tf, dip)
    assert len(g["clusters"]) < len(oracle.find_clusters(tf))


@pytest.mark.parametrize("n_time_bins", [1, 257, 700])
def test_ragged_time_ranges(lib, n_time_bins):
    tf = tpcgen.generate(tpcgen.single_sector(5, n_tracks=60, n_time_bins=n_time_bins,
                                              coll_t0=[n_time_bins - 500.0]))
    check(lib, tf, 10)


def test_dense_sector_unlisted_windows(lib):
    """Windows past the 4096-digit list: the plane is then cleared whole."""
    tf = tpcgen.generate(tpcgen.single_sector(8, n_tracks=3000))
    check(lib, tf, 10)


def test_continuous_pileup(lib):
    """Overlapping collisions of the continuous timeframe (2,000 bins, two sectors)."""
    tf = tpcgen.generate(tpcgen.continuous_tf(3, n_time_bins=2000, n_sectors=2))
    g = check(lib, tf, 10)
    assert len(g["clusters"]) < len(oracle.find_clusters(tf))


def test_full_tpc_all_finder_variants(lib):
    tf = tpcgen.generate(tpcgen.full_tpc(2, n_tracks=4000))
    g = check(lib, tf, 10)
    for flags in (lib.TPC_CTX_DENSE_FINDER, lib.TPC_CTX_FUSED_FINDER):
        d = check(lib, tf, 10, flags=flags)
        assert g["clusters"].tobytes() == d["clusters"].tobytes()


def test_dense_sector_fused_variant(lib):
    tf = tpcgen.generate(tpcgen.single_sector(8, n_tracks=3000))
    check(lib, tf, 10, flags=lib.TPC_CTX_FUSED_FINDER)


def test_rejects_out_of_range(lib):
    tf = tpcgen.generate(tpcgen.single_sector(1, n_tracks=10))
    with pytest.raises(lib.TpcError):
        lib.Reconstructor.for_timeframe(tf, params=params(lib, 1024))
