"""Parity of the optional charge splitting (step 3s, tpc_params.split_charge)
with the oracle: clusters bit for bit (weights, moments and the split flag),
then the CA links, the cluster-to-track map and the tracks built on them, on a
sector, a dense sector, ragged time ranges whose units reach across fragment
edges, with step 2b on as well, and on the full TPC.  The fused and
dense-plane finders refuse the setting (their planes carry 3-bin halos; step
3s needs 5)."""
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


def params(lib, dip=0):
    p = lib.tpc_params_default()
    p.split_charge = 1
    p.ns_min_dip = dip
    return p


def check(lib, tf, dip=0, fit=False):
    orc = oracle.reconstruct(tf, oracle.OracleParams(split_charge=True, ns_min_dip=dip))
    with lib.Reconstructor.for_timeframe(tf, params=params(lib, dip)) as R:
        g = R.run(tf)
    compare_integer(g, orc)
    if fit:
        compare_fit(g, orc)
    split = (g["clusters"]["flags"] & 8) != 0
    return g, split


@pytest.mark.parametrize("seed", [1, 4])
def test_single_sector(lib, seed):
    tf = tpcgen.generate(tpcgen.single_sector(seed, n_tracks=300))
    g, split = check(lib, tf, fit=True)
    assert split.sum() > 50
    plain = oracle.find_clusters(tf)
    assert g["clusters"][~split].tobytes() == plain[~split].tobytes()


def test_dense_sector_with_noise_suppression(lib):
    tf = tpcgen.generate(tpcgen.single_sector(8, n_tracks=3000))
    _, split = check(lib, tf)
    assert split.mean() > 0.2
    check(lib, tf, dip=10)


@pytest.mark.parametrize("n_time_bins", [1, 5, 257, 700, 1030])
def test_ragged_time_ranges(lib, n_time_bins):
    """Peaks within 5 bins of a fragment edge read the neighbouring window's
    digits; the last fragment is ragged."""
    tf = tpcgen.generate(tpcgen.single_sector(5, n_tracks=400, n_time_bins=n_time_bins,
                                              coll_t0=[n_time_bins - 500.0]))
    check(lib, tf)


def test_continuous_pileup(lib):
    """Overlapping collisions of the continuous timeframe (2,000 bins, two
    sectors): pile-up puts more peaks within four pixels of each other."""
    tf = tpcgen.generate(tpcgen.continuous_tf(3, n_time_bins=2000, n_sectors=2))
    _, split = check(lib, tf, fit=True)
    assert split.mean() > 0.02


def test_full_tpc(lib):
    tf = tpcgen.generate(tpcgen.full_tpc(2, n_tracks=4000))
    g, split = check(lib, tf, fit=True)
    assert 0.02 < split.mean() < 0.9


def test_other_finders_refuse(lib):
    tf = tpcgen.generate(tpcgen.single_sector(1, n_tracks=10))
    for flags in (lib.TPC_CTX_DENSE_FINDER, lib.TPC_CTX_FUSED_FINDER):
        with pytest.raises(lib.TpcError) as ei:
            lib.Reconstructor.for_timeframe(tf, params=params(lib), flags=flags)
        assert ei.value.code == -1
    p = params(lib)
    p.split_charge = 2
    with pytest.raises(lib.TpcError):
        lib.Reconstructor.for_timeframe(tf, params=p)


def test_batch_equals_oracle(lib):
    """Uneven events in one batched run (the (event, sector) axis): each event's
    clusters and tracks are the oracle's with charge splitting on."""
    tfs = [tpcgen.generate(tpcgen.single_sector(s, n_tracks=n)) for s, n in [(11, 40), (12, 400), (13, 150)]]
    with lib.Reconstructor.for_timeframe(tfs[0], params=params(lib)) as R:
        batch = R.run_batch(tfs)
    for tf, ev in zip(tfs, batch):
        orc = oracle.reconstruct(tf, oracle.OracleParams(split_charge=True))
        assert ev["clusters"].tobytes() == orc.clusters.tobytes()
        assert np.array_equal(ev["cl2trk"], orc.cl2trk)
        assert np.array_equal(ev["tracks"]["first_cluster"], orc.track_first)
