"""Continuous-readout timeframes at a 50 kHz Pb-Pb-like interaction rate:
collisions with uniform start times whose drift windows overlap.

A short continuous timeframe is compared with the oracle in full, and so are
11,000-bin timeframes of seeds 2-4 sector by sector.  The
full-size one (55,000 time bins, ~2.7e9 digits, ~5.7 GB of ZS pages) runs
through the CUDA path as the benchmark runs it, and every one of its 36
sectors is compared element by element with the oracle run on that sector
alone (every step of the method stays inside a sector), in a spawn pool of
oracle processes; properties that hold at any size check the whole."""
import numpy as np
import pytest

import oracle
import tpcgen
from oracle_pool import oracle_sectors, sector_view
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


def test_short_continuous_parity(lib):
    """2000 bins (~20 overlapping collisions), 2 sectors: full parity."""
    tf = tpcgen.generate(tpcgen.continuous_tf(2, n_time_bins=2000, n_sectors=2))
    orc = oracle.reconstruct(tf)
    with lib.Reconstructor.for_timeframe(tf) as R:
        gpu = R.run(tf)
    compare_integer(gpu, orc)
    compare_fit(gpu, orc)
    assert gpu["counters"]["error_word"] == 0


def check_properties(gpu: dict, tf) -> None:
    cl, tr, m = gpu["clusters"], gpu["tracks"], gpu["cl2trk"]
    assert gpu["counters"]["error_word"] == 0
    # canonical cluster order: (sector, row, t_peak, pad_peak) strictly ascending
    key = (cl["sector"].astype(np.int64) << 40) | (cl["row"].astype(np.int64) << 32) | \
          (cl["t_peak"].astype(np.int64) << 8) | cl["pad_peak"].astype(np.int64)
    assert np.all(np.diff(key) > 0)
    assert int(cl["sector"].max()) < tf.n_sectors and int(cl["t_peak"].max()) < tf.n_time_bins
    # links stay within the neighbouring rows of the same sector and are mutual on chains
    up, down = gpu["up"], gpu["down"]
    has_up = np.nonzero(up >= 0)[0]
    assert np.all(cl["row"][up[has_up]] == cl["row"][has_up] + 1)
    assert np.all(cl["sector"][up[has_up]] == cl["sector"][has_up])
    # tracks: ordered by (sector, lowest cluster), membership agrees with the map
    assert np.all(np.diff(tr["sector"].astype(np.int64) * (1 << 32) + tr["first_cluster"]) > 0)
    on = m >= 0
    assert np.array_equal(np.bincount(m[on], minlength=len(tr)), tr["n_clusters"])
    assert np.all(m[tr["first_cluster"]] == np.arange(len(tr)))
    assert np.all(tr["ndf"][tr["flags"] == 0] > 0)
    assert np.all(np.isfinite(tr["par"]))


def test_continuous_50khz_full_size(lib):
    tf = tpcgen.generate(tpcgen.continuous_tf(1))
    assert tf.n_time_bins == 55000 and tf.pages.nbytes > 3 << 30
    with lib.Reconstructor.for_timeframe(tf, mem_budget=200 << 30) as R:
        gpu = R.run(tf)
    check_properties(gpu, tf)
    n_cl, n_tr = len(gpu["clusters"]), len(gpu["tracks"])
    assert n_cl > 5e7 and n_tr > 2e5, (n_cl, n_tr)
    # every sector element by element against the oracle on that sector alone
    worst = np.zeros(5)
    seen, ncl_sum, ntr_sum = set(), 0, 0
    for k, orc in oracle_sectors(tf, list(range(tf.n_sectors))):
        view = sector_view(gpu, k)
        compare_integer(view, orc)
        rep = compare_fit(view, orc, tf)
        worst = np.maximum(worst, rep["max_rel_par_plain_floor"])
        seen.add(k)
        ncl_sum += len(orc.clusters)
        ntr_sum += len(orc.track_first)
    assert seen == set(range(tf.n_sectors)) and ncl_sum == n_cl and ntr_sum == n_tr
    print("continuous 50 kHz, all sectors: max plain-floor parameter error vs FP64 oracle", worst.tolist())


@pytest.mark.parametrize("seed", [2, 3, 4])
def test_continuous_50khz_other_seeds(lib, seed):
    """The continuous timeframe's other seeds, at 11,000 time bins of the same
    collision law (a fifth of the length, the same occupancy): every sector
    element by element against the oracle, and the properties of the whole."""
    tf = tpcgen.generate(tpcgen.continuous_tf(seed, n_time_bins=11000))
    with lib.Reconstructor.for_timeframe(tf, mem_budget=64 << 30) as R:
        gpu = R.run(tf)
    check_properties(gpu, tf)
    assert len(gpu["clusters"]) > 1e7
    n_cl = n_tr = 0
    for k, orc in oracle_sectors(tf, list(range(tf.n_sectors))):
        view = sector_view(gpu, k)
        compare_integer(view, orc)
        compare_fit(view, orc, tf)
        n_cl += len(orc.clusters)
        n_tr += len(orc.track_first)
    assert n_cl == len(gpu["clusters"]) and n_tr == len(gpu["tracks"])
