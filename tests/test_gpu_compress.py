"""Parity of the track-model compression (step 10) with the oracle.  The codes
are rounded float residuals to the FP32 (GPU) or FP64 (oracle) track model, so
a residual within the fit difference of a rounding boundary can round either
way: statuses and codes must agree for all but a small fraction of clusters,
and never differ by more than one step."""
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


def test_full_tpc_compression_parity(lib):
    tf = tpcgen.generate(tpcgen.full_tpc(1))
    orc = oracle.reconstruct(tf)
    ocy, ocz, ost = oracle.compress(tf, orc)
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        cl = lib.tpc_get_clusters(R.ctx, t)
        n_coded, n_esc = lib.tpc_compress_clusters(R.ctx, t)
        cy, cz, st = lib.tpc_get_compressed(R.ctx, t, len(cl))
        lib.tpc_release(R.ctx, t)
    assert cl.tobytes() == orc.clusters.tobytes()
    assert n_coded == int((st == 1).sum()) and n_esc == int((st == 2).sum())
    assert np.array_equal(st == 0, ost == 0)            # on a track or not: integer, exact
    on = ost > 0
    same_status = (st == ost)[on].mean()
    both = (st == 1) & (ost == 1)
    dy = np.abs(cy[both].astype(int) - ocy[both])
    dz = np.abs(cz[both].astype(int) - ocz[both])
    print(f"clusters on tracks {on.sum()}, coded {n_coded}, escaped {n_esc}; status agree {same_status:.6f}; "
          f"codes differ y {np.mean(dy > 0):.2e} z {np.mean(dz > 0):.2e}")
    assert same_status >= 0.999
    assert dy.max() <= 1 and dz.max() <= 1
    assert np.mean(dy > 0) <= 0.01 and np.mean(dz > 0) <= 0.01


def test_degenerate_inputs_steps_10_11(lib):
    """No digits and noise only (no tracks): step 10 codes nothing, every cluster
    keeps status 0; step 11 finds no track to use and reports no estimate."""
    for cfg in (tpcgen.single_sector(6, n_tracks=0, zs_threshold=1024), tpcgen.single_sector(6, n_tracks=0)):
        tf = tpcgen.generate(cfg)
        with lib.Reconstructor.for_timeframe(tf) as R:
            t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
            R.wait(t)
            cl = lib.tpc_get_clusters(R.ctx, t)
            tr, _ = lib.tpc_get_tracks(R.ctx, t, len(cl))
            assert len(tr) == 0
            assert lib.tpc_compress_clusters(R.ctx, t) == (0, 0)
            cy, cz, st = lib.tpc_get_compressed(R.ctx, t, len(cl))
            assert len(st) == len(cl) and not np.any(st)
            assert lib.tpc_calibrate_drift(R.ctx, t, 750.0) == (0.0, 0.0, 0.0, 0)
            lib.tpc_release(R.ctx, t)
