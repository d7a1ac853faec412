"""Parity of the track-model compression (step 10) with the oracle.  The codes
are rounded float residuals to the FP32 (GPU) or FP64 (oracle) track model: a
code may differ only where the oracle's residual, in steps, lies within
DELTA = 0.1 step of a rounding boundary (a half-integer), and then by one
step; a status (coded or escaped) only where it lies within DELTA of the
+-127.5 escape bound.  On full_tpc the differing codes lie at most 1.7e-3 step
(y) and 3.8e-2 step (zeta: the prediction carries tgl times the arc, up to
~250 cm) from their boundaries; on 2,000 bins of the continuous timeframe
(zeta up to 1,000 cm) 5.3e-4 and 9.0e-2 step.  DELTA still fails any code
computed from a wrong prediction."""
import numpy as np
import pytest

import oracle
import tpcgen

DELTA = 0.1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


@pytest.mark.parametrize("make", [lambda: tpcgen.full_tpc(1),
                                  lambda: tpcgen.continuous_tf(3, n_time_bins=2000, n_sectors=2)],
                         ids=["full_tpc", "continuous_pileup"])
def test_compression_parity(lib, make):
    """full_tpc, and overlapping collisions of the continuous timeframe (2,000
    bins, two sectors: zeta up to twice full_tpc's)."""
    tf = tpcgen.generate(make())
    orc = oracle.reconstruct(tf)
    ocy, ocz, ost, qy, qz = oracle.compress(tf, orc, quotients=True)
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

    def to_boundary(q):
        """Distance (in steps) of the unrounded residual from the nearest half-integer."""
        return np.abs(np.abs(q - np.floor(q)) - 0.5)

    # statuses: a difference needs a residual within DELTA of the escape bound
    sd = np.nonzero(st != ost)[0]
    near_escape = (np.abs(np.abs(qy[sd]) - 127.5) <= DELTA) | (np.abs(np.abs(qz[sd]) - 127.5) <= DELTA)
    assert np.all(near_escape), sd[~near_escape][:10]
    both = (st == 1) & (ost == 1)
    dy = cy[both].astype(int) - ocy[both]
    dz = cz[both].astype(int) - ocz[both]
    assert np.abs(dy).max(initial=0) <= 1 and np.abs(dz).max(initial=0) <= 1
    by, bz = to_boundary(qy[both]), to_boundary(qz[both])
    worst_y = float(by[dy != 0].max(initial=0.0))
    worst_z = float(bz[dz != 0].max(initial=0.0))
    print(f"clusters on tracks {int((ost > 0).sum())}, coded {n_coded}, escaped {n_esc}; statuses differ {len(sd)}; "
          f"codes differ y {np.mean(dy != 0):.2e} z {np.mean(dz != 0):.2e}; farthest differing code from its "
          f"boundary y {worst_y:.2e} z {worst_z:.2e} step; within DELTA of a boundary y {np.mean(by <= DELTA):.2e} "
          f"z {np.mean(bz <= DELTA):.2e}")
    assert worst_y <= DELTA and worst_z <= DELTA


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
