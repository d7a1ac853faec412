"""The scale behind the fit tolerance's sigma term.

The GPU fit is FP32; the oracle's is FP64 on the same integer measurements.
For most parameters the plain bar 1e-4 * max(|p|, floor) is far above what
FP32 rounding does.  q/pT of a short track is the exception: with 10-12
clusters its sigma is ~1 1/GeV, ten times the 0.1 1/GeV floor, so the estimate
is a large multiple of the measurements' sub-micron rounding.  This test
perturbs each measurement of such tracks by one FP32 rounding of its row step
(2^-24 of the step) and refits in FP64: the answer moves by up to a few 1e-6
1/GeV, a few 1e-6 sigma, the order of the 2e-5 sigma the GPU comparison allows
(the FP32 fit takes several roundings per step)."""
import numpy as np

import oracle
import tpcgen

U = 7.8125e-4
DIAG = [0, 2, 5, 9, 14]


def test_one_rounding_per_step_moves_short_tracks_q_over_pt():
    tf = tpcgen.sector_prefix(tpcgen.generate(tpcgen.full_tpc(1)), 6)
    orc = oracle.reconstruct(tf)
    X, Y, Z = oracle.coords(tf, orc.clusters)
    sig = np.sqrt(orc.fits["cov"][:, DIAG])
    short = np.nonzero((sig[:, 4] > 1.0) & (orc.fits["flags"] == 0))[0]
    assert len(short) > 100
    order = np.argsort(orc.cl2trk, kind="stable")
    starts = np.searchsorted(orc.cl2trk[order], np.arange(len(orc.track_first) + 1))
    rng = np.random.default_rng(5)
    moved = []
    for t in short[:150]:
        idx = order[starts[t]:starts[t + 1]]
        x = X[idx] * U
        y = (Y[idx] - Y[idx[0]]) * U
        z = (Z[idx] - Z[idx[0]]) * U
        f0 = oracle.fit_points(x, y, z)
        step_y = np.maximum(np.abs(np.diff(y, prepend=y[0])), 1e-3)
        step_z = np.maximum(np.abs(np.diff(z, prepend=z[0])), 1e-3)
        dq = 0.0
        for _ in range(8):
            f1 = oracle.fit_points(x, y + rng.uniform(-1, 1, len(y)) * 2.0 ** -24 * step_y,
                                   z + rng.uniform(-1, 1, len(z)) * 2.0 ** -24 * step_z)
            dq = max(dq, abs(f1["par"][4] - f0["par"][4]))
        moved.append((dq, dq / sig[t, 4]))
    dq, in_sigma = np.array(moved).T
    # the exact answer itself is uncertain at this level ...
    assert dq.max() > 1e-6 and in_sigma.max() > 1e-6
    # ... which the sigma term (2e-5 sigma) covers several times over
    assert in_sigma.max() < 2e-5
