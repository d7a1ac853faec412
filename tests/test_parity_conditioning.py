"""The conditioning check of the fit comparison (tests/parity.py): the step
by step replay of the oracle's fit reproduces the oracle, rounding the
quantities the FP32 fit stores moves a single-particle track's FP64 answer by
less than the plain 1e-4 bar (so the check cannot loosen the comparison of
such tracks), and moves the answer of a track built from several particles at
50 kHz pile-up by more than the bar."""
import numpy as np
import pytest

import oracle
import tpcgen
from parity import PAR_FLOORS, PAR_RTOL, perturbation_spread


def test_single_particle_tracks_stay_within_the_bar():
    tf = tpcgen.generate(tpcgen.single_sector(1, n_tracks=60))
    res = oracle.reconstruct(tf)
    X, Y, Z = oracle.coords(tf, res.clusters)
    cl2trk = np.asarray(res.cl2trk)
    n_checked = 0
    for t in range(min(len(res.fits), 25)):
        o = res.fits[t]
        if o["flags"] or o["chi2"] > 3 * o["ndf"]:
            continue
        m = np.nonzero(cl2trk == t)[0]
        dpar, _ = perturbation_spread(X[m], Y[m], Z[m], o["par"])   # asserts the replay equals the oracle
        assert np.all(dpar < PAR_RTOL * np.maximum(np.abs(o["par"]), PAR_FLOORS)), (t, dpar)
        n_checked += 1
    assert n_checked >= 10


@pytest.mark.slow
def test_pileup_track_beyond_the_bar():
    """Sector 25 of the 11,000-bin continuous timeframe of seed 2: the track
    whose lowest cluster is the sector's cluster 61,737 (20 clusters, chi2/ndf
    ~1,270) moves by more than 1e-4 of snp under FP32-sized rounding."""
    tf = tpcgen.generate(tpcgen.continuous_tf(2, n_time_bins=11000))
    sec = tpcgen.sector_slice(tf, 25)
    res = oracle.reconstruct(sec)
    t = int(np.nonzero(np.asarray(res.track_first) == 61737)[0][0])
    o = res.fits[t]
    assert o["chi2"] / o["ndf"] > 1000
    m = np.nonzero(np.asarray(res.cl2trk) == t)[0]
    X, Y, Z = oracle.coords(sec, res.clusters[m])
    dpar, _ = perturbation_spread(X, Y, Z, o["par"])
    assert dpar[2] > 2 * PAR_RTOL * max(abs(o["par"][2]), PAR_FLOORS[2])
