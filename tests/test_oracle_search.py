"""The oracle's windowed candidate search (the default) gives exactly what the
plain scan over every candidate gives (search_all = True).

The CA window and the merge's row / time band only skip candidates that a
bound proves would fail the window or residual test, and both searches visit
the rest in the definition's order, so links, chains, ties and merges must be
identical.  Checked on generated timeframes (sparse, dense pile-up, continuous
readout, ragged) and on hand-placed clusters crowded around the bounds."""
import numpy as np
import pytest

import oracle
import tpcgen
from synth import Geom, make_clusters


def both(tf, cl):
    out = []
    for full in (False, True):
        p = oracle.OracleParams(search_all=full)
        up, down, chain = oracle.ca(tf, cl, p)
        cl2trk, first, ncl, passes = oracle.merge(tf, cl, up, down, chain, p)
        out.append((up, down, chain, cl2trk, np.asarray(first), np.asarray(ncl), passes))
    return out


def assert_same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("cfg", [
    lambda: tpcgen.single_sector(1),
    lambda: tpcgen.single_sector(8, n_tracks=3000),
    lambda: tpcgen.continuous_tf(2, n_time_bins=2000, n_sectors=2),
    lambda: tpcgen.single_sector(5, n_tracks=60, n_time_bins=257, coll_t0=[-243.0]),
], ids=["sector", "dense", "continuous", "ragged"])
def test_windowed_search_equals_full_scan_on_generated(cfg):
    tf = tpcgen.generate(cfg())
    cl = oracle.find_clusters(tf)
    a, b = both(tf, cl)
    assert_same(a, b)
    assert int((a[2] >= 0).sum()) > 0


def test_windowed_search_equals_full_scan_at_the_bounds():
    """Clusters on rows 30-40 crowded in y (+-600 u) and in time around each
    other within and just beyond the CA window (about +-4 bins for dX = 960 u:
    (1.1 * 960 + 2560) / 640 + 1), with centroids anywhere in their 5x5 window
    (|Z - 640 t_peak| up to 1280 u); many pairs pass, many fail near the
    bounds, and chains end and restart inside the merge band."""
    rng = np.random.default_rng(11)
    g = Geom(n_sectors=1, n_time_bins=1000)
    pts = []
    for r in range(30, 41):
        for _ in range(60):
            t = int(rng.integers(395, 406))
            Z = (640 * t + int(rng.integers(-256, 257)) * 5)
            pts.append((0, r, int(rng.integers(-300, 301)) * 2, Z))
    cl, _ = make_clusters(g, pts)
    a, b = both(g, cl)
    assert_same(a, b)
    # the window is not vacuous here: some candidate pairs were accepted
    assert int((a[0] >= 0).sum()) > 20


def steep_track(rows, Y0, Z0, dy, dz, R_even, R_odd):
    """Clusters along a straight line (dY, dZ per row) whose time centroids sit
    R/128 bins from their peak bins, alternating between R_even and R_odd."""
    return [(0, r, Y0 + dy * (r - rows[0]), Z0 + dz * (r - rows[0]), R_even if r % 2 == 0 else R_odd)
            for r in rows]


def test_windowed_search_reaches_its_bounds():
    """Tracks with dZ = 640 u per row (dX = 960 u, slope 0.67 < 1.1) whose
    centroids alternate 2 bins before and after their peak bins: consecutive
    peaks are 5 bins apart, the widest the CA window must admit.  A second
    track is broken after row 45 and restarts at row 49 with its peaks 2 bins
    off its centroids, so the merge must look up to 2 bins beyond the
    extrapolated time (plus the residual cut) for the bottom end; a third one
    does the same with the restart's peak 2 bins late instead of early."""
    g = Geom(n_sectors=1, n_time_bins=1000)
    Z0 = 640 * 300
    pts = steep_track(range(30, 60), -4000, Z0, 40, 640, -256, 256)
    pts += steep_track(range(30, 46), 4000, Z0, -40, 640, 256, -256)
    pts += [(0, r, 4000 - 40 * (r - 30), Z0 + 640 * (r - 30), -256 if r % 2 else 256) for r in range(49, 70)]
    # the same with the opposite centroid offsets: the restart's peak lies late
    pts += steep_track(range(30, 46), 12000, Z0, 0, 640, -256, 256)
    pts += [(0, r, 12000, Z0 + 640 * (r - 30), 256 if r % 2 else -256) for r in range(49, 70)]
    cl, order = make_clusters(g, pts)
    inv = np.argsort(order)
    t = cl["t_peak"].astype(int)
    a, b = both(g, cl)
    assert_same(a, b)
    up, down, chain, cl2trk, first, ncl, passes = a
    # the first track is one chain over rows 31-58, with 5-bin steps between peaks
    first_track = inv[:30]
    assert np.all(chain[first_track[1:-1]] == first_track[1])
    assert np.abs(np.diff(t[first_track])).max() == 5
    # the broken one is merged back across its gap: one track of both chains
    assert passes >= 1 and len(set(cl2trk[inv[31:45]]) | set(cl2trk[inv[47:66]])) == 1
    assert len(set(cl2trk[inv[68:82]]) | set(cl2trk[inv[84:103]])) == 1 and cl2trk[inv[68]] >= 0
    # the restarts' bottom clusters (row 50) have peaks 2 bins before / after their centroids
    z = oracle.coords(g, cl)[2]
    assert (640 * t[inv[47]] - z[inv[47]], 640 * t[inv[84]] - z[inv[84]]) == (-1280, 1280)
