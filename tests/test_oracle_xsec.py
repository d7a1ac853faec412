"""Pins of the oracle's cross-sector merge (step 9): the rotation of a track
state between sector frames against its exact map, the multi-frame fit against
an exact helix crossing a sector border, the matching chi2 of two pieces of one
helix, and the links on a generated timeframe against the generator truth."""
import math

import numpy as np
import pytest

import oracle
import tpcgen

KFAC = -0.5 * 0.299792458e-2      # curvature per unit q/pT, 1/cm per 1/GeV
A0, A1 = oracle.sector_alpha(0), oracle.sector_alpha(1)


def test_rotation_round_trip():
    s = np.array([12.3, -40.0, 0.31, 0.7, -1.8])
    s1, x1, _ = oracle.rotate(s, 150.0, A1 - A0)
    s2, x2, _ = oracle.rotate(s1, x1, A0 - A1)
    assert x2 == pytest.approx(150.0, abs=1e-12)
    assert np.allclose(s2, s, rtol=0, atol=1e-12)


@pytest.mark.parametrize("state,x,delta", [([12.3, -40.0, 0.31, 0.7, -1.8], 150.0, math.radians(20)),
                                           ([-20.0, 10.0, -0.2, -0.3, 3.0], 220.0, math.radians(-20)),
                                           ([0.5, 0.0, 0.6, 0.0, 0.4], 90.0, math.radians(20))])
def test_rotation_jacobian_is_the_derivative_of_the_exact_map(state, x, delta):
    """R = d(state at the fixed rotated reference x'0) / d(state): rotate the
    perturbed state exactly, then carry it along its helix back to x'0."""
    s0 = np.array(state, float)
    r0, xr0, R = oracle.rotate(s0, x, delta)

    def exact(s):
        r, xr, _ = oracle.rotate(s, x, delta)
        out, _ = oracle.transport(r, xr0 - xr)
        return out

    h = 1e-6
    num = np.zeros((5, 5))
    for j in range(5):
        dp = np.zeros(5)
        dp[j] = h
        num[:, j] = (exact(s0 + dp) - exact(s0 - dp)) / (2 * h)
    assert np.allclose(num, R, rtol=0, atol=2e-7)


def helix_in_frames(y0, z0, phi0, tgl, qpt, rows_x):
    """Crossings of an exact helix, started at row 0 of sector 0 (local y0,
    direction phi0), with the row planes: in sector 0 while the crossing lies
    in sector 0's wedge, then in sector 1.  Returns x, y (local), z, alpha."""
    k = KFAC * qpt
    ca, sa = math.cos(A0), math.sin(A0)
    P0 = np.array([rows_x[0] * ca - y0 * sa, rows_x[0] * sa + y0 * ca])
    F0 = A0 + phi0

    def point(s):
        F = F0 + k * s
        return P0 + np.array([(math.sin(F) - math.sin(F0)) / k, -(math.cos(F) - math.cos(F0)) / k])

    def local(P, a):
        return P[0] * math.cos(a) + P[1] * math.sin(a), -P[0] * math.sin(a) + P[1] * math.cos(a)

    out = []
    for X in rows_x:
        for a in (A0, A1):
            lo, hi = 0.0, 400.0
            if local(point(hi), a)[0] < X:
                continue
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if local(point(mid), a)[0] < X:
                    lo = mid
                else:
                    hi = mid
            s = 0.5 * (lo + hi)
            xl, yl = local(point(s), a)
            if abs(yl) <= xl * math.tan(math.radians(10.0)):
                out.append((X, yl, z0 + tgl * s, a))
                break
    arr = np.array(out)
    return arr[:, 0], arr[:, 1], arr[:, 2], arr[:, 3]


@pytest.fixture(scope="module")
def crossing():
    rows_x = tpcgen.default_geometry()[1] * 0.05
    y0, z0, phi0, tgl, qpt = 12.0, 30.0, 0.15, -0.4, -2.0
    x, y, z, al = helix_in_frames(y0, z0, phi0, tgl, qpt, rows_x)
    n0 = int(np.sum(al == A0))
    assert n0 >= 10 and len(x) - n0 >= 10, "the helix must cross into the next sector"
    assert np.all(al[:n0] == A0) and np.all(al[n0:] == A1)
    return (x, y, z, al, n0), np.array([y0, z0, math.sin(phi0), tgl, qpt])


def test_multi_frame_fit_exact_helix_closure(crossing):
    (x, y, z, al, n0), want = crossing
    f = oracle.fit_points_xs(x, y, z, al)
    floors = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
    assert f["x"] == pytest.approx(x[0], abs=1e-9)
    assert np.all(np.abs(f["par"] - want) <= 1e-8 * np.maximum(np.abs(want), floors)), (f["par"], want)
    assert f["chi2"] < 1e-10 and f["flags"] == 0 and f["ndf"] == 2 * len(x) - 5


def test_matching_chi2_of_two_pieces_of_one_helix(crossing):
    (x, y, z, al, n0), _ = crossing
    fa = oracle.fit_points(x[:n0], y[:n0], z[:n0])
    fb = oracle.fit_points(x[n0:], y[n0:], z[n0:])
    assert oracle.xs_chi2(fa, A0, fb, A1) < 1e-6
    fb_off = oracle.fit_points(x[n0:], y[n0:] + 0.5, z[n0:])   # a different track, 5 mm away
    assert oracle.xs_chi2(fa, A0, fb_off, A1) > 100.0


def test_cross_sector_links_against_generator_truth():
    """Generator truth (not a parity pin): links join pieces of one generated
    track, and many tracks crossing a border are joined."""
    tf = tpcgen.generate(tpcgen.full_tpc(1))
    r = oracle.reconstruct(tf)
    x = oracle.merge_sectors(tf, r)
    planes = oracle.decode_all(tf)
    lab = np.full(planes.shape, -1, np.int32)
    lab[np.nonzero(planes)] = tf.digit_labels
    cl = r.clusters
    cl_lab = lab[cl["sector"], cl["row"], cl["t_peak"], cl["pad_peak"]]
    track_lab = np.full(len(r.fits), -2)
    for k in range(len(r.fits)):
        v, c = np.unique(cl_lab[r.cl2trk == k], return_counts=True)
        j = int(np.argmax(c))
        if c[j] >= 0.9 * c.sum():
            track_lab[k] = v[j]
    a = np.nonzero(x.link >= 0)[0]
    b = x.link[a]
    same = (track_lab[a] == track_lab[b]) & (track_lab[a] >= 0)
    assert len(a) > 2000 and same.mean() >= 0.98
    # the merged tracks partition the step-8 tracks
    assert x.npieces.sum() == len(r.fits) and len(x.fits) == len(r.fits) - len(a)
    assert np.array_equal(np.bincount(x.cl2trk[x.cl2trk >= 0], minlength=len(x.fits)), x.ncl)
