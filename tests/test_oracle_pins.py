"""Pins of the CPU oracle against facts that do not come from the oracle itself:
an independent re-encoder (ZS round trip), a 3x3 maximum filter (peaks),
closed-form centroids and variances, hand-placed CA / merge geometries, exact
helix closure, finite differences, the information form of the Kalman update,
and pull statistics.  A plausible slip in the oracle (a dropped term, a sign, a
transposed index) breaks at least one of these."""
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle
import tpcgen
from synth import Geom, U_CM, encode_planes, helix_points, make_clusters


# ---------------------------------------------------------------- geometry
def test_geometry_closed_forms():
    npads, row_x = tpcgen.default_geometry()
    assert len(npads) == 152 and npads[0] == 66 and npads[-1] == 138
    assert int(npads.sum()) == 15429 and 36 * int(npads.sum()) == 555444
    assert row_x[0] * 0.05 == pytest.approx(84.85)
    d = np.diff(row_x)
    assert set(d[:63]) == {15} and set(d[63:97]) == {20} and set(d[97:127]) == {24}
    assert set(d[127:]) == {30}


# ---------------------------------------------------------------- ZS
def test_zs_round_trip():
    cfg = tpcgen.single_sector(3, n_tracks=20, n_time_bins=300)
    tf = tpcgen.generate(cfg)
    planes = oracle.decode_all(tf)
    assert int((planes > 0).sum()) == tf.n_digits == len(tf.digit_labels)
    assert planes.max() <= 1023 and planes[planes > 0].min() >= 3
    pages, offs = encode_planes(planes, tf.n_time_bins)
    assert np.array_equal(offs, tf.page_offsets)
    assert np.array_equal(pages, tf.pages)


def test_zs_corrupt_pages_rejected(c1_tf):
    tf = c1_tf
    oracle.decode_all(tf)  # clean input decodes
    for off_in_page, val in [(14, 0x00), (6, 0xFF), (4, 0xFF), (32, 0xFF)]:
        bad = tf.pages.copy()
        # page of (0, 40, 1): pick one that has entries
        k = 40 * 2 + 1
        o = int(tf.page_offsets[k])
        assert bad[o + 4] > 0
        bad[o + off_in_page] = val
        import copy
        t2 = copy.copy(tf)
        t2.pages = bad
        with pytest.raises(oracle.CorruptPage):
            oracle.decode_all(t2)


# ---------------------------------------------------------------- peaks
def _peaks_by_maxfilter(plane, qmin):
    """A pixel is a peak iff its unique key q*BIG - linear_index is the maximum
    of its 3x3 neighbourhood (zero outside the plane) and q >= qmin."""
    T, P = plane.shape
    lin = np.arange(T * P, dtype=np.int64).reshape(T, P)
    big = T * P + 1
    key = plane.astype(np.int64) * big - lin
    key[plane == 0] = -lin[plane == 0]  # q = 0 pixels never beat a q >= qmin pixel
    m = ndimage.maximum_filter(key, size=3, mode="constant", cval=np.iinfo(np.int64).min)
    return (key == m) & (plane >= qmin)


@pytest.mark.parametrize("seed", range(6))
def test_peaks_match_max_filter(seed):
    rng = np.random.default_rng(seed)
    T, P = 16, 8
    # few distinct levels -> many exact ties and plateaus
    plane = rng.choice([0, 0, 3, 9, 10, 10, 11, 12, 40], size=(T, P)).astype(np.uint16)
    if seed == 0:
        plane[:] = 10  # one big plateau: only the lowest index is a peak
    got = oracle.peaks_plane(plane, 10)
    want = _peaks_by_maxfilter(plane, 10)
    assert np.array_equal(got, want)
    # no two peaks are 8-neighbours
    pk = np.argwhere(got)
    for a in range(len(pk)):
        for b in range(a + 1, len(pk)):
            assert np.max(np.abs(pk[a] - pk[b])) > 1
    if seed == 0:
        # every other pixel has a lower-index neighbour of equal charge
        assert got.sum() == 1 and got[0, 0]


def test_plateau_resolves_to_lowest_index():
    plane = np.zeros((5, 6), np.uint16)
    plane[2, 2] = plane[2, 3] = 50
    got = oracle.peaks_plane(plane, 10)
    assert got[2, 2] and not got[2, 3]
    plane[2, 3] = 0
    plane[3, 2] = 50  # same pad, later time: earlier time wins
    got = oracle.peaks_plane(plane, 10)
    assert got[2, 2] and not got[3, 2]


# ---------------------------------------------------------------- clusters
def test_cluster_symmetric_cloud_exact():
    T, P = 20, 12
    plane = np.zeros((T, P), np.uint16)
    t0, p0 = 9, 5
    w = {0: 100, 1: 40, 2: 6}
    for dt in range(-2, 3):
        for dp in range(-2, 3):
            plane[t0 + dt, p0 + dp] = w[abs(dt)] * w[abs(dp)] // 100
    c = oracle.cluster_at(plane, p0, t0)
    assert c["pad_fp"] == 256 * p0
    assert c["time_fp"] == 128 * (t0 + 4)
    assert c["qmax"] == 100
    Q = int(plane.sum())
    assert c["qtot"] == Q
    # closed-form variance of the symmetric weights, 16 * sum q d^2 / Q rounded half up
    var_p = sum(int(plane[t, p]) * (p - p0) ** 2 for t in range(T) for p in range(P)) / Q
    assert c["sigma2_pad"] == math.floor(16 * var_p + 0.5)
    assert c["flags"] == 0


def test_cluster_two_equal_pixels_half_pad():
    plane = np.zeros((10, 10), np.uint16)
    plane[4, 4] = plane[4, 5] = 30
    c = oracle.cluster_at(plane, 4, 4)
    assert c["pad_fp"] == 256 * 4 + 128          # centroid at pad 4.5
    assert c["time_fp"] == 128 * (4 + 4)
    assert c["sigma2_pad"] == 4                  # variance 1/4 -> 16 * 0.25
    assert c["sigma2_time"] == 0


def test_cluster_uniform_3x3_variance():
    plane = np.zeros((10, 10), np.uint16)
    plane[3:6, 3:6] = 20
    plane[4, 4] = 21
    c = oracle.cluster_at(plane, 4, 4)
    # variance of a uniform 3-point set {-1, 0, 1} is 2/3 (perturbed by the +1 at the centre)
    Q = 9 * 20 + 1
    var = 6 * 20 / Q
    assert c["sigma2_pad"] == math.floor(16 * var + 0.5) == c["sigma2_time"]


def test_cluster_outer_rule_and_flags():
    plane = np.zeros((12, 12), np.uint16)
    plane[5, 5] = 100
    plane[5, 6] = 30
    plane[5, 7] = 50     # outer pixel larger than its inner neighbour: excluded
    plane[5, 3] = 20     # outer pixel with an empty inner neighbour (5,4): excluded
    base = plane.copy()
    base[5, 7] = 0
    base[5, 3] = 0
    c = oracle.cluster_at(plane, 5, 5)
    c0 = oracle.cluster_at(base, 5, 5)
    assert c["pad_fp"] == c0["pad_fp"] and c["qtot"] == c0["qtot"] == 130
    assert c["flags"] & 2 and not c0["flags"] & 2
    # an included outer pixel (<= its inner neighbour) moves the centroid
    plane2 = base.copy()
    plane2[5, 7] = 30
    c2 = oracle.cluster_at(plane2, 5, 5)
    assert c2["qtot"] == 160 and c2["pad_fp"] == 256 * 5 + math.floor((2 * 256 * 90 + 160) / 320)
    # another peak inside the 5x5 window
    plane3 = base.copy()
    plane3[7, 7] = 60
    assert oracle.cluster_at(plane3, 5, 5)["flags"] & 4
    # edge pad
    plane4 = np.zeros((12, 12), np.uint16)
    plane4[5, 0] = 40
    assert oracle.cluster_at(plane4, 0, 5)["flags"] & 1


def test_cluster_gaussian_centroid_bound():
    """Noise-free Gaussian cloud (sigma 0.8 pad x 1.0 bin, peak density ~1000 ADC)
    off-centre: the centroid lies within the computed bound of the true centre."""
    from scipy.special import erf
    sp, st = 0.8, 1.0
    for (pc, tc) in [(6.3, 7.8), (6.45, 8.1), (5.9, 7.6)]:
        P, T = 14, 18
        pe = np.arange(P + 1) - 0.5
        te = np.arange(T + 1) - 0.5
        fp = 0.5 * np.diff(erf((pe - pc) / (sp * math.sqrt(2))))
        ft = 0.5 * np.diff(erf((te - tc) / (st * math.sqrt(2))))
        A = 1000 * 2 * math.pi * sp * st
        qc = A * np.outer(ft, fp)                  # continuous-model pixel charges
        q = np.rint(qc).astype(np.int64)
        plane = np.clip(q, 0, 1023).astype(np.uint16)
        t_pk, p_pk = np.unravel_index(np.argmax(plane), plane.shape)
        c = oracle.cluster_at(plane, int(p_pk), int(t_pk))
        pad = c["pad_fp"] / 256.0
        tim = c["time_fp"] / 128.0 - 4
        Q = float(c["qtot"])
        tt, pp = np.meshgrid(np.arange(T) - t_pk, np.arange(P) - p_pk, indexing="ij")
        inside = (np.abs(tt) <= 2) & (np.abs(pp) <= 2)
        # bound per axis: charge left outside the 5x5 times its lever arm, pixel
        # rounding (0.5 ADC per pixel) times its lever arm, and the output quantum
        for (est, true, d, quantum) in [(pad, pc, pp, 1 / 512), (tim, tc, tt, 1 / 256)]:
            bound = ((qc[~inside] * np.abs(d[~inside])).sum()
                     + 0.5 * np.abs(d[inside]).sum()) / Q + quantum
            assert abs(est - true) <= bound < 0.1, (est, true, bound)


# ---------------------------------------------------------------- CA
def _straight_track(geom, s, rows, y0, z0, sy, sz):
    X = 64 * geom.row_x.astype(np.int64)
    pts = []
    for r in rows:
        dx = X[r] - X[rows[0]]
        Y = int(round((y0 + sy * dx) / 2)) * 2
        Z = int(round((z0 + sz * dx) / 5)) * 5
        pts.append((s, r, Y, Z))
    return pts


def test_ca_single_straight_track_one_chain():
    g = Geom(n_sectors=1, n_time_bins=1000)
    pts = _straight_track(g, 0, list(range(152)), 0, 5 * 128 * 500, 0.1, -0.3)
    cl, _ = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    n = len(cl)
    assert np.array_equal(up[:-1], np.arange(1, n)) and up[-1] == -1
    assert np.array_equal(down[1:], np.arange(0, n - 1)) and down[0] == -1
    assert np.all(chain == 0)
    cl2trk, first, ncl, passes = oracle.merge(g, cl, up, down, chain)
    assert list(ncl) == [152] and np.all(cl2trk == 0)


def test_ca_two_tracks_and_noise_paths_disjoint():
    g = Geom(n_sectors=1, n_time_bins=1000)
    rng = np.random.default_rng(5)
    pts = _straight_track(g, 0, list(range(152)), -3000, 5 * 128 * 300, 0.05, 0.2)
    pts += _straight_track(g, 0, list(range(152)), 3000, 5 * 128 * 600, -0.05, -0.2)
    for _ in range(300):
        r = int(rng.integers(0, 152))
        pts.append((0, r, int(rng.integers(-8000, 8000)) * 2, int(rng.integers(5 * 128 * 200, 5 * 128 * 800)) // 5 * 5))
    cl, _ = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    # accepted links form vertex-disjoint paths
    n = len(cl)
    acc_up = np.array([up[c] if up[c] >= 0 and down[up[c]] == c else -1 for c in range(n)])
    tgt = acc_up[acc_up >= 0]
    assert len(np.unique(tgt)) == len(tgt)
    # the two clean tracks survive as the two longest chains
    ids, cnt = np.unique(chain[chain >= 0], return_counts=True)
    assert sorted(cnt)[-2:] == [152, 152]


def test_ca_hand_worked_example():
    """Rows 10, 11, 12 of one sector.  Row 11 holds c at (Y, Z) = (0, 0); row 10
    holds d1 on the straight line and d2 off it; row 12 holds u1 on the line and u2
    slightly off.  dX = 64 * 15 = 960 u between these rows.
    d1 = (-96, -480): slope 0.1 / -0.5; u1 = (96, 480); u2 = (96 + 20, 480).
    Pair (d1, u1): dev = 0 -> score 0, the best.  The deviation of (d1, u2):
    dev_Y = 116*960 - 96*960 = 19200, |dev_Y| <= 256*1920 -> accepted, score 19200^2.
    d2 = (-96 + 600, -480) violates nothing in the window (|dY|=504 <= 960) but
    its deviations are 600*960 = 576000 > 491520 = 256*1920 -> rejected."""
    g = Geom(n_sectors=1, n_time_bins=1000)
    base = 5 * 128 * 400
    pts = [(0, 11, 0, base), (0, 10, -96, base - 480), (0, 10, -96 + 600, base - 480),
           (0, 12, 96, base + 480), (0, 12, 116, base + 480)]
    cl, order = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    inv = np.argsort(order)
    c, d1, d2, u1, u2 = (inv[i] for i in range(5))
    assert up[c] == u1 and down[c] == d1
    # row 10 is not an edge row: its clusters have no rows below -> (-1,-1)
    assert up[d1] == -1 and down[d1] == -1
    # without u1, c pairs with u2 (accepted, score > 0)
    cl2, order2 = make_clusters(g, [pts[i] for i in (0, 1, 2, 4)])
    up2, down2, _ = oracle.ca(g, cl2)
    inv2 = np.argsort(order2)
    assert up2[inv2[0]] == inv2[3] and down2[inv2[0]] == inv2[1]
    # without d1 nothing is accepted (d2 is off the line by 0.47 cm)
    cl3, order3 = make_clusters(g, [pts[i] for i in (0, 2, 3, 4)])
    up3, down3, _ = oracle.ca(g, cl3)
    inv3 = np.argsort(order3)
    assert up3[inv3[0]] == -1 and down3[inv3[0]] == -1


def test_ca_edge_rows():
    g = Geom(n_sectors=1, n_time_bins=1000)
    pts = _straight_track(g, 0, list(range(0, 6)), 0, 5 * 128 * 400, 0.0, 0.0)
    pts += _straight_track(g, 0, list(range(146, 152)), 0, 5 * 128 * 400, 0.0, 0.0)
    cl, _ = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    assert up[0] == 1 and down[0] == -1            # row 0 linked from row 1's down
    assert down[11] == 10 and up[11] == -1         # row 151 mirrors it
    # a segment's inner end (rows 5 and 146 here) has no (down, up) pair, so it
    # keeps no link: the chains are rows 0-4 and 147-151
    assert np.all(chain == np.array([0] * 5 + [-1, -1] + [7] * 5))


# ---------------------------------------------------------------- merge
@pytest.mark.parametrize("missing,expect_one", [(0, True), (1, True), (2, True), (3, True),
                                                (4, False)])
def test_merge_closes_gaps(missing, expect_one):
    """A clean straight track with `missing` rows removed.  The CA drops the two
    clusters next to the hole (an end cluster has no (down, up) pair), so the
    chains end at rows 58 and 61 + missing: gap = missing + 3 rows (missing = 0 is
    a break of the link itself, planted by moving one cluster off the line)."""
    g = Geom(n_sectors=1, n_time_bins=1000)
    rows = list(range(20, 60)) + list(range(60 + missing, 100))
    pts = _straight_track(g, 0, rows, 100, 5 * 128 * 400, 0.2, -0.15)
    if missing == 0:
        # push row 60 off the line by 0.5 cm: rows 59 and 61 lose their pair too
        pts = [(s_, r, Y + (640 if r == 60 else 0), Z) for (s_, r, Y, Z) in pts]
    cl, _ = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    ids, cnt = np.unique(chain[chain >= 0], return_counts=True)
    assert len(ids) == 2
    cl2trk, first, ncl, passes = oracle.merge(g, cl, up, down, chain)
    if expect_one:
        assert list(ncl) == [int(cnt.sum())] and passes == 1
    else:
        assert sorted(ncl) == sorted(cnt) and passes == 0


def test_merge_rejects_offset_segment():
    g = Geom(n_sectors=1, n_time_bins=1000)
    pts = _straight_track(g, 0, list(range(20, 60)), 100, 5 * 128 * 400, 0.2, -0.15)
    upper = _straight_track(g, 0, list(range(61, 100)), 100, 5 * 128 * 400, 0.2, -0.15)
    upper = [(s, r, Y + 2 * 300, Z) for (s, r, Y, Z) in upper]  # 0.47 cm off in y
    cl, _ = make_clusters(g, pts + upper)
    up, down, chain = oracle.ca(g, cl)
    _, cnt = np.unique(chain[chain >= 0], return_counts=True)
    _, _, ncl, passes = oracle.merge(g, cl, up, down, chain)
    assert len(cnt) == 2 and sorted(ncl) == sorted(cnt) and passes == 0


# ---------------------------------------------------------------- fit
def _rows_x():
    _, row_x = tpcgen.default_geometry()
    return row_x * 0.05


@pytest.mark.parametrize("qpt,phi0,tgl", [(1.0 / 0.5, 0.1, -0.5), (-1 / 0.3, -0.2, 0.8),
                                          (1 / 2.0, 0.35, -0.05), (-1 / 0.15, 0.05, 0.3),
                                          (1e-4, 0.0, 0.0)])
def test_fit_exact_helix_closure(qpt, phi0, tgl):
    x = _rows_x()
    k = -0.5 * 0.299792458e-2 * qpt
    x = x[np.abs(np.sin(phi0) + k * (x - x[0])) < 0.9]   # rows the helix reaches
    assert len(x) >= 40
    y0, z0 = 1.5, 40.0
    y, z = helix_points(x, y0, z0, phi0, tgl, qpt)
    f = oracle.fit_points(x, y, z)
    want = np.array([y0, z0, math.sin(phi0), tgl, qpt])
    floors = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
    assert f["x"] == x[0]
    assert np.all(np.abs(f["par"] - want) <= 1e-9 * np.maximum(np.abs(want), floors))
    assert f["chi2"] < 1e-12 and f["ndf"] == 2 * len(x) - 5 and f["flags"] == 0


def test_fit_sign_conventions_against_generator_truth():
    """A positive track in +Bz bends towards -y (F = q v x B), and tgl_zeta on
    side A is -tan(lambda): zeta decreases as |z| grows.  Checked against the
    generator's own helix (global frame) for a seeded single-sector event."""
    tf = tpcgen.generate(tpcgen.single_sector(7, n_tracks=40))
    h = tf.hits
    for tid in range(len(tf.tracks)):
        hh = h[(h["track"] == tid) & (h["leg"] == 0)]
        if len(hh) < 100 or len(np.unique(hh["row"])) != len(hh):
            continue
        hh = np.sort(hh, order="row")
        x = tf.row_x[hh["row"]] * 0.05
        y = (hh["pad"] - 0.5 * (tf.npads[hh["row"]] - 1)) * 0.4
        z = hh["time"] * 0.5
        f = oracle.fit_points(x, y, z)
        tr = tf.tracks[tid]
        assert f["par"][4] == pytest.approx(tr["charge"] / tr["pt"], rel=1e-6)
        assert f["par"][3] == pytest.approx(-math.sinh(tr["eta"]), rel=1e-6, abs=1e-9)
        alpha = math.radians(10.0)
        # local direction at the first hit: phi_local = phi0 - alpha + omega * s
        R = 100 * tr["pt"] / (0.299792458 * 0.5)
        om = -tr["charge"] / R
        X0 = x[0]
        pl0 = tr["phi"] - alpha
        sphi = math.sin(pl0) + om * X0
        assert f["par"][2] == pytest.approx(sphi, rel=1e-6, abs=1e-9)


def test_fit_transport_jacobian_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(40):
        s = np.array([rng.uniform(-10, 10), rng.uniform(-100, 100), rng.uniform(-0.7, 0.7),
                      rng.uniform(-1, 1), rng.uniform(-8, 8)])
        dx = rng.choice([-1, 1]) * rng.uniform(0.3, 30.0)
        ns, F = oracle.transport(s, dx)
        if ns is None:
            continue
        for j in range(5):
            h = 1e-6 * max(abs(s[j]), 1.0)
            sp = s.copy(); sp[j] += h
            sm = s.copy(); sm[j] -= h
            a, _ = oracle.transport(sp, dx)
            b, _ = oracle.transport(sm, dx)
            fd = (a - b) / (2 * h)
            assert np.allclose(F[:, j], fd, rtol=1e-5, atol=1e-7), (j, F[:, j], fd)


def test_fit_update_matches_information_form():
    rng = np.random.default_rng(4)
    p = oracle.OracleParams()
    for _ in range(20):
        A = rng.normal(size=(5, 5))
        C = A @ A.T + 0.1 * np.eye(5)
        s = rng.normal(size=5)
        my, mz = rng.normal(size=2)
        s2, C2, chi2, ok = oracle.update(s, C, my, mz, p)
        H = np.zeros((2, 5)); H[0, 0] = H[1, 1] = 1
        Vi = np.diag([1 / p.sigma_y ** 2, 1 / p.sigma_z ** 2])
        Ci = np.linalg.inv(C)
        Cp = np.linalg.inv(Ci + H.T @ Vi @ H)
        sp = Cp @ (Ci @ s + H.T @ Vi @ np.array([my, mz]))
        assert np.allclose(C2, Cp, rtol=1e-7, atol=1e-12)
        assert np.allclose(s2, sp, rtol=1e-7, atol=1e-10)
        r = np.array([my, mz]) - H @ s
        assert chi2 == pytest.approx(r @ np.linalg.inv(H @ C @ H.T + np.linalg.inv(Vi)) @ r, rel=1e-9)
        assert ok


def test_fit_pulls_unit_normal():
    rng = np.random.default_rng(11)
    p = oracle.OracleParams()
    x = _rows_x()
    pulls, chi2ndf = [], []
    for _ in range(1500):
        qpt = rng.choice([-1, 1]) / rng.uniform(0.3, 3.0)
        phi0 = rng.uniform(-0.3, 0.3)
        tgl = rng.uniform(-1, 1)
        y0, z0 = rng.uniform(-5, 5), rng.uniform(10, 200)
        y, z = helix_points(x, y0, z0, phi0, tgl, qpt)
        y = y + rng.normal(0, p.sigma_y, len(x))
        z = z + rng.normal(0, p.sigma_z, len(x))
        f = oracle.fit_points(x, y, z, p)
        truth = np.array([y0, z0, math.sin(phi0), tgl, qpt])
        d = np.array([f["cov"][0], f["cov"][2], f["cov"][5], f["cov"][9], f["cov"][14]])
        pulls.append((f["par"] - truth) / np.sqrt(d))
        chi2ndf.append(f["chi2"] / f["ndf"])
    pulls = np.array(pulls)
    assert np.all(np.abs(pulls.mean(0)) < 0.1), pulls.mean(0)
    assert np.all(np.abs(pulls.std(0) - 1) < 0.1), pulls.std(0)
    assert abs(np.mean(chi2ndf) - 1) < 0.05


# ---------------------------------------------------------------- whole chain
def test_single_sector_efficiency_against_truth(c1_tf):
    """Generator truth (not a parity pin): findable tracks with pT > 0.2 GeV are
    found, and few reconstructed tracks are fakes."""
    tf = c1_tf
    r = oracle.reconstruct(tf)
    planes = oracle.decode_all(tf)
    lab = np.full(planes.shape, -1, np.int32)
    lab[np.nonzero(planes)] = tf.digit_labels
    cl = r.clusters
    cl_lab = lab[cl["sector"], cl["row"], cl["t_peak"], cl["pad_peak"]]
    found = set()
    fakes = 0
    for k in range(len(r.track_first)):
        ls = cl_lab[r.cl2trk == k]
        v, c = np.unique(ls, return_counts=True)
        j = int(np.argmax(c))
        if c[j] >= 0.9 * len(ls) and v[j] >= 0:
            found.add(int(v[j]))
        else:
            fakes += 1
    h = tf.hits[tf.hits["leg"] == 0]
    nrow = np.bincount(h["track"], minlength=len(tf.tracks))
    findable = np.nonzero((nrow >= 50) & (tf.tracks["pt"] > 0.2))[0]
    eff = np.mean([t in found for t in findable])
    assert len(findable) > 20 and eff >= 0.95
    assert fakes <= 0.1 * len(r.track_first)
