"""Pins of the oracle's decision rules on hand-built inputs whose answer is
worked out by hand in each docstring: the CA tie-breaks (interior and edge
rows), the chain and track length limits, the merge tie-break on both ends,
a merge that needs a second pass, and the fit's circle initialisation.  Each
case is built so that the plausible wrong rule (<= for <, the larger index,
the merged group's id, one pass only, a limit off by one, the wrong three
points) gives a different answer."""
import math

import numpy as np
import pytest

import oracle
from synth import Geom, make_clusters

BASE_Z = 5 * 128 * 400          # Z of time bin 400 (u)


def ca_of(pts, **kw):
    g = Geom(n_sectors=1, n_time_bins=1000)
    cl, order = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl, oracle.OracleParams(**kw))
    inv = np.argsort(order)          # input position -> canonical index
    return cl, inv, up, down, chain


# ---------------------------------------------------------------- CA ties
def test_ca_tie_between_two_lower_clusters_goes_to_the_smaller_d():
    """Rows 10-12 (dX = 960 u each).  c = (0, Z) on row 11; d1 = (-496), d2 =
    (304) on row 10; u1 = (496), u2 = (-304) on row 12, all at the same Z step
    of 480 u per row.  dev_Y = 960 (Y_u + Y_d): (d1, u1) and (d2, u2) score 0,
    the crossed pairs 960 * 800 -> worse.  Tie between (d1, u1) and (d2, u2):
    the smaller d wins, d1 (lower pad), so up = u1 although u2 has the smaller
    index."""
    pts = [(0, 11, 0, BASE_Z), (0, 10, -496, BASE_Z - 480), (0, 10, 304, BASE_Z - 480),
           (0, 12, 496, BASE_Z + 480), (0, 12, -304, BASE_Z + 480)]
    cl, inv, up, down, _ = ca_of(pts)
    c, d1, d2, u1, u2 = inv
    assert d1 < d2 and u2 < u1
    assert (down[c], up[c]) == (d1, u1)


def test_ca_tie_between_two_upper_clusters_goes_to_the_smaller_u():
    """One d = (-96, Z - 480) below c = (0, Z); u1 = (96, Z + 800), u2 = (96,
    Z + 160) above.  dev_Y = 0 for both; dev_Z = 960 (Z_u + Z_d - 2 Z_c) =
    +-960 * 320: equal scores 307200^2 (within the cut 256 * 1920).  u2 is one
    time bin earlier, hence the smaller index, and wins."""
    pts = [(0, 11, 0, BASE_Z), (0, 10, -96, BASE_Z - 480), (0, 12, 96, BASE_Z + 800),
           (0, 12, 96, BASE_Z + 160)]
    cl, inv, up, down, _ = ca_of(pts)
    c, d, u1, u2 = inv
    assert u2 < u1 and (down[c], up[c]) == (d, u2)
    # without the tie the better score wins whatever its index: move u1 onto the line
    pts[2] = (0, 12, 96, BASE_Z + 480)
    cl, inv, up, down, _ = ca_of(pts)
    assert up[inv[0]] == inv[2]


@pytest.mark.parametrize("off1,off2,winner", [(100, 100, "c2"), (100, 150, "c1"), (150, 100, "c2")])
def test_ca_edge_row_zero_takes_the_best_scoring_cluster_above(off1, off2, winner):
    """Row 0 holds d = (0, Z); row 1 holds c1 = (300) and c2 = (-300); row 2
    holds u1 = (600 + off1) and u2 = (-600 - off2).  Each c pairs with (d, its
    own u): dev_Y = +-960 off.  up[d] is the c with down[c] = d and the
    smallest score; on equal scores the smaller index, c2 (lower pad)."""
    pts = [(0, 0, 0, BASE_Z), (0, 1, 300, BASE_Z), (0, 1, -300, BASE_Z),
           (0, 2, 600 + off1, BASE_Z), (0, 2, -600 - off2, BASE_Z)]
    cl, inv, up, down, _ = ca_of(pts)
    d, c1, c2, u1, u2 = inv
    assert c2 < c1
    assert down[c1] == d and down[c2] == d and up[c1] == u1 and up[c2] == u2
    assert up[d] == (c1 if winner == "c1" else c2) and down[d] == -1


@pytest.mark.parametrize("off1,off2,winner", [(100, 100, "c2"), (100, 150, "c1")])
def test_ca_edge_row_last_mirrors_row_zero(off1, off2, winner):
    """Rows 149-151 (dX = 1920 u).  u = (0, Z) on row 151, c1 = (300), c2 =
    (-300) on row 150, d1 = (600 + off1), d2 = (-600 - off2) on row 149:
    dev_Y = 1920 (Y_d - 2 Y_c) = +-1920 off.  down[u] = the c with up[c] = u and
    the smallest score, ties to the smaller index."""
    pts = [(0, 151, 0, BASE_Z), (0, 150, 300, BASE_Z), (0, 150, -300, BASE_Z),
           (0, 149, 600 + off1, BASE_Z), (0, 149, -600 - off2, BASE_Z)]
    cl, inv, up, down, _ = ca_of(pts)
    u, c1, c2, d1, d2 = inv
    assert up[c1] == u and up[c2] == u and down[c1] == d1 and down[c2] == d2
    assert down[u] == (c1 if winner == "c1" else c2) and up[u] == -1


# ---------------------------------------------------------------- chain / track limits
def segment(rows, Y, z_step=0):
    return [(0, r, Y, BASE_Z + z_step * (r - rows[0])) for r in rows]


def test_min_chain_boundary():
    """A straight segment over k rows gives a chain of k - 2 clusters (its end
    clusters have no (down, up) pair): 6 rows -> 4 clusters, dropped; 7 rows
    -> 5 clusters = min_chain, kept."""
    pts = segment(range(20, 26), -6000) + segment(range(30, 37), 6000)
    cl, inv, up, down, chain = ca_of(pts)
    six, seven = inv[:6], inv[6:]
    assert np.all(chain[six] == -1)
    assert np.all(chain[seven[1:-1]] == seven[1]) and chain[seven[0]] == -1 and chain[seven[-1]] == -1
    # with min_chain 4 the 4-chain is kept too
    _, inv4, _, _, chain4 = ca_of(pts, min_chain=4)
    assert np.all(chain4[inv4[1:5]] == inv4[1])


def test_min_track_boundary_single_chains():
    """Chains of 9 (11-row segment) and 10 (12-row segment) clusters: only the
    second becomes a track (min_track = 10)."""
    pts = segment(range(20, 31), -6000) + segment(range(40, 52), 6000)
    g = Geom(n_sectors=1, n_time_bins=1000)
    cl, order = make_clusters(g, pts)
    up, down, chain = oracle.ca(g, cl)
    cl2trk, first, ncl, passes = oracle.merge(g, cl, up, down, chain)
    inv = np.argsort(order)
    assert list(ncl) == [10] and first[0] == inv[12]
    assert np.all(cl2trk[inv[:11]] == -1) and np.all(cl2trk[inv[12:22]] == 0)
    assert cl2trk[inv[11]] == -1 and cl2trk[inv[22]] == -1


# ---------------------------------------------------------------- merge (hand-built chains)
def build_chains(chains):
    """chains: lists of (row, Y, Z) bottom -> top.  Returns the geometry, the
    clusters, the up / down / chain_of arrays the merge reads (each chain
    linked along its list, chain id = canonical index of its bottom cluster),
    and each chain's canonical indices."""
    g = Geom(n_sectors=1, n_time_bins=1000)
    pts = [(0, r, Y, Z) for ch in chains for (r, Y, Z) in ch]
    cl, order = make_clusters(g, pts)
    inv = np.argsort(order)
    n = len(cl)
    up = np.full(n, -1, np.int32)
    down = np.full(n, -1, np.int32)
    chain_of = np.full(n, -1, np.int32)
    idx, k = [], 0
    for ch in chains:
        ii = [int(inv[k + i]) for i in range(len(ch))]
        k += len(ch)
        for a, b in zip(ii, ii[1:]):
            up[a], down[b] = b, a
        chain_of[ii] = ii[0]
        idx.append(ii)
    return g, cl, up, down, chain_of, idx


def chain(rows_body, y_body, end_rows, y_end, top_end=True):
    """A chain whose body (far away, irrelevant to the merge) leads to two end
    clusters on the line Y = y_end at end_rows."""
    body = [(r, y_body, BASE_Z) for r in rows_body]
    ends = [(r, y_end, BASE_Z) for r in end_rows]
    return body + ends if top_end else ends + body


def merged_groups(g, cl, up, down, chain_of, idx, **kw):
    cl2trk, first, ncl, passes = oracle.merge(g, cl, up, down, chain_of, oracle.OracleParams(**kw))
    groups = {}
    for c, ii in enumerate(idx):
        groups.setdefault(int(cl2trk[ii[0]]), []).append(c)
    return sorted(groups.values()), passes, ncl


def test_merge_tie_on_a_top_end_goes_to_the_lower_chain_id():
    """Top end A at rows 43-44 on Y = 0.  Bottom ends B1 (rows 47-48, Y = +100)
    and B2 (rows 49-50, Y = -100): both residuals 100 -> equal scores 2 * 100^2.
    A takes the lower chain id, B1 (its bottom row is lower); B1's and B2's
    only candidate is A, so A-B1 merge and B2 stays alone."""
    A = chain(range(30, 43), -9000, [43, 44], 0)
    B1 = chain(range(49, 60), 7000, [47, 48], 100, top_end=False)
    B2 = chain(range(51, 62), 9000, [49, 50], -100, top_end=False)
    g, cl, up, down, co, idx = build_chains([A, B1, B2])
    assert idx[1][0] < idx[2][0]
    groups, passes, _ = merged_groups(g, cl, up, down, co, idx)
    assert [0, 1] in groups and [2] in groups and passes == 1


def test_merge_tie_on_a_bottom_end_goes_to_the_lower_chain_id():
    """Bottom end B at rows 49-50 on Y = 0.  Top ends A1 (rows 43-44, Y = +100)
    and A2 (rows 45-46, Y = -100), both at residual 100.  A1's root (row 30)
    has a lower index than A2's (row 32): B takes A1."""
    A1 = chain(range(30, 43), -9000, [43, 44], 100)
    A2 = chain(range(32, 45), -7000, [45, 46], -100)
    B = chain(range(51, 62), 9000, [49, 50], 0, top_end=False)
    g, cl, up, down, co, idx = build_chains([A1, A2, B])
    assert idx[0][0] < idx[1][0]
    groups, passes, _ = merged_groups(g, cl, up, down, co, idx)
    assert [0, 2] in groups and [1] in groups


def test_merge_needs_a_second_pass():
    """T3 (top rows 43-44, Y = 0) and D (bottom rows 47-48, Y = 0) score 0 and
    merge in pass 1.  B (bottom rows 49-50, Y = 100) prefers T3 (score 2 *
    100^2) to T1 (top rows 45-46, Y = 300: score 2 * 200^2), but T3 prefers D,
    so B and T1 stay apart in pass 1 (T1 prefers B, not mutual).  In pass 2 T3
    and D are no longer ends: B's best is T1 and T1's is B: they merge.  With
    merge_max_passes = 1 they stay apart."""
    T3 = chain(range(30, 43), -9000, [43, 44], 0)
    T1 = chain(range(32, 45), -7000, [45, 46], 300)
    D = chain(range(49, 60), 7000, [47, 48], 0, top_end=False)
    B = chain(range(51, 62), 9000, [49, 50], 100, top_end=False)
    g, cl, up, down, co, idx = build_chains([T3, T1, D, B])
    groups, passes, _ = merged_groups(g, cl, up, down, co, idx)
    assert groups == [[0, 2], [1, 3]] and passes == 2
    groups1, passes1, _ = merged_groups(g, cl, up, down, co, idx, merge_passes=1)
    assert groups1 == [[0, 2], [1], [3]] and passes1 == 1


@pytest.mark.parametrize("lower,upper,kept", [(5, 5, True), (5, 4, False), (4, 6, True)])
def test_min_track_applies_to_the_merged_total(lower, upper, kept):
    """Two collinear chains (rows 40-... and 50-...) merge; the track is kept
    iff the merged total reaches min_track = 10."""
    A = [(r, 0, BASE_Z) for r in range(45 - lower, 45)]
    B = [(r, 0, BASE_Z) for r in range(48, 48 + upper)]
    g, cl, up, down, co, idx = build_chains([A, B])
    cl2trk, first, ncl, passes = oracle.merge(g, cl, up, down, co)
    assert passes == 1
    assert list(ncl) == ([lower + upper] if kept else [])


# ---------------------------------------------------------------- fit initialisation
@pytest.mark.parametrize("turn", [+1, -1])
def test_fit_initial_state_is_the_circle_through_three_points(turn):
    """fit_passes = 0 returns the initial state.  Points 0, 2, 4 lie on a
    circle of radius 60 cm centred at (100, 50 turn) at angles -110, -90, -70
    degrees (mirrored in y for turn = -1); points 1 and 3 are off the circle
    and must not matter.  Moving towards +x the track turns left (turn = +1):
    curvature +1/60 cm^-1, q/pT = (1/60) / kfac < 0 with kfac = -0.5 c 1e-2.
    The state is at the outermost point: y, zeta of that point, snp = the sine
    of the tangent direction there (angle + 90 degrees, mirrored), tgl =
    (zeta_4 - zeta_0) / (R * 40 degrees)."""
    R, xc, yc = 60.0, 100.0, 50.0 * turn
    th = np.radians([-110.0, -100.0, -90.0, -80.0, -70.0])
    x = xc + R * np.cos(th)
    y = yc + turn * R * np.sin(th)
    y[1] += 5.0
    y[3] -= 7.0
    arc = R * math.radians(40.0)
    z = np.array([20.0, 99.0, 30.0, -50.0, 20.0 + 0.25 * arc])
    f = oracle.fit_points(x, y, z, oracle.OracleParams(fit_passes=0))
    kfac = -0.5 * 0.299792458e-2
    want = [y[4], z[4], turn * math.sin(th[4] + math.pi / 2), 0.25, turn / R / kfac]
    assert f["x"] == x[4]
    assert np.allclose(f["par"], want, rtol=1e-12, atol=1e-12)
