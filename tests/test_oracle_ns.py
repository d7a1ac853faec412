"""Pins of the oracle's optional 5x5 noise suppression (step 2b): hand-worked
planes where the dip between a peak and a higher one two pixels away decides,
the key tie-break direction, the single pass over step 2's peak set, and
invariants on random planes and a generated timeframe."""
import numpy as np
import pytest

import oracle
import tpcgen


def blank(T=14, P=14):
    return np.zeros((T, P), np.uint16)


def peaks(plane, dip):
    return {(int(t), int(p)) for t, p in zip(*np.nonzero(oracle.peaks_plane(plane, 10, dip)))}


def two_peaks(q_mid, mid, pos_small, q_big=100, q_small=20):
    """A peak of q_big at (5, 5), q_small at pos_small and q_mid on the pixel
    between them (seen from the small peak); both are 3x3 peaks."""
    pl = blank()
    pl[5, 5] = q_big
    pl[pos_small] = q_small
    pl[mid] = q_mid
    return pl


@pytest.mark.parametrize("pos,mid", [((5, 7), (5, 6)),      # same time bin, 2 pads away
                                     ((7, 7), (6, 6)),      # diagonal
                                     ((7, 6), (6, 5)),      # knight's move: inner pixel (-1, -1)
                                     ((3, 4), (4, 5)),      # knight's move the other way: (+1, +1)
                                     ((5, 3), (5, 4))])     # lower pad
def test_dip_decides(pos, mid):
    pl = two_peaks(15, mid, pos)    # dip of the small peak: 20 - 15 = 5
    assert peaks(pl, 0) == {(5, 5), pos}
    assert peaks(pl, 5) == {(5, 5), pos}      # 5 < 5 is false: kept
    assert peaks(pl, 6) == {(5, 5)}           # 5 < 6: dropped, the higher peak stays
    pl[mid] = 0                               # a deep valley
    assert peaks(pl, 20) == {(5, 5), pos}
    assert peaks(pl, 21) == {(5, 5)}


def test_equal_charge_tie_goes_to_the_lower_index():
    """Two peaks of 50 two pads apart: the one at the lower (t, p) index has the
    greater key and survives; moving the pair does not change which side wins."""
    pl = blank()
    pl[5, 5] = 50
    pl[5, 7] = 50
    pl[5, 6] = 45
    assert peaks(pl, 0) == {(5, 5), (5, 7)}
    assert peaks(pl, 6) == {(5, 5)}
    pl2 = blank()
    pl2[5, 7] = 50
    pl2[7, 7] = 50
    pl2[6, 7] = 45
    assert peaks(pl2, 6) == {(5, 7)}      # earlier time bin wins


def test_lower_or_distant_peaks_do_not_suppress():
    pl = blank()
    pl[5, 5] = 100
    pl[5, 8] = 90          # three pads away: outside the 5x5
    pl[5, 6] = pl[5, 7] = 80
    # (5, 6), (5, 7) are not peaks (neighbours of 100 / 90); a chain of plateaus
    assert peaks(pl, 0) == {(5, 5), (5, 8)}
    assert peaks(pl, 1000) == {(5, 5), (5, 8)}
    pl = blank()
    pl[5, 5] = 100
    pl[5, 7] = 20
    pl[5, 6] = 19
    assert (5, 5) in peaks(pl, 1000)      # the higher peak never loses to a lower one


def test_single_pass_over_step_2_peaks():
    """100 - 60 - 30 two pads apart, shallow valleys: 60 is dropped because of
    100, and 30 because of 60, although 60 itself does not survive."""
    pl = blank(14, 20)
    pl[5, 3], pl[5, 5], pl[5, 7] = 100, 60, 30
    pl[5, 4], pl[5, 6] = 58, 29
    assert peaks(pl, 0) == {(5, 3), (5, 5), (5, 7)}
    assert peaks(pl, 5) == {(5, 3)}


def test_flag_bit_2_keeps_referring_to_step_2_peaks():
    pl = two_peaks(15, (5, 6), (5, 7))
    c = oracle.cluster_at(pl, 5, 5)
    assert c["flags"] & 4


def test_random_plane_invariants():
    rng = np.random.default_rng(7)
    for _ in range(20):
        pl = (rng.random((24, 20)) < 0.5) * rng.integers(1, 120, (24, 20))
        pl = pl.astype(np.uint16)
        base = peaks(pl, 0)
        assert base == {(int(t), int(p)) for t, p in zip(*np.nonzero(oracle.peaks_plane(pl, 10)))}
        prev = base
        for dip in (1, 5, 20, 200, 1023):
            cur = peaks(pl, dip)
            assert cur <= prev                 # more suppression with a larger dip
            prev = cur
            # every dropped peak has a greater-key step-2 peak on its 5x5 ring
            for t, p in base - cur:
                ring = [(t + dt, p + dp) for dt in range(-2, 3) for dp in range(-2, 3)
                        if max(abs(dt), abs(dp)) == 2 and (t + dt, p + dp) in base]
                assert any((int(pl[n]), -(n[0] * 20 + n[1])) > (int(pl[t, p]), -(t * 20 + p)) for n in ring)
        if base:   # the peak of greatest key survives any dip
            top = max(base, key=lambda c: (int(pl[c]), -(c[0] * 20 + c[1])))
            assert top in prev


def test_timeframe_clusters_are_a_subset_with_identical_records():
    tf = tpcgen.generate(tpcgen.single_sector(3, n_tracks=300))
    a = oracle.find_clusters(tf)
    b = oracle.find_clusters(tf, oracle.OracleParams(ns_min_dip=10))
    assert 0 < len(b) < len(a)
    key = lambda c: (int(c["sector"]), int(c["row"]), int(c["t_peak"]), int(c["pad_peak"]))
    ia = {key(c): i for i, c in enumerate(a)}
    idx = np.array([ia[key(c)] for c in b])
    assert np.all(np.diff(idx) > 0)                       # canonical order kept
    assert a[idx].tobytes() == b.tobytes()                # records unchanged
