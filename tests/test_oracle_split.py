"""Pins of the oracle's optional charge splitting (step 3s): a pixel's charge
goes to the peaks whose 3x3 cores hold it (else to those whose 5x5 outer rings
do), in proportion to their heights.  Hand-worked planes with the sums written
out, the transposed (time) direction, invariants on random dense planes
(conservation: the shares of one pixel never add up to more than its charge
and lose less than one ADC per owner), a two-cloud closure (splitting moves
the centroids toward the true centres) and the timeframe-level identity
(clusters that share nothing keep their records)."""
import math

import numpy as np
import pytest

import oracle
import tpcgen


def R(a, b):
    """floor((2a + b) / (2b)): the record's rounding, half up."""
    return (2 * a + b) // (2 * b)


def row_plane(values, t=5, T=12, P=14):
    """One time bin t holding values (pad -> q); every other pixel empty."""
    pl = np.zeros((T, P), np.uint16)
    for p, q in values.items():
        pl[t, p] = q
    return pl


def test_core_pixel_between_two_peaks_is_shared_by_height():
    """Peaks of 100 (pad 4) and 80 (pad 6), 60 between them.  Pad 5 is in both
    cores: the 100-peak takes floor(60 * 100 / 180) = 33, the 80-peak
    floor(60 * 80 / 180) = 26 (59 of 60 ADC handed out).  Pad 6 is an outer
    pixel of the first cluster and pad 4 one of the second, both above their
    inner pixel (60): excluded by the 5x5 rule, as without splitting.
    First cluster: Q = 40 + 100 + 33 = 173, Sp = -40 + 33 = -7.
    Second: Q = 26 + 80 + 30 = 136, Sp = -26 + 30 = 4."""
    pl = row_plane({3: 40, 4: 100, 5: 60, 6: 80, 7: 30})
    assert oracle.split_share(pl, (4, 5), (5, 5)) == 33
    assert oracle.split_share(pl, (6, 5), (5, 5)) == 26
    assert oracle.split_share(pl, (4, 5), (3, 5)) == 40      # only the first core
    assert oracle.split_share(pl, (4, 5), (4, 5)) == 100     # a peak keeps its own pixel
    a = oracle.cluster_at(pl, 4, 5, split=True)
    b = oracle.cluster_at(pl, 6, 5, split=True)
    assert (a["qtot"], a["pad_fp"]) == (173, 256 * 4 + R(256 * -7, 173))
    assert (b["qtot"], b["pad_fp"]) == (136, 256 * 6 + R(256 * 4, 136))
    assert a["qmax"] == 100 and b["qmax"] == 80
    assert a["flags"] == b["flags"] == 2 | 4 | 8             # excluded, neighbour, split
    # without splitting both count pad 5 whole
    a0 = oracle.cluster_at(pl, 4, 5)
    assert (a0["qtot"], a0["pad_fp"], a0["flags"]) == (200, 256 * 4 + R(256 * 20, 200), 2 | 4)


def test_outer_pixel_in_another_core_goes_to_that_peak():
    """Peaks at pads 4 (100) and 7 (90), three pads apart: neither lies in the
    other's 5x5 window.  Pad 6 (40) is an included outer pixel of the first
    cluster (40 <= 50, its inner pixel), but it lies in the second peak's core
    and in no core of the first: the first cluster counts 0 of it.
    First: Q = 20 + 100 + 50 = 170, Sp = -20 + 50 = 30.  The second cluster is
    unchanged (pad 5 is excluded there by the 5x5 rule; pad 6 and 8 are its own)."""
    pl = row_plane({3: 20, 4: 100, 5: 50, 6: 40, 7: 90, 8: 10})
    assert oracle.split_share(pl, (4, 5), (6, 5)) == 0
    assert oracle.split_share(pl, (7, 5), (6, 5)) == 40
    assert oracle.split_share(pl, (4, 5), (5, 5)) == 50      # pad 5 touches only the first core
    a = oracle.cluster_at(pl, 4, 5, split=True)
    assert (a["qtot"], a["pad_fp"], a["flags"]) == (170, 256 * 4 + R(256 * 30, 170), 8)
    a0 = oracle.cluster_at(pl, 4, 5)
    assert (a0["qtot"], a0["pad_fp"], a0["flags"]) == (210, 256 * 4 + R(256 * 110, 210), 0)
    b = oracle.cluster_at(pl, 7, 5, split=True)
    b0 = oracle.cluster_at(pl, 7, 5)
    assert b.tobytes() == b0.tobytes()
    assert (b["qtot"], b["pad_fp"], b["flags"]) == (140, 256 * 7 + R(256 * -30, 140), 2)


def test_pixel_on_two_outer_rings_only():
    """Peaks at pads 2 (100) and 6 (80), pad 4 (30) two pads from each and in
    neither core: it falls back to the ring owners, floor(30 * 100 / 180) = 16
    and floor(30 * 80 / 180) = 13.
    First: Q = 10 + 100 + 40 + 16 = 166, Sp = -10 + 40 + 2 * 16 = 62.
    Second: Q = 13 + 40 + 80 + 10 = 143, Sp = -2 * 13 - 40 + 10 = -56."""
    pl = row_plane({1: 10, 2: 100, 3: 40, 4: 30, 5: 40, 6: 80, 7: 10})
    assert oracle.split_share(pl, (2, 5), (4, 5)) == 16
    assert oracle.split_share(pl, (6, 5), (4, 5)) == 13
    a = oracle.cluster_at(pl, 2, 5, split=True)
    b = oracle.cluster_at(pl, 6, 5, split=True)
    assert (a["qtot"], a["pad_fp"], a["flags"]) == (166, 256 * 2 + R(256 * 62, 166), 8)
    assert (b["qtot"], b["pad_fp"], b["flags"]) == (143, 256 * 6 + R(256 * -56, 143), 8)


def test_time_direction():
    """The first example turned by 90 degrees: the shares move time_fp and
    sigma2_time exactly as they moved pad_fp (St = -7 over Q = 173)."""
    pl = row_plane({3: 40, 4: 100, 5: 60, 6: 80, 7: 30}).T.copy()   # pad 5, time bins 3..7
    a = oracle.cluster_at(pl, 5, 4, split=True)
    assert (a["qtot"], a["pad_fp"]) == (173, 256 * 5)
    assert a["time_fp"] == 128 * (4 + 4) + R(128 * -7, 173)
    Stt = 40 + 33
    assert a["sigma2_time"] == min(255, R(16 * (Stt * 173 - 49), 173 * 173))


def test_isolated_clusters_unchanged():
    """Peaks five or more pixels apart share nothing: every record equals the
    record without splitting and carries no split flag."""
    rng = np.random.default_rng(3)
    pl = np.zeros((40, 40), np.uint16)
    w = np.array([0.1, 0.4, 1.0, 0.4, 0.1])
    for t0 in range(4, 36, 6):
        for p0 in range(4, 36, 6):
            amp = rng.uniform(50, 900)
            pl[t0 - 2:t0 + 3, p0 - 2:p0 + 3] = np.rint(amp * np.outer(w, w * rng.uniform(0.8, 1.2, 5)))
    fl = oracle.peaks_plane(pl)
    assert fl.sum() == 36
    for t, p in zip(*np.nonzero(fl)):
        a = oracle.cluster_at(pl, int(p), int(t), split=True)
        b = oracle.cluster_at(pl, int(p), int(t))
        assert not a["flags"] & 8
        assert a.tobytes() == b.tobytes()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_shares_conserve_charge(seed):
    """Dense random plane: for every pixel x, the owners' shares add up to at
    most q(x) and to more than q(x) - |owners| (one floor each); a pixel with a
    single owner goes to it whole; peaks that do not own x get 0."""
    rng = np.random.default_rng(seed)
    T, P = 24, 24
    pl = rng.integers(0, 120, size=(T, P)).astype(np.uint16)
    fl = oracle.peaks_plane(pl)
    peaks = [(int(p), int(t)) for t, p in zip(*np.nonzero(fl))]
    assert len(peaks) > 30
    total = np.zeros((T, P), np.int64)
    owners = np.zeros((T, P), np.int64)
    for (pc, tc) in peaks:
        for dt in range(-2, 3):
            for dp in range(-2, 3):
                px, pt = pc + dp, tc + dt
                if not (0 <= px < P and 0 <= pt < T):
                    continue
                w = oracle.split_share(pl, (pc, tc), (px, pt))
                assert 0 <= w <= pl[pt, px]
                total[pt, px] += w
                owners[pt, px] += w > 0
    q = pl.astype(np.int64)
    covered = owners > 0
    assert (total <= q).all()
    # the owners of a covered pixel: each takes a floor share, so less than one ADC each is lost
    near = np.zeros_like(covered)
    for (pc, tc) in peaks:
        near[max(0, tc - 2):tc + 3, max(0, pc - 2):pc + 3] = True
    pos = near & (q > 0)
    lost = (q - total)[pos]
    assert (lost < 9).all()                       # at most 9 owners in a 5x5 (peaks are never adjacent)
    single = pos & (owners == 1) & (total == q)
    assert single.sum() > 0.5 * pos.sum()


def test_two_cloud_closure():
    """Two noise-free Gaussian clouds (sigma 0.8 pad, 1.0 bin) three pads apart:
    without splitting each cluster counts the other cloud's core pixel on its
    outer ring and is pulled toward it; splitting hands that pixel to the other
    peak, and the pad centroids move from ~0.35 pad off the true centres to
    within 0.06 (what is left: each cloud's tail on the other's core pixel)."""
    from scipy.special import erf
    sp, st = 0.8, 1.0
    P, T = 20, 16
    pe = np.arange(P + 1) - 0.5
    te = np.arange(T + 1) - 0.5
    centres = [(7.1, 7.9), (10.05, 8.0)]
    qc = np.zeros((T, P))
    A = 600 * 2 * math.pi * sp * st
    for pc, tc in centres:
        fp = 0.5 * np.diff(erf((pe - pc) / (sp * math.sqrt(2))))
        ft = 0.5 * np.diff(erf((te - tc) / (st * math.sqrt(2))))
        qc += A * np.outer(ft, fp)
    pl = np.clip(np.rint(qc), 0, 1023).astype(np.uint16)
    fl = oracle.peaks_plane(pl)
    pk = sorted((int(p), int(t)) for t, p in zip(*np.nonzero(fl)))
    assert [p for p, _ in pk] == [7, 10]
    for (p, t), (pc, tc) in zip(pk, centres):
        a = oracle.cluster_at(pl, p, t, split=True)
        b = oracle.cluster_at(pl, p, t)
        err_split = abs(a["pad_fp"] / 256 - pc)
        err_plain = abs(b["pad_fp"] / 256 - pc)
        assert a["flags"] & 8
        assert err_split < 0.06 and err_split < 0.25 * err_plain, (err_split, err_plain)


def test_timeframe_split_changes_only_flagged_clusters():
    """A generated sector: splitting keeps the cluster set (same peaks, same
    order) and every record without the split flag; flagged clusters never gain
    charge."""
    tf = tpcgen.generate(tpcgen.single_sector(5))
    a = oracle.find_clusters(tf)
    b = oracle.find_clusters(tf, oracle.OracleParams(split_charge=True))
    assert len(a) == len(b)
    for k in ("row", "t_peak", "pad_peak", "sector", "qmax"):
        assert (a[k] == b[k]).all()
    fl = (b["flags"] & 8) != 0
    assert 0.02 < fl.mean() < 0.9
    assert a[~fl].tobytes() == b[~fl].tobytes()
    assert (b["qtot"][fl] <= a["qtot"][fl]).all()
    assert ((a["flags"][fl] | 8) == b["flags"][fl]).all()
