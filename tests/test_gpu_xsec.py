"""Parity of the cross-sector merge (step 9) with the oracle.

Its decisions are float: the GPU matches on its FP32 fits with an FP32 chi2,
the oracle on FP64 ones, so a decision near the cut or between near-equal
candidates can go either way.  Links must be identical except where the oracle
marks the decision borderline (a candidate chi2 within 1 % of the cut, or a
runner-up within 1 % of the best, for the piece or a partner it has on either
side); the merged tracks whose pieces agree must contain the same clusters, and
their refitted parameters agree with the FP64 refit within the fit
tolerance."""
import numpy as np
import pytest

import oracle
import tpcgen
from parity import COV_RTOL, PAR_RTOL, param_allowance

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def gpu_merge(lib, tf):
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        cl = lib.tpc_get_clusters(R.ctx, t)
        tr, m = lib.tpc_get_tracks(R.ctx, t, len(cl))
        n = lib.tpc_merge_sectors(R.ctx, t)
        mt, mm, link = lib.tpc_get_merged_tracks(R.ctx, t, len(cl), len(tr))
        lib.tpc_release(R.ctx, t)
    assert len(mt) == n
    return cl, tr, m, mt, mm, link


def test_full_tpc_cross_sector_parity(lib):
    check_parity(lib, tpcgen.generate(tpcgen.full_tpc(1)), min_multi=1000)


def test_continuous_timeframe_cross_sector_parity(lib):
    """2000 bins of the 50 kHz continuous timeframe: the candidate search runs
    over several zeta bins per sector, and pieces of different collisions
    overlap in time."""
    check_parity(lib, tpcgen.generate(tpcgen.continuous_tf(1, n_time_bins=2000)), min_multi=300)


def check_parity(lib, tf, min_multi):
    orc = oracle.reconstruct(tf)
    ox = oracle.merge_sectors(tf, orc)
    cl, tr, m, mt, mm, link = gpu_merge(lib, tf)
    assert cl.tobytes() == orc.clusters.tobytes() and np.array_equal(m, orc.cl2trk)
    diff = np.nonzero(link != ox.link)[0]
    # a differing decision must be a borderline one in the oracle's own numbers
    oprev = np.full(len(link), -1)
    oprev[ox.link[ox.link >= 0]] = np.nonzero(ox.link >= 0)[0]
    gprev = np.full(len(link), -1)
    gprev[link[link >= 0]] = np.nonzero(link >= 0)[0]

    def explained(t):
        cand = {t, ox.link[t], link[t], oprev[t], gprev[t]} - {-1}
        return any(ox.borderline[c] for c in cand)
    unexplained = [int(t) for t in diff if not explained(t)]
    print("links: oracle", int((ox.link >= 0).sum()), "gpu", int((link >= 0).sum()), "differ", len(diff),
          "borderline pieces", int(ox.borderline.sum()))
    assert not unexplained, [(t, ox.link[t], link[t], ox.best_chi2[t]) for t in unexplained[:10]]
    # merged tracks whose pieces agree: same clusters, refit within tolerance;
    # piece chains by root on both sides
    def chains(lk):
        prev = np.full(len(lk), -1)
        prev[lk[lk >= 0]] = np.nonzero(lk >= 0)[0]
        out = []
        for r in np.nonzero(prev < 0)[0]:
            c, t = [], r
            while t >= 0:
                c.append(int(t))
                t = lk[t]
            out.append(tuple(c))
        return out
    oc, gc = chains(ox.link), chains(link)
    assert len(oc) == len(ox.fits) and len(gc) == len(mt)
    common = set(oc) & set(gc)
    assert len(common) >= len(oc) - 2 * len(diff)
    oi = {c: i for i, c in enumerate(oc)}
    gi = {c: i for i, c in enumerate(gc)}
    multi = [c for c in common if len(c) > 1]
    assert len(multi) > min_multi
    diag = [0, 2, 5, 9, 14]
    worst = np.zeros(5)
    worst_cov = 0.0
    nflag = 0
    for c in multi:
        o, g = ox.fits[oi[c]], mt[gi[c]]
        assert g["flags"] & lib.TPC_TRK_XSECTOR
        assert g["n_clusters"] == ox.ncl[oi[c]] and g["first_cluster"] == ox.first[oi[c]]
        if o["flags"] or (int(g["flags"]) & ~lib.TPC_TRK_XSECTOR):
            nflag += 1
            continue
        allow = param_allowance(o["par"][None], o["cov"][None], [o["chi2"]], [o["ndf"]], [o["flags"]])[0]
        rel = np.abs(g["par"].astype(float) - o["par"]) / allow * PAR_RTOL
        worst = np.maximum(worst, rel)
        assert g["x"] == pytest.approx(o["x"], rel=1e-5)
        cd = np.abs(g["cov"].astype(float) - o["cov"])
        k = 0
        for i in range(5):
            for j in range(i + 1):
                worst_cov = max(worst_cov, cd[k] / np.sqrt(o["cov"][diag[i]] * o["cov"][diag[j]]))
                k += 1
    print("merged refit precision vs FP64:", worst.tolist(), "cov", worst_cov, "flagged", nflag)
    assert nflag <= 0.01 * len(multi)
    assert np.all(worst <= PAR_RTOL) and worst_cov <= COV_RTOL
    # the cluster-to-track map of the merged tracks follows the chains
    g_of = np.zeros(len(link), np.int64)
    for i, c in enumerate(gc):
        g_of[list(c)] = i
    assert np.array_equal(mm, np.where(m >= 0, g_of[np.maximum(m, 0)], -1))


def test_batch_merge_equals_events_alone(lib):
    tfs = [tpcgen.generate(tpcgen.full_tpc(60 + i, n_tracks=3000)) for i in range(2)]
    alone = [gpu_merge(lib, tf) for tf in tfs]
    with lib.Reconstructor.for_timeframe(tfs[0]) as R:
        t, keep = lib.tpc_submit_batch(R.ctx, [(tf.pages, tf.page_offsets) for tf in tfs], tfs[0].n_time_bins)
        R.wait(t)
        cs, ts = lib.tpc_get_batch_info(R.ctx, t)
        ncl, ntr = int(cs[-1]), int(ts[-1])
        lib.tpc_merge_sectors(R.ctx, t)
        mt, mm, link = lib.tpc_get_merged_tracks(R.ctx, t, ncl, ntr)
        lib.tpc_release(R.ctx, t)
    off = 0
    for e, (cl, tr, m, amt, amm, alink) in enumerate(alone):
        lk = link[ts[e]:ts[e + 1]].copy()
        lk[lk >= 0] -= int(ts[e])
        assert np.array_equal(lk, alink)
        sub = mt[off:off + len(amt)].copy()
        sub["first_cluster"] -= int(cs[e])
        assert sub.tobytes() == amt.tobytes()
        mp = mm[cs[e]:cs[e + 1]].copy()
        mp[mp >= 0] -= off
        assert np.array_equal(mp, amm)
        off += len(amt)
    assert off == len(mt)


def test_degenerate_inputs(lib):
    """No digits, noise only, and one sector (no neighbouring sector to enter):
    step 9 links nothing and every piece is its own merged track, unchanged."""
    cases = [tpcgen.single_sector(6, n_tracks=0, zs_threshold=1024),
             tpcgen.single_sector(6, n_tracks=0),
             tpcgen.single_sector(1)]
    for cfg in cases:
        tf = tpcgen.generate(cfg)
        cl, tr, m, mt, mm, link = gpu_merge(lib, tf)
        assert len(mt) == len(tr)
        assert np.all(np.asarray(link) < 0)
        if len(tr):
            assert np.array_equal(mt["par"], tr["par"]) and np.array_equal(mt["cov"], tr["cov"])
            assert np.array_equal(mt["n_clusters"], tr["n_clusters"])
            assert np.array_equal(mm, m)
            assert not np.any(mt["flags"] & lib.TPC_TRK_XSECTOR)
