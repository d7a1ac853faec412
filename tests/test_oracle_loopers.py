"""Pins of the oracle's looper-leg join (step 9b).

The looping test against the circle traced point by point; links of the legs
of one looper built turn by turn from an exact helix (one turn on: the same
transverse state, zeta advanced by tgl 2 pi / |k|), in any index order; ties;
legs that must not link; the matching chi2 of true pairs drawn from known
covariances against the chi2 distribution with 5 degrees of freedom (which a
wrong or missing Jacobian entry of the turn advance, or of the transport to a
common x, would break); the covariance scaling; the borderline flag; and the
links on a generated timeframe against the generator truth."""
import math
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
import tpcgen
from synth import Geom, make_clusters

KFAC = -0.5 * 0.299792458e-2      # curvature per unit q/pT, 1/cm per 1/GeV
CUT = oracle.LoopParams().chi2_cut


def fit_rec(par, x=85.0, cov=None, chi2=5.0, ndf=10, flags=0):
    f = np.zeros(1, oracle.FIT_DTYPE)[0]
    f["par"] = par
    f["x"] = x
    C = np.diag([4e-4, 9e-4, 4e-6, 1e-6, 2.5e-3]) if cov is None else np.asarray(cov, float)
    f["cov"] = [C[i, j] for i in range(5) for j in range(i + 1)]
    f["chi2"], f["ndf"], f["n_used"], f["flags"] = chi2, ndf, (ndf + 5) // 2, flags
    return f


def turn_length(par):
    return 2 * math.pi / abs(KFAC * par[4])


def advance(par, m=1):
    """The same transverse state m turns on: zeta + m tgl 2 pi / |k|."""
    out = np.array(par, float)
    out[1] += m * par[3] * turn_length(par)
    return out


def fake_result(sectors, fits):
    """One cluster per track in the given sectors, so that the join sees the
    tracks' sectors; the fits are given directly."""
    g = Geom(n_sectors=max(sectors) + 1)
    cl, order = make_clusters(g, [(s, 0, 0, 640 * (10 + i)) for i, s in enumerate(sectors)])
    c2t = np.full(len(cl), -1, np.int32)
    c2t[np.argsort(order)] = np.arange(len(sectors))
    return g, SimpleNamespace(clusters=cl, cl2trk=c2t, fits=np.array(fits, oracle.FIT_DTYPE))


def join(sectors, fits, **kw):
    g, res = fake_result(sectors, fits)
    return oracle.join_loopers(g, res, loop=oracle.LoopParams(**kw))


def traced_reach(x, y, snp, qpt):
    """Largest distance from the axis of the circle through (x, y) with
    direction asin(snp) and curvature k, traced along its arc."""
    k = KFAC * qpt
    f0 = math.asin(snp)
    s = np.linspace(0.0, 2 * math.pi / abs(k), 200001)
    px = x + (np.sin(f0 + k * s) - math.sin(f0)) / k
    py = y - (np.cos(f0 + k * s) - math.cos(f0)) / k
    return float(np.hypot(px, py).max())


A = np.array([3.0, 20.0, 0.3, 0.15, -9.0])     # pT 0.11 GeV: R = 73 cm, loops


@pytest.mark.parametrize("x,y,snp,qpt", [(85.0, 3.0, 0.3, -9.0), (120.0, -20.0, -0.6, 12.0),
                                         (200.0, 30.0, 0.1, -3.0), (90.0, 0.0, 0.0, 5.0)])
def test_reach_against_the_traced_circle(x, y, snp, qpt):
    f = fit_rec([y, 0.0, snp, 0.1, qpt], x=x, cov=np.zeros((5, 5)))
    r = traced_reach(x, y, snp, qpt)
    assert oracle.loops(f, r * (1 + 1e-6)) and not oracle.loops(f, r * (1 - 1e-6))


def test_reach_takes_q_over_pt_three_sigma_up_with_the_scaled_covariance():
    """sigma(q/pT) = 0.2, chi2/ndf = 4: the circle of |q/pT| + 3 * 0.2 * 2."""
    C = np.zeros((5, 5))
    C[4, 4] = 0.04
    f = fit_rec([3.0, 0.0, 0.3, 0.1, -4.0], cov=C, chi2=40.0, ndf=10)
    r = traced_reach(85.0, 3.0, 0.3, -4.0 - 1.2)
    assert oracle.loops(f, r * (1 + 1e-6)) and not oracle.loops(f, r * (1 - 1e-6))
    assert r < traced_reach(85.0, 3.0, 0.3, -4.0) - 20.0


def test_legs_of_successive_turns_link_in_a_chain():
    fits = [fit_rec(A), fit_rec(advance(A, 1)), fit_rec(advance(A, 2)), fit_rec(advance(A, 1))]
    c2, m = oracle.loop_pair(fits[0], fits[1])
    assert m == 1 and c2 == pytest.approx(0.0, abs=1e-12)
    assert oracle.loop_pair(fits[0], fits[2])[1] == 2
    r = join([0, 0, 0, 1], fits)
    # the fourth leg is in another sector: no candidate
    assert r.next.tolist() == [1, 2, -1, -1] and r.prev.tolist() == [-1, 0, 1, -1] and r.n_links == 2


def test_direction_follows_the_fitted_motion_in_any_index_order():
    """Indices C = 0, A = 1, B = 2 (A, B, C on successive turns): the pair (C, A)
    is computed with C first, so m = -2, directed A -> C; next picks the least
    |m|, so the chain is A -> B -> C whatever the indices."""
    fits = [fit_rec(advance(A, 2)), fit_rec(A), fit_rec(advance(A, 1))]
    assert oracle.loop_pair(fits[0], fits[1])[1] == -2
    r = join([0, 0, 0], fits)
    assert r.next.tolist() == [-1, 2, 0] and r.prev.tolist() == [2, -1, 1]
    # a track running towards -zeta (tgl < 0): its next leg has lower zeta
    Am = A * np.array([1, 1, 1, -1, 1])
    r = join([0, 0], [fit_rec(advance(Am, 1)), fit_rec(Am)])
    assert advance(Am, 1)[1] < Am[1] and r.next.tolist() == [-1, 0]


def test_equal_candidates_go_to_the_lower_index():
    fits = [fit_rec(A), fit_rec(advance(A, 1)), fit_rec(advance(A, 1))]
    r = join([0, 0, 0], fits)
    # legs 1 and 2 are identical (m = 0 between them: no pair); 0 links to 1
    assert r.next.tolist() == [1, -1, -1] and r.prev.tolist() == [-1, 0, -1]
    # the tie is leg 0's decision: its two best candidates have equal chi2
    assert r.borderline.tolist() == [1, 0, 0]


def test_legs_of_different_loopers_do_not_link():
    B = advance(A, 1)
    other_pt = B * np.array([1, 1, 1, 1, 1.1])            # q/pT 10 % off, sigma 0.05
    other_charge = B * np.array([1, 1, -1, 1, -1])        # opposite curvature
    shifted = B + np.array([0.5, 0, 0, 0, 0])             # 5 mm away in y, sigma 0.02
    for b in (other_pt, other_charge, shifted):
        r = join([0, 0], [fit_rec(A), fit_rec(b)])
        assert r.n_links == 0 and r.next.tolist() == [-1, -1]
    # a flagged fit, and a track whose circle reaches beyond the loop radius
    assert join([0, 0], [fit_rec(A), fit_rec(B, flags=1)]).n_links == 0
    stiff = np.array([3.0, 20.0, 0.3, 0.15, -1.0])        # R = 667 cm
    assert join([0, 0], [fit_rec(stiff), fit_rec(advance(stiff, 1))]).n_links == 0


def test_tgl_of_opposite_signs_is_no_pair():
    """Even with a tgl error that lets the chi2 pass, legs whose tgl differ in
    sign are no pair: a chain's legs share the sign, so zeta advances one way
    along it."""
    C = np.diag([4e-4, 9e-4, 4e-6, 0.04, 2.5e-3])          # sigma(tgl) = 0.2
    b = advance(A, 1)
    b[3] = -0.01
    assert oracle.loop_pair(fit_rec(A, cov=C), fit_rec(b, cov=C))[0] == -1.0
    b[3] = 0.01
    c2, m = oracle.loop_pair(fit_rec(A, cov=C), fit_rec(b, cov=C))
    assert m == 1 and 0.0 <= c2 < CUT


def test_turn_count_rounds_to_the_nearest_and_stays_in_range():
    S = A[3] * turn_length(A)
    for q, m in ((1.49, 1), (1.51, 2), (-1.51, -2), (4.49, 4), (0.49, None), (4.51, None), (-4.6, None)):
        b = A.copy()
        b[1] += q * S
        c2, mm = oracle.loop_pair(fit_rec(A), fit_rec(b))
        if m is None:
            assert c2 == -1.0
        else:
            assert mm == m and c2 > 0.0


def random_cov(rng, sd):
    L = np.tril(rng.normal(size=(5, 5)) * 0.4) + np.eye(5)
    C = L @ L.T
    d = np.sqrt(np.diag(C))
    return C / np.outer(d, d) * np.outer(sd, sd)


@pytest.mark.parametrize("xb", [85.0, 97.5])
def test_true_pairs_give_chi2_with_five_degrees_of_freedom(xb):
    """A = truth + N(0, C_A), B = truth one turn on (carried to x_B first when
    x_B > x_A) + N(0, C_B): the chi2 must follow chi2(5).  sigma(tgl) and
    sigma(q/pT) times the turn length dominate the zeta residual (0.46 cm and
    0.4 cm against sigma(zeta) 0.03 cm), so a wrong Jacobian of the turn advance
    would shift the mean far from 5."""
    rng = np.random.default_rng(3)
    CA = random_cov(rng, [0.02, 0.03, 0.002, 1e-3, 0.05])
    CB = random_cov(rng, [0.03, 0.04, 0.003, 1.5e-3, 0.07])
    tb = A.copy()
    if xb != 85.0:
        tb, _ = oracle.transport(A, xb - 85.0)
    tb = advance(tb, 1)
    LA, LB = np.linalg.cholesky(CA), np.linalg.cholesky(CB)
    chi2 = []
    for _ in range(4000):
        fa = fit_rec(A + LA @ rng.normal(size=5), cov=CA)
        fb = fit_rec(tb + LB @ rng.normal(size=5), x=xb, cov=CB)
        c2, m = oracle.loop_pair(fa, fb)
        assert m == 1
        chi2.append(c2)
    chi2 = np.array(chi2)
    # mean 5, standard error sqrt(10 / 4000) = 0.05; 95 % quantile of chi2(5) 11.07
    assert abs(chi2.mean() - 5.0) < 0.25, chi2.mean()
    assert abs(np.mean(chi2 > 11.0705) - 0.05) < 0.012


def test_covariances_are_scaled_by_chi2_per_ndf():
    b = advance(A, 1) + np.array([0.02, 0.05, 0.001, 0.0005, 0.03])
    c1, _ = oracle.loop_pair(fit_rec(A, chi2=5, ndf=10), fit_rec(b, chi2=8, ndf=10))
    c4, _ = oracle.loop_pair(fit_rec(A, chi2=40, ndf=10), fit_rec(b, chi2=40, ndf=10))
    assert c4 == pytest.approx(c1 / 4.0, rel=1e-12)


def test_borderline_marks_a_chi2_near_the_cut():
    """Only y differs, covariances diagonal and both legs at one x: chi2 =
    dy^2 / (C_A,yy + C_B,yy); 0.5 % above the cut is no link but borderline,
    5 % above is neither."""
    for over, border in ((1.005, 1), (1.05, 0)):
        dy = math.sqrt(CUT * over * 8e-4)
        r = join([0, 0], [fit_rec(A), fit_rec(advance(A, 1) + np.array([dy, 0, 0, 0, 0]))])
        assert r.n_links == 0 and r.borderline.tolist() == [border, border]


def test_generated_looper_links_against_generator_truth():
    """Generator truth (not a parity pin): the legs a link joins carry the same
    majority label (one generated track), and the join finds thousands."""
    tf = tpcgen.generate(tpcgen.full_tpc(1))
    r = oracle.reconstruct(tf)
    lr = oracle.join_loopers(tf, r)
    planes = oracle.decode_all(tf)
    lab = np.full(planes.shape, -1, np.int32)
    lab[np.nonzero(planes)] = tf.digit_labels
    del planes
    cl = r.clusters
    cl_lab = lab[cl["sector"], cl["row"], cl["t_peak"], cl["pad_peak"]]
    order = np.argsort(r.cl2trk, kind="stable")
    starts = np.searchsorted(r.cl2trk[order], np.arange(len(r.fits) + 1))
    major = np.full(len(r.fits), -2)
    for t in range(len(r.fits)):
        v, c = np.unique(cl_lab[order[starts[t]:starts[t + 1]]], return_counts=True)
        major[t] = v[np.argmax(c)]
    f = np.nonzero(lr.next >= 0)[0]
    same = (major[f] == major[lr.next[f]]) & (major[f] >= 0)
    print(f"looper links {len(f)}, same generated track {same.mean():.4f}, borderline {int(lr.borderline.sum())}")
    assert len(f) > 2000 and same.mean() >= 0.95
    # links are mutual, chains never branch and never close into a cycle
    assert np.all(lr.prev[lr.next[f]] == f)
    assert len(set(lr.next[f].tolist())) == len(f)
    seen = np.zeros(len(r.fits), bool)
    for t in np.nonzero(lr.prev < 0)[0]:
        while t >= 0 and not seen[t]:
            seen[t] = True
            t = lr.next[t]
    assert seen.all()
