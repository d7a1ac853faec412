"""Comparison of the CUDA path's results with the oracle's.

Integers (clusters, CA links, chains, cluster-to-track map, track membership,
track flags, ndf) must be bit-exact.  Track parameters must agree with the FP64
oracle within

    1e-4 * max(|p|, floor_p) * A  +  2e-5 * sigma_p * max(1, chi2 / ndf)

floors y, zeta 1 cm; snp, tgl 0.1; q/pT 0.1 1/GeV; sigma_p, chi2 and ndf the
oracle's own.  The first term is the plain bar.  The second is what FP32
rounding does where a parameter is barely measured or the track does not fit
its clusters: q/pT of a 10-cluster track has sigma ~1 1/GeV, and one FP32
rounding of each row-to-row step of the measurements moves the exact FP64
answer by up to ~3e-6 sigma (the FP32 fit, with a few roundings per step,
by ~1e-5 sigma); on a track built from several particles (chi2/ndf in the
hundreds or thousands at 50 kHz pile-up) every update moves the state by many
sigma and the FP32 answer follows a rounding-dependent path: an FP32
emulation of the fit under four rounding patterns scatters by up to 5e-6
sigma per unit of chi2/ndf (1.2e-4 to 1.8e-3 relative in q/pT for a track of
chi2/ndf 5,000).  A = 1, except for tracks whose fit stopped
(TPC_TRK_STOPPED): their state is that at the stop, next to |snp| = 0.999,
where the state's sensitivity to rounding grows as 1 / cos^3 phi, so A = (1 -
snp^2)^(-3/2).  Covariances must agree within 1e-3 * sqrt(C_ii C_jj) * A.
Every track is compared; only tracks flagged TPC_TRK_NOT_PD on both sides would
be left out of the parameter comparison.

Some tracks built from several particles are more sensitive than the chi2/ndf
term allows (at 50 kHz pile-up, one of 18,116 tracks of a sector: chi2/ndf
1,270, whose FP64 snp moves by 0.070 sigma when the quantities the FP32 fit stores are
rounded, against 0.067 sigma between the GPU and the oracle).  Given the
timeframe (compare_fit's tf), a track outside the bounds above is measured
against the oracle itself: the oracle's own transport and update are replayed
step by step for that track, and after each of them every state entry and
every entry of the covariance's U D U^T factors (the FP32 fit's
representation) is multiplied by (1 + e), |e| <= 2^-24, one rounding of each
stored quantity per step where the FP32 fit has several, over 32 seeded
patterns; the track passes if each of its parameters (and covariance entries)
lies within the bounds above or differs from the oracle's by no more than the
largest deviation of those patterns.  On single-particle tracks that spread stays below the plain bar
(q/pT up to half of it), so the check cannot loosen their comparison.
"""
from __future__ import annotations

import numpy as np

PAR_FLOORS = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
PAR_RTOL = 1e-4
COV_RTOL = 1e-3
SIGMA_FRAC = 2e-5
TRI = [(i, j) for i in range(5) for j in range(i + 1)]


def cluster_bytes(a):
    return np.ascontiguousarray(a).view(np.uint8).reshape(len(a), 16)


def compare_integer(gpu: dict, orc) -> None:
    gcl, ocl = gpu["clusters"], orc.clusters
    assert len(gcl) == len(ocl), f"cluster count {len(gcl)} != oracle {len(ocl)}"
    gb, ob = cluster_bytes(gcl), cluster_bytes(ocl)
    bad = np.nonzero(np.any(gb != ob, axis=1))[0]
    assert len(bad) == 0, f"{len(bad)} clusters differ, first {bad[:5]}: gpu {gcl[bad[:2]]} oracle {ocl[bad[:2]]}"
    for k in ("up", "down", "chain_of", "cl2trk"):
        g, o = gpu[k], getattr(orc, k)
        bad = np.nonzero(g != o)[0]
        assert len(bad) == 0, f"{k}: {len(bad)} differ, first {bad[:5]} gpu {g[bad[:5]]} oracle {o[bad[:5]]}"
    tr = gpu["tracks"]
    assert len(tr) == len(orc.track_first)
    assert np.array_equal(tr["first_cluster"], orc.track_first)
    assert np.array_equal(tr["n_clusters"], orc.track_ncl)


def stop_conditioning(par, flags):
    """A of the module docstring: 1, or (1 - snp^2)^(-3/2) for a stopped fit."""
    snp2 = np.minimum(np.asarray(par)[:, 2] ** 2, 0.999 ** 2)
    return np.where(np.asarray(flags) & 1, (1.0 - snp2) ** -1.5, 1.0)


def param_allowance(par, cov, chi2, ndf, flags):
    """The allowed |diff| of each parameter (see the module docstring) for
    oracle states par [n, 5], covariances cov [n, 15] (lower triangle), chi2,
    ndf and flags [n]."""
    diag = [0, 2, 5, 9, 14]
    sig = np.sqrt(cov[:, diag])
    A = stop_conditioning(par, flags)
    s = np.maximum(1.0, np.asarray(chi2, np.float64) / np.maximum(np.asarray(ndf, np.float64), 1.0))
    return PAR_RTOL * np.maximum(np.abs(par), PAR_FLOORS) * A[:, None] + SIGMA_FRAC * sig * s[:, None]


def fit_errors(gpu_tracks, fits):
    """Per-parameter |diff| in units of the allowed error times 1e-4 (<= 1e-4
    passes), the plain-floor relative error, and the cov deviation in units of
    sqrt(C_ii C_jj), over the tracks whose covariance is positive definite on
    both sides (flags must already be equal)."""
    ok = ((gpu_tracks["flags"] & 2) == 0) & ((fits["flags"] & 2) == 0)
    gp = gpu_tracks["par"][ok].astype(np.float64)
    op = fits["par"][ok]
    diag = [0, 2, 5, 9, 14]
    allow = param_allowance(op, fits["cov"][ok], fits["chi2"][ok], fits["ndf"][ok], fits["flags"][ok])
    rel = np.abs(gp - op) / allow * PAR_RTOL
    rel_plain = np.abs(gp - op) / np.maximum(np.abs(op), PAR_FLOORS)
    gc = gpu_tracks["cov"][ok].astype(np.float64)
    oc = fits["cov"][ok]
    cond = stop_conditioning(op, fits["flags"][ok])
    cov_dev = np.zeros((ok.sum(), 15))
    for m, (i, j) in enumerate(TRI):
        cov_dev[:, m] = np.abs(gc[:, m] - oc[:, m]) / np.sqrt(oc[:, diag[i]] * oc[:, diag[j]]) / cond
    return rel, cov_dev, ok, rel_plain


PERTURB_EPS = 2.0 ** -24
PERTURB_PATTERNS = 32
U_CM = 7.8125e-4


def _ud(C):
    """C = U D U^T with U unit upper triangular (the GPU fit's representation)."""
    n = 5
    Uu, D = np.eye(n), np.zeros(n)
    for j in range(n - 1, -1, -1):
        D[j] = C[j, j] - sum(D[k] * Uu[j, k] ** 2 for k in range(j + 1, n))
        for i in range(j):
            Uu[i, j] = (C[i, j] - sum(D[k] * Uu[i, k] * Uu[j, k] for k in range(j + 1, n))) / D[j]
    return Uu, D


def _fit_replay(x, y, z, P, rng=None, eps=PERTURB_EPS):
    """The oracle's FP64 fit of points (cm, ascending x), step by step through
    its own transport and update (three passes inward / outward / inward, the
    covariance reset each pass, a stopped transport ending its pass).  With
    rng, after each transport and update every state entry and every entry of
    the covariance's U D U^T factors is multiplied by (1 + e), |e| <= eps: the
    rounding of the quantities the FP32 fit stores.  Returns (state, covariance)."""
    import oracle
    n = len(x)
    i1, i2, i3 = 0, (n - 1) // 2, n - 1
    ax, ay = x[i2] - x[i1], y[i2] - y[i1]
    bx, by = x[i3] - x[i2], y[i3] - y[i2]
    cx, cy = x[i3] - x[i1], y[i3] - y[i1]
    la, lb, lc = np.hypot(ax, ay), np.hypot(bx, by), np.hypot(cx, cy)
    k = 2.0 * (ax * cy - ay * cx) / (la * lb * lc)
    half = np.arcsin(min(1.0, max(-1.0, k * lc / 2.0)))
    phic = np.arctan2(cy, cx)
    arc = lc * (1.0 + (k * lc) ** 2 / 24.0) if abs(k * lc) < 1e-3 else 2.0 * half / k
    kfac = -P.bz * 0.299792458 * 1e-2          # curvature (1/cm) per q/pT (1/GeV)
    s = np.array([y[i3], z[i3], np.sin(phic + half), (z[i3] - z[i1]) / arc, k / kfac])

    def jig_s(a):
        return a if rng is None else a * (1.0 + rng.uniform(-eps, eps, size=a.shape))

    def jig_c(C):
        if rng is None:
            return C
        Uu, D = _ud(C)
        Uu = Uu * (1.0 + rng.uniform(-eps, eps, size=Uu.shape))
        np.fill_diagonal(Uu, 1.0)
        D = D * (1.0 + rng.uniform(-eps, eps, size=5))
        return Uu @ np.diag(D) @ Uu.T
    xcur = x[n - 1]
    C = None
    for p in range(P.fit_passes):
        C = np.diag(np.array(P.c0, np.float64))
        inward = p % 2 == 0
        for j in range(n):
            i = n - 1 - j if inward else j
            if x[i] != xcur:
                ns, F = oracle.transport(s, x[i] - xcur, P)
                if ns is None:
                    break
                C = jig_c(F @ C @ F.T)
                s = jig_s(ns)
                xcur = x[i]
            s, C, _, _ = oracle.update(s, C, y[i], z[i], P)
            s = jig_s(s)
            C = jig_c(C)
    return s, C


def perturbation_spread(X, Y, Z, oracle_par, params=None, patterns=PERTURB_PATTERNS, seed=1):
    """Largest deviations of the oracle's fit of one track (integer cluster
    coordinates X, Y, Z in u, ascending row) under FP32-sized rounding of its
    steps: (per parameter, per lower-triangle covariance entry), absolute.  The
    unperturbed replay must reproduce the oracle's parameters."""
    import oracle
    P = params or oracle.OracleParams()
    X, Y, Z = (np.asarray(a, np.int64) for a in (X, Y, Z))
    x, y, z = X * U_CM, (Y - Y[0]) * U_CM, (Z - Z[0]) * U_CM
    s0, C0 = _fit_replay(x, y, z, P)
    par0 = s0 + np.array([Y[0] * U_CM, Z[0] * U_CM, 0.0, 0.0, 0.0])
    assert np.allclose(par0, oracle_par, rtol=1e-9, atol=1e-9), (par0, oracle_par)
    rng = np.random.default_rng(seed)
    dpar = np.zeros(5)
    dcov = np.zeros(15)
    for _ in range(patterns):
        s, C = _fit_replay(x, y, z, P, rng)
        dpar = np.maximum(dpar, np.abs(s - s0))
        dcov = np.maximum(dcov, np.abs(np.array([C[i, j] - C0[i, j] for i, j in TRI])))
    return dpar, dcov


def _conditioning_pass(gpu_tracks, orc, tf, tracks) -> list:
    """For each track index in tracks: whether its parameters and covariance lie
    within the oracle's own FP32-sized rounding spread (module docstring)."""
    import oracle
    cl2trk = np.asarray(orc.cl2trk)
    out = []
    for t in tracks:
        members = np.nonzero(cl2trk == t)[0]
        X, Y, Z = oracle.coords(tf, orc.clusters[members])
        o = orc.fits[t]
        dpar, dcov = perturbation_spread(X, Y, Z, o["par"])
        g = gpu_tracks[t]
        dp = np.abs(g["par"].astype(np.float64) - o["par"])
        dc = np.abs(g["cov"].astype(np.float64) - o["cov"])
        # a parameter within the bounds above stays accepted; the others must
        # lie within the spread
        dpar = np.maximum(dpar, param_allowance(o["par"][None], o["cov"][None], [o["chi2"]], [o["ndf"]],
                                                [o["flags"]])[0])
        cov_ok = (dc <= np.maximum(dcov, COV_RTOL * np.sqrt([o["cov"][[0, 2, 5, 9, 14][i]] * o["cov"][[0, 2, 5, 9, 14][j]]
                                                            for i, j in TRI]))).all()
        out.append(dict(track=int(t), ok=bool((dp <= dpar).all() and cov_ok),
                        dev_over_spread=(dp / np.maximum(dpar, 1e-300)).tolist()))
    return out


def compare_fit(gpu: dict, orc, tf=None) -> dict:
    tr, fits = gpu["tracks"], orc.fits
    # the GPU's flags carry only the step-8 bits here (XSECTOR belongs to step 9)
    gflags = tr["flags"].astype(np.int64) & 3
    oflags = fits["flags"].astype(np.int64)
    bad = np.nonzero(gflags != oflags)[0]
    assert len(bad) == 0, f"{len(bad)} track flags differ, first {bad[:5]}: gpu {gflags[bad[:5]]} oracle {oflags[bad[:5]]}"
    assert np.array_equal(tr["ndf"], fits["ndf"]), "ndf differ"
    rel, cov_dev, ok, rel_plain = fit_errors(tr, fits)
    assert np.allclose(tr["x"], fits["x"], rtol=1e-6)
    report = {"max_rel_par": rel.max(0).tolist() if len(rel) else [0] * 5,
              "max_rel_par_plain_floor": rel_plain.max(0).tolist() if len(rel) else [0] * 5,
              "frac_plain_floor_over_1e-4": float((rel_plain > PAR_RTOL).any(1).mean()) if len(rel) else 0.0,
              "max_cov_dev": float(cov_dev.max()) if cov_dev.size else 0.0,
              "n_tracks": int(len(tr)), "n_compared": int(ok.sum()),
              "n_stopped": int((oflags & 1).sum()), "n_not_pd": int(((oflags & 2) != 0).sum())}
    if not np.all(rel <= PAR_RTOL):
        idx = np.nonzero(ok)[0]
        worst = np.argsort(rel.max(1))[::-1][:5]
        diag = [0, 2, 5, 9, 14]
        report["worst"] = [dict(track=int(idx[w]), n_clusters=int(tr["n_clusters"][idx[w]]),
                                first_cluster=int(tr["first_cluster"][idx[w]]),
                                gpu=tr["par"][idx[w]].tolist(), oracle=fits["par"][idx[w]].tolist(),
                                sigma=np.sqrt(fits["cov"][idx[w]][diag]).tolist(),
                                chi2_ndf=float(fits["chi2"][idx[w]] / max(fits["ndf"][idx[w]], 1)),
                                flags=int(fits["flags"][idx[w]]),
                                n_fp64=int(tr["n_fp64"][idx[w]])) for w in worst]
    out_par = ~np.all(rel <= PAR_RTOL, axis=1)
    out_cov = ~np.all(cov_dev <= COV_RTOL, axis=1)
    if tf is not None and (out_par | out_cov).any() and (out_par | out_cov).sum() <= 50:
        # outside the bounds: within the oracle's own FP32-sized rounding spread?
        idx = np.nonzero(ok)[0]
        checked = _conditioning_pass(tr, orc, tf, idx[out_par | out_cov])
        report["conditioning_checked"] = checked
        passed = np.array([c["ok"] for c in checked])
        keep = np.ones(len(rel), bool)
        keep[np.nonzero(out_par | out_cov)[0][passed]] = False
        rel, cov_dev, ids = rel[keep], cov_dev[keep], idx[keep]
    else:
        ids = np.nonzero(ok)[0]
    assert np.all(rel <= PAR_RTOL), f"params beyond 1e-4: {report}"
    if not np.all(cov_dev <= COV_RTOL):
        w = ids[int(np.argmax(cov_dev.max(1)))]
        report["worst_cov"] = dict(track=int(w), n_clusters=int(tr["n_clusters"][w]), flags=int(fits["flags"][w]),
                                   chi2_ndf=float(fits["chi2"][w] / max(fits["ndf"][w], 1)),
                                   oracle_par=fits["par"][w].tolist(), gpu_cov=tr["cov"][w].tolist(),
                                   oracle_cov=fits["cov"][w].tolist())
    assert np.all(cov_dev <= COV_RTOL), f"cov beyond 1e-3: {report}"
    return report
