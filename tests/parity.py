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


def compare_fit(gpu: dict, orc) -> dict:
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
    assert np.all(rel <= PAR_RTOL), f"params beyond 1e-4: {report}"
    if not np.all(cov_dev <= COV_RTOL):
        idx = np.nonzero(ok)[0]
        w = idx[int(np.argmax(cov_dev.max(1)))]
        report["worst_cov"] = dict(track=int(w), n_clusters=int(tr["n_clusters"][w]), flags=int(fits["flags"][w]),
                                   chi2_ndf=float(fits["chi2"][w] / max(fits["ndf"][w], 1)),
                                   oracle_par=fits["par"][w].tolist(), gpu_cov=tr["cov"][w].tolist(),
                                   oracle_cov=fits["cov"][w].tolist())
    assert np.all(cov_dev <= COV_RTOL), f"cov beyond 1e-3: {report}"
    return report
