"""Comparison of the CUDA path's results with the oracle's.

Integers (clusters, CA links, chains, cluster-to-track map, track membership)
must be bit-exact.  Track parameters must agree with the FP64 oracle within
1e-4 * max(|p|, floor_p) + 1e-3 * sigma_p: floors y, zeta 1 cm; snp, tgl 0.1;
q/pT 0.1 1/GeV; sigma_p the oracle's own standard deviation of the parameter.
The sigma term only matters where the fit is ill-conditioned (short or nearly
straight tracks whose curvature is barely measured): there, rounding the
measurements alone to FP32 moves the exact FP64 answer by up to ~2e-4 sigma_p,
more than 1e-4 of the plain floor, so no FP32 fit can meet the plain bound.
Covariances must agree within 1e-3 * sqrt(C_ii C_jj)."""
from __future__ import annotations

import numpy as np

PAR_FLOORS = np.array([1.0, 1.0, 0.1, 0.1, 0.1])
PAR_RTOL = 1e-4
COV_RTOL = 1e-3
SIGMA_FRAC = 1e-3
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


def fit_errors(gpu_tracks, fits):
    """Per-parameter max |diff| / max(|p|, floor) and max cov deviation in units
    of sqrt(C_ii C_jj); tracks flagged by either side are excluded."""
    ok = (gpu_tracks["flags"] == 0) & (fits["flags"] == 0)
    gp = gpu_tracks["par"][ok].astype(np.float64)
    op = fits["par"][ok]
    diag = [0, 2, 5, 9, 14]
    sig = np.sqrt(fits["cov"][ok][:, diag])
    # error in units of the allowed error (<= 1 passes)
    rel = np.abs(gp - op) / (np.maximum(np.abs(op), PAR_FLOORS) + SIGMA_FRAC / PAR_RTOL * sig) 
    rel_plain = np.abs(gp - op) / np.maximum(np.abs(op), PAR_FLOORS)
    gc = gpu_tracks["cov"][ok].astype(np.float64)
    oc = fits["cov"][ok]
    cov_dev = np.zeros((ok.sum(), 15))
    for m, (i, j) in enumerate(TRI):
        cov_dev[:, m] = np.abs(gc[:, m] - oc[:, m]) / np.sqrt(oc[:, diag[i]] * oc[:, diag[j]])
    return rel, cov_dev, ok, rel_plain


def compare_fit(gpu: dict, orc, min_ok_fraction: float = 0.99) -> dict:
    tr, fits = gpu["tracks"], orc.fits
    assert np.array_equal(tr["ndf"][(tr["flags"] == 0) & (fits["flags"] == 0)],
                          fits["ndf"][(tr["flags"] == 0) & (fits["flags"] == 0)])
    rel, cov_dev, ok, rel_plain = fit_errors(tr, fits)
    assert ok.mean() >= min_ok_fraction if len(ok) else True, f"flagged fraction {1 - ok.mean()}"
    assert np.allclose(tr["x"], fits["x"], rtol=1e-6)
    report = {"max_rel_par": rel.max(0).tolist() if len(rel) else [0] * 5,
              "max_rel_par_plain_floor": rel_plain.max(0).tolist() if len(rel) else [0] * 5,
              "frac_plain_floor_over_1e-4": float((rel_plain > PAR_RTOL).any(1).mean()) if len(rel) else 0.0,
              "max_cov_dev": float(cov_dev.max()) if cov_dev.size else 0.0,
              "n_tracks": int(len(tr)), "n_compared": int(ok.sum())}
    if not np.all(rel <= PAR_RTOL):
        idx = np.nonzero(ok)[0]
        worst = np.argsort(rel.max(1))[::-1][:5]
        diag = [0, 2, 5, 9, 14]
        report["worst"] = [dict(track=int(idx[w]), n_clusters=int(tr["n_clusters"][idx[w]]),
                                first_cluster=int(tr["first_cluster"][idx[w]]),
                                gpu=tr["par"][idx[w]].tolist(), oracle=fits["par"][idx[w]].tolist(),
                                sigma=np.sqrt(fits["cov"][idx[w]][diag]).tolist(),
                                n_fp64=int(tr["n_fp64"][idx[w]])) for w in worst]
    assert np.all(rel <= PAR_RTOL), f"params beyond 1e-4: {report}"
    assert np.all(cov_dev <= COV_RTOL), f"cov beyond 1e-3: {report}"
    return report
