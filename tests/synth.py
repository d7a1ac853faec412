"""Hand-built inputs for the oracle's pin tests: clusters placed at chosen
integer coordinates, and a geometry-only stand-in for a generated timeframe."""
from __future__ import annotations

import numpy as np

import oracle
import tpcgen

U_CM = 7.8125e-4


class Geom:
    """Duck-types the fields of tpcgen.Timeframe the oracle needs, with no pages."""

    def __init__(self, n_sectors=1, n_time_bins=1000, npads=None, row_x=None):
        g_np, g_x = tpcgen.default_geometry()
        self.npads = g_np if npads is None else np.asarray(npads, np.int32)
        self.row_x = g_x if row_x is None else np.asarray(row_x, np.int32)
        self.n_sectors = n_sectors
        self.n_time_bins = n_time_bins
        nf = (n_time_bins + 255) // 256
        self.pages = np.zeros(0, np.uint8)
        self.page_offsets = np.zeros(n_sectors * len(self.npads) * nf, np.uint64)

    @property
    def n_rows(self):
        return len(self.npads)


def make_clusters(geom: Geom, pts):
    """pts: iterable of (sector, row, Y, Z) with Y even and Z a multiple of 5 (u
    units).  Returns clusters sorted in canonical order and the permutation."""
    rec = []
    for (s, r, Y, Z) in pts:
        assert Y % 2 == 0 and Z % 5 == 0
        np_ = int(geom.npads[r])
        pad_fp = Y // 2 + 128 * (np_ - 1)
        zi = Z // 5
        t_peak = int(round(zi / 128.0))
        f = t_peak // 256
        time_fp = zi - 128 * 256 * f + 512
        assert 0 <= pad_fp < 65536 and 0 <= time_fp < 65536
        pad_peak = int(round(pad_fp / 256.0))
        rec.append((pad_fp, time_fp, 50, 300, 16, 16, 0, r, t_peak, max(0, min(np_ - 1, pad_peak)), s))
    cl = np.array(rec, dtype=oracle.CLUSTER_DTYPE)
    key = (cl["sector"].astype(np.int64) * 256 + cl["row"]) * 65536 * 256 + \
        cl["t_peak"].astype(np.int64) * 256 + cl["pad_peak"]
    order = np.argsort(key, kind="stable")
    return cl[order], order


def helix_points(x_rows, y0, z0, phi0, tgl, qpt, bz=0.5):
    """Exact crossings of a helix with the planes x = x_rows (cm, ascending), in
    the sector-local frame, starting at x_rows[0] with local direction phi0.
    Parametrised by the direction angle: x(phi) = x0 + (sin phi - sin phi0)/k,
    y(phi) = y0 - (cos phi - cos phi0)/k, arc s = (phi - phi0)/k, zeta = z0 + tgl s."""
    k = -bz * 0.299792458e-2 * qpt
    x0 = x_rows[0]
    ys, zs = [], []
    for x in x_rows:
        if abs(k) < 1e-12:
            y = y0 + (x - x0) * np.tan(phi0)
            s = (x - x0) / np.cos(phi0)
        else:
            sphi = np.sin(phi0) + k * (x - x0)
            phi = np.arcsin(sphi)
            y = y0 - (np.cos(phi) - np.cos(phi0)) / k
            s = (phi - phi0) / k
        ys.append(y)
        zs.append(z0 + tgl * s)
    return np.array(ys), np.array(zs)
