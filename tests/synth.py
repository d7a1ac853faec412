"""Hand-built inputs for the oracle's pin tests: clusters placed at chosen
integer coordinates, and a geometry-only stand-in for a generated timeframe."""
from __future__ import annotations

import numpy as np

import oracle
import tpcgen

U_CM = 7.8125e-4


def encode_planes(planes, n_time_bins, npads=None):
    """Encode dense planes [s, r, t, p] to the documented ZS page format,
    written from the format's description alone (independent of the generator's
    encoder).  npads: pads per row (default: the default geometry's)."""
    out = bytearray()
    offs = []
    S, R, T, _ = planes.shape
    if npads is None:
        npads, _ = tpcgen.default_geometry()
    nf = (n_time_bins + 255) // 256
    for s in range(S):
        for r in range(R):
            np_ = int(npads[r])
            for f in range(nf):
                ents, runs, adcs = [], [], []
                lo = hi = None
                for tt in range(256):
                    t = 256 * f + tt
                    if tt == 253 and hi is None:
                        hi = (len(ents), len(runs), len(adcs))
                    if t < n_time_bins:
                        row = planes[s, r, t, :np_]
                        nz = np.nonzero(row)[0]
                        if len(nz):
                            # maximal runs of consecutive pads
                            splits = np.nonzero(np.diff(nz) > 1)[0] + 1
                            groups = np.split(nz, splits)
                            ents.append((tt, len(groups)))
                            for g in groups:
                                runs.append((int(g[0]), len(g)))
                                adcs.extend(int(v) for v in row[g])
                    if tt == 2:
                        lo = (len(ents), len(runs), len(adcs))
                if hi is None:
                    hi = (len(ents), len(runs), len(adcs))
                body = 32 + 2 * len(ents) + 2 * len(runs)
                body = (body + 3) // 4 * 4
                nw = (len(adcs) + 2) // 3
                ln = (body + 4 * nw + 15) // 16 * 16
                pg = bytearray(ln)
                pg[0:4] = ln.to_bytes(4, "little")
                pg[4:6] = len(ents).to_bytes(2, "little")
                pg[6:8] = len(runs).to_bytes(2, "little")
                pg[8:10] = len(adcs).to_bytes(2, "little")
                pg[10], pg[11] = s, r
                pg[12:14] = f.to_bytes(2, "little")
                pg[14:16] = (0x5A53).to_bytes(2, "little")
                for i, v in enumerate(lo + hi):
                    pg[16 + 2 * i:18 + 2 * i] = v.to_bytes(2, "little")
                o = 32
                for (t, n) in ents:
                    pg[o], pg[o + 1] = t, n
                    o += 2
                for (p, n) in runs:
                    pg[o], pg[o + 1] = p, n
                    o += 2
                for w in range(nw):
                    word = 0
                    for k in range(3):
                        if 3 * w + k < len(adcs):
                            word |= adcs[3 * w + k] << (10 * k)
                    pg[body + 4 * w:body + 4 * w + 4] = word.to_bytes(4, "little")
                offs.append(len(out))
                out += pg
    return np.frombuffer(bytes(out), np.uint8), np.array(offs, np.uint64)


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
    units), or (sector, row, Y, Z, R) with the time centroid R/128 bins from the
    peak bin (|R| <= 256, as step 3 allows; (Z - 5 R) a multiple of 640); by
    default the peak is the bin nearest to the centroid.  Returns clusters
    sorted in canonical order and the permutation."""
    rec = []
    for pt in pts:
        s, r, Y, Z = pt[:4]
        assert Y % 2 == 0 and Z % 5 == 0
        np_ = int(geom.npads[r])
        pad_fp = Y // 2 + 128 * (np_ - 1)
        zi = Z // 5
        if len(pt) == 5:
            R = pt[4]
            assert abs(R) <= 256 and (Z - 5 * R) % 640 == 0
            t_peak = (Z - 5 * R) // 640
        else:
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
