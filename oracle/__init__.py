"""CPU oracle of the TPC timeframe reconstruction — TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import this package.  The library (``paper_2208_07412_b300``)
never does, and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, exact integers, FP64 fit; built
``-O2`` without fast-math).  This module only marshals arguments.  What each
function computes, and the passage it follows, is stated in ``oracle.c``: the
paper (section "Hardware and data flow") says that the EPN GPUs run the full
online TPC reconstruction on zero-suppressed data but defines no algorithm, so
the oracle writes out the library's documented definition in its plainest form.

Parity status: decode, peaks, clusters, CA, merge and fit are pinned by the
``-m "not gpu"`` tests (round trip, 3x3 maximum filter, closed forms,
hand-worked examples, gap closure, exact-helix closure, finite differences,
information-form update, pulls).  Tracking efficiency / fake rate against the
generator truth: parity unpinned (the paper prints no figure).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CLUSTER_DTYPE = np.dtype([("pad_fp", "<u2"), ("time_fp", "<u2"), ("qmax", "<u2"), ("qtot", "<u2"),
                          ("sigma2_pad", "u1"), ("sigma2_time", "u1"), ("flags", "u1"),
                          ("row", "u1"), ("t_peak", "<u2"), ("pad_peak", "u1"), ("sector", "u1")])
assert CLUSTER_DTYPE.itemsize == 16

FIT_DTYPE = np.dtype([("par", "<f8", (5,)), ("x", "<f8"), ("cov", "<f8", (15,)), ("chi2", "<f8"),
                      ("ndf", "<i4"), ("n_used", "<i4"), ("flags", "<i4"), ("pad", "<i4")])
assert FIT_DTYPE.itemsize == 8 * 22 + 16

U_CM = 7.8125e-4


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared",
                               "-fPIC", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Input(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("npads", ctypes.c_void_p), ("row_x", ctypes.c_void_p),
                ("n_time_bins", ctypes.c_int32), ("pages", ctypes.c_void_p),
                ("pages_bytes", ctypes.c_uint64), ("page_offsets", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("q_peak_min", ctypes.c_int32), ("sy_num", ctypes.c_int32),
                ("sy_den", ctypes.c_int32), ("sz_num", ctypes.c_int32),
                ("sz_den", ctypes.c_int32), ("ca_cut", ctypes.c_int32),
                ("min_chain", ctypes.c_int32), ("merge_cut", ctypes.c_int32),
                ("gap_min", ctypes.c_int32), ("gap_max", ctypes.c_int32),
                ("merge_passes", ctypes.c_int32), ("min_track", ctypes.c_int32),
                ("fit_passes", ctypes.c_int32), ("ns_min_dip", ctypes.c_int32), ("bz", ctypes.c_double),
                ("sigma_y", ctypes.c_double), ("sigma_z", ctypes.c_double),
                ("c0", ctypes.c_double * 5), ("search_all", ctypes.c_int32),
                ("split_charge", ctypes.c_int32)]


@dataclass
class OracleParams:
    """The oracle's own copy of the reconstruction constants."""
    q_peak_min: int = 10
    sy_num: int = 1
    sy_den: int = 1
    sz_num: int = 11
    sz_den: int = 10
    ca_cut: int = 256          # 0.2 cm in u
    min_chain: int = 5
    merge_cut: int = 384       # 0.3 cm in u
    gap_min: int = 1
    gap_max: int = 6
    merge_passes: int = 8
    min_track: int = 10
    fit_passes: int = 3
    ns_min_dip: int = 0        # 5x5 noise suppression (step 2b): 0 off
    bz: float = 0.5
    sigma_y: float = 0.02
    sigma_z: float = 0.03
    c0: tuple = (4.0, 4.0, 0.25, 1.0, 100.0)
    search_all: bool = False   # CA / merge visit every candidate (no time window)
    split_charge: bool = False  # step 3s: pixels near several peaks share their charge

    def _c(self) -> _Params:
        p = _Params()
        for k in ("q_peak_min", "sy_num", "sy_den", "sz_num", "sz_den", "ca_cut", "min_chain",
                  "merge_cut", "gap_min", "gap_max", "merge_passes", "min_track", "fit_passes", "ns_min_dip",
                  "search_all", "split_charge"):
            setattr(p, k, int(getattr(self, k)))
        p.bz, p.sigma_y, p.sigma_z = self.bz, self.sigma_y, self.sigma_z
        for i in range(5):
            p.c0[i] = self.c0[i]
        return p


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_decode_row.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P]
        L.orc_decode_all.argtypes = [_P, _P, ctypes.c_int]
        L.orc_find_clusters.argtypes = [_P, _P, _P, ctypes.c_int64]
        L.orc_find_clusters.restype = ctypes.c_int64
        L.orc_peaks_plane.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
        L.orc_peaks_plane_ns.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]
        L.orc_entropy_encode.argtypes = [ctypes.c_int64, _P, _P, _P, _P, _P, ctypes.c_int64]
        L.orc_entropy_encode.restype = ctypes.c_int64
        L.orc_cluster_at.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, _P]
        L.orc_split_share.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int]
        L.orc_ca.argtypes = [_P, _P, _P, ctypes.c_int64, _P, _P, _P]
        L.orc_merge.argtypes = [_P, _P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_int64, _P]
        L.orc_merge.restype = ctypes.c_int64
        L.orc_fit_all.argtypes = [_P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P]
        L.orc_fit_points.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.orc_fit_track.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P]
        L.orc_transport.argtypes = [_P, _P, ctypes.c_double, _P, _P]
        L.orc_update.argtypes = [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P]
        L.orc_update.restype = ctypes.c_double
        L.orc_rotate.argtypes = [_P, _P, _P, ctypes.c_double, _P]
        L.orc_xs_chi2.argtypes = [_P, _P, ctypes.c_double, _P, ctypes.c_double]
        L.orc_xs_chi2.restype = ctypes.c_double
        L.orc_fit_points_xs.argtypes = [_P, ctypes.c_int, _P, _P, _P, _P, _P]
        L.orc_merge_sectors.argtypes = [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P,
                                        _P, _P, _P, _P, _P]
        L.orc_merge_sectors.restype = ctypes.c_int64
        L.orc_join_loopers.argtypes = [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P, _P]
        L.orc_join_loopers.restype = ctypes.c_int64
        L.orc_loop_pair.argtypes = [_P, _P, _P, _P, _P]
        L.orc_loop_pair.restype = ctypes.c_double
        L.orc_loops.argtypes = [_P, _P, ctypes.c_double]
        L.orc_loops.restype = ctypes.c_int
        L.orc_compress.argtypes = [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P]
        L.orc_compress.restype = ctypes.c_int64
        L.orc_calibrate_drift.argtypes = [_P, _P, _P, ctypes.c_int64, ctypes.c_double, _P, _P, _P]
        L.orc_calibrate_drift.restype = ctypes.c_int64
        _lib = L
    return _lib


class _In:
    """Keeps the numpy buffers of one oracle input alive."""

    def __init__(self, pages, page_offsets, npads, row_x, n_sectors, n_time_bins):
        self.pages = np.ascontiguousarray(pages, dtype=np.uint8)
        self.offs = np.ascontiguousarray(page_offsets, dtype=np.uint64)
        self.npads = np.ascontiguousarray(npads, dtype=np.int32)
        self.row_x = np.ascontiguousarray(row_x, dtype=np.int32)
        s = _Input()
        s.n_sectors, s.n_rows = int(n_sectors), int(len(self.npads))
        s.npads, s.row_x = self.npads.ctypes.data, self.row_x.ctypes.data
        s.n_time_bins = int(n_time_bins)
        s.pages = self.pages.ctypes.data if self.pages.size else None
        s.pages_bytes = int(self.pages.size)
        s.page_offsets = self.offs.ctypes.data
        self.s = s

    @classmethod
    def from_tf(cls, tf):
        return cls(tf.pages, tf.page_offsets, tf.npads, tf.row_x, tf.n_sectors, tf.n_time_bins)

    @property
    def ref(self):
        return ctypes.byref(self.s)


class CorruptPage(Exception):
    pass


def decode_all(tf) -> np.ndarray:
    """Dense planes [sector, row, t, pad] (pads padded to the widest row)."""
    L = _load()
    inp = _In.from_tf(tf)
    npmax = int(inp.npads.max())
    out = np.zeros((tf.n_sectors, len(inp.npads), tf.n_time_bins, npmax), dtype=np.uint16)
    if L.orc_decode_all(inp.ref, out.ctypes.data, npmax) != 0:
        raise CorruptPage("corrupt ZS page")
    return out


def peaks_plane(plane: np.ndarray, q_peak_min: int = 10, ns_min_dip: int = 0) -> np.ndarray:
    """Peak flags of one dense plane q[t, pad] (after step 2b's noise
    suppression when ns_min_dip > 0)."""
    L = _load()
    plane = np.ascontiguousarray(plane, dtype=np.uint16)
    T, np_ = plane.shape
    fl = np.zeros((T, np_), dtype=np.uint8)
    if ns_min_dip:
        L.orc_peaks_plane_ns(plane.ctypes.data, np_, T, q_peak_min, ns_min_dip, fl.ctypes.data)
    else:
        L.orc_peaks_plane(plane.ctypes.data, np_, T, q_peak_min, fl.ctypes.data)
    return fl.astype(bool)


def cluster_at(plane: np.ndarray, pad: int, t: int, q_peak_min: int = 10, split: bool = False) -> np.void:
    L = _load()
    plane = np.ascontiguousarray(plane, dtype=np.uint16)
    T, np_ = plane.shape
    out = np.zeros(1, dtype=CLUSTER_DTYPE)
    L.orc_cluster_at(plane.ctypes.data, np_, T, pad, t, q_peak_min, int(split), out.ctypes.data)
    return out[0]


def split_share(plane: np.ndarray, peak: tuple, pixel: tuple, q_peak_min: int = 10) -> int:
    """Step 3s: the charge of pixel (pad, t) that the cluster of the peak
    (pad, t) counts when charge splitting is on."""
    L = _load()
    plane = np.ascontiguousarray(plane, dtype=np.uint16)
    T, np_ = plane.shape
    return int(L.orc_split_share(plane.ctypes.data, np_, T, q_peak_min, peak[0], peak[1], pixel[0], pixel[1]))


def find_clusters(tf, params: OracleParams | None = None) -> np.ndarray:
    L = _load()
    p = (params or OracleParams())._c()
    inp = _In.from_tf(tf)
    n = L.orc_find_clusters(inp.ref, ctypes.byref(p), None, 0)
    if n < 0:
        raise CorruptPage("corrupt ZS page")
    out = np.zeros(n, dtype=CLUSTER_DTYPE)
    L.orc_find_clusters(inp.ref, ctypes.byref(p), out.ctypes.data if n else None, n)
    return out


def coords(tf, clusters: np.ndarray):
    """Integer (X, Y, Z) in u = 7.8125 um (restated here from the same definition
    for convenience of the tests; the C code is what the other functions use)."""
    npads = np.asarray(tf.npads, dtype=np.int64)
    row_x = np.asarray(tf.row_x, dtype=np.int64)
    r = clusters["row"].astype(np.int64)
    f = clusters["t_peak"].astype(np.int64) // 256
    Y = 2 * (clusters["pad_fp"].astype(np.int64) - 128 * (npads[r] - 1))
    Z = 5 * (128 * 256 * f + clusters["time_fp"].astype(np.int64) - 512)
    X = 64 * row_x[r]
    return X, Y, Z


def ca(tf, clusters: np.ndarray, params: OracleParams | None = None):
    L = _load()
    p = (params or OracleParams())._c()
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(clusters, dtype=CLUSTER_DTYPE)
    n = len(cl)
    up = np.full(n, -1, np.int32)
    down = np.full(n, -1, np.int32)
    chain = np.full(n, -1, np.int32)
    L.orc_ca(inp.ref, ctypes.byref(p), cl.ctypes.data if n else None, n, up.ctypes.data,
             down.ctypes.data, chain.ctypes.data)
    return up, down, chain


def merge(tf, clusters, up, down, chain_of, params: OracleParams | None = None):
    L = _load()
    p = (params or OracleParams())._c()
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(clusters, dtype=CLUSTER_DTYPE)
    n = len(cl)
    cl2trk = np.full(n, -1, np.int32)
    cap = max(1, n // 5 + 1)
    first = np.zeros(cap, np.int64)
    ncl = np.zeros(cap, np.int64)
    passes = ctypes.c_int32(0)
    up = np.ascontiguousarray(up, np.int32)
    down = np.ascontiguousarray(down, np.int32)
    chain_of = np.ascontiguousarray(chain_of, np.int32)
    nt = L.orc_merge(inp.ref, ctypes.byref(p), cl.ctypes.data if n else None, n, up.ctypes.data,
                     down.ctypes.data, chain_of.ctypes.data, cl2trk.ctypes.data, first.ctypes.data,
                     ncl.ctypes.data, cap, ctypes.byref(passes))
    return cl2trk, first[:nt].copy(), ncl[:nt].copy(), int(passes.value)


def fit_all(tf, clusters, cl2trk, n_tracks, params: OracleParams | None = None) -> np.ndarray:
    L = _load()
    p = (params or OracleParams())._c()
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(clusters, dtype=CLUSTER_DTYPE)
    out = np.zeros(max(n_tracks, 1), dtype=FIT_DTYPE)
    cl2trk = np.ascontiguousarray(cl2trk, np.int32)
    L.orc_fit_all(inp.ref, ctypes.byref(p), cl.ctypes.data if len(cl) else None, len(cl),
                  cl2trk.ctypes.data, n_tracks, out.ctypes.data)
    return out[:n_tracks]


def fit_points(x, y, z, params: OracleParams | None = None) -> np.void:
    """FP64 fit of points (cm), ascending x."""
    L = _load()
    p = (params or OracleParams())._c()
    x = np.ascontiguousarray(x, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    z = np.ascontiguousarray(z, np.float64)
    out = np.zeros(1, dtype=FIT_DTYPE)
    L.orc_fit_points(ctypes.byref(p), len(x), x.ctypes.data, y.ctypes.data, z.ctypes.data,
                     out.ctypes.data)
    return out[0]


def transport(state, dx, params: OracleParams | None = None):
    """Exact helix transport; returns (new_state, F) or (None, None) if stopped."""
    L = _load()
    p = (params or OracleParams())._c()
    s = np.ascontiguousarray(state, np.float64)
    o = np.zeros(5)
    F = np.zeros(25)
    rc = L.orc_transport(ctypes.byref(p), s.ctypes.data, float(dx), o.ctypes.data, F.ctypes.data)
    if rc:
        return None, None
    return o, F.reshape(5, 5)


def update(state, C, my, mz, params: OracleParams | None = None):
    """One Kalman update; returns (state', C', chi2, pd_ok)."""
    L = _load()
    p = (params or OracleParams())._c()
    s = np.array(state, np.float64)
    Cm = np.array(C, np.float64).reshape(25).copy()
    ok = ctypes.c_int(0)
    chi2 = L.orc_update(ctypes.byref(p), s.ctypes.data, Cm.ctypes.data, float(my), float(mz),
                        ctypes.byref(ok))
    return s, Cm.reshape(5, 5), chi2, bool(ok.value)


class _XsParams(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_double), ("edge_cm", ctypes.c_double), ("dz_cm", ctypes.c_double)]


@dataclass
class XsParams:
    """Cross-sector merge constants."""
    chi2_cut: float = 100.0
    edge_cm: float = 6.0
    dz_cm: float = 250.0       # the drift length: pieces of one track lie within it in zeta

    def _c(self) -> _XsParams:
        return _XsParams(float(self.chi2_cut), float(self.edge_cm), float(self.dz_cm))


def sector_alpha(s: int) -> float:
    return ((s % 18) + 0.5) * np.deg2rad(20.0)


def rotate(state, x, delta, params: OracleParams | None = None):
    """Express a state at x in a frame rotated by -delta (delta = alpha_old -
    alpha_new); returns (state', x', R) or (None, None, None)."""
    L = _load()
    p = (params or OracleParams())._c()
    s = np.array(state, np.float64)
    xx = ctypes.c_double(float(x))
    R = np.zeros(25)
    if L.orc_rotate(ctypes.byref(p), s.ctypes.data, ctypes.byref(xx), float(delta), R.ctypes.data):
        return None, None, None
    return s, xx.value, R.reshape(5, 5)


def xs_chi2(fa, alpha_a, fb, alpha_b, params: OracleParams | None = None) -> float:
    L = _load()
    p = (params or OracleParams())._c()
    a = np.ascontiguousarray(np.array([fa], dtype=FIT_DTYPE))
    b = np.ascontiguousarray(np.array([fb], dtype=FIT_DTYPE))
    return L.orc_xs_chi2(ctypes.byref(p), a.ctypes.data, float(alpha_a), b.ctypes.data, float(alpha_b))


def fit_points_xs(x, y, z, alpha, params: OracleParams | None = None) -> np.void:
    """FP64 fit of points (cm) in several sector frames (alpha per point)."""
    L = _load()
    p = (params or OracleParams())._c()
    arrs = [np.ascontiguousarray(a, np.float64) for a in (x, y, z, alpha)]
    out = np.zeros(1, dtype=FIT_DTYPE)
    L.orc_fit_points_xs(ctypes.byref(p), len(arrs[0]), *(a.ctypes.data for a in arrs), out.ctypes.data)
    return out[0]


@dataclass
class XsResult:
    link: np.ndarray        # [n_tracks] outer piece or -1
    best_chi2: np.ndarray   # [n_tracks] best candidate chi2 as the inner piece, or -1
    group_of: np.ndarray    # [n_tracks] merged track of every piece
    fits: np.ndarray        # [n_merged]
    first: np.ndarray       # [n_merged] lowest-row cluster of the innermost piece
    ncl: np.ndarray         # [n_merged]
    npieces: np.ndarray     # [n_merged]
    cl2trk: np.ndarray      # [n_clusters] merged track or -1
    borderline: np.ndarray  # [n_tracks] 1 where the piece's decision is within 1 % of flipping


def merge_sectors(tf, res, params: OracleParams | None = None, xs: XsParams | None = None) -> XsResult:
    """Cross-sector merge of an OracleResult's tracks (step 9)."""
    L = _load()
    p = (params or OracleParams())._c()
    xp = (xs or XsParams())._c()
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(res.clusters)
    c2t = np.ascontiguousarray(res.cl2trk, np.int32)
    fits = np.ascontiguousarray(res.fits)
    nt = len(fits)
    link = np.zeros(max(nt, 1), np.int32)
    best = np.zeros(max(nt, 1), np.float64)
    grp = np.zeros(max(nt, 1), np.int32)
    gfit = np.zeros(max(nt, 1), FIT_DTYPE)
    gf = np.zeros(max(nt, 1), np.int32)
    gn = np.zeros(max(nt, 1), np.int32)
    gp = np.zeros(max(nt, 1), np.int32)
    bl = np.zeros(max(nt, 1), np.int8)
    ng = L.orc_merge_sectors(inp.ref, ctypes.byref(p), ctypes.byref(xp), cl.ctypes.data if len(cl) else None,
                             len(cl), c2t.ctypes.data if len(c2t) else None, nt,
                             fits.ctypes.data if nt else None, link.ctypes.data, best.ctypes.data,
                             grp.ctypes.data, gfit.ctypes.data, gf.ctypes.data, gn.ctypes.data, gp.ctypes.data,
                             bl.ctypes.data)
    new_c2t = np.where(c2t >= 0, grp[np.maximum(c2t, 0)], -1).astype(np.int32)
    return XsResult(link[:nt].copy(), best[:nt].copy(), grp[:nt].copy(), gfit[:ng].copy(), gf[:ng].copy(),
                    gn[:ng].copy(), gp[:ng].copy(), new_c2t, bl[:nt].copy())


class _LoopParams(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_double), ("loop_radius_cm", ctypes.c_double),
                ("max_turns", ctypes.c_int32), ("pad", ctypes.c_int32)]


@dataclass
class LoopParams:
    """Step 9b (looper legs): chi2 cut of a leg pair, radius within which a
    fitted circle counts as looping (the 250 cm outer field cage + 10 %), and
    the largest number of turns between two joined legs."""
    chi2_cut: float = 30.0
    loop_radius_cm: float = 275.0
    max_turns: int = 4

    def _c(self) -> _LoopParams:
        return _LoopParams(self.chi2_cut, self.loop_radius_cm, self.max_turns, 0)


@dataclass
class LoopResult:
    next: np.ndarray        # [n_tracks] the following leg (further along the fitted motion) or -1
    prev: np.ndarray        # [n_tracks] the preceding leg or -1
    next_chi2: np.ndarray   # [n_tracks] chi2 of the link to next, or -1
    borderline: np.ndarray  # [n_tracks] 1 where a decision about the track is within 1 % of flipping
    n_links: int


def join_loopers(tf, res, params: OracleParams | None = None, loop: LoopParams | None = None) -> LoopResult:
    """Looper-leg join of an OracleResult's tracks (step 9b)."""
    L = _load()
    p = (params or OracleParams())._c()
    lp = (loop or LoopParams())._c()
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(res.clusters)
    c2t = np.ascontiguousarray(res.cl2trk, np.int32)
    fits = np.ascontiguousarray(res.fits)
    nt = len(fits)
    nxt = np.zeros(max(nt, 1), np.int32)
    prv = np.zeros(max(nt, 1), np.int32)
    c2 = np.zeros(max(nt, 1), np.float64)
    bl = np.zeros(max(nt, 1), np.int8)
    n = L.orc_join_loopers(inp.ref, ctypes.byref(p), ctypes.byref(lp), cl.ctypes.data if len(cl) else None, len(cl),
                           c2t.ctypes.data if len(c2t) else None, nt, fits.ctypes.data if nt else None,
                           nxt.ctypes.data, prv.ctypes.data, c2.ctypes.data, bl.ctypes.data)
    return LoopResult(nxt[:nt].copy(), prv[:nt].copy(), c2[:nt].copy(), bl[:nt].copy(), int(n))


def loop_pair(fa, fb, params: OracleParams | None = None, loop: LoopParams | None = None) -> tuple[float, int]:
    """Step 9b's matching chi2 of two fitted legs (FIT_DTYPE records) and the
    signed number of turns from A to B; chi2 -1 when the pair is no candidate."""
    L = _load()
    p = (params or OracleParams())._c()
    lp = (loop or LoopParams())._c()
    a = np.ascontiguousarray(np.asarray(fa, FIT_DTYPE).reshape(1))
    b = np.ascontiguousarray(np.asarray(fb, FIT_DTYPE).reshape(1))
    m = ctypes.c_int(0)
    c2 = float(L.orc_loop_pair(ctypes.byref(p), ctypes.byref(lp), a.ctypes.data, b.ctypes.data, ctypes.byref(m)))
    return c2, int(m.value)


def loops(fit, r_out_cm: float, params: OracleParams | None = None) -> bool:
    """Step 9b's looping test: the fitted circle lies within r_out_cm."""
    L = _load()
    p = (params or OracleParams())._c()
    a = np.ascontiguousarray(np.asarray(fit, FIT_DTYPE).reshape(1))
    return bool(L.orc_loops(ctypes.byref(p), a.ctypes.data, float(r_out_cm)))


class _CmpParams(ctypes.Structure):
    _fields_ = [("step_y", ctypes.c_double), ("step_z", ctypes.c_double)]


STEP_Y = 0.4 / 32     # 1/32 pad, cm
STEP_Z = 0.5 / 32     # 1/32 time bin, cm


def compress(tf, res, step_y: float = STEP_Y, step_z: float = STEP_Z, params: OracleParams | None = None,
             quotients: bool = False):
    """Track-model compression of the clusters on an OracleResult's tracks
    (step 10).  Returns (code_y, code_z, status) per cluster, and with
    quotients=True also the residuals in steps before rounding (NaN where no
    prediction was made)."""
    L = _load()
    p = (params or OracleParams())._c()
    cp = _CmpParams(float(step_y), float(step_z))
    inp = _In.from_tf(tf)
    cl = np.ascontiguousarray(res.clusters)
    n = len(cl)
    c2t = np.ascontiguousarray(res.cl2trk, np.int32)
    fits = np.ascontiguousarray(res.fits)
    cy = np.zeros(max(n, 1), np.int8)
    cz = np.zeros(max(n, 1), np.int8)
    st = np.zeros(max(n, 1), np.uint8)
    qy = np.zeros(max(n, 1), np.float64)
    qz = np.zeros(max(n, 1), np.float64)
    L.orc_compress(inp.ref, ctypes.byref(p), ctypes.byref(cp), cl.ctypes.data if n else None, n,
                   c2t.ctypes.data if n else None, len(fits), fits.ctypes.data if len(fits) else None,
                   cy.ctypes.data, cz.ctypes.data, st.ctypes.data, qy.ctypes.data, qz.ctypes.data)
    if quotients:
        return cy[:n].copy(), cz[:n].copy(), st[:n].copy(), qy[:n].copy(), qz[:n].copy()
    return cy[:n].copy(), cz[:n].copy(), st[:n].copy()


ZETA_PER_BIN = 0.5   # cm of the drift coordinate per time bin (Z = 640 u per bin)


def calibrate_drift(res, t0_bins: float, drift_length_cm: float = 250.0, params: OracleParams | None = None):
    """Drift calibration from an OracleResult's tracks (step 11).  Returns
    (t_vertex_bins, eps_vd, t0_from_vertex_bins, n_used)."""
    L = _load()
    p = (params or OracleParams())._c()
    fits = np.ascontiguousarray(res.fits)
    ncl = np.ascontiguousarray(res.track_ncl, np.int32)
    nt = len(fits)
    tv = ctypes.c_double(0.0)
    per = np.zeros(max(nt, 1))
    used = np.zeros(max(nt, 1), np.uint8)
    n = L.orc_calibrate_drift(ctypes.byref(p), fits.ctypes.data if nt else None, ncl.ctypes.data if nt else None,
                              nt, ZETA_PER_BIN, ctypes.byref(tv), per.ctypes.data, used.ctypes.data)
    full = drift_length_cm / ZETA_PER_BIN
    eps = full / (tv.value - t0_bins) - 1.0 if n else float("nan")
    return tv.value, eps, tv.value - full, int(n)


@dataclass
class OracleResult:
    clusters: np.ndarray
    up: np.ndarray
    down: np.ndarray
    chain_of: np.ndarray
    cl2trk: np.ndarray
    track_first: np.ndarray
    track_ncl: np.ndarray
    fits: np.ndarray
    merge_passes: int = 0
    times: dict = field(default_factory=dict)


def reconstruct(tf, params: OracleParams | None = None) -> OracleResult:
    """The whole pipeline, stage by stage."""
    import time
    times = {}
    t = time.perf_counter()
    cl = find_clusters(tf, params)
    times["find"] = time.perf_counter() - t
    t = time.perf_counter()
    up, down, chain = ca(tf, cl, params)
    times["ca"] = time.perf_counter() - t
    t = time.perf_counter()
    cl2trk, first, ncl, passes = merge(tf, cl, up, down, chain, params)
    times["merge"] = time.perf_counter() - t
    t = time.perf_counter()
    fits = fit_all(tf, cl, cl2trk, len(first), params)
    times["fit"] = time.perf_counter() - t
    return OracleResult(cl, up, down, chain, cl2trk, first, ncl, fits, passes, times)


def entropy_encode(code_y, code_z, status):
    """Step 10c: canonical-Huffman stream of the coded clusters' codes.
    Returns (lengths [2, 256] of the y and z alphabets, bits, words)."""
    L = _load()
    cy = np.ascontiguousarray(code_y, np.int8)
    cz = np.ascontiguousarray(code_z, np.int8)
    st = np.ascontiguousarray(status, np.uint8)
    n = len(st)
    lens = np.zeros(512, np.uint8)
    nbits = L.orc_entropy_encode(n, cy.ctypes.data, cz.ctypes.data, st.ctypes.data, lens.ctypes.data, None, 0)
    words = np.zeros(max(1, (nbits + 31) // 32), np.uint32)
    L.orc_entropy_encode(n, cy.ctypes.data, cz.ctypes.data, st.ctypes.data, lens.ctypes.data,
                         words.ctypes.data, len(words))
    return lens.reshape(2, 256), int(nbits), words[: (nbits + 31) // 32]
