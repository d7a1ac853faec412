"""Seeded synthetic TPC timeframe generator (input module).

Produces the ZS pages the reconstruction consumes, plus the generator truth
(tracks, hits, per-digit labels).  It is the one module shared by the CUDA
path's tests and the oracle's tests: it holds the detector description and the
input simulation, and none of the reconstruction arithmetic.

Workload recipes (all seeded):
  single_sector     one sector, 500 time bins, 150 tracks from the vertex
  full_tpc          36 sectors, 1000 time bins, 10,000 tracks (5 % loopers)
  batch_event       one event of a batch: 36 sectors, 1000 bins, M tracks
  continuous_tf     50 kHz continuous timeframe: 55,000 bins, Poisson(550) collisions
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpcgen.c")
_LIB = os.path.join(_HERE, "libtpcgen.so")

N_ROWS = 152
N_SECTORS = 36
FRAG = 256


def build(force: bool = False) -> str:
    """Compile libtpcgen.so in place (gcc -O2 -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


# ------------------------------------------------------------------ geometry
def default_geometry():
    """Row layout of the synthetic TPC: 152 rows, npads(r) = 66 + floor(72 r / 151),
    pad pitch 0.4 cm, row pitch 7.5 / 10 / 12 / 15 mm over rows 0-62 / 63-96 /
    97-126 / 127-151, x(0) = 84.85 cm.  Returns (npads, row_x) with row_x in units
    of 0.05 cm."""
    npads = np.array([66 + (72 * r) // 151 for r in range(N_ROWS)], dtype=np.int32)
    pitch = np.empty(N_ROWS, dtype=np.int32)
    pitch[0:63] = 15
    pitch[63:97] = 20
    pitch[97:127] = 24
    pitch[127:152] = 30
    row_x = np.empty(N_ROWS, dtype=np.int32)
    row_x[0] = 1697
    for r in range(1, N_ROWS):
        row_x[r] = row_x[r - 1] + pitch[r - 1]
    return npads, row_x


# ------------------------------------------------------------------ ctypes
class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64), ("n_sectors", ctypes.c_int32), ("n_rows", ctypes.c_int32),
        ("npads", ctypes.c_void_p), ("row_x", ctypes.c_void_p), ("n_time_bins", ctypes.c_int32),
        ("n_collisions", ctypes.c_int32), ("coll_t0", ctypes.c_void_p),
        ("coll_ntracks", ctypes.c_void_p), ("looper_frac", ctypes.c_double),
        ("pt_min", ctypes.c_double), ("pt_mean_excess", ctypes.c_double),
        ("looper_pt_min", ctypes.c_double), ("looper_pt_max", ctypes.c_double),
        ("eta_min", ctypes.c_double), ("eta_max", ctypes.c_double),
        ("phi_min", ctypes.c_double), ("phi_max", ctypes.c_double), ("bz", ctypes.c_double),
        ("drift_length", ctypes.c_double), ("bin_cm", ctypes.c_double),
        ("outer_radius", ctypes.c_double), ("sigma_pad", ctypes.c_double),
        ("sigma_time", ctypes.c_double), ("landau_mpv", ctypes.c_double),
        ("landau_xi", ctypes.c_double), ("amp_cap", ctypes.c_double),
        ("noise_sigma", ctypes.c_double), ("zs_threshold", ctypes.c_int32),
        ("max_turns", ctypes.c_int32), ("want_labels", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
    ]


class _Result(ctypes.Structure):
    _fields_ = [
        ("pages", ctypes.c_void_p), ("pages_bytes", ctypes.c_uint64),
        ("page_offsets", ctypes.c_void_p), ("n_pages", ctypes.c_int64),
        ("n_digits", ctypes.c_int64), ("digit_labels", ctypes.c_void_p),
        ("n_tracks", ctypes.c_int64), ("tracks", ctypes.c_void_p),
        ("n_hits", ctypes.c_int64), ("hits", ctypes.c_void_p),
    ]


TRACK_DTYPE = np.dtype([("pt", "f8"), ("phi", "f8"), ("eta", "f8"), ("t0", "f8"),
                        ("charge", "i4"), ("collision", "i4"), ("looper", "i4"), ("n_hits", "i4")])
HIT_DTYPE = np.dtype([("pad", "f8"), ("time", "f8"), ("amp", "f4"), ("sector", "i4"),
                      ("row", "i4"), ("track", "i4"), ("leg", "i4")], align=True)
assert TRACK_DTYPE.itemsize == 48 and HIT_DTYPE.itemsize == 40

_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        _lib.tpcgen_generate.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.POINTER(_Result))]
        _lib.tpcgen_generate.restype = ctypes.c_int
        _lib.tpcgen_free.argtypes = [ctypes.POINTER(_Result)]
        _lib.tpcgen_sample_landau.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_void_p]
    return _lib


@dataclass
class GenConfig:
    seed: int = 1
    n_sectors: int = N_SECTORS
    n_time_bins: int = 1000
    coll_t0: list = field(default_factory=lambda: [250.0])
    coll_ntracks: list = field(default_factory=lambda: [10000])
    looper_frac: float = 0.0
    pt_min: float = 0.1
    pt_mean_excess: float = 0.5
    looper_pt_min: float = 0.05
    looper_pt_max: float = 0.10
    eta_min: float = -0.9
    eta_max: float = 0.9
    phi_min: float = 0.0
    phi_max: float = 2 * math.pi
    bz: float = 0.5
    drift_length: float = 250.0
    bin_cm: float = 0.5
    outer_radius: float = 250.0
    sigma_pad: float = 0.8
    sigma_time: float = 1.0
    landau_mpv: float = 60.0
    landau_xi: float = 6.0
    amp_cap: float = 1200.0
    noise_sigma: float = 1.0
    zs_threshold: int = 3
    max_turns: int = 20
    want_labels: bool = True
    n_threads: int = 0
    npads: np.ndarray | None = None
    row_x: np.ndarray | None = None
    name: str = "custom"


@dataclass
class Timeframe:
    """One generated timeframe: ZS pages + page table + generator truth."""
    pages: np.ndarray          # uint8, 16-byte aligned length
    page_offsets: np.ndarray   # uint64 [n_sectors * n_rows * n_fragments]
    n_time_bins: int
    n_sectors: int
    npads: np.ndarray
    row_x: np.ndarray
    n_digits: int
    digit_labels: np.ndarray | None
    tracks: np.ndarray
    hits: np.ndarray
    config: GenConfig

    @property
    def n_rows(self) -> int:
        return int(len(self.npads))

    @property
    def n_fragments(self) -> int:
        return (self.n_time_bins + FRAG - 1) // FRAG


def generate(cfg: GenConfig) -> Timeframe:
    lib = _load()
    npads, row_x = default_geometry() if cfg.npads is None else (cfg.npads, cfg.row_x)
    npads = np.ascontiguousarray(npads, dtype=np.int32)
    row_x = np.ascontiguousarray(row_x, dtype=np.int32)
    t0 = np.ascontiguousarray(cfg.coll_t0, dtype=np.float64)
    ntr = np.ascontiguousarray(cfg.coll_ntracks, dtype=np.int32)
    c = _Config()
    c.seed = cfg.seed
    c.n_sectors = cfg.n_sectors
    c.n_rows = len(npads)
    c.npads = npads.ctypes.data
    c.row_x = row_x.ctypes.data
    c.n_time_bins = cfg.n_time_bins
    c.n_collisions = len(t0)
    c.coll_t0 = t0.ctypes.data
    c.coll_ntracks = ntr.ctypes.data
    for k in ("looper_frac", "pt_min", "pt_mean_excess", "looper_pt_min", "looper_pt_max",
              "eta_min", "eta_max", "phi_min", "phi_max", "bz", "drift_length", "bin_cm",
              "outer_radius", "sigma_pad", "sigma_time", "landau_mpv", "landau_xi", "amp_cap",
              "noise_sigma"):
        setattr(c, k, float(getattr(cfg, k)))
    c.zs_threshold = cfg.zs_threshold
    c.max_turns = cfg.max_turns
    c.want_labels = int(cfg.want_labels)
    c.n_threads = cfg.n_threads
    res = ctypes.POINTER(_Result)()
    rc = lib.tpcgen_generate(ctypes.byref(c), ctypes.byref(res))
    if rc != 0:
        raise RuntimeError(f"tpcgen_generate failed ({rc})")
    try:
        r = res.contents
        nb = int(r.pages_bytes)
        pages = np.empty(max(nb, 16), dtype=np.uint8)[:nb]
        if nb:
            ctypes.memmove(pages.ctypes.data, r.pages, nb)
        offs = np.empty(int(r.n_pages), dtype=np.uint64)
        ctypes.memmove(offs.ctypes.data, r.page_offsets, offs.nbytes)
        labels = None
        if cfg.want_labels:
            labels = np.empty(int(r.n_digits), dtype=np.int32)
            if labels.size:
                ctypes.memmove(labels.ctypes.data, r.digit_labels, labels.nbytes)
        tracks = np.empty(int(r.n_tracks), dtype=TRACK_DTYPE)
        if tracks.size:
            ctypes.memmove(tracks.ctypes.data, r.tracks, tracks.nbytes)
        # per-hit truth only where digit labels are asked for (a continuous
        # timeframe has ~1.4e8 hits)
        hits = np.empty(int(r.n_hits) if cfg.want_labels else 0, dtype=HIT_DTYPE)
        if hits.size:
            ctypes.memmove(hits.ctypes.data, r.hits, hits.nbytes)
        return Timeframe(pages=pages, page_offsets=offs, n_time_bins=cfg.n_time_bins,
                         n_sectors=cfg.n_sectors, npads=npads, row_x=row_x,
                         n_digits=int(r.n_digits), digit_labels=labels, tracks=tracks, hits=hits,
                         config=cfg)
    finally:
        lib.tpcgen_free(res)


def sample_landau(seed: int, n: int, mpv: float = 60.0, xi: float = 6.0) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    lib.tpcgen_sample_landau(seed, n, mpv, xi, out.ctypes.data)
    return out


# ------------------------------------------------------------------ workloads
def single_sector(seed: int = 1, n_tracks: int = 150, **kw) -> GenConfig:
    """One sector (sector 0, side A), 500 time bins, tracks from the vertex with
    eta in [0, 0.9) and phi uniform within the sector (+-10 deg around 10 deg)."""
    d = dict(seed=seed, n_sectors=1, n_time_bins=500, coll_t0=[0.0], coll_ntracks=[n_tracks],
             eta_min=0.0, eta_max=0.9, phi_min=0.0, phi_max=math.radians(20.0),
             name="single_sector")
    d.update(kw)
    return GenConfig(**d)


def full_tpc(seed: int = 1, n_tracks: int = 10000, **kw) -> GenConfig:
    """36 sectors, 1000 time bins, one central collision at T0 = 250 bins with
    n_tracks tracks, 5 % of them low-pT loopers (pT 50-100 MeV)."""
    d = dict(seed=seed, n_sectors=36, n_time_bins=1000, coll_t0=[250.0], coll_ntracks=[n_tracks],
             looper_frac=0.05, name="full_tpc")
    d.update(kw)
    return GenConfig(**d)


def batch_multiplicities(seed: int, n_events: int = 64, lo: int = 200, hi: int = 20000):
    """Log-uniform multiplicities of a batch of uneven events."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_events))).astype(int)


def pp_tf(seed: int = 1, n_time_bins: int = 55000, rate_per_bin: float = 0.2, mean_tracks: float = 30.0,
          **kw) -> GenConfig:
    """pp-like continuous timeframe: 1 MHz interaction rate (0.2 collisions per
    200 ns time bin, Poisson), multiplicity per collision Poisson(mean_tracks)."""
    rng = np.random.default_rng(seed + 0x99)
    n = rng.poisson(rate_per_bin * n_time_bins)
    t0 = np.sort(rng.uniform(0.0, n_time_bins, size=n))
    m = rng.poisson(mean_tracks, size=n).astype(int)
    d = dict(seed=seed, n_sectors=36, n_time_bins=n_time_bins, coll_t0=list(t0),
             coll_ntracks=list(m), looper_frac=0.05, want_labels=False, name="pp_tf")
    d.update(kw)
    return GenConfig(**d)


def continuous_tf(seed: int = 1, n_time_bins: int = 55000, rate_per_bin: float = 0.01,
                  **kw) -> GenConfig:
    """50 kHz continuous timeframe: Poisson(rate * bins) collisions with uniform
    start times; multiplicity M = floor(15000 U^7.82) per collision."""
    rng = np.random.default_rng(seed + 0x5EED)
    n = rng.poisson(rate_per_bin * n_time_bins)
    t0 = np.sort(rng.uniform(0.0, n_time_bins, size=n))
    m = np.floor(15000.0 * rng.uniform(0.0, 1.0, size=n) ** 7.82).astype(int)
    d = dict(seed=seed, n_sectors=36, n_time_bins=n_time_bins, coll_t0=list(t0),
             coll_ntracks=list(m), looper_frac=0.05, want_labels=False, name="continuous_tf")
    d.update(kw)
    return GenConfig(**d)


def time_prefix(tf: Timeframe, n_fragments: int) -> Timeframe:
    """The first n_fragments 256-bin fragments of every (sector, row) of a
    timeframe as a timeframe of their own (pages copied in window order; a
    page's header keeps its fragment number, and the last kept fragment simply
    has no next neighbour)."""
    import copy
    nf_old = tf.n_fragments
    k = max(1, min(int(n_fragments), nf_old))
    if k == nf_old:
        return tf
    offs = tf.page_offsets.astype(np.int64)
    ends = np.append(offs[1:], len(tf.pages))
    idx = (np.arange(tf.n_sectors * tf.n_rows)[:, None] * nf_old + np.arange(k)[None, :]).ravel()
    lens = ends[idx] - offs[idx]
    new_offs = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64)
    pages = np.concatenate([tf.pages[offs[i]:ends[i]] for i in idx]) if len(idx) else tf.pages[:0]
    s = copy.copy(tf)
    s.pages, s.page_offsets = pages, new_offs
    s.n_time_bins = min(tf.n_time_bins, 256 * k)
    s.digit_labels = None
    s.tracks, s.hits = tf.tracks[:0], tf.hits[:0]
    return s


def sector_slice(tf: Timeframe, sector: int) -> Timeframe:
    """One sector of a timeframe as a single-sector timeframe of its own: it
    becomes sector 0 (the sector byte at offset 10 of every page header is
    rewritten) and the offsets are rebased to its first page, which keeps their
    16-byte alignment."""
    import copy
    nw = tf.n_rows * tf.n_fragments
    a = int(tf.page_offsets[sector * nw])
    b = int(tf.page_offsets[(sector + 1) * nw]) if (sector + 1) * nw < len(tf.page_offsets) else len(tf.pages)
    s = copy.copy(tf)
    s.page_offsets = tf.page_offsets[sector * nw:(sector + 1) * nw] - np.uint64(a)
    s.pages = tf.pages[a:b].copy()
    s.pages[s.page_offsets.astype(np.int64) + 10] = 0
    s.n_sectors = 1
    s.digit_labels = None           # no generator truth: the slice is input only
    s.tracks, s.hits = tf.tracks[:0], tf.hits[:0]
    return s


def sector_prefix(tf: Timeframe, n_sectors: int) -> Timeframe:
    """The first n_sectors sectors of a timeframe as a timeframe of their own.
    Pages are laid out window by window with the sector outermost, so these
    sectors' pages are a prefix of the page array and keep their offsets."""
    import copy
    n_sectors = min(n_sectors, tf.n_sectors)
    s = copy.copy(tf)
    nwin = n_sectors * tf.n_rows * tf.n_fragments
    s.page_offsets = tf.page_offsets[:nwin].copy()
    end = int(tf.page_offsets[nwin]) if nwin < len(tf.page_offsets) else len(tf.pages)
    s.pages = tf.pages[:end]
    s.n_sectors = n_sectors
    s.digit_labels = None
    return s
