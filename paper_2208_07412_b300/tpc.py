"""Thin ctypes binding of the C ABI in include/tpc.h (argument marshalling only).

Every function keeps the C name.  Host buffers are numpy arrays; device
buffers are torch CUDA tensors (used only for their memory and streams).  All
reconstruction work runs in the CUDA kernels of libtpc_b300.so: if that library
is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_P = ctypes.c_void_p
_u64 = ctypes.c_uint64

TPC_OK = 0
ERRORS = {-1: "TPC_E_INVAL", -2: "TPC_E_NOMEM", -3: "TPC_E_BUSY", -4: "TPC_E_CUDA",
          -5: "TPC_E_CORRUPT", -6: "TPC_E_NOTREADY", -7: "TPC_E_TIMEOUT",
          -8: "TPC_E_OVERFLOW", -9: "TPC_E_DEVICE", -10: "TPC_E_NOTFOUND"}
TPC_STATE_QUEUED, TPC_STATE_RUNNING, TPC_STATE_INPUT_RELEASED, TPC_STATE_DONE, TPC_STATE_FAILED = range(5)
TPC_TF_DEVICE_INPUT = 1
TPC_TF_NOWAIT = 2
TPC_CTX_STAGE_TIMING = 1
TPC_CTX_NO_GRAPHS = 2
TPC_CTX_DENSE_FINDER = 4
TPC_CTX_FUSED_FINDER = 8
STAGES = ("find", "ca", "merge", "fit")

CLUSTER_DTYPE = np.dtype([("pad_fp", "<u2"), ("time_fp", "<u2"), ("qmax", "<u2"), ("qtot", "<u2"),
                          ("sigma2_pad", "u1"), ("sigma2_time", "u1"), ("flags", "u1"),
                          ("row", "u1"), ("t_peak", "<u2"), ("pad_peak", "u1"), ("sector", "u1")])
TRACK_DTYPE = np.dtype([("par", "<f4", (5,)), ("x", "<f4"), ("alpha", "<f4"), ("chi2", "<f4"),
                        ("cov", "<f4", (15,)), ("ndf", "<i4"), ("n_clusters", "<i4"),
                        ("first_cluster", "<i4"), ("sector", "<i2"), ("flags", "<u2"),
                        ("n_fp64", "<i4")])
assert CLUSTER_DTYPE.itemsize == 16 and TRACK_DTYPE.itemsize == 112


class TpcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class tpc_geometry_desc(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("npads", _P), ("row_x", _P)]


class tpc_params(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint32), ("q_peak_min", ctypes.c_int32),
                ("ca_slope_y_num", ctypes.c_int32), ("ca_slope_y_den", ctypes.c_int32),
                ("ca_slope_z_num", ctypes.c_int32), ("ca_slope_z_den", ctypes.c_int32),
                ("ca_cut", ctypes.c_int32), ("min_chain", ctypes.c_int32),
                ("merge_cut", ctypes.c_int32), ("merge_gap_min", ctypes.c_int32),
                ("merge_gap_max", ctypes.c_int32), ("merge_max_passes", ctypes.c_int32),
                ("min_track", ctypes.c_int32), ("fit_passes", ctypes.c_int32),
                ("ns_min_dip", ctypes.c_int32), ("bz", ctypes.c_double),
                ("sigma_y", ctypes.c_double), ("sigma_z", ctypes.c_double),
                ("c0", ctypes.c_double * 5), ("fp32_pd_margin", ctypes.c_double),
                ("split_charge", ctypes.c_int32)]


class tpc_tuning(ctypes.Structure):
    _fields_ = [("find_threads", ctypes.c_int32), ("find_ctas_per_sm", ctypes.c_int32),
                ("ca_blocks_per_sm", ctypes.c_int32), ("elem_blocks_per_sm", ctypes.c_int32),
                ("fit_threads", ctypes.c_int32), ("fit_blocks_per_sm", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class tpc_xs_params(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_double), ("edge_cm", ctypes.c_double), ("dz_cm", ctypes.c_double)]


class tpc_loop_params(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_double), ("loop_radius_cm", ctypes.c_double),
                ("max_turns", ctypes.c_int32), ("pad", ctypes.c_int32)]


class tpc_cmp_params(ctypes.Structure):
    _fields_ = [("step_y_cm", ctypes.c_double), ("step_z_cm", ctypes.c_double)]


class tpc_timeframe_desc(ctypes.Structure):
    _fields_ = [("pages", _P), ("pages_bytes", _u64), ("page_offsets", _P),
                ("n_time_bins", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


EXPORTS = ("tpc_params_default", "tpc_create_geometry", "tpc_destroy_geometry", "tpc_create_context",
           "tpc_destroy_context", "tpc_submit_timeframe", "tpc_poll", "tpc_get_clusters",
           "tpc_get_tracks", "tpc_get_links", "tpc_get_device_results", "tpc_get_stage_times",
           "tpc_get_counters", "tpc_release", "tpc_last_error", "tpc_find_clusters_noalloc",
           "tpc_submit_batch", "tpc_get_batch_info", "tpc_get_event_clusters", "tpc_get_event_tracks",
           "tpc_get_tuning", "tpc_set_tuning", "tpc_autotune", "tpc_merge_sectors", "tpc_get_merged_tracks",
           "tpc_join_loopers", "tpc_get_looper_links", "tpc_compress_clusters", "tpc_get_compressed", "tpc_entropy_encode", "tpc_calibrate_drift", "tpc_measure_fma_peak")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libtpc_b300.so (building it in place if it is missing and nvcc is
    available).  Raises if the library cannot be loaded: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB) and build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libtpc_b300.so is not built (run paper_2208_07412_b300/build.py)")
    L = ctypes.CDLL(_build.LIB)
    L.tpc_params_default.argtypes = [ctypes.POINTER(tpc_params)]
    L.tpc_create_geometry.argtypes = [ctypes.POINTER(tpc_geometry_desc), ctypes.POINTER(_P)]
    L.tpc_destroy_geometry.argtypes = [_P]
    L.tpc_destroy_geometry.restype = None
    L.tpc_create_context.argtypes = [_P, ctypes.POINTER(tpc_params), ctypes.c_int, _u64, ctypes.c_int, _P,
                                     ctypes.c_uint32, ctypes.POINTER(_P)]
    L.tpc_destroy_context.argtypes = [_P]
    L.tpc_destroy_context.restype = None
    L.tpc_submit_timeframe.argtypes = [_P, ctypes.POINTER(tpc_timeframe_desc), ctypes.POINTER(_u64)]
    L.tpc_poll.argtypes = [_P, _u64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]
    L.tpc_get_clusters.argtypes = [_P, _u64, _P, _u64, ctypes.POINTER(_u64)]
    L.tpc_get_tracks.argtypes = [_P, _u64, _P, _u64, ctypes.POINTER(_u64), _P]
    L.tpc_get_links.argtypes = [_P, _u64, _P, _P, _P]
    L.tpc_get_device_results.argtypes = [_P, _u64, ctypes.POINTER(_P), ctypes.POINTER(_u64),
                                         ctypes.POINTER(_P), ctypes.POINTER(_u64), ctypes.POINTER(_P)]
    L.tpc_get_stage_times.argtypes = [_P, _u64, _P]
    L.tpc_get_counters.argtypes = [_P, _u64, _P, ctypes.c_int]
    L.tpc_release.argtypes = [_P, _u64]
    L.tpc_find_clusters_noalloc.argtypes = [_P, ctypes.POINTER(tpc_params), ctypes.c_int, _P, _u64, _P,
                                            ctypes.c_uint32, _P, _u64, ctypes.POINTER(_u64), _P]
    L.tpc_submit_batch.argtypes = [_P, ctypes.POINTER(tpc_timeframe_desc), ctypes.c_uint32, ctypes.POINTER(_u64)]
    L.tpc_get_batch_info.argtypes = [_P, _u64, ctypes.POINTER(ctypes.c_uint32), _P, _P]
    L.tpc_get_event_clusters.argtypes = [_P, _u64, ctypes.c_uint32, _P, _u64, ctypes.POINTER(_u64)]
    L.tpc_get_event_tracks.argtypes = [_P, _u64, ctypes.c_uint32, _P, _u64, ctypes.POINTER(_u64), _P]
    L.tpc_get_tuning.argtypes = [_P, ctypes.POINTER(tpc_tuning)]
    L.tpc_set_tuning.argtypes = [_P, ctypes.POINTER(tpc_tuning)]
    L.tpc_autotune.argtypes = [_P, ctypes.POINTER(tpc_timeframe_desc), ctypes.c_int, ctypes.POINTER(tpc_tuning)]
    L.tpc_merge_sectors.argtypes = [_P, _u64, ctypes.POINTER(tpc_xs_params), ctypes.POINTER(_u64)]
    L.tpc_get_merged_tracks.argtypes = [_P, _u64, _P, _u64, ctypes.POINTER(_u64), _P, _P]
    L.tpc_join_loopers.argtypes = [_P, _u64, ctypes.POINTER(tpc_loop_params), ctypes.POINTER(_u64)]
    L.tpc_get_looper_links.argtypes = [_P, _u64, _P, _P, ctypes.POINTER(_u64)]
    L.tpc_compress_clusters.argtypes = [_P, _u64, ctypes.POINTER(tpc_cmp_params), ctypes.POINTER(_u64),
                                        ctypes.POINTER(_u64)]
    L.tpc_get_compressed.argtypes = [_P, _u64, _P, _P, _P]
    L.tpc_entropy_encode.argtypes = [_P, _u64, _P, _P, _P, _P, ctypes.POINTER(_u64), _P, _u64]
    L.tpc_calibrate_drift.argtypes = [_P, _u64, ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(_u64)]
    L.tpc_measure_fma_peak.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.tpc_last_error.argtypes = []
    L.tpc_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("tpc_destroy_geometry", "tpc_destroy_context", "tpc_last_error"):
            getattr(L, name).restype = ctypes.c_int32
    _lib = L
    return L


def _check(rc):
    if rc != TPC_OK:
        raise TpcError(rc, load().tpc_last_error().decode())
    return rc


# ------------------------------------------------------------------ C-named wrappers
def tpc_params_default() -> tpc_params:
    p = tpc_params()
    _check(load().tpc_params_default(ctypes.byref(p)))
    return p


def tpc_create_geometry(npads, row_x, n_sectors: int):
    npads = np.ascontiguousarray(npads, np.int32)
    row_x = np.ascontiguousarray(row_x, np.int32)
    d = tpc_geometry_desc(int(n_sectors), len(npads), npads.ctypes.data, row_x.ctypes.data)
    out = _P()
    _check(load().tpc_create_geometry(ctypes.byref(d), ctypes.byref(out)))
    return out


def tpc_destroy_geometry(g):
    load().tpc_destroy_geometry(g)


def tpc_create_context(geom, params: tpc_params | None = None, device: int = 0, mem_budget: int = 0,
                       n_slots: int = 1, stream: int | None = None, flags: int = 0):
    out = _P()
    _check(load().tpc_create_context(geom, ctypes.byref(params) if params is not None else None, device,
                                     mem_budget, n_slots, stream, flags, ctypes.byref(out)))
    return out


def tpc_destroy_context(ctx):
    load().tpc_destroy_context(ctx)


def _ptr(a):
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def tpc_submit_timeframe(ctx, pages, page_offsets, n_time_bins: int, flags: int = 0) -> int:
    """pages / page_offsets: numpy arrays (host) or torch CUDA tensors (device,
    TPC_TF_DEVICE_INPUT is then set).  The caller keeps them alive until the
    ticket reaches TPC_STATE_INPUT_RELEASED."""
    d, _keep = _desc(pages, page_offsets, n_time_bins, flags)
    t = _u64()
    _check(load().tpc_submit_timeframe(ctx, ctypes.byref(d), ctypes.byref(t)))
    return int(t.value)


def _desc(pages, page_offsets, n_time_bins: int, flags: int = 0):
    """Descriptor of one timeframe; also returns the arrays it points into
    (keep them alive while the descriptor is in use)."""
    if hasattr(pages, "data_ptr"):
        if pages.is_cuda:
            flags |= TPC_TF_DEVICE_INPUT
        nbytes = pages.numel() * pages.element_size()
    else:
        pages = np.ascontiguousarray(pages, np.uint8)
        page_offsets = np.ascontiguousarray(page_offsets, np.uint64)
        nbytes = pages.nbytes
    return tpc_timeframe_desc(_ptr(pages), nbytes, _ptr(page_offsets), int(n_time_bins), flags), (pages, page_offsets)


def tpc_submit_batch(ctx, events, n_time_bins: int) -> tuple[int, list]:
    """events: [(pages, page_offsets[, n_time_bins]), ...] as for
    tpc_submit_timeframe (n_time_bins: the argument unless given per event).
    Returns (ticket, keep): keep holds the arrays the descriptors point into;
    keep it alive until TPC_STATE_INPUT_RELEASED."""
    descs, keep = [], []
    for ev in events:
        pages, offs, *rest = ev
        d, k = _desc(pages, offs, rest[0] if rest else n_time_bins)
        descs.append(d)
        keep.append(k)
    arr = (tpc_timeframe_desc * len(descs))(*descs)
    t = _u64()
    _check(load().tpc_submit_batch(ctx, arr, len(descs), ctypes.byref(t)))
    return int(t.value), keep


def tpc_get_batch_info(ctx, ticket: int):
    """Returns (cluster_start, track_start), each n_events + 1 long."""
    L = load()
    n = ctypes.c_uint32()
    _check(L.tpc_get_batch_info(ctx, ticket, ctypes.byref(n), None, None))
    cs = np.zeros(n.value + 1, np.uint64)
    ts = np.zeros(n.value + 1, np.uint64)
    _check(L.tpc_get_batch_info(ctx, ticket, ctypes.byref(n), cs.ctypes.data, ts.ctypes.data))
    return cs, ts


def tpc_get_event_clusters(ctx, ticket: int, event: int) -> np.ndarray:
    L = load()
    n = _u64()
    _check(L.tpc_get_event_clusters(ctx, ticket, event, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, CLUSTER_DTYPE)
    if n.value:
        _check(L.tpc_get_event_clusters(ctx, ticket, event, out.ctypes.data, n.value, ctypes.byref(n)))
    return out


def tpc_get_event_tracks(ctx, ticket: int, event: int, n_clusters: int):
    """Returns (tracks, cluster_to_track) of one event, indices relative to it."""
    L = load()
    n = _u64()
    _check(L.tpc_get_event_tracks(ctx, ticket, event, None, 0, ctypes.byref(n), None))
    out = np.zeros(n.value, TRACK_DTYPE)
    m = np.zeros(n_clusters, np.int32)
    _check(L.tpc_get_event_tracks(ctx, ticket, event, out.ctypes.data if n.value else None, n.value,
                                  ctypes.byref(n), m.ctypes.data if n_clusters else None))
    return out, m


def tpc_get_tuning(ctx) -> dict:
    t = tpc_tuning()
    _check(load().tpc_get_tuning(ctx, ctypes.byref(t)))
    return t.as_dict()


def tpc_set_tuning(ctx, **kw) -> None:
    """Set launch-configuration fields (the others keep their current values)."""
    t = tpc_tuning()
    _check(load().tpc_get_tuning(ctx, ctypes.byref(t)))
    for k, v in kw.items():
        setattr(t, k, int(v))
    _check(load().tpc_set_tuning(ctx, ctypes.byref(t)))


def tpc_autotune(ctx, pages, page_offsets, n_time_bins: int, reps: int = 3) -> dict:
    """Tune the context's launch configuration on a sample timeframe; returns it."""
    d, _keep = _desc(pages, page_offsets, n_time_bins)
    t = tpc_tuning()
    _check(load().tpc_autotune(ctx, ctypes.byref(d), int(reps), ctypes.byref(t)))
    return t.as_dict()


TPC_TRK_STOPPED = 1
TPC_TRK_NOT_PD = 2
TPC_TRK_XSECTOR = 4


def tpc_merge_sectors(ctx, ticket: int, chi2_cut: float = 100.0, edge_cm: float = 6.0, dz_cm: float = 250.0) -> int:
    """Cross-sector merge of a finished ticket; returns the number of tracks after it."""
    n = _u64()
    xp = tpc_xs_params(float(chi2_cut), float(edge_cm), float(dz_cm))
    _check(load().tpc_merge_sectors(ctx, ticket, ctypes.byref(xp), ctypes.byref(n)))
    return int(n.value)


def tpc_get_merged_tracks(ctx, ticket: int, n_clusters: int, n_tracks: int):
    """Returns (merged tracks, cluster_to_track, link per step-8 track)."""
    L = load()
    n = _u64()
    _check(L.tpc_get_merged_tracks(ctx, ticket, None, 0, ctypes.byref(n), None, None))
    out = np.zeros(n.value, TRACK_DTYPE)
    m = np.zeros(n_clusters, np.int32)
    link = np.zeros(n_tracks, np.int32)
    _check(L.tpc_get_merged_tracks(ctx, ticket, out.ctypes.data if n.value else None, n.value, ctypes.byref(n),
                                   m.ctypes.data if n_clusters else None, link.ctypes.data if n_tracks else None))
    return out, m, link


def tpc_join_loopers(ctx, ticket: int, chi2_cut: float = 30.0, loop_radius_cm: float = 275.0,
                     max_turns: int = 4) -> int:
    """Looper-leg join (step 9b) of a finished ticket; returns the number of links."""
    n = _u64()
    lp = tpc_loop_params(float(chi2_cut), float(loop_radius_cm), int(max_turns), 0)
    _check(load().tpc_join_loopers(ctx, ticket, ctypes.byref(lp), ctypes.byref(n)))
    return int(n.value)


def tpc_get_looper_links(ctx, ticket: int):
    """Returns (next, prev): per step-8 track the linked following / preceding leg or -1."""
    L = load()
    n = _u64()
    _check(L.tpc_get_looper_links(ctx, ticket, None, None, ctypes.byref(n)))
    nxt = np.zeros(n.value, np.int32)
    prv = np.zeros(n.value, np.int32)
    if n.value:
        _check(L.tpc_get_looper_links(ctx, ticket, nxt.ctypes.data, prv.ctypes.data, ctypes.byref(n)))
    return nxt, prv


def tpc_compress_clusters(ctx, ticket: int, step_y_cm: float = 0.4 / 32, step_z_cm: float = 0.5 / 32):
    """Track-model compression of a finished ticket; returns (n_coded, n_escaped)."""
    a, b = _u64(), _u64()
    cp = tpc_cmp_params(float(step_y_cm), float(step_z_cm))
    _check(load().tpc_compress_clusters(ctx, ticket, ctypes.byref(cp), ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def tpc_get_compressed(ctx, ticket: int, n_clusters: int):
    """Returns (code_y, code_z, status) per cluster."""
    cy = np.zeros(max(n_clusters, 1), np.int8)
    cz = np.zeros(max(n_clusters, 1), np.int8)
    st = np.zeros(max(n_clusters, 1), np.uint8)
    _check(load().tpc_get_compressed(ctx, ticket, cy.ctypes.data, cz.ctypes.data, st.ctypes.data))
    return cy[:n_clusters], cz[:n_clusters], st[:n_clusters]


def tpc_entropy_encode(ctx, ticket: int, codes=None, fetch: bool = True):
    """Step 10c on a finished ticket: (lengths [2, 256], n_bits, words).
    codes: None for the ticket's step-10 codes, or (code_y, code_z, status)
    arrays of n_clusters entries that replace them.  fetch=False encodes
    without copying the stream to host memory (words is then None)."""
    L = load()
    nb = _u64()
    lens = np.zeros(512, np.uint8)
    args = [None, None, None]
    if codes is not None:
        args = [np.ascontiguousarray(codes[0], np.int8), np.ascontiguousarray(codes[1], np.int8),
                np.ascontiguousarray(codes[2], np.uint8)]
    keep = [a if a is None or len(a) else np.zeros(1, a.dtype) for a in args]   # no clusters: a dummy entry
    ptrs = [a.ctypes.data if a is not None else None for a in keep]
    _check(L.tpc_entropy_encode(ctx, ticket, *ptrs, lens.ctypes.data, ctypes.byref(nb), None, 0))
    n = int(nb.value)
    if not fetch:
        return lens.reshape(2, 256), n, None
    words = np.zeros(max(1, (n + 31) // 32), np.uint32)
    _check(L.tpc_entropy_encode(ctx, ticket, None, None, None, None, ctypes.byref(nb), words.ctypes.data,
                                len(words)))
    return lens.reshape(2, 256), n, words[: (n + 31) // 32]


def tpc_calibrate_drift(ctx, ticket: int, t0_bins: float, drift_length_cm: float = 250.0):
    """Drift calibration of a finished ticket: (t_vertex_bins, eps_vd, t0_from_vertex, n_used)."""
    tv, eps, t0, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), _u64()
    _check(load().tpc_calibrate_drift(ctx, ticket, float(t0_bins), float(drift_length_cm), ctypes.byref(tv),
                                      ctypes.byref(eps), ctypes.byref(t0), ctypes.byref(n)))
    return tv.value, eps.value, t0.value, int(n.value)


def tpc_poll(ctx, ticket: int, timeout_us: int = 0xFFFFFFFF) -> int:
    st = ctypes.c_int32(-1)
    _check(load().tpc_poll(ctx, ticket, timeout_us, ctypes.byref(st)))
    return int(st.value)


def tpc_get_clusters(ctx, ticket: int) -> np.ndarray:
    L = load()
    n = _u64()
    _check(L.tpc_get_clusters(ctx, ticket, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, CLUSTER_DTYPE)
    if n.value:
        _check(L.tpc_get_clusters(ctx, ticket, out.ctypes.data, n.value, ctypes.byref(n)))
    return out


def tpc_get_tracks(ctx, ticket: int, n_clusters: int | None = None):
    """Returns (tracks, cluster_to_track)."""
    L = load()
    n = _u64()
    _check(L.tpc_get_tracks(ctx, ticket, None, 0, ctypes.byref(n), None))
    if n_clusters is None:
        nc = _u64()
        _check(L.tpc_get_clusters(ctx, ticket, None, 0, ctypes.byref(nc)))
        n_clusters = nc.value
    out = np.zeros(n.value, TRACK_DTYPE)
    m = np.zeros(n_clusters, np.int32)
    _check(L.tpc_get_tracks(ctx, ticket, out.ctypes.data if n.value else None, n.value, ctypes.byref(n),
                            m.ctypes.data if n_clusters else None))
    return out, m


def tpc_get_links(ctx, ticket: int, n_clusters: int):
    up = np.zeros(n_clusters, np.int32)
    down = np.zeros(n_clusters, np.int32)
    chain = np.zeros(n_clusters, np.int32)
    if n_clusters:
        _check(load().tpc_get_links(ctx, ticket, up.ctypes.data, down.ctypes.data, chain.ctypes.data))
    return up, down, chain


def tpc_get_device_results(ctx, ticket: int):
    cl, ncl, tr, ntr, m = _P(), _u64(), _P(), _u64(), _P()
    _check(load().tpc_get_device_results(ctx, ticket, ctypes.byref(cl), ctypes.byref(ncl), ctypes.byref(tr),
                                         ctypes.byref(ntr), ctypes.byref(m)))
    return cl.value, ncl.value, tr.value, ntr.value, m.value


def tpc_get_stage_times(ctx, ticket: int) -> dict:
    ms = np.zeros(4, np.float32)
    _check(load().tpc_get_stage_times(ctx, ticket, ms.ctypes.data))
    return dict(zip(STAGES, ms.tolist()))


COUNTERS = ("clusters", "chains", "tracks", "clusters_on_tracks", "fp64_redos", "merge_passes",
            "error_word", "zs_bytes", "kernel_launches", "runs")


def tpc_get_counters(ctx, ticket: int) -> dict:
    out = np.zeros(10, np.uint64)
    _check(load().tpc_get_counters(ctx, ticket, out.ctypes.data, 10))
    return dict(zip(COUNTERS, (int(v) for v in out)))


def tpc_release(ctx, ticket: int):
    _check(load().tpc_release(ctx, ticket))


def tpc_find_clusters_noalloc(geom, pages, page_offsets, n_time_bins: int, clusters, device: int = 0,
                              params: tpc_params | None = None, stream: int | None = None) -> int:
    """Allocation-free finder: pages, page_offsets and clusters are torch CUDA
    tensors owned by the caller (clusters: uint8 tensor of 16 * cap bytes).
    Returns the number of clusters written."""
    n = _u64()
    cap = clusters.numel() * clusters.element_size() // 16
    _check(load().tpc_find_clusters_noalloc(geom, ctypes.byref(params) if params is not None else None, device,
                                            pages.data_ptr(), pages.numel() * pages.element_size(),
                                            page_offsets.data_ptr(), int(n_time_bins), clusters.data_ptr(),
                                            cap, ctypes.byref(n), stream))
    return int(n.value)


def tpc_measure_fma_peak(device: int = 0, reps: int = 5) -> float:
    """Measured FP32 FMA throughput of the device (FLOP/s)."""
    v = ctypes.c_double()
    _check(load().tpc_measure_fma_peak(int(device), int(reps), ctypes.byref(v)))
    return float(v.value)


def tpc_last_error() -> str:
    return load().tpc_last_error().decode()


# ------------------------------------------------------------------ convenience
class Reconstructor:
    """Owns one geometry + context; forwards to the C-named wrappers."""

    def __init__(self, npads, row_x, n_sectors, params: tpc_params | None = None, device: int = 0,
                 mem_budget: int = 0, n_slots: int = 1, stream: int | None = None, flags: int = 0):
        self.geom = tpc_create_geometry(npads, row_x, n_sectors)
        self.ctx = None
        try:
            self.ctx = tpc_create_context(self.geom, params, device, mem_budget, n_slots, stream, flags)
        except BaseException:
            tpc_destroy_geometry(self.geom)
            self.geom = None
            raise

    @classmethod
    def for_timeframe(cls, tf, **kw):
        return cls(tf.npads, tf.row_x, tf.n_sectors, **kw)

    def submit(self, pages, page_offsets, n_time_bins, flags: int = 0) -> int:
        return tpc_submit_timeframe(self.ctx, pages, page_offsets, n_time_bins, flags)

    def wait(self, ticket: int, timeout_us: int = 0xFFFFFFFF) -> int:
        return tpc_poll(self.ctx, ticket, timeout_us)

    def run(self, tf):
        """Submit a generated timeframe, wait, fetch everything, release."""
        t = self.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        try:
            self.wait(t)
            cl = tpc_get_clusters(self.ctx, t)
            up, down, chain = tpc_get_links(self.ctx, t, len(cl))
            tracks, m = tpc_get_tracks(self.ctx, t, len(cl))
            ctr = tpc_get_counters(self.ctx, t)
        finally:
            tpc_release(self.ctx, t)
        return dict(clusters=cl, up=up, down=down, chain_of=chain, tracks=tracks, cl2trk=m, counters=ctr)

    def run_batch(self, tfs):
        """Submit generated timeframes (same n_time_bins) as one batch, wait,
        fetch each event's results (indices relative to the event), release."""
        t, keep = tpc_submit_batch(self.ctx, [(tf.pages, tf.page_offsets) for tf in tfs], tfs[0].n_time_bins)
        try:
            self.wait(t)
            out = []
            for e in range(len(tfs)):
                cl = tpc_get_event_clusters(self.ctx, t, e)
                tracks, m = tpc_get_event_tracks(self.ctx, t, e, len(cl))
                out.append(dict(clusters=cl, tracks=tracks, cl2trk=m))
            ctr = tpc_get_counters(self.ctx, t)
            for o in out:
                o["counters"] = ctr
        finally:
            tpc_release(self.ctx, t)
            del keep
        return out

    def close(self):
        if self.ctx:
            tpc_destroy_context(self.ctx)
            self.ctx = None
        if self.geom:
            tpc_destroy_geometry(self.geom)
            self.geom = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
