"""CPU-side checks of the C-ABI library: it builds, loads, exports every
function include/tpc.h declares, and validates its arguments without a GPU."""
import os
import re

import numpy as np
import pytest

import tpcgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:tpc_status|void|const char\*)\s+(tpc_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    from paper_2208_07412_b300 import tpc
    L = tpc.load()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(tpc.EXPORTS)


def test_params_defaults():
    from paper_2208_07412_b300 import tpc
    p = tpc.tpc_params_default()
    assert (p.q_peak_min, p.ca_cut, p.min_chain, p.merge_cut, p.min_track, p.fit_passes) == (10, 256, 5, 384, 10, 3)
    assert (p.ca_slope_z_num, p.ca_slope_z_den, p.merge_gap_min, p.merge_gap_max) == (11, 10, 1, 6)
    assert list(p.c0) == [4.0, 4.0, 0.25, 1.0, 100.0] and p.bz == 0.5
    assert p.fp32_pd_margin == 0.0 and p.split_charge == 0 and p.version == 3


def test_geometry_validation():
    from paper_2208_07412_b300 import tpc
    npads, row_x = tpcgen.default_geometry()
    g = tpc.tpc_create_geometry(npads, row_x, 36)
    tpc.tpc_destroy_geometry(g)
    bad_x = row_x.copy()
    bad_x[10] = bad_x[9]
    with pytest.raises(tpc.TpcError):
        tpc.tpc_create_geometry(npads, bad_x, 36)
    bad_p = npads.copy()
    bad_p[0] = 300
    with pytest.raises(tpc.TpcError):
        tpc.tpc_create_geometry(bad_p, row_x, 36)


def test_context_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2208_07412_b300 import tpc
    npads, row_x = tpcgen.default_geometry()
    g = tpc.tpc_create_geometry(npads, row_x, 36)
    with pytest.raises(tpc.TpcError):
        tpc.tpc_create_context(g)
    tpc.tpc_destroy_geometry(g)


def test_record_layouts_match_header():
    from paper_2208_07412_b300 import tpc
    import oracle
    assert tpc.CLUSTER_DTYPE.itemsize == 16 and tpc.TRACK_DTYPE.itemsize == 112
    assert tpc.CLUSTER_DTYPE.names == oracle.CLUSTER_DTYPE.names
    assert np.dtype(tpc.CLUSTER_DTYPE).fields["sector"][1] == 15
