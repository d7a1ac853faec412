"""The allocation-free finder entry point, for callers that cannot allocate
device memory (a budget owned by another framework, or a loop that must never
reach cudaMalloc and its implicit device synchronisation).  Its clusters must
equal those of the regular entry point, call after call: the scratch array it
shares between calls keeps the previous call's contents and must be cleared
each time.  Collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import oracle
import tpcgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def reference_clusters(tpc, tf):
    with tpc.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        cl = tpc.tpc_get_clusters(R.ctx, t)
        tpc.tpc_release(R.ctx, t)
    return cl


@pytest.mark.parametrize("make", [lambda: tpcgen.single_sector(4), lambda: tpcgen.full_tpc(2)])
def test_noalloc_matches_regular_entry_point_twice(lib, make):
    import torch
    tf = tpcgen.generate(make())
    want = reference_clusters(lib, tf)
    pages = torch.from_numpy(tf.pages).cuda()
    offs = torch.from_numpy(tf.page_offsets.view(np.int64)).cuda()
    geom = lib.tpc_create_geometry(tf.npads, tf.row_x, tf.n_sectors)
    try:
        for _ in range(2):   # the second call must not see the first call's scratch
            out = torch.zeros(16 * (len(want) + 64), dtype=torch.uint8, device="cuda")
            n = lib.tpc_find_clusters_noalloc(geom, pages, offs, tf.n_time_bins, out)
            assert n == len(want)
            got = out[: 16 * n].cpu().numpy().view(lib.CLUSTER_DTYPE)
            assert got.tobytes() == want.tobytes()
    finally:
        lib.tpc_destroy_geometry(geom)


def test_noalloc_rejects_too_many_windows(lib):
    import torch
    npads, row_x = tpcgen.default_geometry()
    geom = lib.tpc_create_geometry(npads, row_x, 36)
    try:
        pages = torch.zeros(64, dtype=torch.uint8, device="cuda")
        offs = torch.zeros(1, dtype=torch.int64, device="cuda")
        out = torch.zeros(16 * 64, dtype=torch.uint8, device="cuda")
        with pytest.raises(lib.TpcError) as ei:   # 36 x 152 x 12 fragments > 65,536 windows
            lib.tpc_find_clusters_noalloc(geom, pages, offs, 12 * 256, out)
        assert ei.value.code == -1
    finally:
        lib.tpc_destroy_geometry(geom)


def test_noalloc_noise_suppression_matches_oracle(lib):
    """Step 2b through the allocation-free entry point."""
    import torch
    tf = tpcgen.generate(tpcgen.single_sector(9, n_tracks=400))
    want = oracle.find_clusters(tf, oracle.OracleParams(ns_min_dip=10))
    p = lib.tpc_params_default()
    p.ns_min_dip = 10
    geom = lib.tpc_create_geometry(tf.npads, tf.row_x, tf.n_sectors)
    try:
        pages = torch.from_numpy(tf.pages).cuda()
        offs = torch.from_numpy(tf.page_offsets.view(np.int64)).cuda()
        out = torch.zeros(16 * (len(want) + 64), dtype=torch.uint8, device="cuda")
        n = lib.tpc_find_clusters_noalloc(geom, pages, offs, tf.n_time_bins, out, params=p)
        torch.cuda.synchronize()
    finally:
        lib.tpc_destroy_geometry(geom)
    assert n == len(want)
    assert out[:16 * n].cpu().numpy().tobytes() == want.tobytes()
