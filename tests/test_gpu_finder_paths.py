"""The two-pass finder's three ways through a unit, each checked bit for bit
against the oracle on hand-built planes: the digit list (at most 4096 digits
and 1024 own peaks), the list whose own peaks overflow their room and are
ranked in pixel order instead (isolated digits on every other pad of every
other time bin: ~1,056 own peaks from ~1,155 digits), and the pixel scan of a
unit with more digits than the list takes (every pixel charged).  Random
planes at occupancies around the list's capacity mix the three.  Each with
step 2b and step 3s on as well."""
from types import SimpleNamespace

import numpy as np
import pytest

import oracle
from synth import encode_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def make_tf(planes, npads):
    T = planes.shape[2]
    pages, offs = encode_planes(planes, T, npads)
    n_rows = planes.shape[1]
    return SimpleNamespace(pages=pages, page_offsets=offs, n_time_bins=T, n_sectors=1,
                           npads=np.asarray(npads, np.int32),
                           row_x=(1697 + 15 * np.arange(n_rows)).astype(np.int32))


def check(lib, tf, dip=0, split=False):
    want = oracle.find_clusters(tf, oracle.OracleParams(ns_min_dip=dip, split_charge=split))
    p = lib.tpc_params_default()
    p.ns_min_dip = dip
    p.split_charge = int(split)
    with lib.Reconstructor.for_timeframe(tf, params=p) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        got = lib.tpc_get_clusters(R.ctx, t)
        lib.tpc_release(R.ctx, t)
    assert len(got) == len(want)
    assert got.tobytes() == want.tobytes()
    return want


VARIANTS = [dict(), dict(dip=10), dict(split=True), dict(dip=10, split=True)]


@pytest.mark.parametrize("v", VARIANTS)
def test_own_peaks_overflow_the_list(lib, v):
    T, npads = 600, [66, 66, 66]
    planes = np.zeros((1, 3, T, 66), np.uint16)
    planes[0, :, 0::2, 0::2] = 50
    planes[0, 1, 1::4, 1::2] = 4          # low digits between them in the second row
    want = check(lib, make_tf(planes, npads), **v)
    assert len(want) >= 3 * 300 * 33 - 100


@pytest.mark.parametrize("v", VARIANTS)
def test_every_pixel_charged(lib, v):
    rng = np.random.default_rng(5)
    T, npads = 520, [138, 100, 70]
    planes = rng.integers(1, 200, size=(1, 3, T, 138)).astype(np.uint16)
    planes[0, 1, :, 100:] = 0
    planes[0, 2, :, 70:] = 0
    check(lib, make_tf(planes, npads), **v)


@pytest.mark.parametrize("occ", [0.2, 0.3, 0.4, 0.5])
@pytest.mark.parametrize("v", VARIANTS[::3])
def test_random_occupancy(lib, occ, v):
    rng = np.random.default_rng(int(occ * 100))
    T, npads = 700, [138, 66, 120]
    planes = np.zeros((1, 3, T, 138), np.uint16)
    mask = rng.random(planes.shape) < occ
    planes[mask] = rng.integers(3, 300, size=int(mask.sum()))
    for r, n in enumerate(npads):
        planes[0, r, :, n:] = 0
    check(lib, make_tf(planes, npads), **v)
