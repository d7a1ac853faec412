"""Parity of the entropy coding of the step-10 codes (step 10c) with the
oracle: on the oracle's own codes (given to the library in place of the
ticket's), the GPU's codeword lengths and stream must equal the oracle's bit
for bit, on a sector, the full TPC, the hand-worked alphabet, a lone symbol, a
histogram that needs the length limit and a timeframe with nothing coded.  On
the ticket's own step-10 codes the stream must decode back to them."""
import numpy as np
import pytest

import oracle
import tpcgen
from test_oracle_entropy import decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2208_07412_b300 import tpc
    tpc.load()
    return tpc


def gpu_encode(lib, tf, codes=None):
    with lib.Reconstructor.for_timeframe(tf) as R:
        t = R.submit(tf.pages, tf.page_offsets, tf.n_time_bins)
        R.wait(t)
        n = len(lib.tpc_get_clusters(R.ctx, t))
        if codes is None:
            lib.tpc_compress_clusters(R.ctx, t)
        else:
            codes = tuple(np.resize(np.asarray(c), n) if len(c) != n else c for c in codes)
        out = lib.tpc_entropy_encode(R.ctx, t, codes)
        mine = lib.tpc_get_compressed(R.ctx, t, n)
        lib.tpc_release(R.ctx, t)
    return out, mine


def same(got, want):
    (gl, gn, gw), (ol, on, ow) = got, want
    assert gn == on
    assert (gl == ol).all()
    assert gw.tobytes() == ow.tobytes()


@pytest.mark.parametrize("make", [lambda: tpcgen.single_sector(3, n_tracks=300), lambda: tpcgen.full_tpc(2, n_tracks=3000),
                                  lambda: tpcgen.continuous_tf(3, n_time_bins=2000, n_sectors=2)])
def test_oracle_codes(lib, make):
    tf = tpcgen.generate(make())
    res = oracle.reconstruct(tf)
    codes = oracle.compress(tf, res)
    got, _ = gpu_encode(lib, tf, codes)
    same(got, oracle.entropy_encode(*codes))
    assert got[1] > 0


def synthetic(n, rng, kind):
    cy = np.zeros(n, np.int8)
    cz = np.zeros(n, np.int8)
    st = np.zeros(n, np.uint8)
    if kind == "hand":
        v = np.array([0, 0, 1, 0, -1, 0, 2, 1, 0], np.int8)
        idx = np.sort(rng.choice(n, size=len(v), replace=False))
        cy[idx] = v
        cz[idx] = v
        st[idx] = 1
    elif kind == "lone":
        st[::7] = 1
        cy[:] = -5
        cz[:] = 3
    elif kind == "fib":
        fib = [1, 1]
        while len(fib) < 28:             # 832,039 symbols, a Huffman tree 27 deep without the limit
            fib.append(fib[-1] + fib[-2])
        seq = np.repeat(np.arange(-14, 14), fib)
        assert len(seq) < n
        rng.shuffle(seq)
        cy[: len(seq)] = seq
        st[: len(seq)] = 1
        st[len(seq):] = rng.choice([0, 2], size=n - len(seq))
    elif kind == "wide":
        cy[:] = np.clip(np.rint(rng.normal(0, 40, n)), -127, 127)
        cz[:] = np.clip(np.rint(rng.laplace(0, 2, n)), -127, 127)
        st[:] = rng.choice([0, 1, 1, 2], size=n)
    return cy, cz, st


@pytest.mark.parametrize("kind", ["hand", "lone", "fib", "wide"])
def test_synthetic_codes(lib, kind):
    tf = tpcgen.generate(tpcgen.full_tpc(1) if kind == "fib" else tpcgen.single_sector(1))
    n = len(oracle.find_clusters(tf))
    codes = synthetic(n, np.random.default_rng(7), kind)
    got, _ = gpu_encode(lib, tf, codes)
    want = oracle.entropy_encode(*codes)
    same(got, want)
    if kind == "fib":
        assert got[0][0].max() <= 24


def test_nothing_coded(lib):
    tf = tpcgen.generate(tpcgen.single_sector(1))
    n = len(oracle.find_clusters(tf))
    codes = (np.zeros(n, np.int8), np.zeros(n, np.int8), np.full(n, 2, np.uint8))
    got, _ = gpu_encode(lib, tf, codes)
    assert got[1] == 0 and (got[0] == 0).all()


def test_ticket_codes_round_trip(lib):
    tf = tpcgen.generate(tpcgen.full_tpc(1, n_tracks=3000))
    (lens, nbits, words), (cy, cz, st) = gpu_encode(lib, tf)
    coded = st == 1
    assert coded.sum() > 100000
    for k, c in enumerate((cy, cz)):
        counts = np.bincount(c[coded].astype(np.int64) + 128, minlength=256)
        assert ((lens[k] > 0) == (counts > 0)).all()
        assert abs(sum(2.0 ** -int(l) for l in lens[k] if l) - 1.0) < 1e-12
    assert nbits == int(sum((np.bincount(c[coded].astype(np.int64) + 128, minlength=256) * lens[k]).sum()
                            for k, c in enumerate((cy, cz))))
    got = decode(lens, words, nbits, int(coded.sum()))
    assert (got[:, 0] == cy[coded]).all() and (got[:, 1] == cz[coded]).all()
