"""Pins of the oracle's entropy coding of the step-10 codes (step 10c):
a hand-worked alphabet with its canonical codewords and stream written out,
the prefix code's completeness (Kraft sum 1), optimality (the stream's length
equals the textbook Huffman cost, computed here with a heap), the length limit
on a Fibonacci histogram, a decode of the stream back to the codes by a decoder
written here from the stream's description, and on a generated timeframe the
stream within one bit per symbol of the codes' Shannon entropy."""
import heapq
import math

import numpy as np
import pytest

import oracle
import tpcgen


def decode(lens, words, nbits, n_coded):
    """Decode n_coded (y, z) pairs from the stream: canonical codewords rebuilt
    from the lengths (ordered by (length, symbol)), bits read MSB first."""
    tables = []
    for k in range(2):
        syms = sorted((int(lens[k][s]), s) for s in range(256) if lens[k][s])
        table, code, prev = {}, 0, 0
        for i, (l, s) in enumerate(syms):
            code = 0 if i == 0 else (code + 1) << (l - prev)
            table[(l, code)] = s
            prev = l
        tables.append(table)
    bits = [(int(words[b // 32]) >> (31 - b % 32)) & 1 for b in range(nbits)]
    out, b = [], 0
    for _ in range(n_coded):
        pair = []
        for k in range(2):
            code, l = 0, 0
            while (l, code) not in tables[k]:
                code = (code << 1) | bits[b]
                b += 1
                l += 1
                assert l <= 24
            pair.append(tables[k][(l, code)] - 128)
        out.append(pair)
    assert b == nbits
    return np.array(out, np.int64).reshape(-1, 2)


def heap_cost(counts):
    """Textbook Huffman cost (sum of the merged weights); ties do not change it."""
    h = [int(c) for c in counts if c]
    if len(h) == 1:
        return h[0]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    return cost


def test_hand_worked_alphabet():
    """Codes 0 x5, +1 x2, -1 x1, +2 x1 (symbols 128, 129, 127, 130).  Queue A by
    (count, symbol): 127, 130, 129, 128.  Merges: 127 + 130 -> n1 (2); leaf 129
    (2) before n1 (2) on the tie, then n1 -> n2 (4); n2 before leaf 128 (5) ->
    root.  Lengths 128: 1, 129: 2, 127: 3, 130: 3; canonical codewords 0, 10,
    110, 111; 15 bits per component."""
    cy = np.array([0, 0, 1, 0, -1, 0, 2, 1, 0], np.int8)
    st = np.ones(9, np.uint8)
    lens, nbits, words = oracle.entropy_encode(cy, cy, st)
    assert {s: int(lens[0][s]) for s in range(256) if lens[0][s]} == {127: 3, 128: 1, 129: 2, 130: 3}
    assert nbits == 30
    cw = {0: "0", 1: "10", -1: "110", 2: "111"}
    stream = "".join(cw[int(c)] * 2 for c in cy)   # y codeword then z codeword
    assert stream == "".join(str((int(words[b // 32]) >> (31 - b % 32)) & 1) for b in range(nbits))
    assert int(words[0]) & 0x3 == 0                # zero padding


def test_escaped_and_untracked_clusters_take_no_bits():
    cy = np.array([5, 5, 7, -3], np.int8)
    cz = np.array([1, 1, 1, 1], np.int8)
    lens, nbits, _ = oracle.entropy_encode(cy, cz, np.array([1, 0, 2, 1], np.uint8))
    assert int(lens[0][128 + 7]) == 0 and int(lens[0][128 + 5]) == 1 and int(lens[0][128 - 3]) == 1
    assert int(lens[1][129]) == 1 and nbits == 4


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_complete_optimal_and_decodable(seed):
    rng = np.random.default_rng(seed)
    n = 5000
    cy = np.clip(np.rint(rng.normal(0, 6 * seed, n)), -127, 127).astype(np.int8)
    cz = np.clip(np.rint(rng.laplace(0, 3, n)), -127, 127).astype(np.int8)
    st = rng.choice([0, 1, 1, 1, 2], size=n).astype(np.uint8)
    lens, nbits, words = oracle.entropy_encode(cy, cz, st)
    coded = st == 1
    for k, c in enumerate((cy, cz)):
        counts = np.bincount(c[coded].astype(np.int64) + 128, minlength=256)
        assert ((lens[k] > 0) == (counts > 0)).all()
        assert math.isclose(sum(2.0 ** -int(l) for l in lens[k] if l), 1.0)
        assert int((counts * lens[k]).sum()) == heap_cost(counts)
    got = decode(lens, words, nbits, int(coded.sum()))
    assert (got[:, 0] == cy[coded]).all() and (got[:, 1] == cz[coded]).all()


def test_length_limit():
    """Fibonacci counts over 30 symbols: the plain Huffman tree is 29 deep;
    the halving keeps every length within 24 (at the price of more bits than
    the unlimited optimum) and the code prefix-free."""
    fib = [1, 1]
    while len(fib) < 30:
        fib.append(fib[-1] + fib[-2])
    cy = np.repeat(np.arange(-15, 15), fib).astype(np.int8)
    st = np.ones(len(cy), np.uint8)
    lens, nbits, words = oracle.entropy_encode(cy, np.zeros_like(cy), st)
    assert lens[0].max() <= 24
    assert int((np.array(fib) * lens[0][113:143]).sum()) > heap_cost(fib)
    assert sum(2.0 ** -int(l) for l in lens[0] if l) <= 1.0
    got = decode(lens, words, nbits, len(cy))
    assert (got[:, 0] == cy).all()


def test_timeframe_codes_within_a_bit_of_the_entropy():
    tf = tpcgen.generate(tpcgen.single_sector(3, n_tracks=300))
    res = oracle.reconstruct(tf)
    cy, cz, st = oracle.compress(tf, res)
    lens, nbits, words = oracle.entropy_encode(cy, cz, st)
    coded = st == 1
    n = int(coded.sum())
    assert n > 10000
    h = 0.0
    for c in (cy, cz):
        p = np.bincount(c[coded].astype(np.int64) + 128, minlength=256) / n
        h -= (p[p > 0] * np.log2(p[p > 0])).sum() * n
    assert h <= nbits < h + 2 * n
    got = decode(lens, words, nbits, n)
    assert (got[:, 0] == cy[coded]).all() and (got[:, 1] == cz[coded]).all()
