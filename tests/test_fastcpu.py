"""The CPU restatement of the paper's fast algorithms (oracle/fastcpu.c),
used only for comparison timings, is pinned to the oracle: its transforms,
derivative, encoder and decoder give the oracle's results."""
import itertools

import numpy as np
import pytest

from oracle import fastcpu as FC
from oracle import oracle as O


def rnd(rows, cols, seed, r):
    return np.random.default_rng(seed).integers(0, 1 << r, size=(rows, cols), dtype=np.uint16)


@pytest.mark.parametrize("r,lgh,l", [(8, 1, 0), (8, 3, 8), (8, 5, 96), (8, 8, 0), (16, 4, 48), (16, 9, 1024),
                                     (16, 6, 0)])
def test_transforms_match_the_oracle(r, lgh, l):
    h = 1 << lgh
    d = rnd(h, 3, seed=lgh + l, r=r)
    assert np.array_equal(FC.transform(r, l, d), O.fft(r, l, d))
    assert np.array_equal(FC.transform(r, l, FC.transform(r, l, d), inverse=True), d)
    assert np.array_equal(FC.transform(r, l, d, inverse=True), O.ifft(r, l, d))


@pytest.mark.parametrize("r,lgh", [(8, 1), (8, 4), (8, 8), (16, 5), (16, 7)])
def test_derivative_matches_the_oracle(r, lgh):
    d = rnd(1 << lgh, 3, seed=100 + lgh, r=r)
    assert np.array_equal(FC.derivative(r, d), O.derivative(r, d))


@pytest.mark.parametrize("r,n,k", [(8, 32, 16), (8, 256, 64), (16, 64, 32), (16, 1024, 256), (8, 8, 8)])
def test_encode_and_decode_match_the_oracle(r, n, k):
    cw = np.zeros((n, 4), dtype=np.uint16)
    cw[:k] = rnd(k, 4, seed=n + k, r=r)
    enc = FC.rs_encode(r, n, k, cw)
    assert np.array_equal(enc, O.rs_encode(r, n, k, cw))
    g = np.random.default_rng(n)
    for e in sorted({0, min(1, n - k), (n - k) // 2, n - k}):
        erased = np.zeros(n, dtype=np.uint8)
        erased[g.choice(n, e, replace=False)] = 1
        bad = enc.copy()
        bad[erased != 0] = 0xBEEF % (1 << r)
        assert np.array_equal(FC.rs_decode(r, n, k, bad, erased), enc)


def test_decode_every_pattern_of_8_4():
    r, n, k = 8, 8, 4
    cw = np.zeros((n, 2), dtype=np.uint16)
    cw[:k] = rnd(k, 2, seed=84, r=r)
    enc = FC.rs_encode(r, n, k, cw)
    for e in range(n - k + 1):
        for rows in itertools.combinations(range(n), e):
            erased = np.zeros(n, dtype=np.uint8)
            erased[list(rows)] = 1
            bad = enc.copy()
            bad[erased != 0] = 0
            assert np.array_equal(FC.rs_decode(r, n, k, bad, erased), enc), rows
    erased = np.ones(n, dtype=np.uint8)
    with pytest.raises(ValueError):
        FC.rs_decode(r, n, k, enc, erased)  # more than n - k erasures


def test_full_size_encode_matches_the_oracle_on_sampled_rows():
    """n = 65536, k = 32768 over GF(2^16): four parity rows of one column, the
    first, second, a middle and the last, against the oracle's Lagrange
    evaluation."""
    from paper_1404_3458_gb300 import workloads as WL

    n, k = 65536, 32768
    msg = np.zeros((n, 1), dtype=np.uint16)
    msg[:k, 0] = O.to_elems(WL.shards(k, 2, seed=WL.SEED_BASE + 9), 16)[:, 0]
    enc = FC.rs_encode(16, n, k, msg)
    rows = k + np.array([0, 1, 12345, n - k - 1])
    assert np.array_equal(enc[rows], O.rs_encode(16, n, k, msg, rows=rows)[rows])
