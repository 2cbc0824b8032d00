"""Pins for the oracle's field arithmetic (Sec. II.A; Appendix for alpha).

The oracle's fast product (log/exp tables) is checked against its bitwise
carry-less product, and both against hand-derived powers of alpha."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_powers():
    rows = []
    with open(os.path.join(GOLDEN, "alpha_powers.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                r, e, v = (int(x) for x in line.split())
                rows.append((r, e, v))
    return rows


@pytest.mark.parametrize("r,e,v", _golden_powers())
def test_alpha_powers_golden(r, e, v):
    acc = 1
    for _ in range(e):
        acc = O.gf_mul_bitwise(r, acc, 2)
    assert acc == v
    assert O.gf_exp(r, e) == v


@pytest.mark.parametrize("r", [8, 16])
def test_alpha_is_primitive(r):
    # the library refuses to load unless alpha = x has order 2^r - 1; check again
    M = (1 << r) - 1
    assert O.lib().orc_field_ok(r) == 0
    assert O.gf_exp(r, M) == 1
    # no smaller order: alpha^(M/p) != 1 for each prime p | M
    primes = {8: [3, 5, 17], 16: [3, 5, 17, 257]}[r]
    for p in primes:
        assert O.gf_exp(r, M // p) != 1


def test_gf8_table_product_matches_bitwise_exhaustive():
    a = np.repeat(np.arange(256, dtype=np.uint16), 256)
    b = np.tile(np.arange(256, dtype=np.uint16), 256)
    fast = O.gf_mul_vec(8, a, b)
    slow = np.array([O.gf_mul_bitwise(8, int(x), int(y)) for x, y in zip(a, b)], dtype=np.uint16)
    assert np.array_equal(fast, slow)


def test_gf16_table_product_matches_bitwise_sampled():
    g = np.random.default_rng(7)
    a = g.integers(0, 65536, 4000, dtype=np.uint16)
    b = g.integers(0, 65536, 4000, dtype=np.uint16)
    fast = O.gf_mul_vec(16, a, b)
    slow = np.array([O.gf_mul_bitwise(16, int(x), int(y)) for x, y in zip(a, b)], dtype=np.uint16)
    assert np.array_equal(fast, slow)


@pytest.mark.parametrize("r", [8, 16])
def test_inverse_and_log_exp_roundtrip(r):
    q = 1 << r
    a = np.arange(1, q, dtype=np.uint16)
    inv = np.array([O.gf_inv(r, int(x)) for x in a], dtype=np.uint16)
    assert np.all(O.gf_mul_vec(r, a, inv) == 1)
    logs = np.array([O.gf_log(r, int(x)) for x in a])
    assert sorted(logs.tolist()) == list(range(q - 1))
    assert all(O.gf_exp(r, int(lg)) == int(x) for x, lg in zip(a[:: max(1, q // 997)], logs[:: max(1, q // 997)]))


def test_gf8_distributive_and_associative_exhaustive_pairs():
    g = np.random.default_rng(3)
    a = np.repeat(np.arange(256, dtype=np.uint16), 256)
    b = np.tile(np.arange(256, dtype=np.uint16), 256)
    for c in g.integers(0, 256, 6):
        c = np.uint16(c)
        lhs = O.gf_mul_vec(8, a, b ^ c)
        rhs = O.gf_mul_vec(8, a, b) ^ O.gf_mul_vec(8, a, np.full_like(a, c))
        assert np.array_equal(lhs, rhs)
        lhs = O.gf_mul_vec(8, O.gf_mul_vec(8, a, b), np.full_like(a, c))
        rhs = O.gf_mul_vec(8, a, O.gf_mul_vec(8, b, np.full_like(a, c)))
        assert np.array_equal(lhs, rhs)
