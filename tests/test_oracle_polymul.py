"""Pins for the oracle's product in the basis (Sec. VI.A)."""
import numpy as np
import pytest

from oracle import oracle as O


@pytest.mark.parametrize("r,lgh", [(8, 2), (8, 5), (8, 7), (16, 4)])
def test_product_evaluates_to_product_of_values(r, lgh):
    """At every point the product polynomial equals the product of the two
    factors' values (direct evaluation, independent of the monomial route);
    with 2h <= 2^r points in the evaluation set this fixes the product."""
    h = 1 << lgh
    g = np.random.default_rng(h + r)
    a = g.integers(0, 1 << r, (h, 2)).astype(np.uint16)
    b = g.integers(0, 1 << r, (h, 2)).astype(np.uint16)
    c = O.poly_mul(r, a, b)
    pad = lambda x: np.vstack([x, np.zeros_like(x)])
    rows = np.arange(2 * h) if r == 8 else g.choice(1 << r, 48, replace=False)
    for l in ([0, 2 * h] if 4 * h <= (1 << r) else [0]):
        va = O.fft(r, l, pad(a), rows=rows % (2 * h) if r == 16 else rows)
        vb = O.fft(r, l, pad(b), rows=rows % (2 * h) if r == 16 else rows)
        vc = O.fft(r, l, c, rows=rows % (2 * h) if r == 16 else rows)
        assert np.array_equal(vc, O.gf_mul_vec(r, va, vb))
    if r == 8:  # and at every element of the field
        for x in range(256):
            ea = 0
            eb = 0
            ec = 0
            for i in range(h):
                ea ^= O.gf_mul(r, int(a[i, 0]), O.X(r, i, x))
                eb ^= O.gf_mul(r, int(b[i, 0]), O.X(r, i, x))
            for i in range(2 * h):
                ec ^= O.gf_mul(r, int(c[i, 0]), O.X(r, i, x))
            assert ec == O.gf_mul(r, ea, eb)


def test_unit_and_degree():
    r, h = 8, 16
    g = np.random.default_rng(1)
    a = g.integers(0, 256, (h, 3)).astype(np.uint16)
    one = np.zeros((h, 3), dtype=np.uint16)
    one[0] = 1  # X_0 = 1
    c = O.poly_mul(r, a, one)
    assert np.array_equal(c[:h], a) and not c[h:].any()
    # X_i * X_j with disjoint bit sets is X_{i+j} (product of distinct W factors)
    e = lambda i: np.eye(h, dtype=np.uint16)[:, [i]]
    assert np.array_equal(O.poly_mul(r, e(5), e(10))[:, 0], np.eye(2 * h, dtype=np.uint16)[15])
    # degree of the product is the sum of the degrees
    x = np.zeros((h, 1), dtype=np.uint16)
    y = np.zeros((h, 1), dtype=np.uint16)
    x[:7, 0] = g.integers(1, 256, 7)
    y[:10, 0] = g.integers(1, 256, 10)
    p = O.poly_mul(r, x, y)[:, 0]
    assert p[6 + 9] != 0 and not p[16:].any()
