"""Pins for the transform oracle (Sec. III): direct evaluation against Horner
evaluation of the same polynomial written in the monomial basis, the paper's
recursion and op counts, and the inverse."""
import numpy as np
import pytest

from oracle import butterfly as B
from oracle import oracle as O


def monomial_to_X(r, lgh, p):
    """Coefficients in X_0..X_{h-1} of the monomial polynomial p (deg < h), by
    the triangular solve that deg X_i = i allows (Sec. II.C)."""
    h = 1 << lgh
    Xs = [O.X_poly(r, lgh, i) for i in range(h)]
    rem = [int(v) for v in p] + [0] * (h - len(p))
    d = [0] * h
    for i in range(h - 1, -1, -1):
        e = O.gf_mul(r, rem[i], O.gf_inv(r, int(Xs[i][i])))
        d[i] = e
        if e:
            for m in range(i + 1):
                rem[m] ^= O.gf_mul(r, e, int(Xs[i][m]))
    assert not any(rem)
    return d


@pytest.mark.parametrize("r,lgh,l", [(8, 3, 0), (8, 4, 0), (8, 4, 48), (8, 6, 128), (8, 3, 3),
                                     (16, 4, 0), (16, 4, 4096 + 16), (16, 5, 65504)])
def test_transform_is_evaluation_of_monomial_polynomial(r, lgh, l):
    """A random polynomial of degree < h, converted to the X basis, transforms
    to its Horner values at w_c + w_l."""
    h = 1 << lgh
    g = np.random.default_rng(lgh * 1000 + l)
    p = g.integers(0, 1 << r, h)
    d = np.array(monomial_to_X(r, lgh, p), dtype=np.uint16)[:, None]
    out = O.fft(r, l, d)[:, 0]
    assert [int(v) for v in out] == [O.poly_eval(r, p, c ^ l) for c in range(h)]


@pytest.mark.parametrize("lgh", range(1, 9))
def test_paper_recursion_equals_direct_evaluation_gf8(lgh):
    """Sec. III.C recursion, every shift l that is a multiple of h (and a few
    others) on random columns, against direct evaluation."""
    r, h = 8, 1 << lgh
    g = np.random.default_rng(lgh)
    shifts = list(range(0, 256, h))
    if lgh <= 3:
        shifts += [1, 3, 5]
    for l in shifts[:: max(1, len(shifts) // 16)]:
        d = g.integers(0, 256, h).astype(np.uint16)
        ref = O.fft(r, l, d[:, None])[:, 0].tolist()
        vals, _, _ = B.transform_sets(r, d, l)
        assert vals == ref
        assert B.transform_inplace(r, d, l) == ref


@pytest.mark.parametrize("r,lgh,l", [(16, 4, 0), (16, 5, 96), (16, 6, 4096)])
def test_paper_recursion_equals_direct_evaluation_gf16(r, lgh, l):
    h = 1 << lgh
    d = np.random.default_rng(5).integers(0, 1 << r, h).astype(np.uint16)
    ref = O.fft(r, l, d[:, None])[:, 0].tolist()
    assert B.transform_sets(r, d, l)[0] == ref
    assert B.transform_inplace(r, d, l) == ref


@pytest.mark.parametrize("r,lgh", [(8, l) for l in range(1, 8)] + [(16, 8), (16, 10)])
def test_operation_counts(r, lgh):
    """A(h) = h lg h, M(h) = h/2 lg h; with zero shift A_0 = h lg h - h + 1,
    M_0 = h/2 lg h - h + 1 (Sec. III.D)."""
    h = 1 << lgh
    d = list(range(h))
    _, a, m = B.transform_sets(r, d, h)  # a nonzero shift that is a multiple of h
    assert (a, m) == (h * lgh, h // 2 * lgh)
    _, a0, m0 = B.transform_sets(r, d, 0)
    assert (a0, m0) == (h * lgh - h + 1, h // 2 * lgh - h + 1)


@pytest.mark.parametrize("r,lgh,l", [(8, 1, 0), (8, 4, 0), (8, 5, 32), (8, 7, 128), (8, 8, 0),
                                     (16, 6, 0), (16, 7, 1280)])
def test_inverse_roundtrip(r, lgh, l):
    h = 1 << lgh
    g = np.random.default_rng(lgh + l)
    x = g.integers(0, 1 << r, (h, 3)).astype(np.uint16)
    assert np.array_equal(O.ifft(r, l, O.fft(r, l, x)), x)
    assert np.array_equal(O.fft(r, l, O.ifft(r, l, x)), x)


@pytest.mark.parametrize("lgh,l", [(3, 0), (5, 64), (6, 0)])
def test_inverse_network_matches_inverse_oracle(lgh, l):
    h = 1 << lgh
    v = np.random.default_rng(h).integers(0, 256, h).astype(np.uint16)
    assert B.inverse_inplace(8, v, l) == O.ifft(8, l, v[:, None])[:, 0].tolist()


def test_sampled_rows_equal_full():
    x = np.random.default_rng(1).integers(0, 65536, (64, 5)).astype(np.uint16)
    full = O.fft(16, 192, x)
    rows = [63, 0, 17]
    assert np.array_equal(O.fft(16, 192, x, rows=rows), full[rows])
