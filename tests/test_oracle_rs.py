"""Pins for the encode/decode and locator oracles (Sec. V, Appendix)."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_1404_3458_gb300 import workloads as WL


def vandermonde_solve(r, xs, ys):
    """Monomial coefficients of the interpolant through (xs, ys): Gaussian
    elimination on the Vandermonde system (textbook, independent of the
    oracle's barycentric form)."""
    k = len(xs)
    A = [[0] * k + [int(y)] for y in ys]
    for row, x in enumerate(xs):
        p = 1
        for m in range(k):
            A[row][m] = p
            p = O.gf_mul(r, p, int(x))
    for c in range(k):
        piv = next(i for i in range(c, k) if A[i][c])
        A[c], A[piv] = A[piv], A[c]
        s = O.gf_inv(r, A[c][c])
        A[c] = [O.gf_mul(r, v, s) for v in A[c]]
        for i in range(k):
            if i != c and A[i][c]:
                f = A[i][c]
                A[i] = [a ^ O.gf_mul(r, f, b) for a, b in zip(A[i], A[c])]
    return [A[i][k] for i in range(k)]


@pytest.mark.parametrize("r,n,k", [(8, 8, 4), (8, 16, 8), (8, 16, 12), (16, 16, 4), (8, 32, 6)])
def test_encode_matches_vandermonde_horner(r, n, k):
    g = np.random.default_rng(n * 31 + k)
    cw = np.zeros((n, 3), dtype=np.uint16)
    cw[:k] = g.integers(0, 1 << r, (k, 3))
    out = O.rs_encode(r, n, k, cw)
    assert np.array_equal(out[:k], cw[:k])  # systematic prefix (eq. F(i)=m_i)
    for col in range(3):
        coeffs = vandermonde_solve(r, list(range(k)), cw[:k, col])
        for t in range(n):
            assert int(out[t, col]) == O.poly_eval(r, coeffs, t)


@pytest.mark.parametrize("r,n,k", [(8, 32, 16), (8, 64, 8), (16, 64, 32)])
def test_codeword_has_degree_below_k(r, n, k):
    """The X-basis coefficients of the whole codeword vanish at indices >= k."""
    g = np.random.default_rng(k)
    cw = np.zeros((n, 2), dtype=np.uint16)
    cw[:k] = g.integers(0, 1 << r, (k, 2))
    coef = O.ifft(r, 0, O.rs_encode(r, n, k, cw))
    assert not coef[k:].any()
    assert coef[:k].any()


def test_mds_exhaustive_8_4():
    """Every erasure pattern with at most n-k = 4 erasures on (8,4) over GF(2^8),
    including all C(8,4) = 70 choices of k survivors, decodes back."""
    r, n, k = 8, 8, 4
    g = np.random.default_rng(84)
    cw = np.zeros((n, 4), dtype=np.uint16)
    cw[:k] = g.integers(0, 256, (k, 4))
    cw = O.rs_encode(r, n, k, cw)
    patterns = 0
    for e in range(0, n - k + 1):
        for erased in itertools.combinations(range(n), e):
            m = np.zeros(n, dtype=np.uint8)
            m[list(erased)] = 1
            bad = cw.copy()
            bad[m == 1] = g.integers(0, 256, (e, 4))
            assert np.array_equal(O.rs_decode(r, n, k, bad, m), cw)
            patterns += 1
    assert patterns == 163


@pytest.mark.parametrize("r,n,k,e", [(8, 32, 16, 16), (8, 16, 12, 3), (16, 256, 128, 128), (16, 64, 48, 10)])
def test_decode_random_patterns(r, n, k, e):
    g = np.random.default_rng(n + e)
    cw = np.zeros((n, 2), dtype=np.uint16)
    cw[:k] = g.integers(0, 1 << r, (k, 2))
    cw = O.rs_encode(r, n, k, cw)
    m = WL.erasure_mask(n, e, seed=n * 7 + e)
    bad = cw.copy()
    bad[m == 1] = 0
    assert np.array_equal(O.rs_decode(r, n, k, bad, m), cw)


def test_decode_refuses_too_many_erasures():
    m = np.zeros(8, dtype=np.uint8)
    m[:5] = 1
    with pytest.raises(RuntimeError):
        O.rs_decode(8, 8, 4, np.zeros((8, 1), dtype=np.uint16), m)


@pytest.mark.parametrize("r,n,e", [(8, 32, 16), (8, 256, 100), (16, 64, 30)])
def test_locator_matches_expanded_polynomial(r, n, e):
    """pi[j] is Pi(w_j) off E and Pi'(w_j) on E, where Pi(x) = prod_{y in E}(x+y)
    is multiplied out and differentiated term by term (Appendix)."""
    m = WL.erasure_mask(n, e, seed=e)
    pi = O.locator(r, n, m)
    poly = [1]
    for y in np.nonzero(m)[0]:
        nxt = [0] * (len(poly) + 1)
        for i, c in enumerate(poly):
            nxt[i + 1] ^= c
            nxt[i] ^= O.gf_mul(r, c, int(y))
        poly = nxt
    dpoly = [poly[i + 1] if (i + 1) % 2 else 0 for i in range(len(poly) - 1)]
    for j in range(n):
        if m[j]:
            assert O.poly_eval(r, poly, j) == 0
            assert int(pi[j]) == O.poly_eval(r, dpoly, j)
        else:
            assert int(pi[j]) == O.poly_eval(r, poly, j) != 0


def fwht_mod(v, M):
    v = [int(x) % M for x in v]
    h = 1
    while h < len(v):
        for i in range(0, len(v), 2 * h):
            for j in range(i, i + h):
                a, b = v[j], v[j + h]
                v[j], v[j + h] = (a + b) % M, (a - b) % M
        h *= 2
    return v


@pytest.mark.parametrize("r,n,e", [(8, 256, 40), (8, 32, 16), (8, 64, 1), (16, 256, 128), (16, 1024, 300)])
def test_locator_by_logical_convolution(r, n, e):
    """The Appendix algorithm, eq. Rnmathrmw, with n-point FWHTs mod 2^r - 1:
    Log Pi = n^-1 FWHT(FWHT(R) * FWHT(L)), n^-1 = 2^(r - lg n) mod 2^r - 1
    (reading for n < 2^r), Log(0) = 0; it reproduces the direct product."""
    Mod = (1 << r) - 1
    lgn = n.bit_length() - 1
    m = WL.erasure_mask(n, e, seed=3 * e + 1)
    R = [int(x) for x in m]
    L = [0] + [O.gf_log(r, y) for y in range(1, n)]
    P = [a * b % Mod for a, b in zip(fwht_mod(R, Mod), fwht_mod(L, Mod))]
    C = [c * pow(2, r - lgn, Mod) % Mod for c in fwht_mod(P, Mod)]
    pi = O.locator(r, n, m)
    assert [O.gf_exp(r, c) for c in C] == [int(x) for x in pi]
