"""Pins for the derivative oracle (Sec. IV): the paper's closed form and its
worked examples, which the oracle (monomial route) never uses."""
import numpy as np
import pytest

from oracle import oracle as O


def unit(h, i):
    v = np.zeros((h, 1), dtype=np.uint16)
    v[i, 0] = 1
    return v


@pytest.mark.parametrize("r", [8, 16])
def test_derivative_of_X_power_of_two_is_Wprime(r):
    """X_{2^l} = W_l / W_l(w_{2^l}), whose derivative is the constant W'_l."""
    lgh = 5
    h = 1 << lgh
    for l in range(lgh):
        out = O.derivative(r, unit(h, 1 << l))[:, 0]
        expect = np.zeros(h, dtype=np.uint16)
        expect[0] = O.Wprime(r, l)
        assert np.array_equal(out, expect)


@pytest.mark.parametrize("r", [8, 16])
def test_X13_example(r):
    """X'_13 = W'_0 X_12 + W'_2 X_9 + W'_3 X_5 (Sec. IV.A example)."""
    out = O.derivative(r, unit(16, 13))[:, 0]
    expect = np.zeros(16, dtype=np.uint16)
    expect[12] = O.Wprime(r, 0)
    expect[9] = O.Wprime(r, 2)
    expect[5] = O.Wprime(r, 3)
    assert np.array_equal(out, expect)


def test_h8_worked_example():
    """The h = 8 example of Sec. IV.B with B_i = prod_{j in I_i} W'_j."""
    r = 8
    M = lambda a, b: O.gf_mul(r, a, b)
    Wp = [O.Wprime(r, j) for j in range(3)]
    Bc = []
    for i in range(8):
        acc = 1
        for j in range(3):
            if (i >> j) & 1:
                acc = M(acc, Wp[j])
        Bc.append(acc)
    g = np.random.default_rng(8)
    for _ in range(20):
        d = [int(v) for v in g.integers(0, 256, 8)]
        dd = [M(d[i], Bc[i]) for i in range(8)]
        div = lambda s, i: M(s, O.gf_inv(r, Bc[i]))
        expect = [div(dd[1] ^ dd[2] ^ dd[4], 0), div(dd[3] ^ dd[5], 1), div(dd[3] ^ dd[6], 2),
                  div(dd[7], 3), div(dd[5] ^ dd[6], 4), div(dd[7], 5), div(dd[7], 6), 0]
        out = O.derivative(r, np.array(d, dtype=np.uint16)[:, None])[:, 0].tolist()
        assert out == expect


@pytest.mark.parametrize("r,lgh", [(8, 6), (8, 8), (16, 6)])
def test_closed_form(r, lgh):
    """eq. D'_h(x)-2: coefficient j is sum over l not in I_j (l < lg h) of
    W'_l d_{j+2^l}."""
    h = 1 << lgh
    g = np.random.default_rng(h + r)
    d = g.integers(0, 1 << r, (h, 2)).astype(np.uint16)
    out = O.derivative(r, d)
    Wp = [O.Wprime(r, l) for l in range(lgh)]
    for col in range(2):
        for j in range(h):
            s = 0
            for l in range(lgh):
                if not (j >> l) & 1:
                    s ^= O.gf_mul(r, Wp[l], int(d[j + (1 << l), col]))
            assert int(out[j, col]) == s


def test_derivative_values_match_monomial_derivative():
    """Evaluations: ([D]')(x) equals the Horner value of the term-by-term
    derivative of the monomial expansion, at every x in GF(2^8)."""
    r, lgh = 8, 4
    h = 1 << lgh
    d = np.random.default_rng(2).integers(0, 256, h).astype(np.uint16)
    # monomial expansion of [D](x)
    p = [0] * h
    for i in range(h):
        Xi = O.X_poly(r, lgh, i)
        for m in range(i + 1):
            p[m] ^= O.gf_mul(r, int(d[i]), int(Xi[m]))
    dp = [p[m + 1] if (m + 1) % 2 else 0 for m in range(h - 1)]
    e = O.derivative(r, d[:, None])[:, 0]
    for x in range(256):
        lhs = 0
        for i in range(h):
            lhs ^= O.gf_mul(r, int(e[i]), O.X(r, i, x))
        assert lhs == O.poly_eval(r, dp, x)
