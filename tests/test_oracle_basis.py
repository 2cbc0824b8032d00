"""Pins for W_j, X_i and W'_l (Sec. II.B-C, Lemma 1, Lemma 3, the h=8 example)."""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def W_table(r, j, xs):
    return np.array([O.W(r, j, int(x)) for x in xs], dtype=np.int64)


@pytest.mark.parametrize("j", range(8))
def test_W_vanishes_exactly_on_subspace_gf8(j):
    w = W_table(8, j, range(256))
    zeros = np.nonzero(w == 0)[0]
    assert zeros.tolist() == list(range(1 << j))  # W_j(w_i) = 0 iff i < 2^j (eq. w_j)


@pytest.mark.parametrize("j", range(8))
def test_lemma1_linearity_exhaustive_gf8(j):
    w = W_table(8, j, range(256))
    x = np.arange(256)[:, None]
    y = np.arange(256)[None, :]
    assert np.array_equal(w[x ^ y], w[x] ^ w[y])  # W_j(x+y) = W_j(x) + W_j(y)


@pytest.mark.parametrize("r,j", [(8, j) for j in range(8)] + [(16, j) for j in range(9)])
def test_W_is_linearized_polynomial(r, j):
    """Lemma 1, eq. W_i(x): the monomial expansion of prod (x + w_a) has terms
    only at degrees 2^i, i <= j, and is monic of degree 2^j."""
    c = O.W_poly(r, j)
    assert c.size == (1 << j) + 1 and c[-1] == 1
    support = set(np.nonzero(c)[0].tolist())
    assert support <= {1 << i for i in range(j + 1)}
    # the expansion evaluates (Horner) to the direct product
    g = np.random.default_rng(j)
    for x in g.integers(0, 1 << r, 5):
        assert O.poly_eval(r, c, int(x)) == O.W(r, j, int(x))


@pytest.mark.parametrize("r,l", [(8, l) for l in range(8)] + [(16, l) for l in range(10)])
def test_lemma3_Wprime(r, l):
    """W_l'(x) is the constant prod_{j=1}^{2^l-1} w_j: it is the coefficient of
    x^1 in the expansion, and W'_l divides it by W_l(w_{2^l}) (eq. W-l)."""
    c = O.W_poly(r, l)
    num = 1
    for a in range(1, 1 << l):
        num = O.gf_mul_bitwise(r, num, a)
    assert int(c[1]) == num
    assert O.gf_mul(r, O.Wprime(r, l), O.W(r, l, 1 << l)) == num


@pytest.mark.parametrize("r", [8, 16])
def test_X_degree_and_normalisation(r):
    lgh = 5
    for i in range(1 << lgh):
        c = O.X_poly(r, lgh, i)
        assert c.size == i + 1 and c[i] != 0  # deg X_i = i (Sec. II.C)
        for x in (0, 1, 5, 17, (1 << r) - 3):
            assert O.poly_eval(r, c, x) == O.X(r, i, x)
    for j in range(r):
        assert O.X(r, 1 << j, 1 << j) == 1  # X_{2^j}(w_{2^j}) = W_j(w_{2^j}) / W_j(w_{2^j})


def test_h8_recursive_expansion():
    """The worked h = 8 expansion of [D_8](x) into Delta_2, Delta_1, Delta_0
    (eq. P_j^i(x)rec example) agrees with sum_i d_i X_i(x) at every point."""
    r = 8
    g = np.random.default_rng(11)
    d = [int(v) for v in g.integers(0, 256, 8)]
    M = lambda a, b: O.gf_mul(r, a, b)
    for x in range(256):
        hw = [M(O.W(r, j, x), O.gf_inv(r, O.W(r, j, 1 << j))) for j in range(3)]
        direct = 0
        for i in range(8):
            direct ^= M(d[i], O.X(r, i, x))
        nested = (d[0] ^ M(d[4], hw[2]) ^ M(hw[1], d[2] ^ M(d[6], hw[2]))) ^ M(
            hw[0], d[1] ^ M(d[5], hw[2]) ^ M(hw[1], d[3] ^ M(d[7], hw[2])))
        assert direct == nested


def test_transform_h4_golden():
    """Hand-derived X_i(w_c + w_l) for h = 4 in GF(2^8)."""
    with open(os.path.join(GOLDEN, "transform_h4_gf8.txt")) as f:
        rows = [list(map(int, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")]
    for l, c, *xs in rows:
        assert [O.X(8, i, c ^ l) for i in range(4)] == xs
        # and through the transform oracle, column by column
        eye = np.eye(4, dtype=np.uint16)
        out = O.fft(8, l, eye, rows=[c])
        assert out[0].tolist() == xs
