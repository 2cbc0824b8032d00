"""The paper's fast transform, written in its own set notation, for pinning.

TEST INFRASTRUCTURE ONLY.  This is not the plain-definition oracle (that is
``oracle.fft``, direct evaluation); it restates the algorithm of Sec. III.C so
that the tests can check three things against the direct evaluation:

* the recursion from Psi(i+1, m, l) and Psi(i+1, m+2^i, l) to Psi(i, m, l)
  (eqs. Deltajimcoplusl and Deltajimcoplusloplusi2) reproduces
  [D_h](w_c + w_l) for every c < h;
* the operation counts of Sec. III.D: A(h) = h lg h additions and
  M(h) = (h/2) lg h multiplications, or A_0(h) = h lg h - h + 1 and
  M_0(h) = (h/2) lg h - h + 1 when the shift is zero (eq. Deltajim0);
* the reading that Fig. 1 (whose image is missing from the paper) is the
  in-place, natural-order butterfly network: element t of an h-vector pairs
  with t + 2^i at level i, with factor W_i(w_j + w_l)/W_i(w_{2^i}) where j is
  t with its low i+1 bits cleared; levels run from lg h - 1 down to 0 for the
  transform and from 0 up for its inverse (Sec. III.E).

Pure Python on one column of small h; the field products come from the
oracle's tables.
"""
from __future__ import annotations

from . import oracle as O


def _factor(r: int, i: int, point: int) -> int:
    """W_i(point) / W_i(w_{2^i})."""
    return O.gf_mul(r, O.W(r, i, point), O.gf_inv(r, O.W(r, i, 1 << i)))


def transform_sets(r: int, d, l: int):
    """Psi_h^l[D_h] by the recursion on the sets Psi(i, m, l).

    Returns (values, additions, multiplications).  Psi(i, m, l) is held as a
    dict c -> Delta_i^m(w_c + w_l) over c in {b 2^i}."""
    h = len(d)
    lgh = h.bit_length() - 1
    assert 1 << lgh == h
    adds = muls = 0
    psi = {m: {0: int(d[m])} for m in range(h)}  # Psi(lg h, m, l) = {d_m}
    for i in range(lgh - 1, -1, -1):
        nxt = {}
        for m in range(1 << i):
            lo, hi = psi[m], psi[m + (1 << i)]
            out = {}
            for c in range(0, h, 1 << (i + 1)):
                u, v = lo[c], hi[c]
                if c ^ l == 0:  # w_c + w_l = 0: Delta_i^m(0) = Delta_{i+1}^m(0)
                    x0 = u
                else:
                    x0 = u ^ O.gf_mul(r, _factor(r, i, c ^ l), v)
                    adds += 1
                    muls += 1
                x1 = x0 ^ v
                adds += 1
                out[c] = x0
                out[c + (1 << i)] = x1
            nxt[m] = out
        psi = nxt
    vals = [psi[0][c] for c in range(h)]
    return vals, adds, muls


def transform_inplace(r: int, d, l: int):
    """The same transform as an in-place natural-order butterfly network."""
    a = [int(x) for x in d]
    h = len(a)
    lgh = h.bit_length() - 1
    for i in range(lgh - 1, -1, -1):
        s = 1 << i
        for j in range(0, h, 2 * s):
            f = _factor(r, i, j ^ l)
            for t in range(j, j + s):
                a[t] ^= O.gf_mul(r, f, a[t + s])
                a[t + s] ^= a[t]
    return a


def inverse_inplace(r: int, v, l: int):
    """Inverse network: levels 0 .. lg h - 1, each butterfly undone (Sec. III.E)."""
    a = [int(x) for x in v]
    h = len(a)
    lgh = h.bit_length() - 1
    for i in range(lgh):
        s = 1 << i
        for j in range(0, h, 2 * s):
            f = _factor(r, i, j ^ l)
            for t in range(j, j + s):
                a[t + s] ^= a[t]
                a[t] ^= O.gf_mul(r, f, a[t + s])
    return a
