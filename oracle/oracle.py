"""ctypes wrapper around ``oracle.c``, the plain CPU oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function here
marshals numpy arrays into the C routines, each of which computes its result
from the paper's plain definition; see ``oracle.c`` for the citations.

Element matrices are ``uint16`` arrays of shape ``[rows, cols]`` in both fields.
``to_elems`` / ``from_elems`` convert shard bytes ``uint8 [rows, S]`` to that form
(GF(2^16) elements are little-endian ``uint16``; GF(2^8) elements are bytes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "lib", "to_elems", "from_elems", "gf_mul", "gf_mul_bitwise", "gf_inv", "gf_exp",
    "gf_log", "gf_mul_vec", "W", "Wprime", "X", "W_poly", "X_poly", "fft", "ifft", "derivative",
    "rs_encode", "rs_decode", "locator", "poly_eval", "poly_mul",
]


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` beside it (gcc, -O2)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32, i32, i64, vp = ctypes.c_uint32, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        sig = {
            "orc_field_ok": (ctypes.c_int, [ctypes.c_int]),
            "orc_gf_mul_bitwise": (u32, [ctypes.c_int, u32, u32]),
            "orc_gf_mul": (u32, [ctypes.c_int, u32, u32]),
            "orc_gf_inv": (u32, [ctypes.c_int, u32]),
            "orc_gf_exp": (u32, [ctypes.c_int, u32]),
            "orc_gf_log": (u32, [ctypes.c_int, u32]),
            "orc_gf_mul_vec": (None, [ctypes.c_int, vp, vp, vp, i64]),
            "orc_W": (u32, [ctypes.c_int, ctypes.c_int, u32]),
            "orc_Wprime": (u32, [ctypes.c_int, ctypes.c_int]),
            "orc_X": (u32, [ctypes.c_int, ctypes.c_int, u32]),
            "orc_W_poly": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp]),
            "orc_X_poly": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32, vp]),
            "orc_fft": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32, vp, vp, i64, vp, i32]),
            "orc_ifft": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, u32, vp, vp, i64]),
            "orc_derivative": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, i64]),
            "orc_rs_encode": (ctypes.c_int, [ctypes.c_int, u32, u32, vp, i64, vp, i32]),
            "orc_rs_decode": (ctypes.c_int, [ctypes.c_int, u32, u32, vp, vp, i64, vp, i32]),
            "orc_locator": (ctypes.c_int, [ctypes.c_int, u32, vp, vp]),
            "orc_poly_mul": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, vp, vp, vp, i64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        for r in (8, 16):
            if L.orc_field_ok(r) != 0:
                raise RuntimeError(f"oracle: alpha = x is not primitive in GF(2^{r})")
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


# --------------------------------------------------------------------------- shards <-> elements

def to_elems(shards: np.ndarray, r: int) -> np.ndarray:
    """uint8 [rows, S] shard bytes -> uint16 [rows, S/(r/8)] field elements."""
    a = np.ascontiguousarray(shards, dtype=np.uint8)
    if r == 16:
        return a.view("<u2").astype(np.uint16)
    return a.astype(np.uint16)


def from_elems(elems: np.ndarray, r: int) -> np.ndarray:
    """Inverse of ``to_elems``."""
    e = np.ascontiguousarray(elems, dtype=np.uint16)
    if r == 16:
        return e.astype("<u2").view(np.uint8).reshape(e.shape[0], -1)
    return e.astype(np.uint8)


# --------------------------------------------------------------------------- field

def gf_mul(r: int, a: int, b: int) -> int:
    return int(lib().orc_gf_mul(r, a, b))


def gf_mul_bitwise(r: int, a: int, b: int) -> int:
    return int(lib().orc_gf_mul_bitwise(r, a, b))


def gf_inv(r: int, a: int) -> int:
    return int(lib().orc_gf_inv(r, a))


def gf_exp(r: int, i: int) -> int:
    return int(lib().orc_gf_exp(r, i))


def gf_log(r: int, a: int) -> int:
    return int(lib().orc_gf_log(r, a))


def gf_mul_vec(r: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint16)
    b = np.ascontiguousarray(np.broadcast_to(b, a.shape), dtype=np.uint16)
    out = np.empty_like(a)
    lib().orc_gf_mul_vec(r, _ptr(a), _ptr(b), _ptr(out), a.size)
    return out


def poly_eval(r: int, coeffs, x: int) -> int:
    """Horner evaluation of sum_m coeffs[m] x^m (monomial basis)."""
    acc = 0
    for c in reversed(list(coeffs)):
        acc = gf_mul(r, acc, x) ^ int(c)
    return acc


# --------------------------------------------------------------------------- basis

def W(r: int, j: int, x: int) -> int:
    """W_j(x) = prod_{a<2^j} (x + w_a)."""
    return int(lib().orc_W(r, j, x))


def Wprime(r: int, l: int) -> int:
    """W'_l = prod_{j=1}^{2^l-1} w_j / W_l(w_{2^l}) (Lemma 3, eq. W-l)."""
    return int(lib().orc_Wprime(r, l))


def X(r: int, i: int, x: int) -> int:
    """X_i(x) = prod_{j in I_i} W_j(x) / W_j(w_{2^j})."""
    return int(lib().orc_X(r, i, x))


def W_poly(r: int, j: int) -> np.ndarray:
    out = np.zeros((1 << j) + 1, dtype=np.uint32)
    _check(lib().orc_W_poly(r, j, _ptr(out)), "W_poly")
    return out


def X_poly(r: int, lgh: int, i: int) -> np.ndarray:
    out = np.zeros(i + 1, dtype=np.uint32)
    _check(lib().orc_X_poly(r, lgh, i, _ptr(out)), "X_poly")
    return out


# --------------------------------------------------------------------------- transforms

def fft(r: int, l: int, data: np.ndarray, rows=None) -> np.ndarray:
    """Psi_h^l by direct evaluation.  data: uint16 [h, cols].  With ``rows``,
    only those output rows are evaluated (returned in that order)."""
    d = np.ascontiguousarray(data, dtype=np.uint16)
    h, cols = d.shape
    lgh = h.bit_length() - 1
    assert 1 << lgh == h
    if rows is None:
        out = np.empty_like(d)
        _check(lib().orc_fft(r, lgh, l, _ptr(d), _ptr(out), cols, None, 0), "fft")
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int32)
        out = np.empty((rr.size, cols), dtype=np.uint16)
        _check(lib().orc_fft(r, lgh, l, _ptr(d), _ptr(out), cols, _ptr(rr), rr.size), "fft")
    return out


def ifft(r: int, l: int, data: np.ndarray) -> np.ndarray:
    """(Psi_h^l)^-1 by Gaussian elimination on the evaluation matrix."""
    d = np.ascontiguousarray(data, dtype=np.uint16)
    h, cols = d.shape
    lgh = h.bit_length() - 1
    assert 1 << lgh == h
    out = np.empty_like(d)
    _check(lib().orc_ifft(r, lgh, l, _ptr(d), _ptr(out), cols), "ifft")
    return out


def derivative(r: int, data: np.ndarray) -> np.ndarray:
    """Formal derivative of [D_h], in the X basis, via the monomial basis."""
    d = np.ascontiguousarray(data, dtype=np.uint16)
    h, cols = d.shape
    lgh = h.bit_length() - 1
    assert 1 << lgh == h
    out = np.empty_like(d)
    _check(lib().orc_derivative(r, lgh, _ptr(d), _ptr(out), cols), "derivative")
    return out


# --------------------------------------------------------------------------- RS code

def rs_encode(r: int, n: int, k: int, codeword: np.ndarray, rows=None) -> np.ndarray:
    """Fill parity rows (all of [k, n), or just ``rows``) of a copy of ``codeword``
    (uint16 [n, cols], message in rows 0..k-1) by Lagrange interpolation."""
    cw = np.array(codeword, dtype=np.uint16, order="C", copy=True)
    assert cw.shape[0] == n
    if rows is None:
        _check(lib().orc_rs_encode(r, n, k, _ptr(cw), cw.shape[1], None, 0), "rs_encode")
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int32)
        _check(lib().orc_rs_encode(r, n, k, _ptr(cw), cw.shape[1], _ptr(rr), rr.size), "rs_encode")
    return cw


def rs_decode(r: int, n: int, k: int, codeword: np.ndarray, erased: np.ndarray, rows=None) -> np.ndarray:
    """Recover erased rows (all, or the erased ones among ``rows``) of a copy of
    ``codeword`` by re-interpolation from the first k survivors."""
    cw = np.array(codeword, dtype=np.uint16, order="C", copy=True)
    m = np.ascontiguousarray(erased, dtype=np.uint8)
    assert cw.shape[0] == n and m.size == n
    if rows is None:
        rc = lib().orc_rs_decode(r, n, k, _ptr(cw), _ptr(m), cw.shape[1], None, 0)
    else:
        rr = np.ascontiguousarray(rows, dtype=np.int32)
        rc = lib().orc_rs_decode(r, n, k, _ptr(cw), _ptr(m), cw.shape[1], _ptr(rr), rr.size)
    _check(rc, "rs_decode")
    return cw


def locator(r: int, n: int, erased: np.ndarray) -> np.ndarray:
    """pi[j] = prod_{y in E, y != j} (w_j + w_y): Pi(j) off E, Pi'(j) on E."""
    m = np.ascontiguousarray(erased, dtype=np.uint8)
    out = np.empty(n, dtype=np.uint32)
    _check(lib().orc_locator(r, n, _ptr(m), _ptr(out)), "locator")
    return out


def poly_mul(r: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Coefficients (2h rows, X basis) of the product of the polynomials with
    X-basis coefficients a and b (h rows each), via the monomial basis."""
    A = np.ascontiguousarray(a, dtype=np.uint16)
    Bm = np.ascontiguousarray(b, dtype=np.uint16)
    h, cols = A.shape
    lgh = h.bit_length() - 1
    assert 1 << lgh == h and Bm.shape == A.shape
    out = np.empty((2 * h, cols), dtype=np.uint16)
    _check(lib().orc_poly_mul(r, lgh, _ptr(A), _ptr(Bm), _ptr(out), cols), "poly_mul")
    return out
