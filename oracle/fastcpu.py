"""ctypes wrapper around ``fastcpu.c``: the paper's O(h lg h) algorithms on one
CPU core.

TEST AND BASELINE INFRASTRUCTURE ONLY, like the oracle beside it, and not the
oracle: it runs the paper's butterflies, derivative and locator on a CPU
core, as the paper's own timings did, so that the method's CPU speed can be
set beside the paper's figures (Sec. VI.B: about 1.12 s to encode and 3.06 s
to decode n = 2^16, k = 2^15 on an Intel Core i7-950) and beside the GPU
library.  The tests pin it to the oracle.

``python -m oracle.fastcpu`` times one encode and one decode of n = 65536,
k = 32768 with 32768 random erasures over GF(2^16), one element per symbol
(the paper's setting) and 2048 elements per symbol (the GPU workload's 4 KiB
shards), on one core, and prints one JSON line.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fastcpu.c")
_LIB = os.path.join(_HERE, "libfastcpu.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``fastcpu.c`` into ``libfastcpu.so`` beside it (gcc, -O2)."""
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
        i, u32, i64, vp = ctypes.c_int, ctypes.c_uint32, ctypes.c_int64, ctypes.c_void_p
        for name, args in {"fc_transform": [i, u32, u32, i, vp, i64], "fc_derivative": [i, u32, vp, i64],
                           "fc_encode": [i, u32, u32, vp, i64], "fc_decode": [i, u32, u32, vp, vp, i64]}.items():
            fn = getattr(L, name)
            fn.restype = i
            fn.argtypes = args
        _lib = L
    return _lib


def _mat(a) -> np.ndarray:
    m = np.array(a, dtype=np.uint16, order="C", copy=True)
    assert m.ndim == 2
    return m


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"fastcpu {what}: status {rc}")


def transform(r: int, l: int, data, inverse: bool = False) -> np.ndarray:
    """Psi_h^l (or its inverse) of the h rows of ``data`` (uint16 [h, cols])."""
    m = _mat(data)
    _check(lib().fc_transform(r, m.shape[0], l, int(inverse), m.ctypes.data, m.shape[1]), "transform")
    return m


def derivative(r: int, data) -> np.ndarray:
    """Coefficients of the formal derivative of [D_h] (Sec. IV)."""
    m = _mat(data)
    _check(lib().fc_derivative(r, m.shape[0], m.ctypes.data, m.shape[1]), "derivative")
    return m


def rs_encode(r: int, n: int, k: int, codeword) -> np.ndarray:
    """Algorithm 1 (k a power of two): parity rows k..n-1 of a copy of ``codeword``."""
    m = _mat(codeword)
    _check(lib().fc_encode(r, n, k, m.ctypes.data, m.shape[1]), "encode")
    return m


def rs_decode(r: int, n: int, k: int, codeword, erased) -> np.ndarray:
    """Algorithm 2: the erased rows of a copy of ``codeword`` recovered."""
    m = _mat(codeword)
    e = np.ascontiguousarray(np.asarray(erased, dtype=np.uint8).reshape(-1))
    _check(lib().fc_decode(r, n, k, m.ctypes.data, e.ctypes.data, m.shape[1]), "decode")
    return m


def _time(cols: int, seed: int = 0):
    import time

    r, n, k = 16, 65536, 32768
    transform(r, 0, np.zeros((2, 1), dtype=np.uint16))  # field tables built before timing
    g = np.random.default_rng(seed)
    cw = np.zeros((n, cols), dtype=np.uint16)
    cw[:k] = g.integers(0, 1 << 16, size=(k, cols), dtype=np.uint16)
    t0 = time.perf_counter()
    enc = rs_encode(r, n, k, cw)
    t1 = time.perf_counter()
    erased = np.zeros(n, dtype=np.uint8)
    erased[g.choice(n, n - k, replace=False)] = 1
    bad = enc.copy()
    bad[erased != 0] = 0
    t2 = time.perf_counter()
    dec = rs_decode(r, n, k, bad, erased)
    t3 = time.perf_counter()
    assert np.array_equal(dec, enc)
    return t1 - t0, t3 - t2


if __name__ == "__main__":
    import json
    import platform

    e1, d1 = _time(1)
    e2, d2 = _time(2048)
    print(json.dumps({"n": 65536, "k": 32768, "erasures": 32768, "field": "GF(2^16)", "cores": 1,
                      "machine": platform.machine(),
                      "one_element_per_symbol": {"encode_s": round(e1, 4), "decode_s": round(d1, 4)},
                      "4KiB_shards": {"encode_s": round(e2, 3), "decode_s": round(d2, 3),
                                      "shard_data_gbs": round(2 * 32768 * 4096 / (e2 + d2) / 1e9, 4)}}))
