"""Thin Python binding of the liblch C ABI (``include/lch.h``).

Argument marshalling only: every step of every call runs in the CUDA kernels
of ``liblch.so``.  Data arguments are CUDA ``torch.uint8`` tensors of shape
``[rows, shard_bytes]`` (contiguous, 16-byte aligned); calls are enqueued on
torch's current CUDA stream unless a stream is given.  The library is loaded
from this package directory; if it is missing or fails to load, every call
raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblch.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "lch.h")

LCH_OK, LCH_EINVAL, LCH_ETOOMANY, LCH_ENOMEM, LCH_ECUDA, LCH_ETIMEDOUT = 0, 1, 2, 3, 4, 5
GF8, GF16 = 8, 16

_lib = None

BATCH_ENCODE, BATCH_DECODE = 0, 1


class Codeword(ctypes.Structure):
    """struct lch_codeword of include/lch.h."""

    _fields_ = [("n", ctypes.c_uint32), ("k", ctypes.c_uint32), ("field", ctypes.c_int),
                ("reserved", ctypes.c_uint32), ("shard_bytes", ctypes.c_size_t), ("shards", ctypes.c_void_p),
                ("erasure_mask", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    """struct lch_tuning of include/lch.h."""

    _fields_ = [("split", ctypes.c_uint32), ("lg_tile_low", ctypes.c_uint32), ("lg_tile_high", ctypes.c_uint32),
                ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {"split": int(self.split), "lg_tile_low": int(self.lg_tile_low),
                "lg_tile_high": int(self.lg_tile_high), "ms": float(self.ms)}


class LchError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def declared_functions():
    """Names of the entry points that include/lch.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return re.findall(r"LCH_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)


def load() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblch.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, sz, i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
    sigs = {
        "lch_ctx_create": (i, [ctypes.POINTER(vp), i]),
        "lch_ctx_destroy": (None, [vp]),
        "lch_fft": (i, [vp, i, u32, u32, vp, sz, vp]),
        "lch_ifft": (i, [vp, i, u32, u32, vp, sz, vp]),
        "lch_derivative": (i, [vp, i, u32, vp, sz, vp]),
        "rs_encode": (i, [vp, u32, u32, i, vp, sz, vp]),
        "rs_decode": (i, [vp, u32, u32, i, vp, sz, vp, vp]),
        "rs_decode_packed": (i, [vp, u32, u32, i, vp, vp, sz, vp, vp]),
        "lch_strerror": (ctypes.c_char_p, [i]),
        "lch_last_error": (ctypes.c_char_p, []),
        "lch_launch_count": (ctypes.c_uint64, [vp]),
        "lch_derivative_noalloc": (i, [i, u32, vp, sz, vp]),
        "lch_poly_mul": (i, [vp, i, u32, vp, vp, vp, sz, vp]),
        "lch_batch_create": (i, [vp, i, vp, u32, ctypes.POINTER(vp)]),
        "lch_batch_run": (i, [vp, vp, vp]),
        "lch_batch_bytes": (i, [vp, i, vp, u32, ctypes.POINTER(sz)]),
        "lch_batch_create_in": (i, [vp, i, vp, u32, vp, sz, vp, ctypes.POINTER(vp)]),
        "lch_batch_status": (i, [vp, vp]),
        "lch_batch_tasks": (u32, [vp]),
        "lch_batch_destroy": (None, [vp]),
        "lch_profile_enable": (i, [vp, i]),
        "lch_profile_read": (i, [vp, i, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]),
        "lch_autotune": (i, [vp, i, u32, sz, vp, ctypes.POINTER(Tuning)]),
        "lch_batch_set_wait_limit": (i, [vp, u32]),
        "lch_rows_gather": (i, [vp, vp, vp, u32, sz, vp]),
        "lch_rows_scatter": (i, [vp, vp, vp, u32, sz, vp]),
        "lch_batch_selftest_stall": (i, [vp, vp]),
        "lch_tune_set": (i, [vp, i, u32, sz, ctypes.POINTER(Tuning)]),
        "lch_tune_get": (i, [vp, i, u32, sz, ctypes.POINTER(Tuning)]),
        "lch_set_bitslice": (i, [vp, i]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return load().lch_last_error().decode()


def _check(status: int):
    if status != LCH_OK:
        raise LchError(status, last_error())


def _stream_handle(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _buf(t, rows=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8:
        raise TypeError("expected a CUDA uint8 tensor of shape [rows, shard_bytes]")
    if t.dim() != 2 or not t.is_contiguous():
        raise ValueError("expected a contiguous 2-D tensor [rows, shard_bytes]")
    if rows is not None and t.shape[0] != rows:
        raise ValueError(f"expected {rows} rows, got {t.shape[0]}")
    return ctypes.c_void_p(t.data_ptr()), t.shape[1]


def derivative_noalloc(field: int, buf, stream=None):
    """lch_derivative_noalloc: the formal derivative of the h rows of ``buf``
    in place, on the tensor's current device, without any device allocation
    (for callers that cannot call cudaMalloc).  h * shard_bytes <= 16 MiB."""
    p, S = _buf(buf)
    _check(load().lch_derivative_noalloc(field, buf.shape[0], p, S, _stream_handle(stream)))


def _rows_args(src, dst, idx):
    import torch

    for t in (src, dst):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.uint8 or t.dim() != 2 \
                or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA uint8 tensors [rows, shard_bytes]")
    if src.shape[1] != dst.shape[1]:
        raise ValueError("src and dst must have the same shard_bytes")
    if not isinstance(idx, torch.Tensor) or not idx.is_cuda or idx.dtype != torch.int32 or idx.dim() != 1 \
            or not idx.is_contiguous():
        raise TypeError("expected a contiguous CUDA int32 index tensor")
    return ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), ctypes.c_void_p(idx.data_ptr()), \
        idx.numel(), src.shape[1]


def rows_gather(src, dst, idx, stream=None):
    """lch_rows_gather: dst[i] = src[idx[i]] (rows); idx a CUDA int32 tensor."""
    ps, pd, pi, cnt, S = _rows_args(src, dst, idx)
    if dst.shape[0] < cnt:
        raise ValueError("dst has fewer rows than idx")
    _check(load().lch_rows_gather(ps, pd, pi, cnt, S, _stream_handle(stream)))


def rows_scatter(src, dst, idx, stream=None):
    """lch_rows_scatter: dst[idx[i]] = src[i] (rows); idx a CUDA int32 tensor."""
    ps, pd, pi, cnt, S = _rows_args(src, dst, idx)
    if src.shape[0] < cnt:
        raise ValueError("src has fewer rows than idx")
    _check(load().lch_rows_scatter(ps, pd, pi, cnt, S, _stream_handle(stream)))


def _codeword_array(codewords, keep):
    """ctypes array of struct lch_codeword; host masks are appended to `keep`."""
    arr = (Codeword * max(1, len(codewords)))()
    for i, (n, k, field, shards, mask) in enumerate(codewords):
        p, S = _buf(shards, n)
        m = None
        if mask is not None:
            m = np.ascontiguousarray(np.asarray(mask, dtype=np.uint8).reshape(-1))
            if m.size != n:
                raise ValueError(f"codeword {i}: erasure mask must have n={n} entries")
            keep.append(m)
        arr[i] = Codeword(n, k, field, 0, S, p.value, None if m is None else m.ctypes.data)
    return arr


class Batch:
    """A planned batch of codewords (lch_batch_create); run() enqueues one
    persistent launch, status() waits and reports."""

    def __init__(self, ctx, op, codewords, mem=None, stream=None):
        """codewords: list of (n, k, field, shards_tensor, erasure_mask or None).
        mem: optional CUDA uint8 tensor holding the batch's device memory
        (see batch_bytes); the batch then allocates nothing."""
        self._ctx = ctx
        self._keep = []
        arr = self._array(codewords)
        h = ctypes.c_void_p()
        if mem is None:
            _check(load().lch_batch_create(ctx._h, op, arr, len(codewords), ctypes.byref(h)))
        else:
            self._keep.append(mem)
            _check(load().lch_batch_create_in(ctx._h, op, arr, len(codewords), ctypes.c_void_p(mem.data_ptr()),
                                              mem.numel(), _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def _array(self, codewords):
        return _codeword_array(codewords, self._keep)

    @property
    def tasks(self) -> int:
        return int(load().lch_batch_tasks(self._h))

    def run(self, stream=None):
        _check(load().lch_batch_run(self._ctx._h, self._h, _stream_handle(stream)))

    def status(self):
        _check(load().lch_batch_status(self._ctx._h, self._h))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lch_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """A liblch context on one CUDA device (owns tables and scratch)."""

    def __init__(self, device: int = 0):
        L = load()
        h = ctypes.c_void_p()
        _check(L.lch_ctx_create(ctypes.byref(h), int(device)))
        self._h = h
        self.device = device

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().lch_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(load().lch_launch_count(self._h))

    def profile_enable(self, on: bool = True):
        _check(load().lch_profile_enable(self._h, int(on)))

    def profile(self, kind: int) -> dict:
        """Launches, summed device ms, algorithmic bytes and field
        multiplications of one kernel kind since profiling was enabled (see
        lch_profile_read)."""
        n, ms, by, mu = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().lch_profile_read(self._h, kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by),
                                       ctypes.byref(mu)))
        return {"launches": int(n.value), "ms": float(ms.value), "bytes": int(by.value), "mults": int(mu.value)}

    def batch(self, op: int, codewords, mem=None, stream=None) -> "Batch":
        return Batch(self, op, codewords, mem=mem, stream=stream)

    def batch_set_wait_limit(self, wait_us: int):
        """lch_batch_set_wait_limit: per-task dependency wait limit of later
        batch runs."""
        _check(load().lch_batch_set_wait_limit(self._h, int(wait_us)))

    def batch_selftest_stall(self, stream=None) -> int:
        """lch_batch_selftest_stall: the status of a batch run whose one task
        can never start (LCH_ETIMEDOUT when the wait gave up as designed)."""
        return int(load().lch_batch_selftest_stall(self._h, _stream_handle(stream)))

    def batch_bytes(self, op: int, codewords) -> int:
        """Device bytes a batch of these codewords needs (lch_batch_bytes)."""
        keep = []
        arr = _codeword_array(codewords, keep)
        out = ctypes.c_size_t()
        _check(load().lch_batch_bytes(self._h, op, arr, len(codewords), ctypes.byref(out)))
        return int(out.value)

    def autotune(self, field: int, h: int, shard_bytes: int, stream=None) -> dict:
        """lch_autotune: time candidate pass plans for (field, h, shard_bytes),
        keep the fastest on this context and return it."""
        t = Tuning()
        _check(load().lch_autotune(self._h, field, h, shard_bytes, _stream_handle(stream), ctypes.byref(t)))
        return t.as_dict()

    def tune_set(self, field: int, h: int, shard_bytes: int, plan: dict | None):
        """lch_tune_set: install a plan (a dict as autotune returns), or None
        to go back to the default plan."""
        if plan is None:
            _check(load().lch_tune_set(self._h, field, h, shard_bytes, None))
            return
        t = Tuning(int(plan["split"]), int(plan["lg_tile_low"]), int(plan["lg_tile_high"]), float(plan.get("ms", 0.0)))
        _check(load().lch_tune_set(self._h, field, h, shard_bytes, ctypes.byref(t)))

    def tune_get(self, field: int, h: int, shard_bytes: int):
        """lch_tune_get: the plan installed for (field, h, shard_bytes) as a
        dict, or None when there is none."""
        t = Tuning()
        if load().lch_tune_get(self._h, field, h, shard_bytes, ctypes.byref(t)) != LCH_OK:
            return None
        return t.as_dict()

    def set_bitslice(self, on: bool):
        """lch_set_bitslice: GF(2^16) transforms as bit-sliced passes (True)
        or split-table passes (False, the default); the results are the same."""
        _check(load().lch_set_bitslice(self._h, int(bool(on))))

    # Sec. III: Psi_h^l and its inverse, in place on h rows.
    def fft(self, field: int, l: int, buf, stream=None):
        p, S = _buf(buf)
        _check(load().lch_fft(self._h, field, buf.shape[0], l, p, S, _stream_handle(stream)))

    def ifft(self, field: int, l: int, buf, stream=None):
        p, S = _buf(buf)
        _check(load().lch_ifft(self._h, field, buf.shape[0], l, p, S, _stream_handle(stream)))

    # Sec. IV: formal derivative, in place on h rows.
    def derivative(self, field: int, buf, stream=None):
        p, S = _buf(buf)
        _check(load().lch_derivative(self._h, field, buf.shape[0], p, S, _stream_handle(stream)))

    # Sec. VI.A: c (2h rows) = coefficients of [a](x) [b](x); a, b: h rows.
    def poly_mul(self, field: int, a, b, c, stream=None):
        pa, S = _buf(a)
        pb, _ = _buf(b, a.shape[0])
        pc, _ = _buf(c, 2 * a.shape[0])
        _check(load().lch_poly_mul(self._h, field, a.shape[0], pa, pb, pc, S, _stream_handle(stream)))

    # Sec. V, Algorithm 1.
    def rs_encode(self, n: int, k: int, field: int, shards, stream=None):
        p, S = _buf(shards, n)
        _check(load().rs_encode(self._h, n, k, field, p, S, _stream_handle(stream)))

    # Sec. V, Algorithm 2.  erasure_mask: n bytes on the host, nonzero = erased.
    def rs_decode(self, n: int, k: int, field: int, shards, erasure_mask, stream=None):
        p, S = _buf(shards, n)
        m = np.ascontiguousarray(np.asarray(erasure_mask, dtype=np.uint8).reshape(-1))
        if m.size != n:
            raise ValueError(f"erasure mask must have n={n} entries")
        _check(load().rs_decode(self._h, n, k, field, p, S, m.ctypes.data, _stream_handle(stream)))

    # Algorithm 2 from the received shards alone: `received` holds the
    # n - |E| surviving shards in row order, `recovered` gets the |E| erased
    # ones in row order; the codeword is never assembled.
    def rs_decode_packed(self, n: int, k: int, field: int, received, recovered, erasure_mask, stream=None):
        m = np.ascontiguousarray(np.asarray(erasure_mask, dtype=np.uint8).reshape(-1))
        if m.size != n:
            raise ValueError(f"erasure mask must have n={n} entries")
        ne = int(np.count_nonzero(m))
        pr, S = _buf(received, n - ne)
        po, S2 = _buf(recovered, ne)
        if S2 != S:
            raise ValueError("received and recovered shards differ in size")
        _check(load().rs_decode_packed(self._h, n, k, field, pr, po, S, m.ctypes.data, _stream_handle(stream)))
