"""The C ABI loads, exports every entry point include/lch.h declares, and
rejects bad arguments on the host before touching a GPU (no compute calls)."""
import ctypes

import pytest

from paper_1404_3458_gb300 import build as B
from paper_1404_3458_gb300 import lch


@pytest.fixture(scope="module")
def L():
    B.build()
    return lch.load()


def test_exports_every_declared_symbol(L):
    names = lch.declared_functions()
    assert set(names) >= {"lch_ctx_create", "lch_ctx_destroy", "lch_fft", "lch_ifft", "lch_derivative",
                          "rs_encode", "rs_decode", "lch_strerror", "lch_last_error", "lch_launch_count"}
    for name in names:
        assert hasattr(L, name), name


def test_strerror(L):
    assert L.lch_strerror(0) == b"success"
    assert L.lch_strerror(lch.LCH_ETOOMANY) == b"more erasures than n - k"
    assert L.lch_strerror(99) == b"unknown status"


FAKE = ctypes.c_void_p(0x10000)       # 16-byte aligned, never dereferenced
MISALIGNED = ctypes.c_void_p(0x10008)


@pytest.mark.parametrize("args,needle", [
    ((None, 33, 16, 8, FAKE, 1024, None), "n must be a power of two"),
    ((None, 512, 16, 8, FAKE, 1024, None), "at most 2^8"),
    ((None, 32, 0, 8, FAKE, 1024, None), "1 <= k <= n"),
    ((None, 32, 33, 8, FAKE, 1024, None), "1 <= k <= n"),
    ((None, 32, 16, 12, FAKE, 1024, None), "field must be"),
    ((None, 32, 16, 8, FAKE, 1000, None), "multiple of 16"),
    ((None, 32, 16, 8, FAKE, 0, None), "multiple of 16"),
    ((None, 32, 16, 8, MISALIGNED, 1024, None), "16-byte aligned"),
    ((None, 32, 16, 8, None, 1024, None), "NULL"),
    ((None, 32, 16, 8, FAKE, 1024, None), "ctx is NULL"),
])
def test_encode_argument_checks(L, args, needle):
    assert L.rs_encode(*args) == lch.LCH_EINVAL
    assert needle in lch.last_error()


def test_decode_packed_argument_checks(L):
    mask = (ctypes.c_uint8 * 32)()
    mask[3] = 1
    assert L.rs_decode_packed(None, 32, 16, 8, FAKE, FAKE, 1024, None, None) == lch.LCH_EINVAL
    assert "erasure_mask is NULL" in lch.last_error()
    assert L.rs_decode_packed(None, 32, 16, 8, FAKE, None, 1024, mask, None) == lch.LCH_EINVAL
    assert "NULL" in lch.last_error()
    assert L.rs_decode_packed(None, 32, 16, 8, MISALIGNED, FAKE, 1024, mask, None) == lch.LCH_EINVAL
    assert "16-byte aligned" in lch.last_error()
    assert L.rs_decode_packed(None, 32, 16, 8, FAKE, FAKE, 1000, mask, None) == lch.LCH_EINVAL
    assert L.rs_decode_packed(None, 32, 16, 8, FAKE, FAKE, 1024, mask, None) == lch.LCH_EINVAL
    assert "ctx is NULL" in lch.last_error()
    # no erasures: nothing to do, whatever the buffers
    assert L.rs_decode_packed(None, 32, 16, 8, None, None, 1024, (ctypes.c_uint8 * 32)(), None) == lch.LCH_OK


def test_decode_and_transform_argument_checks(L):
    mask = (ctypes.c_uint8 * 32)()
    assert L.rs_decode(None, 32, 16, 8, FAKE, 1024, None, None) == lch.LCH_EINVAL
    assert "erasure_mask is NULL" in lch.last_error()
    assert L.rs_decode(None, 65536 * 2, 16, 16, FAKE, 1024, mask, None) == lch.LCH_EINVAL
    assert L.lch_fft(None, 16, 256, 65536, FAKE, 64, None) == lch.LCH_EINVAL
    assert "shift l" in lch.last_error()
    assert L.lch_ifft(None, 8, 3, 0, FAKE, 64, None) == lch.LCH_EINVAL
    assert L.lch_derivative(None, 16, 1 << 17, FAKE, 64, None) == lch.LCH_EINVAL
    assert L.lch_fft(None, 16, 256, 0, FAKE, 64, None) == lch.LCH_EINVAL
    assert "ctx is NULL" in lch.last_error()
    assert L.lch_launch_count(None) == 0
    L.lch_ctx_destroy(None)  # ignored


def test_python_binding_refuses_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(lch, "_lib", None)
    monkeypatch.setattr(lch, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        lch.load()


def test_utility_entry_points_check_arguments(L):
    """Host-side checks of the entry points outside the paper (no GPU call is
    made before a failing check)."""
    vp = ctypes.c_void_p
    assert L.lch_strerror(lch.LCH_ETIMEDOUT) == b"a batch task gave up waiting"
    t = lch.Tuning()
    assert L.lch_autotune(None, 16, 1024, 64, None, ctypes.byref(t)) == lch.LCH_EINVAL
    assert L.lch_autotune(vp(1), 16, 1000, 64, None, ctypes.byref(t)) == lch.LCH_EINVAL   # h not a power of two
    assert L.lch_autotune(vp(1), 16, 1024, 40, None, ctypes.byref(t)) == lch.LCH_EINVAL   # shard bytes
    assert L.lch_tune_set(None, 16, 1024, 64, None) == lch.LCH_EINVAL
    assert L.lch_tune_get(None, 16, 1024, 64, ctypes.byref(t)) == lch.LCH_EINVAL
    assert L.lch_batch_set_wait_limit(None, 1000) == lch.LCH_EINVAL
    assert L.lch_batch_selftest_stall(None, None) == lch.LCH_EINVAL
    assert L.lch_rows_gather(None, vp(16), vp(16), 4, 64, None) == lch.LCH_EINVAL
    assert L.lch_rows_scatter(vp(16), vp(16), vp(16), 4, 40, None) == lch.LCH_EINVAL
    assert L.lch_rows_scatter(vp(8), vp(16), vp(16), 4, 64, None) == lch.LCH_EINVAL      # misaligned
    assert L.lch_rows_gather(None, None, None, 0, 64, None) == lch.LCH_OK                 # count 0: no-op


def test_binding_refuses_host_tensors_before_any_call():
    """The Python binding marshals only CUDA uint8 tensors: host tensors and
    wrong shapes are refused before the library is called."""
    import numpy as np
    import torch

    with pytest.raises(TypeError):
        lch._buf(torch.zeros((4, 16), dtype=torch.uint8))            # host memory
    with pytest.raises(TypeError):
        lch._buf(np.zeros((4, 16), dtype=np.uint8))                   # not a tensor
    with pytest.raises(TypeError):
        lch.rows_gather(torch.zeros((4, 16), dtype=torch.uint8), torch.zeros((4, 16), dtype=torch.uint8),
                        torch.zeros(4, dtype=torch.int32))
    with pytest.raises(TypeError):
        lch.derivative_noalloc(16, torch.zeros((8, 16), dtype=torch.uint8))


C_CLIENT = r"""
#include "lch.h"
#include <stdio.h>
#include <string.h>

int main(void) {
    unsigned char mask[32] = {0};
    mask[3] = 1;
    void *fake = (void *)0x10000;                       /* never dereferenced */
    if (rs_decode(0, 32, 16, LCH_GF8, fake, 1024, mask, 0) != LCH_EINVAL) return 1;
    if (!strstr(lch_last_error(), "ctx is NULL")) return 2;
    if (rs_encode(0, 33, 16, LCH_GF8, fake, 1024, 0) != LCH_EINVAL) return 3;
    if (rs_decode_packed(0, 32, 16, LCH_GF8, fake, fake, 1000, mask, 0) != LCH_EINVAL) return 4;
    if (strcmp(lch_strerror(LCH_ETOOMANY), "more erasures than n - k") != 0) return 5;
    lch_ctx *ctx = 0;
    int rc = lch_ctx_create(&ctx, 0);                   /* LCH_OK with a GPU, LCH_ECUDA without */
    if (rc == LCH_OK) lch_ctx_destroy(ctx);
    else if (rc != LCH_ECUDA) return 6;
    printf("ok\n");
    return 0;
}
"""


def test_header_is_a_plain_c_abi(L, tmp_path):
    """include/lch.h compiles as C99 with warnings as errors, and a C program
    links liblch.so and gets the documented argument checks (no compute)."""
    import os
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lch.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.dirname(lch.HEADER),
                    str(src), "-L", libdir, "-llch", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
