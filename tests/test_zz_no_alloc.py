"""lch_derivative_noalloc: the formal derivative for callers that cannot
allocate device memory (their allocator owns the device heap, or their host
forbids allocation).  It must give the same bytes as lch_derivative, which uses
context scratch; its own scratch is a fixed 16 MiB device array shared by every
call.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import build as B
from paper_1404_3458_gb300 import lch
from paper_1404_3458_gb300 import workloads as WL

FAKE = ctypes.c_void_p(0x10000)


def test_noalloc_host_checks():
    """Arguments are checked on the host before any CUDA call."""
    B.build()
    L = lch.load()
    assert L.lch_derivative_noalloc(16, 8192, FAKE, 2048 + 16, None) == lch.LCH_EINVAL
    assert "16 MiB" in lch.last_error()
    assert L.lch_derivative_noalloc(16, 3, FAKE, 64, None) == lch.LCH_EINVAL
    assert L.lch_derivative_noalloc(9, 4, FAKE, 64, None) == lch.LCH_EINVAL
    assert L.lch_derivative_noalloc(8, 4, FAKE, 40, None) == lch.LCH_EINVAL


@pytest.mark.gpu
def test_noalloc_matches_lch_derivative_on_consecutive_calls(ctx):
    import torch

    # two GF(2^16) calls in a row (the second fills the whole 16 MiB scratch,
    # so stale contents of the first would show), then a GF(2^8) call
    for i, (r, h, S) in enumerate([(16, 4096, 1024), (16, 8192, 2048), (8, 256, 1040)]):
        host = WL.shards(h, S, seed=7000 + i)
        ref = to_dev(host)
        ctx.derivative(r, ref)
        got = to_dev(host)
        lch.derivative_noalloc(r, got)
        torch.cuda.synchronize()
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy()), (r, h, S)


@pytest.mark.gpu
@pytest.mark.parametrize("r,lgh,S", [(16, 12, 4096), (16, 13, 2048), (16, 13, 2032), (8, 8, 1040)])
def test_noalloc_matches_oracle(ctx, r, lgh, S):
    """The allocation-free derivative against the oracle's derivative
    (Sec. IV.B, computed through the monomial basis) on sampled element
    columns, at the sizes the 16 MiB scratch admits."""
    import torch

    h = 1 << lgh
    host = WL.shards(h, S, seed=7100 + lgh + S)
    got = to_dev(host)
    lch.derivative_noalloc(r, got)
    torch.cuda.synchronize()
    cols = elem_cols(S, r, 6, seed=lgh + S)
    assert np.array_equal(elems(got.cpu().numpy(), r, cols), O.derivative(r, elems(host, r, cols)))
