"""GPU parity of the bit-sliced GF(2^16) transform passes: against the oracle
(direct evaluation, Gaussian elimination, Lagrange encoding) and, byte for
byte, against the split-table passes on the same inputs.  Shard sizes cover
one and several 2 KB column tiles, ragged last tiles (S = 64 * odd) and tiles
narrower than a warp's 32 chunks; h covers one to three passes."""
import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

R = 16


def _both(ctx, fn):
    """fn(ctx) with the bit-sliced passes, then with the split-table ones (the
    default, restored afterwards)."""
    ctx.set_bitslice(True)
    try:
        a = fn(ctx)
    finally:
        ctx.set_bitslice(False)
    return a, fn(ctx)


@pytest.mark.parametrize("lgh,l,S", [(1, 0, 64), (2, 6, 128), (3, 0, 2048), (5, 32, 2112), (6, 0, 192),
                                     (7, 128, 4096), (9, 0, 2176), (11, 2048, 640), (12, 0, 4096),
                                     (13, 8192, 2048), (15, 0, 1088), (16, 0, 64)])
def test_fft_ifft_sliced(ctx, lgh, l, S):
    import torch

    h = 1 << lgh
    host = WL.shards(h, S, seed=9000 + lgh + S)

    def run(c):
        dev = to_dev(host)
        c.fft(R, l, dev)
        out = dev.clone()
        c.ifft(R, l, dev)
        torch.cuda.synchronize()
        return out.cpu().numpy(), dev.cpu().numpy()

    (f_bs, back_bs), (f_tab, _) = _both(ctx, run)
    assert np.array_equal(f_bs, f_tab)          # same bytes as the split-table passes
    assert np.array_equal(back_bs, host)        # Psi^-1 (Psi x) = x on every byte
    cols = elem_cols(S, R, 5, seed=lgh)
    rows = None if h <= 512 else np.random.default_rng(lgh).choice(h, 40, replace=False)
    expect = O.fft(R, l, elems(host, R, cols), rows=rows)
    assert np.array_equal(elems(f_bs, R, cols) if rows is None else elems(f_bs, R, cols)[rows], expect)
    if h <= 256:
        dev = to_dev(host)
        ctx.set_bitslice(True)
        try:
            ctx.ifft(R, l, dev)
        finally:
            ctx.set_bitslice(False)
        assert np.array_equal(elems(dev.cpu().numpy(), R, cols), O.ifft(R, l, elems(host, R, cols)))


@pytest.mark.parametrize("n,k,S", [(512, 256, 2048), (1024, 512, 2112), (4096, 1024, 640), (2048, 1536, 4096),
                                   (8192, 4096, 128), (65536, 32768, 64)])
def test_encode_decode_sliced(ctx, n, k, S):
    import torch

    host = np.zeros((n, S), dtype=np.uint8)
    host[:k] = WL.shards(k, S, seed=9100 + n + k + S)
    mask = WL.erasure_mask(n, n - k, seed=9200 + n)

    def run(c):
        dev = to_dev(host)
        c.rs_encode(n, k, R, dev)
        enc = dev.cpu().numpy()
        dev[torch.from_numpy(mask.astype(bool)).cuda()] = 0x3C
        c.rs_decode(n, k, R, dev, mask)
        torch.cuda.synchronize()
        return enc, dev.cpu().numpy()

    (enc_bs, dec_bs), (enc_tab, _) = _both(ctx, run)
    assert np.array_equal(enc_bs, enc_tab)
    assert np.array_equal(dec_bs, enc_bs)
    if k > 4096:
        return  # the oracle's O(k^2) weights; this size is covered by the byte comparison above
    cols = elem_cols(S, R, 3, seed=n)
    rows = np.sort(np.random.default_rng(n).choice(np.arange(k, n), min(48, n - k), replace=False))
    want = O.rs_encode(R, n, k, elems(host, R, cols), rows=rows)
    assert np.array_equal(elems(enc_bs, R, cols)[rows], want[rows])
