"""GPU parity: lch_fft / lch_ifft / lch_derivative against the CPU oracle,
bit-exact, at sizes spanning several tiles with ragged column tails."""
import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FFT_CASES = [
    # (r, lg h, shift l, shard bytes)
    (8, 0, 0, 16), (8, 1, 0, 16), (8, 3, 0, 48), (8, 4, 16, 1024), (8, 5, 96, 208),
    (8, 8, 0, 4112), (8, 6, 3, 64), (8, 7, 128, 144),
    (16, 1, 2, 16), (16, 4, 0, 2064), (16, 7, 65408, 1040), (16, 8, 256, 4096),
    (16, 9, 0, 336), (16, 10, 1024, 128), (16, 12, 4096, 80), (16, 5, 7, 48),
]


@pytest.mark.parametrize("r,lgh,l,S", FFT_CASES)
def test_fft_matches_direct_evaluation(ctx, r, lgh, l, S):
    h = 1 << lgh
    host = WL.shards(h, S, seed=1000 + lgh * 7 + l % 97 + S)
    dev = to_dev(host)
    ctx.fft(r, l, dev)
    got = elems(dev.cpu().numpy(), r)
    cols = elem_cols(S, r, 24, seed=lgh)
    rows = None if h <= 1024 else np.random.default_rng(h).choice(h, 96, replace=False)
    expect = O.fft(r, l, elems(host, r, cols), rows=rows)
    assert np.array_equal(got[:, cols] if rows is None else got[rows][:, cols], expect)


@pytest.mark.parametrize("r,lgh,l,S", [c for c in FFT_CASES if c[1] <= 9])
def test_ifft_matches_elimination(ctx, r, lgh, l, S):
    h = 1 << lgh
    host = WL.shards(h, S, seed=2000 + lgh + S)
    dev = to_dev(host)
    ctx.ifft(r, l, dev)
    got = elems(dev.cpu().numpy(), r)
    cols = elem_cols(S, r, 12, seed=lgh + 1)
    assert np.array_equal(got[:, cols], O.ifft(r, l, elems(host, r, cols)))


@pytest.mark.parametrize("r,lgh,l,S", [(16, 13, 0, 64), (16, 16, 0, 32), (16, 15, 32768, 48), (8, 8, 0, 16)])
def test_large_transforms_sampled(ctx, r, lgh, l, S):
    """Large h: the oracle evaluates the GPU's IFFT output at sampled points
    (they must reproduce the input), and checks sampled FFT rows directly."""
    import torch

    h = 1 << lgh
    host = WL.shards(h, S, seed=3000 + lgh)
    dev = to_dev(host)
    ctx.ifft(r, l, dev)
    coef = dev.cpu().numpy()
    rows = np.random.default_rng(lgh).choice(h, 24, replace=False)
    cols = elem_cols(S, r, 6, seed=lgh)
    assert np.array_equal(O.fft(r, l, elems(coef, r, cols), rows=rows), elems(host, r, cols)[rows])
    ctx.fft(r, l, dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), host)  # Psi o Psi^-1 = id on every byte


@pytest.mark.parametrize("r,lgh,S", [(8, 0, 16), (8, 1, 32), (8, 3, 48), (8, 8, 1040), (16, 4, 64),
                                     (16, 9, 80), (16, 10, 32)])
def test_derivative_matches_oracle(ctx, r, lgh, S):
    h = 1 << lgh
    host = WL.shards(h, S, seed=4000 + lgh + S)
    dev = to_dev(host)
    ctx.derivative(r, dev)
    got = elems(dev.cpu().numpy(), r)
    cols = elem_cols(S, r, 8, seed=lgh)
    assert np.array_equal(got[:, cols], O.derivative(r, elems(host, r, cols)))


@pytest.mark.parametrize("lgh,S", [(12, 4096), (13, 4112), (13, 8192)])
def test_derivative_full_size_forms(ctx, lgh, S):
    """Sec. IV.B at sizes where the derivative runs as two persistent passes
    over the two bit groups (several column tiles per row group, ragged last
    tile at S = 4112), against the oracle's monomial-basis derivative on
    sampled element columns."""
    r, h = 16, 1 << lgh
    host = WL.shards(h, S, seed=4500 + lgh + S)
    dev = to_dev(host)
    ctx.derivative(r, dev)
    cols = elem_cols(S, r, 6, seed=lgh + S)
    got = elems(dev.cpu().numpy(), r, cols)
    assert np.array_equal(got, O.derivative(r, elems(host, r, cols)))


@pytest.mark.parametrize("lgh", list(range(8, 17)))
def test_roundtrip_config2_sizes(ctx, lgh):
    """lch_fft / lch_ifft round trips at h = 2^8 .. 2^16 in GF(2^16) with
    64 KiB shards (4 KiB for h >= 2^15, which would otherwise need 2-4 GB):
    every byte returns, and sampled transform values match direct evaluation."""
    import torch

    r, h = 16, 1 << lgh
    S = 65536 if lgh <= 14 else 4096
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4000 + lgh)
    dev = torch.randint(0, 256, (h, S), dtype=torch.uint8, device="cuda", generator=gen)
    orig = dev.clone()
    cols = elem_cols(S, r, 4, seed=lgh)
    byte_cols = np.concatenate([[2 * c, 2 * c + 1] for c in cols])
    coef = orig[:, torch.from_numpy(byte_cols).cuda()].cpu().numpy()
    ctx.fft(r, 0, dev)
    rows = np.random.default_rng(lgh).choice(h, 16, replace=False)
    got = dev[torch.from_numpy(rows).cuda()][:, torch.from_numpy(byte_cols).cuda()].cpu().numpy()
    assert np.array_equal(O.to_elems(got, r), O.fft(r, 0, O.to_elems(coef, r), rows=rows))
    ctx.ifft(r, 0, dev)
    torch.cuda.synchronize()
    assert torch.equal(dev, orig)
