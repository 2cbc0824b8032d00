"""GPU parity: lch_poly_mul (Sec. VI.A) against the oracle's product through
the monomial basis, and at large h against products of sampled values."""
import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r,h,S", [(8, 1, 16), (8, 4, 16), (8, 64, 48), (8, 128, 1024), (16, 16, 64),
                                   (16, 256, 80), (16, 512, 32)])
def test_poly_mul_matches_oracle(ctx, r, h, S):
    import torch

    a = WL.shards(h, S, seed=h + S)
    b = WL.shards(h, S, seed=h + S + 1)
    c = torch.empty((2 * h, S), dtype=torch.uint8, device="cuda")
    ctx.poly_mul(r, to_dev(a), to_dev(b), c)
    torch.cuda.synchronize()
    cols = elem_cols(S, r, 6, seed=h)
    expect = O.poly_mul(r, elems(a, r, cols), elems(b, r, cols))
    assert np.array_equal(elems(c.cpu().numpy(), r)[:, cols], expect)


def test_poly_mul_large_sampled(ctx):
    import torch

    r, h, S = 16, 32768, 32
    a = WL.shards(h, S, seed=5)
    b = WL.shards(h, S, seed=6)
    c = torch.empty((2 * h, S), dtype=torch.uint8, device="cuda")
    ctx.poly_mul(r, to_dev(a), to_dev(b), c)
    torch.cuda.synchronize()
    cols = elem_cols(S, r, 3, seed=1)
    pad = lambda x: np.vstack([elems(x, r, cols), np.zeros((h, cols.size), dtype=np.uint16)])
    rows = np.random.default_rng(2).choice(2 * h, 12, replace=False)
    va, vb = O.fft(r, 0, pad(a), rows=rows), O.fft(r, 0, pad(b), rows=rows)
    vc = O.fft(r, 0, elems(c.cpu().numpy(), r, cols), rows=rows)
    assert np.array_equal(vc, O.gf_mul_vec(r, va, vb))
