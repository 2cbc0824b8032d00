"""The serving loop: host logic on the CPU (allocator, arrivals) and, on the
GPU, that every request's result is the same alone and in the mix, and equal
to the oracle's encoding (Algorithm 1: the codeword is F(w_0..w_{n-1}) with
F(w_i) = m_i for i < k) or the oracle's recovered rows (Algorithm 2) on sampled
element columns."""
import numpy as np
import pytest

from helpers import elem_cols, elems
from oracle import oracle as O
from paper_1404_3458_gb300 import lch
from paper_1404_3458_gb300 import serve as SV
from paper_1404_3458_gb300 import workloads as WL


def test_arena_first_fit_and_merge():
    a = SV.Arena(4096)
    x = a.alloc(100)   # 256
    y = a.alloc(1000)  # 1024
    z = a.alloc(2816)  # the rest
    assert (x, y, z) == (0, 256, 1280) and a.alloc(1) == -1
    a.release(y, 1000)
    assert a.alloc(2000) == -1 and a.alloc(512) == 256
    a.release(x, 100)
    a.release(256, 512)
    a.release(z, 2816)
    assert a.free == [(0, 4096)] and a.used == 0


def test_poisson_arrivals():
    t = SV.poisson_arrivals(1000.0, 20000, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 20000 - 1e-3) < 5e-5  # mean gap 1/rate


def _requests(ctx, count, rate, seed):
    """Seeded requests; expect[i] is the single-call CUDA result and
    oracle[i] = (cols, rows): the oracle's n rows of sampled element columns."""
    import torch

    g = np.random.default_rng(seed)
    arr = SV.poisson_arrivals(rate, count, seed)
    reqs, expect, oracle = [], [], []
    for i in range(count):
        n = int(g.choice([32, 64, 256, 1024]))
        field = 8 if n <= 256 else 16
        k = n * int(g.choice([2, 1, 3])) // 4
        S = int(g.choice([64, 256, 1024]))
        host = np.zeros((n, S), dtype=np.uint8)
        host[:k] = WL.shards(k, S, seed=seed * 1000 + i)
        dev = torch.from_numpy(host).cuda()
        cols = elem_cols(S, field, 3, seed=seed + i)
        if g.random() < 0.7:
            op, mask = lch.BATCH_ENCODE, None
            alone = dev.clone()
            ctx.rs_encode(n, k, field, alone)
            # every row of the sampled columns: message rows kept, parity rows
            # the interpolant's values
            oracle.append((cols, O.rs_encode(field, n, k, elems(host, field, cols))))
        else:
            op = lch.BATCH_DECODE
            ctx.rs_encode(n, k, field, dev)
            mask = WL.erasure_mask(n, int(g.integers(0, n - k + 1)), seed=i)
            alone = dev.clone()
            dev[torch.from_numpy(mask.astype(bool)).cuda()] = 0xEE
            # the oracle decodes its own encoding, damaged the same way
            damaged = O.rs_encode(field, n, k, elems(host, field, cols))
            damaged[mask == 1] = 0xEEEE if field == 16 else 0xEE
            oracle.append((cols, O.rs_decode(field, n, k, damaged, mask)))
            tmp = dev.clone()
            ctx.rs_decode(n, k, field, tmp, mask)
            assert torch.equal(tmp, alone)
        reqs.append(SV.Request(i, op, field, n, k, S, float(arr[i]), mask=mask, payload=dev))
        expect.append(alone)
    torch.cuda.synchronize()
    return reqs, expect, oracle


def _check_oracle(reqs, got, oracle):
    for r, (cols, want) in zip(reqs, oracle):
        served = elems(got[r.rid].cpu().numpy(), r.field, cols)
        assert np.array_equal(served, want), ("oracle", r.rid, r.op, r.n, r.k, r.shard_bytes)


@pytest.mark.gpu
@pytest.mark.parametrize("budget_mb,rate,min_batch,max_direct,max_batch_bytes",
                         [(64, 20000.0, 16, 4, 0), (8, 200000.0, 16, 4, 0), (64, 200000.0, 2, 0, 0),
                          (16, 50000.0, 4, 1, 0), (64, 200000.0, 2, 0, 1 << 19)])
def test_served_results_equal_alone(ctx, budget_mb, rate, min_batch, max_direct, max_batch_bytes):
    import torch

    reqs, expect, oracle = _requests(ctx, 60, rate, seed=budget_mb + min_batch + max_batch_bytes)
    got = {}
    server = SV.Server(ctx, budget_mb << 20, max_inflight=2, max_batch=32, min_batch=min_batch,
                       max_direct=max_direct, max_batch_bytes=max_batch_bytes)
    stats = server.run(reqs, on_done=lambda r: got.__setitem__(r.rid, r.buf.clone()))
    torch.cuda.synchronize()
    assert len(got) == len(reqs)
    for r, e in zip(reqs, expect):
        assert torch.equal(got[r.rid], e), (r.rid, r.op, r.n, r.k, r.shard_bytes)
    _check_oracle(reqs, got, oracle)
    assert stats["requests"] == 60 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["batches"] + stats["direct_calls"] == stats["launch_groups"]
    if max_direct == 0:
        # everything went out in batches, several requests per launch
        assert stats["direct_calls"] == 0 and stats["batches"] < len(reqs)


@pytest.mark.gpu
def test_plain_loop_results_equal_alone(ctx):
    import torch

    reqs, expect, oracle = _requests(ctx, 24, 5000.0, seed=7)
    got = {}
    SV.serve_plain(ctx, reqs, 32 << 20, on_done=lambda r: got.__setitem__(r.rid, r.buf.clone()))
    torch.cuda.synchronize()
    for r, e in zip(reqs, expect):
        assert torch.equal(got[r.rid], e)
    _check_oracle(reqs, got, oracle)
