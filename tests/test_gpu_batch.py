"""GPU parity for batches (one persistent launch over many codewords): every
codeword of a mixed batch must come out byte-identical to the single-codeword
entry points and to the oracle, alone or in the mix, including under CUDA-graph
replay."""
import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import lch
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

# (field, n, k, shard bytes): both fields, single- and two-pass transforms,
# k a power of two, k not a power of two (shortened), k = 1 and k = n, ragged S.
SHAPES = [(8, 8, 4, 16), (8, 32, 16, 1024), (8, 256, 64, 48), (8, 128, 96, 80), (8, 64, 1, 32),
          (16, 64, 32, 512), (16, 512, 128, 208), (16, 1024, 768, 64), (16, 2048, 1024, 32),
          (16, 8192, 4096, 16), (16, 256, 256, 64), (16, 4096, 3072, 48), (16, 16, 12, 2064)]


def messages(seed=0):
    out = []
    for i, (r, n, k, S) in enumerate(SHAPES):
        host = np.zeros((n, S), dtype=np.uint8)
        host[:k] = WL.shards(k, S, seed=seed + 31 * i)
        out.append(host)
    return out


def test_batch_encode_matches_single_and_oracle(ctx):
    import torch

    hosts = messages()
    devs = [to_dev(h) for h in hosts]
    b = ctx.batch(lch.BATCH_ENCODE, [(n, k, r, d, None) for (r, n, k, S), d in zip(SHAPES, devs)])
    assert b.tasks > 0
    b.run()
    b.status()
    for (r, n, k, S), h, d in zip(SHAPES, hosts, devs):
        single = to_dev(h)
        ctx.rs_encode(n, k, r, single)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        assert np.array_equal(got, single.cpu().numpy()), (r, n, k, S)
        cols = elem_cols(S, r, 3, seed=n)
        rows = np.arange(k, n)[:: max(1, (n - k) // 16)] if k < n else None
        if rows is not None:
            ref = O.rs_encode(r, n, k, elems(h, r, cols), rows=rows)
            assert np.array_equal(elems(got, r, cols)[rows], ref[rows]), (r, n, k, S)
    b.close()


def test_batch_decode_recovers_every_codeword(ctx):
    import torch

    hosts = messages(seed=100)
    cws = []
    for (r, n, k, S), h in zip(SHAPES, hosts):
        d = to_dev(h)
        ctx.rs_encode(n, k, r, d)
        torch.cuda.synchronize()
        cws.append(d.cpu().numpy())
    g = np.random.default_rng(5)
    masks, devs = [], []
    for i, ((r, n, k, S), cw) in enumerate(zip(SHAPES, cws)):
        e = [0, 1, n - k, int(g.integers(0, n - k + 1))][i % 4]
        m = WL.erasure_mask(n, e, seed=i)
        bad = cw.copy()
        bad[m == 1] = 0xC3
        masks.append(m)
        devs.append(to_dev(bad))
    b = ctx.batch(lch.BATCH_DECODE, [(n, k, r, d, m) for (r, n, k, S), d, m in zip(SHAPES, devs, masks)])
    b.run()
    b.status()
    for (r, n, k, S), cw, d in zip(SHAPES, cws, devs):
        assert np.array_equal(d.cpu().numpy(), cw), (r, n, k, S)
    b.close()


def test_batch_graph_replay(ctx):
    """The run is recorded once in a CUDA graph and replayed on fresh damage."""
    import torch

    shapes = [(16, 1024, 512, 256), (8, 64, 32, 1024), (16, 8192, 4096, 32)]
    cws, devs, masks = [], [], []
    for i, (r, n, k, S) in enumerate(shapes):
        host = np.zeros((n, S), dtype=np.uint8)
        host[:k] = WL.shards(k, S, seed=900 + i)
        d = to_dev(host)
        ctx.rs_encode(n, k, r, d)
        torch.cuda.synchronize()
        cws.append(d.cpu().numpy())
        devs.append(d)
        masks.append(WL.erasure_mask(n, n - k, seed=77 + i))
    b = ctx.batch(lch.BATCH_DECODE, [(n, k, r, d, m) for (r, n, k, S), d, m in zip(shapes, devs, masks)])
    stream = torch.cuda.Stream()
    b.run(stream)  # warm run outside capture
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.run(stream)
    for fill in (0x00, 0x7E):
        for d, m in zip(devs, masks):
            d[torch.from_numpy(m.astype(bool)).cuda()] = fill
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        b.status()
        for cw, d in zip(cws, devs):
            assert np.array_equal(d.cpu().numpy(), cw)
    b.close()


def test_batch_refusals(ctx):
    n, k, S = 64, 32, 64
    d = to_dev(np.zeros((n, S), dtype=np.uint8))
    m = np.zeros(n, dtype=np.uint8)
    m[: n - k + 1] = 1
    with pytest.raises(lch.LchError) as ei:
        ctx.batch(lch.BATCH_DECODE, [(n, k, 16, d, m)])
    assert ei.value.status == lch.LCH_ETOOMANY
    big = to_dev(np.zeros((16384, 16), dtype=np.uint8))
    with pytest.raises(lch.LchError) as ei:
        ctx.batch(lch.BATCH_ENCODE, [(16384, 8192, 16, big, None)])
    assert ei.value.status == lch.LCH_EINVAL and "n <= 8192" in str(ei.value)
    empty = ctx.batch(lch.BATCH_ENCODE, [])
    empty.run()
    empty.status()
    assert empty.tasks == 0


def test_batch_wait_gives_up_and_context_recovers():
    """Failure path of the persistent kernel: a task whose dependency is
    never met waits at most the context's limit, the run reports
    LCH_ETIMEDOUT, and the same context then runs a batch correctly."""
    import time

    import torch

    c = lch.Context(0)
    try:
        c.batch_set_wait_limit(20000)  # 20 ms
        t0 = time.perf_counter()
        assert c.batch_selftest_stall() == lch.LCH_ETIMEDOUT
        assert time.perf_counter() - t0 < 5.0
        with pytest.raises(lch.LchError):
            c.batch_set_wait_limit(0)
        r, n, k, S = 16, 256, 128, 64
        host = np.zeros((n, S), dtype=np.uint8)
        host[:k] = WL.shards(k, S, seed=123)
        d = to_dev(host)
        b = c.batch(lch.BATCH_ENCODE, [(n, k, r, d, None)])
        b.run()
        b.status()
        cols = elem_cols(S, r, 4, seed=2)
        assert np.array_equal(elems(d.cpu().numpy(), r)[:, cols], O.rs_encode(r, n, k, elems(host, r, cols)))
        torch.cuda.synchronize()
    finally:
        c.close()


def test_batch_of_the_measured_mix():
    """The batched workload's own distributions (n = 2^6..2^13, k/n in
    {1/2, 1/4, 3/4}, both fields, 512 B..16 KiB shards, uniform erasure
    counts): a 24-codeword sample of the mix, encoded and then decoded in two
    batches on autotuned plans; sampled parity rows against the oracle, and
    every decoded codeword byte-identical to its encoding."""
    import torch

    from paper_1404_3458_gb300 import tuning

    c = lch.Context(0)
    try:
        specs = WL.batch_workload(24, seed=WL.SEED_BASE + 44)
        shapes = set()
        for (r, n, k, S, e) in specs:
            shapes.add((r, n, S))
            if k & (k - 1) == 0 and k >= 2:
                shapes.add((r, k, S))
        tuning.tune(c, sorted(shapes))
        hosts, devs = [], []
        for i, (r, n, k, S, e) in enumerate(specs):
            host = np.zeros((n, S), dtype=np.uint8)
            host[:k] = WL.shards(k, S, seed=600 + i)
            hosts.append(host)
            devs.append(to_dev(host))
        b = c.batch(lch.BATCH_ENCODE, [(n, k, r, d, None) for (r, n, k, S, e), d in zip(specs, devs)])
        b.run()
        b.status()
        cws = [d.clone() for d in devs]
        for i, ((r, n, k, S, e), host, d) in enumerate(zip(specs, hosts, devs)):
            cols = elem_cols(S, r, 2, seed=i)
            rows = k + np.random.default_rng(i).choice(n - k, min(n - k, 6), replace=False)
            expect = O.rs_encode(r, n, k, elems(host, r, cols), rows=rows)
            got = elems(d.cpu().numpy(), r)
            assert np.array_equal(got[rows][:, cols], expect[rows]), (i, r, n, k, S)
        masks = [WL.erasure_mask(n, e, 700 + i) for i, (r, n, k, S, e) in enumerate(specs)]
        for d, m in zip(devs, masks):
            d[torch.from_numpy(m != 0).cuda()] = 0x3C
        b = c.batch(lch.BATCH_DECODE, [(n, k, r, d, m) for (r, n, k, S, e), d, m in zip(specs, devs, masks)])
        b.run()
        b.status()
        for d, cw in zip(devs, cws):
            assert torch.equal(d, cw)
    finally:
        c.close()
