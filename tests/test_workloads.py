"""The seeded input generators (paper_1404_3458_gb300/workloads.py) produce
the documented shapes and distributions, reproducibly: the measured
single-codeword workloads, erasure sets of exactly the stated size, bursts,
and the batched mix."""
import numpy as np

from paper_1404_3458_gb300 import workloads as WL


def test_single_codeword_workloads():
    w = WL.WORKLOADS
    assert (w["small_gf8"].field, w["small_gf8"].n, w["small_gf8"].k, w["small_gf8"].shard_bytes) == (8, 32, 16, 1024)
    assert (w["medium_gf16"].field, w["medium_gf16"].n, w["medium_gf16"].k,
            w["medium_gf16"].shard_bytes) == (16, 256, 128, 65536)
    assert (w["large_gf16"].field, w["large_gf16"].n, w["large_gf16"].k,
            w["large_gf16"].shard_bytes) == (16, 65536, 32768, 4096)
    for v in w.values():
        assert v.erasures == v.n - v.k


def test_shards_and_masks_are_seeded_and_exact():
    a, b = WL.shards(16, 64, seed=3), WL.shards(16, 64, seed=3)
    assert a.shape == (16, 64) and a.dtype == np.uint8 and np.array_equal(a, b)
    assert not np.array_equal(a, WL.shards(16, 64, seed=4))
    for n, e in ((32, 0), (32, 16), (65536, 32768), (8, 8)):
        m = WL.erasure_mask(n, e, seed=n + e)
        assert m.dtype == np.uint8 and m.size == n and int(m.sum()) == e
        assert np.array_equal(m, WL.erasure_mask(n, e, seed=n + e))
    m = WL.burst_mask(64, 16, 10)
    assert int(m.sum()) == 16 and m[10:26].all() and not m[:10].any() and not m[26:].any()
    s = WL.random_burst_start(65536, 32768, seed=1)
    assert 0 <= s <= 32768


def test_batched_mix_distributions():
    specs = WL.batch_workload(4096)
    assert specs == WL.batch_workload(4096)
    ns = {n for (_, n, _, _, _) in specs}
    assert ns == {1 << u for u in range(6, 14)}
    assert {S for (_, _, _, S, _) in specs} == {512, 2048, 8192, 16384}
    for field, n, k, S, e in specs:
        assert field == (8 if n <= 256 else 16)
        assert 4 * k in (2 * n, n, 3 * n)
        assert 0 <= e <= n - k
    ratios = {4 * k // n for (_, n, k, _, _) in specs}
    assert ratios == {1, 2, 3}
