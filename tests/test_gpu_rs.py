"""GPU parity: rs_encode / rs_decode against the CPU oracle, bit-exact, on
the measured workloads (small_gf8, medium_gf16, large_gf16) and edge cases."""
import itertools

import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import lch
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def message(n, k, S, seed):
    host = np.zeros((n, S), dtype=np.uint8)
    host[:k] = WL.shards(k, S, seed)
    return host


def gpu_encode(ctx, r, n, k, host):
    dev = to_dev(host)
    ctx.rs_encode(n, k, r, dev)
    return dev.cpu().numpy()


def gpu_decode(ctx, r, n, k, cw, mask, fill=0x5A):
    bad = cw.copy()
    bad[mask != 0] = fill
    dev = to_dev(bad)
    ctx.rs_decode(n, k, r, dev, mask)
    return dev.cpu().numpy()


@pytest.mark.parametrize("r,n,k,S", [(8, 32, 16, 1024), (8, 8, 4, 16), (8, 256, 128, 48), (8, 64, 16, 4112),
                                     (16, 64, 32, 2064), (16, 256, 64, 208), (8, 16, 1, 32), (16, 16, 16, 16),
                                     (8, 64, 48, 80), (16, 128, 96, 64), (8, 32, 3, 16), (16, 512, 500, 32)])
def test_encode_matches_oracle(ctx, r, n, k, S):
    host = message(n, k, S, seed=n + k + S)
    got = gpu_encode(ctx, r, n, k, host)
    cols = elem_cols(S, r, 32, seed=n)
    expect = O.rs_encode(r, n, k, elems(host, r, cols))
    assert np.array_equal(elems(got, r)[:, cols], expect)
    assert np.array_equal(got[:k], host[:k])


def test_small_gf8_workload_full(ctx):
    w = WL.WORKLOADS["small_gf8"]
    host = message(w.n, w.k, w.shard_bytes, w.seed)
    cw = gpu_encode(ctx, w.field, w.n, w.k, host)
    expect = O.from_elems(O.rs_encode(w.field, w.n, w.k, elems(host, w.field)), w.field)
    assert np.array_equal(cw, expect)
    mask = WL.erasure_mask(w.n, w.erasures, w.seed)
    assert np.array_equal(gpu_decode(ctx, w.field, w.n, w.k, cw, mask), cw)
    # the oracle recovers the same rows from the same survivors
    bad = cw.copy()
    bad[mask == 1] = 0
    ref = O.from_elems(O.rs_decode(w.field, w.n, w.k, elems(bad, w.field), mask), w.field)
    assert np.array_equal(ref, cw)


def test_exhaustive_8_4_all_patterns(ctx):
    """Every pattern of at most 4 erasures on (8,4) over GF(2^8): 163 decodes."""
    r, n, k, S = 8, 8, 4, 32
    cw = gpu_encode(ctx, r, n, k, message(n, k, S, seed=84))
    count = 0
    for e in range(n - k + 1):
        for erased in itertools.combinations(range(n), e):
            mask = np.zeros(n, dtype=np.uint8)
            mask[list(erased)] = 1
            assert np.array_equal(gpu_decode(ctx, r, n, k, cw, mask), cw), erased
            count += 1
    assert count == 163


@pytest.mark.parametrize("r,n,k,S", [(16, 2, 1, 32), (8, 4, 2, 16), (16, 4, 1, 48), (16, 8, 6, 4112)])
def test_tiny_codes_all_patterns(ctx, r, n, k, S):
    """Codes of 2 to 8 rows: every erasure pattern the code can repair, against
    the oracle's encode (the whole decode runs as one fused launch here)."""
    host = message(n, k, S, seed=n + k + S)
    cw = gpu_encode(ctx, r, n, k, host)
    cols = elem_cols(S, r, 8, seed=n)
    assert np.array_equal(elems(cw, r)[:, cols], O.rs_encode(r, n, k, elems(host, r, cols)))
    for e in range(n - k + 1):
        for erased in itertools.combinations(range(n), e):
            mask = np.zeros(n, dtype=np.uint8)
            mask[list(erased)] = 1
            assert np.array_equal(gpu_decode(ctx, r, n, k, cw, mask), cw), erased


@pytest.mark.parametrize("r,n,k,S,e", [(8, 32, 16, 1024, 16), (8, 32, 16, 1024, 5), (8, 256, 128, 48, 128),
                                       (16, 64, 32, 2064, 32), (16, 1024, 512, 32, 512), (16, 8192, 4096, 16, 4000),
                                       (8, 64, 48, 80, 16), (16, 128, 96, 64, 1), (16, 4096, 2048, 48, 2048)])
def test_decode_matches_oracle(ctx, r, n, k, S, e):
    host = message(n, k, S, seed=5 * n + e)
    cw = gpu_encode(ctx, r, n, k, host)
    mask = WL.erasure_mask(n, e, seed=n * 3 + e)
    got = gpu_decode(ctx, r, n, k, cw, mask)
    assert np.array_equal(got, cw)
    cols = elem_cols(S, r, 4, seed=e)
    bad = elems(cw, r, cols)
    bad[mask == 1] = 0
    rows = np.nonzero(mask)[0][:64]
    ref = O.rs_decode(r, n, k, bad, mask, rows=rows)
    assert np.array_equal(elems(got, r, cols)[rows], ref[rows])


def test_decode_edge_cases(ctx):
    r, n, k, S = 16, 64, 32, 64
    cw = gpu_encode(ctx, r, n, k, message(n, k, S, seed=9))
    # zero erasures: a no-op, even on corrupted data
    dev = to_dev(cw)
    ctx.rs_decode(n, k, r, dev, np.zeros(n, np.uint8))
    assert np.array_equal(dev.cpu().numpy(), cw)
    # more than n - k erasures: refused, buffer untouched
    mask = np.zeros(n, np.uint8)
    mask[: n - k + 1] = 1
    dev = to_dev(cw)
    with pytest.raises(lch.LchError) as ei:
        ctx.rs_decode(n, k, r, dev, mask)
    assert ei.value.status == lch.LCH_ETOOMANY
    assert np.array_equal(dev.cpu().numpy(), cw)
    # all message rows erased, and all parity rows erased
    for mask in (WL.burst_mask(n, n - k, 0), WL.burst_mask(n, n - k, k)):
        assert np.array_equal(gpu_decode(ctx, r, n, k, cw, mask), cw)


def test_medium_gf16_workload(ctx):
    w = WL.WORKLOADS["medium_gf16"]
    host = message(w.n, w.k, w.shard_bytes, w.seed)
    cw = gpu_encode(ctx, w.field, w.n, w.k, host)
    cols = elem_cols(w.shard_bytes, w.field, 48, seed=2)
    assert np.array_equal(elems(cw, w.field, cols), O.rs_encode(w.field, w.n, w.k, elems(host, w.field, cols)))
    mask = WL.erasure_mask(w.n, w.erasures, w.seed)
    assert np.array_equal(gpu_decode(ctx, w.field, w.n, w.k, cw, mask), cw)


@pytest.mark.parametrize("r,n,k,S", [(16, 256, 128, 65424), (16, 256, 128, 65488), (8, 256, 64, 40000),
                                     (16, 128, 64, 175728)])
def test_fused_decode_slicing_tail(ctx, r, n, k, S):
    """The fused short-codeword decode is persistent over column slices; the
    columns left after whole rounds of the grid go as half-width slices, the
    last of them partial or (when S ends early in its slice) empty.  Every
    erased row against the codeword, sampled columns against the oracle."""
    host = message(n, k, S, seed=S + n)
    cw = gpu_encode(ctx, r, n, k, host)
    mask = WL.erasure_mask(n, n - k, seed=S)
    got = gpu_decode(ctx, r, n, k, cw, mask)
    assert np.array_equal(got, cw)
    cols = elem_cols(S, r, 6, seed=1)
    bad = elems(cw, r, cols)
    bad[mask == 1] = 0
    rows = np.nonzero(mask)[0][:64]
    ref = O.rs_decode(r, n, k, bad, mask, rows=rows)
    assert np.array_equal(elems(got, r, cols)[rows], ref[rows])


@pytest.mark.parametrize("r,n,k,S", [(16, 16, 8, 528), (16, 32, 16, 1040), (16, 32, 8, 4112), (16, 128, 64, 2064),
                                     (8, 32, 16, 1040), (8, 128, 32, 4112)])
@pytest.mark.parametrize("kind", ["one", "most", "burst_head", "burst_tail"])
def test_fused_decode_patterns(ctx, r, n, k, S, kind):
    """The fused decode in both of its forms (GF(2^16): element-lane
    transforms with the Pi and 1/Pi' steps inside their first and last
    rounds, one round per transform up to 16 rows, two above; GF(2^8): a pass
    per step), for one erasure, n - k random ones, and bursts at either end
    of the codeword; every erased row against the oracle's encoding and
    sampled columns against the oracle's decode."""
    host = message(n, k, S, seed=31 * n + k)
    cw = gpu_encode(ctx, r, n, k, host)
    if kind == "one":
        mask = WL.erasure_mask(n, 1, seed=n)
    elif kind == "most":
        mask = WL.erasure_mask(n, n - k, seed=n + 1)
    elif kind == "burst_head":
        mask = WL.burst_mask(n, n - k, 0)
    else:
        mask = WL.burst_mask(n, n - k, k)
    got = gpu_decode(ctx, r, n, k, cw, mask)
    assert np.array_equal(got, cw)
    cols = elem_cols(S, r, 4, seed=k)
    bad = elems(cw, r, cols)
    bad[mask == 1] = 0
    rows = np.nonzero(mask)[0][:32]
    ref = O.rs_decode(r, n, k, bad, mask, rows=rows)
    assert np.array_equal(elems(got, r, cols)[rows], ref[rows])


def test_fused_decode_cached_locator_wide_shards():
    """A shortened code (k not a power of two) encodes by a decode with the
    cached locator, whose records each CTA of the fused decode builds for
    every slice it walks; wide shards take the half-width tail as well."""
    ctx2 = lch.Context(0)
    try:
        r, n, k, S = 16, 256, 200, 65424
        host = message(n, k, S, seed=4242)
        got = gpu_encode(ctx2, r, n, k, host)
        cols = elem_cols(S, r, 6, seed=3)
        assert np.array_equal(elems(got, r)[:, cols], O.rs_encode(r, n, k, elems(host, r, cols)))
    finally:
        ctx2.close()


def test_large_gf16_workload(ctx):
    """n = 65536, k = 32768, 4 KiB shards: all 32768 parity rows of 4 element
    columns (the first, the last and two seeded ones) against the oracle's
    Lagrange evaluation, then random and burst erasures of n - k rows recovered
    on every byte."""
    w = WL.WORKLOADS["large_gf16"]
    host = message(w.n, w.k, w.shard_bytes, w.seed)
    cw = gpu_encode(ctx, w.field, w.n, w.k, host)
    assert np.array_equal(cw[: w.k], host[: w.k])
    cols = elem_cols(w.shard_bytes, w.field, 4, seed=3)
    ref = O.rs_encode(w.field, w.n, w.k, elems(host, w.field, cols))
    assert np.array_equal(elems(cw, w.field, cols), ref)
    for mask in (WL.erasure_mask(w.n, w.erasures, w.seed),
                 WL.burst_mask(w.n, w.erasures, 0),
                 WL.burst_mask(w.n, w.erasures, WL.random_burst_start(w.n, w.erasures, w.seed))):
        assert np.array_equal(gpu_decode(ctx, w.field, w.n, w.k, cw, mask), cw)


def test_large_gf16_encode_matches_the_cpu_restatement(ctx):
    """n = 65536, k = 32768, 4 KiB shards: all 32768 parity rows of 64 element
    columns against the CPU restatement of the paper's fast algorithms
    (oracle/fastcpu.c, itself pinned to the oracle, at this size too)."""
    from oracle import fastcpu as FC

    w = WL.WORKLOADS["large_gf16"]
    host = message(w.n, w.k, w.shard_bytes, w.seed + 1)
    cw = gpu_encode(ctx, w.field, w.n, w.k, host)
    cols = elem_cols(w.shard_bytes, w.field, 64, seed=11)
    assert np.array_equal(elems(cw, w.field, cols), FC.rs_encode(w.field, w.n, w.k, elems(host, w.field, cols)))


def test_shortened_encode_reuses_cached_locator():
    """k not a power of two: the locator of E = {k..n-1} is computed once per
    (field, n, k) and reused by later calls and by batches; every use gives the
    oracle's parity."""
    ctx2 = lch.Context(0)
    try:
        for r, n, k, S in [(16, 1024, 768, 96), (8, 128, 96, 48)]:
            for rep in range(2):
                host = message(n, k, S, seed=7000 + rep + n)
                got = gpu_encode(ctx2, r, n, k, host)
                cols = elem_cols(S, r, 8, seed=rep)
                assert np.array_equal(elems(got, r)[:, cols], O.rs_encode(r, n, k, elems(host, r, cols)))
            hosts = [message(n, k, S, seed=7100 + i) for i in range(2)]
            devs = [to_dev(h) for h in hosts]
            b = ctx2.batch(lch.BATCH_ENCODE, [(n, k, r, d, None) for d in devs])
            b.run()
            b.status()
            for h, d in zip(hosts, devs):
                assert np.array_equal(d.cpu().numpy(), gpu_encode(ctx2, r, n, k, h))
    finally:
        ctx2.close()


@pytest.mark.parametrize("r,n,k,S", [(16, 65536, 1, 16), (16, 4096, 2, 48), (8, 256, 4, 32), (16, 65536, 16, 16),
                                     (16, 65536, 1024, 32), (8, 256, 128, 16), (16, 8192, 512, 80)])
def test_encode_many_cosets(ctx, r, n, k, S):
    """Algorithm 1 with many parity cosets (all cosets run as one pass set;
    k = 1 is a broadcast): sampled parity rows against the oracle, message
    rows untouched."""
    host = message(n, k, S, seed=9000 + n + k)
    got = gpu_encode(ctx, r, n, k, host)
    assert np.array_equal(got[:k], host[:k])
    cols = elem_cols(S, r, 4, seed=k)
    g = np.random.default_rng(n + k)
    rows = np.unique(np.concatenate([[k, n - 1], k + g.choice(n - k, min(n - k, 40), replace=False)]))
    expect = O.rs_encode(r, n, k, elems(host, r, cols), rows=rows)
    assert np.array_equal(elems(got, r)[rows][:, cols], expect[rows])


@pytest.mark.parametrize("r,n,k,S,kind", [(8, 32, 16, 1024, "random"), (8, 8, 4, 16, "random"),
                                          (16, 256, 64, 208, "random"), (16, 1024, 512, 48, "burst"),
                                          (16, 4096, 3072, 64, "random"), (16, 65536, 32768, 32, "random"),
                                          (16, 65536, 32768, 16, "burst"), (8, 64, 48, 80, "random")])
def test_decode_packed_matches_in_place(ctx, r, n, k, S, kind):
    """rs_decode_packed, from the surviving shards alone, recovers exactly the
    erased rows that rs_decode restores in place (and the true codeword)."""
    import torch

    cw = gpu_encode(ctx, r, n, k, message(n, k, S, seed=n + S))
    e = n - k
    mask = WL.erasure_mask(n, e, seed=n + 7) if kind == "random" else WL.burst_mask(n, e, (n - e) // 3)
    erased = np.nonzero(mask)[0]
    surv = np.nonzero(mask == 0)[0]
    received = to_dev(np.ascontiguousarray(cw[surv]))
    recovered = torch.full((len(erased), S), 0xC3, dtype=torch.uint8, device="cuda")
    ctx.rs_decode_packed(n, k, r, received, recovered, mask)
    assert np.array_equal(recovered.cpu().numpy(), cw[erased])
    assert np.array_equal(received.cpu().numpy(), cw[surv])  # only read
    assert np.array_equal(gpu_decode(ctx, r, n, k, cw, mask)[erased], cw[erased])


def test_decode_packed_edge_cases(ctx):
    import torch

    r, n, k, S = 16, 64, 32, 64
    cw = gpu_encode(ctx, r, n, k, message(n, k, S, seed=11))
    # no erasures: nothing to do
    empty = torch.empty((0, S), dtype=torch.uint8, device="cuda")
    ctx.rs_decode_packed(n, k, r, to_dev(cw), empty, np.zeros(n, np.uint8))
    # more than n - k erasures: refused, nothing written
    mask = np.zeros(n, np.uint8)
    mask[: n - k + 1] = 1
    out = torch.zeros((n - k + 1, S), dtype=torch.uint8, device="cuda")
    with pytest.raises(lch.LchError) as ei:
        ctx.rs_decode_packed(n, k, r, to_dev(cw[n - k + 1:]), out, mask)
    assert ei.value.status == lch.LCH_ETOOMANY
    assert not out.any()
    # a single erasure, in each position of a short code
    for j in (0, 31, 63):
        mask = np.zeros(n, np.uint8)
        mask[j] = 1
        out = torch.empty((1, S), dtype=torch.uint8, device="cuda")
        ctx.rs_decode_packed(n, k, r, to_dev(np.delete(cw, j, axis=0)), out, mask)
        assert np.array_equal(out.cpu().numpy()[0], cw[j])


def test_rows_gather_scatter_round_trip():
    """lch_rows_scatter / lch_rows_gather move whole rows by a device index
    array: scattering the survivors of a codeword into a fresh buffer and
    decoding restores it; gathering the erased rows returns exactly them."""
    import torch

    r, n, k, S = 16, 256, 128, 208
    host = message(n, k, S, seed=4242)
    cw = gpu_encode(lch.Context(0), r, n, k, host)
    mask = WL.erasure_mask(n, n - k, seed=17)
    surv = np.nonzero(mask == 0)[0].astype(np.int32)
    eras = np.nonzero(mask)[0].astype(np.int32)
    packed = to_dev(cw[surv])
    dev = torch.full((n, S), 0x77, dtype=torch.uint8, device="cuda")
    lch.rows_scatter(packed, dev, torch.from_numpy(surv).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy()[surv], cw[surv])
    c = lch.Context(0)
    c.rs_decode(n, k, r, dev, mask)
    out = torch.empty((eras.size, S), dtype=torch.uint8, device="cuda")
    lch.rows_gather(dev, out, torch.from_numpy(eras).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), cw[eras])
    c.close()


def _pattern(n, kind):
    """Erasure patterns that make a decode's low passes skip row groups:
    aligned and unaligned bursts, erasures in two runs of groups, and one
    group in four wholly erased (more runs than the skipping handles)."""
    m = np.zeros(n, dtype=np.uint8)
    if kind == "burst_aligned":
        m[n // 4:3 * n // 4] = 1
    elif kind == "burst_unaligned":
        m[100:100 + n // 2] = 1
    elif kind == "two_runs":
        m[:64] = 1
        m[n // 2:n // 2 + 64] = 1
    elif kind == "scattered_groups":
        for g in range(0, n // 64, 4):
            m[g * 64:(g + 1) * 64] = 1
    elif kind == "tail":
        m[3 * n // 4:] = 1
    return m


@pytest.mark.parametrize("n,S", [(4096, 128), (65536, 64)])
@pytest.mark.parametrize("kind", ["burst_aligned", "burst_unaligned", "two_runs", "scattered_groups", "tail"])
def test_decode_with_skipped_row_groups(ctx, n, S, kind):
    """Algorithm 2 with the low transform passes restricted to the row groups
    they must touch: every byte of the codeword comes back, alone and (for
    n <= 8192) in a batch, whose planner skips the same groups."""
    import torch

    r, k = 16, n // 2
    cw = gpu_encode(ctx, r, n, k, message(n, k, S, seed=n + len(kind)))
    mask = _pattern(n, kind)
    assert 0 < mask.sum() <= n - k
    assert np.array_equal(gpu_decode(ctx, r, n, k, cw, mask), cw)
    if n > 8192:
        return  # batches take n <= 2^13
    bad = cw.copy()
    bad[mask != 0] = 0x77
    dev = to_dev(bad)
    b = ctx.batch(lch.BATCH_DECODE, [(n, k, r, dev, mask)])
    b.run()
    b.status()
    b.close()
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), cw)


@pytest.mark.parametrize("n,k,S", [(4096, 3072, 80), (8192, 5000, 32)])
def test_shortened_encode_with_skipped_groups(ctx, n, k, S):
    """k not a power of two: the parity rows are the erasures {k..n-1}, a tail
    burst, so the decoder's low passes skip most groups; the parity must still
    be the oracle's interpolant on sampled columns, alone and in a batch."""
    import torch

    host = message(n, k, S, seed=n + k)
    got = gpu_encode(ctx, 16, n, k, host)
    cols = elem_cols(S, 16, 3, seed=k)
    rows = np.sort(np.random.default_rng(k).choice(np.arange(k, n), 40, replace=False))
    want = O.rs_encode(16, n, k, elems(host, 16, cols), rows=rows)
    assert np.array_equal(elems(got, 16, cols)[rows], want[rows])
    dev = to_dev(host)
    b = ctx.batch(lch.BATCH_ENCODE, [(n, k, 16, dev, None)])
    b.run()
    b.status()
    b.close()
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), got)


@pytest.mark.parametrize("lgk,S", [(9, 48), (10, 4112), (11, 64), (12, 2064), (13, 16), (14, 80)])
def test_encode_one_coset_fused_middle(ctx, lgk, S):
    """n = 2k with lg k > 8: Algorithm 1's two middle passes run as one
    (the inverse's levels 8 .. lg k - 1, then the coset's), for every depth
    of that fused pass from 1 to 6 levels; sampled parity rows against the
    oracle's Lagrange evaluation, ragged column tiles included."""
    k = 1 << lgk
    n = 2 * k
    host = message(n, k, S, seed=lgk + S)
    got = gpu_encode(ctx, 16, n, k, host)
    cols = elem_cols(S, 16, 4, seed=lgk)
    rows = np.sort(np.random.default_rng(lgk).choice(np.arange(k, n), 32, replace=False))
    want = O.rs_encode(16, n, k, elems(host, 16, cols), rows=rows)
    assert np.array_equal(elems(got, 16, cols)[rows], want[rows])
    assert np.array_equal(got[:k], host[:k])
