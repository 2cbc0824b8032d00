"""GPU parity under autotuned and hand-set pass plans (lch_autotune,
lch_tune_set): the level split and column-tile widths change only the speed,
so every plan must give the oracle's results bit for bit, through the direct
calls and through batches planned afterwards."""
import numpy as np
import pytest

from helpers import elem_cols, elems, to_dev
from oracle import oracle as O
from paper_1404_3458_gb300 import lch
from paper_1404_3458_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


@pytest.fixture()
def tctx():
    """A context of its own, so that its plans never reach other tests."""
    c = lch.Context(0)
    yield c
    c.close()


def plans_for(r, lgh, S):
    """Hand-set plans: every split with both passes <= 8 levels, each with the
    narrowest (16-byte), a 64-byte and a 256-byte column tile (from 256 bytes
    up the persistent pass splits its CTA into two column halves)."""
    out = []
    splits = [lgh] if lgh <= 8 else [a for a in range(1, 9) if 1 <= lgh - a <= 8]
    for a in splits:
        b = lgh - a
        for lo, hi in ((4, 4 if b else 0), (6, 6 if b else 0), (8, 8 if b else 0)):
            cap = max(4, int(np.ceil(np.log2(S))))
            out.append({"split": a, "lg_tile_low": min(lo, cap), "lg_tile_high": min(hi, cap) if b else 0})
    return out


@pytest.mark.parametrize("r,lgh,l,S", [(8, 8, 0, 4112), (16, 10, 1024, 336), (16, 12, 0, 80), (8, 5, 96, 208)])
def test_fft_ifft_exact_under_every_plan(tctx, r, lgh, l, S):
    import torch

    h = 1 << lgh
    host = WL.shards(h, S, seed=5000 + lgh + S)
    cols = elem_cols(S, r, 8, seed=lgh)
    rows = None if h <= 1024 else np.random.default_rng(h).choice(h, 48, replace=False)
    expect = O.fft(r, l, elems(host, r, cols), rows=rows)
    for plan in plans_for(r, lgh, S):
        tctx.tune_set(r, h, S, plan)
        dev = to_dev(host)
        tctx.fft(r, l, dev)
        got = elems(dev.cpu().numpy(), r)
        got = got[:, cols] if rows is None else got[rows][:, cols]
        assert np.array_equal(got, expect), plan
        tctx.ifft(r, l, dev)
        torch.cuda.synchronize()
        assert np.array_equal(dev.cpu().numpy(), host), plan


def test_autotune_plan_is_valid_and_exact(tctx):
    r, n, k, S = 16, 1024, 512, 1040
    for h in (k, n):
        p = tctx.autotune(r, h, S)
        lgh = h.bit_length() - 1
        assert 1 <= p["split"] <= min(lgh, 8) and lgh - p["split"] <= 8
        assert 4 <= p["lg_tile_low"] <= 12 and p["ms"] > 0
        assert (p["lg_tile_high"] == 0) == (p["split"] == lgh)
    host = np.zeros((n, S), dtype=np.uint8)
    host[:k] = WL.shards(k, S, seed=77)
    dev = to_dev(host)
    tctx.rs_encode(n, k, r, dev)
    cw = dev.cpu().numpy()
    cols = elem_cols(S, r, 6, seed=3)
    rows = k + np.random.default_rng(5).choice(n - k, 40, replace=False)  # parity rows
    expect = O.rs_encode(r, n, k, elems(host, r, cols), rows=rows)
    assert np.array_equal(elems(cw, r)[rows][:, cols], expect[rows])
    assert np.array_equal(cw[:k], host[:k])
    mask = WL.erasure_mask(n, n - k, seed=9)
    bad = cw.copy()
    bad[mask != 0] = 0xA5
    dev = to_dev(bad)
    tctx.rs_decode(n, k, r, dev, mask)
    assert np.array_equal(dev.cpu().numpy(), cw)


def test_batches_follow_installed_plans(tctx):
    """Batches planned after lch_tune_set use the plan (tile widths capped to
    the batch kernel's shared memory) and stay exact."""
    r, n, k, S = 16, 512, 256, 208
    tctx.tune_set(r, k, S, {"split": 8, "lg_tile_low": 4, "lg_tile_high": 0})
    tctx.tune_set(r, n, S, {"split": 3, "lg_tile_low": 8, "lg_tile_high": 4})
    hosts = []
    for i in range(3):
        host = np.zeros((n, S), dtype=np.uint8)
        host[:k] = WL.shards(k, S, seed=900 + i)
        hosts.append(host)
    devs = [to_dev(h) for h in hosts]
    b = tctx.batch(lch.BATCH_ENCODE, [(n, k, r, d, None) for d in devs])
    b.run()
    b.status()
    cws = [d.cpu().numpy() for d in devs]
    cols = elem_cols(S, r, 5, seed=1)
    for host, cw in zip(hosts, cws):
        assert np.array_equal(elems(cw, r)[:, cols], O.rs_encode(r, n, k, elems(host, r, cols)))
    masks = [WL.erasure_mask(n, n - k, seed=40 + i) for i in range(3)]
    bads = []
    for cw, m in zip(cws, masks):
        bad = cw.copy()
        bad[m != 0] = 0
        bads.append(to_dev(bad))
    b = tctx.batch(lch.BATCH_DECODE, [(n, k, r, d, m) for d, m in zip(bads, masks)])
    b.run()
    b.status()
    for d, cw in zip(bads, cws):
        assert np.array_equal(d.cpu().numpy(), cw)


@pytest.mark.parametrize("plan", [
    {"split": 0, "lg_tile_low": 6, "lg_tile_high": 6},    # empty low pass
    {"split": 9, "lg_tile_low": 6, "lg_tile_high": 6},    # pass of 9 levels
    {"split": 2, "lg_tile_low": 6, "lg_tile_high": 6},    # high pass of 10 levels
    {"split": 6, "lg_tile_low": 3, "lg_tile_high": 6},    # tile below 16 bytes
    {"split": 6, "lg_tile_low": 6, "lg_tile_high": 13},   # tile above 4 KiB
])
def test_tune_set_rejects_invalid_plans(tctx, plan):
    with pytest.raises(lch.LchError) as e:
        tctx.tune_set(16, 1 << 12, 4096, plan)
    assert e.value.status == lch.LCH_EINVAL


def test_tune_set_none_restores_defaults(tctx):
    import torch

    r, h, S = 8, 256, 64
    host = WL.shards(h, S, seed=31)
    tctx.tune_set(r, h, S, {"split": 8, "lg_tile_low": 4, "lg_tile_high": 0})
    a = to_dev(host)
    tctx.fft(r, 0, a)
    tctx.tune_set(r, h, S, None)
    b = to_dev(host)
    tctx.fft(r, 0, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_large_gf16_with_autotuned_plans(tctx):
    """The measured workload (n = 65536, k = 32768, 4 KiB shards) under the
    autotuned plans that bench.py uses: sampled parity rows against the
    oracle, then a decode of 32768 random erasures restores every byte."""
    import torch

    w = WL.WORKLOADS["large_gf16"]
    r, n, k, S = w.field, w.n, w.k, w.shard_bytes
    for h in (k, n):
        tctx.autotune(r, h, S)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(77)
    dev = torch.zeros((n, S), dtype=torch.uint8, device="cuda")
    dev[:k] = torch.randint(0, 256, (k, S), dtype=torch.uint8, device="cuda", generator=gen)
    tctx.rs_encode(n, k, r, dev)
    cw = dev.clone()
    cols = elem_cols(S, r, 3, seed=5)
    byte_cols = torch.from_numpy(np.concatenate([[2 * c, 2 * c + 1] for c in cols])).cuda()
    rows = k + np.random.default_rng(6).choice(n - k, 12, replace=False)
    msg = O.to_elems(dev[:, byte_cols].cpu().numpy(), r)
    msg[k:] = 0
    expect = O.rs_encode(r, n, k, msg, rows=rows)
    assert np.array_equal(O.to_elems(dev[:, byte_cols].cpu().numpy(), r)[rows], expect[rows])
    mask = WL.erasure_mask(n, n - k, w.seed + 100)
    dev[torch.from_numpy(mask != 0).cuda()] = 0x5A
    tctx.rs_decode(n, k, r, dev, mask)
    torch.cuda.synchronize()
    assert torch.equal(dev, cw)
