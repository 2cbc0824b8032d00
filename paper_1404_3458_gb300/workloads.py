"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no field arithmetic and nothing of the method: it only draws
shard bytes and erasure sets from numpy's PCG64 generator, with the shapes of
the workloads the library is measured on.

Workload shapes (field, n, k, shard bytes, erasures):

* ``small_gf8``:   GF(2^8),  n=32,    k=16,    S=1 KiB,  16 random erasures
* ``medium_gf16``: GF(2^16), n=256,   k=128,   S=64 KiB, 128 random erasures
* ``large_gf16``:  GF(2^16), n=65536, k=32768, S=4 KiB,  32768 random erasures
  (or a contiguous burst of 32768)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 1404_3458


@dataclass(frozen=True)
class Workload:
    name: str
    field: int          # r: 8 or 16
    n: int
    k: int
    shard_bytes: int
    erasures: int
    seed: int


WORKLOADS = {
    "small_gf8": Workload("small_gf8", 8, 32, 16, 1024, 16, SEED_BASE + 1),
    "medium_gf16": Workload("medium_gf16", 16, 256, 128, 65536, 128, SEED_BASE + 2),
    "large_gf16": Workload("large_gf16", 16, 65536, 32768, 4096, 32768, SEED_BASE + 3),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def shards(rows: int, shard_bytes: int, seed: int) -> np.ndarray:
    """uint8 [rows, shard_bytes], uniform random bytes (uniform uint16 elements
    when read little-endian)."""
    return rng(seed).integers(0, 256, size=(rows, shard_bytes), dtype=np.uint8)


def erasure_mask(n: int, count: int, seed: int) -> np.ndarray:
    """uint8 [n]: exactly ``count`` positions set, drawn uniformly (a seeded
    random permutation, i.e. a Fisher-Yates sample)."""
    m = np.zeros(n, dtype=np.uint8)
    if count:
        m[rng(seed).permutation(n)[:count]] = 1
    return m


def burst_mask(n: int, count: int, start: int) -> np.ndarray:
    """uint8 [n]: the contiguous run [start, start+count) set, no wrap-around."""
    assert 0 <= start and start + count <= n
    m = np.zeros(n, dtype=np.uint8)
    m[start:start + count] = 1
    return m


def random_burst_start(n: int, count: int, seed: int) -> int:
    return int(rng(seed).integers(0, n - count + 1))


def batch_workload(count: int, seed: int = SEED_BASE + 4):
    """The batched mix: `count` codewords with n = 2^u, u uniform in 6..13,
    k/n drawn from {1/2, 1/4, 3/4}, GF(2^8) when n <= 256 else GF(2^16),
    shard bytes from {512, 2048, 8192, 16384} and an erasure count uniform in
    [0, n-k].  Returns a list of (field, n, k, shard_bytes, erasures)."""
    g = rng(seed)
    out = []
    for _ in range(count):
        n = 1 << int(g.integers(6, 14))
        k = n * [2, 1, 3][int(g.integers(0, 3))] // 4
        field = 8 if n <= 256 else 16
        S = [512, 2048, 8192, 16384][int(g.integers(0, 4))]
        e = int(g.integers(0, n - k + 1))
        out.append((field, n, k, S, e))
    return out
