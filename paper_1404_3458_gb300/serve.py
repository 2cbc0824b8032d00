"""A serving loop for encode and decode requests with continuous batching.

Requests arrive open-loop (their arrival times are fixed in advance, e.g. a
Poisson stream) and are served on one GPU:

* admission: a request is admitted only when its codeword buffer and its
  share of batch scratch fit in a device-memory budget (an arena carved once
  from the device; nothing is allocated per request);
* direct calls: while fewer than `max_direct` of them are in flight, a waiting
  request is launched at once as its own rs_encode/rs_decode call on a
  stream of its own, so a lightly loaded server answers as fast as one call;
* continuous batching: once that stream is full and at least `min_batch`
  requests wait, a free launch slot takes the waiting requests in arrival
  order, up to `max_batch` of them and `max_batch_bytes` of codeword data,
  and plans them into one batch per operation (lch_batch_create_in, memory
  from the arena), launched as a single persistent kernel while up to
  `max_inflight` earlier batches are still running on other streams;
* retirement: completed calls and batches are detected by polling their CUDA
  events; their requests get a completion time and their arena memory is
  released.

`serve_plain` is the reference policy: the same arrivals and budget, but each
request is its own rs_encode/rs_decode call on one stream.

The field tables and the FWHT(log) tables stay resident on the context; the
per-request state (shards, erasure masks, scratch) lives in the arena.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field as dfield

import numpy as np

from . import lch

ALIGN = 256


@dataclass
class Request:
    rid: int
    op: int               # lch.BATCH_ENCODE or lch.BATCH_DECODE
    field: int
    n: int
    k: int
    shard_bytes: int
    arrival: float        # seconds from the start of the run
    mask: np.ndarray | None = None
    payload: object = None  # device uint8 tensor [n, S] copied in on admission (None: left as is)
    # filled in by the server
    buf: object = None
    offset: int = -1
    admitted: float = -1.0
    done: float = -1.0

    @property
    def shard_data(self) -> int:
        """Shard bytes the request encodes (k S) or recovers (|E| S)."""
        if self.op == lch.BATCH_ENCODE:
            return self.k * self.shard_bytes
        return int(self.mask.sum()) * self.shard_bytes


class Arena:
    """First-fit allocator over one device block (offsets, 256-byte aligned)."""

    def __init__(self, size: int):
        self.size = size
        self.free = [(0, size)]  # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes: int) -> int:
        need = (max(nbytes, 1) + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= need:
                if ln == need:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + need, ln - need)
                self.used += need
                return off
        return -1

    def release(self, off: int, nbytes: int):
        need = (max(nbytes, 1) + ALIGN - 1) // ALIGN * ALIGN
        self.used -= need
        self.free.append((off, need))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of `count` requests of a Poisson stream."""
    g = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(g.exponential(1.0 / rate, size=count))


def _estimate(r: Request) -> int:
    """Device bytes a request may need while in flight: its buffer, batch
    scratch (k S for the encode of Algorithm 1, at most 2 n S for a decode or
    an encode with k not a power of two) and its share of the task queue."""
    nS = r.n * r.shard_bytes
    if r.op == lch.BATCH_ENCODE and r.k & (r.k - 1) == 0:
        return nS + r.k * r.shard_bytes + 16 * r.n + 65536
    return 3 * nS + 16 * r.n + 65536


@dataclass
class _Inflight:
    event: object
    slot: int
    batches: list
    requests: list
    blocks: list = dfield(default_factory=list)


class Server:
    def __init__(self, ctx: "lch.Context", budget_bytes: int, max_inflight: int = 3, max_batch: int = 1024,
                 min_batch: int = 16, max_direct: int = 32, prefer_batch: bool = False,
                 max_batch_bytes: int = 2 * 10**9):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.arena = Arena(budget_bytes)
        self.mem = torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.min_batch = min_batch
        self.max_direct = max_direct
        self.prefer_batch = prefer_batch  # a backlog of min_batch goes to a free slot before the direct stream
        # codeword bytes (n S summed) one batch may take, 0 = no limit.  A
        # batch completes as a whole, so without a bound a deep backlog goes
        # out as one long batch whose requests all wait for its end; too
        # small a bound gives up the batch kernel's efficiency.
        self.max_batch_bytes = max_batch_bytes
        self.streams = [torch.cuda.Stream() for _ in range(max_inflight)]
        # A lone request skips batch planning and runs as a single-codeword
        # call; each launch slot has its own context so those calls never
        # share context scratch across streams.
        self.slot_ctx = [lch.Context(ctx.device) for _ in range(max_inflight)]
        # direct calls: one stream and one context of their own
        self.direct_stream = torch.cuda.Stream()
        self.direct_ctx = lch.Context(ctx.device)

    def prewarm(self, shapes):
        """Build, before serving, what each context builds on first use for
        these (field, n, k, shard_bytes) shapes: field tables, FWHT(log)
        tables, shortened-code locators and scratch of the largest size (a
        first use synchronises the device, which would stall the loop).  Pass
        plans installed on the server's main context are copied to the
        contexts of the direct calls and of the launch slots."""
        torch = self.torch
        seen = sorted(set(shapes), key=lambda t: t[1] * t[3], reverse=True)
        for field, n, k, S in seen:
            for h in {n, k}:
                if h < 2 or h & (h - 1):
                    continue
                plan = self.ctx.tune_get(field, h, S)
                if plan is not None:
                    for c in [self.direct_ctx] + self.slot_ctx:
                        c.tune_set(field, h, S, plan)
        for field, n, k, S in seen:
            buf = torch.zeros((n, S), dtype=torch.uint8, device="cuda")
            mask = np.zeros(n, dtype=np.uint8)
            mask[k:] = 1
            for c in [self.ctx, self.direct_ctx] + self.slot_ctx:
                c.rs_encode(n, k, field, buf)
                if k < n:
                    c.rs_decode(n, k, field, buf, mask)
            del buf
        torch.cuda.synchronize()

    def _view(self, off: int, n: int, S: int):
        return self.mem[off:off + n * S].view(n, S)

    def _admit(self, r: Request) -> bool:
        off = self.arena.alloc(r.n * r.shard_bytes)
        if off < 0:
            return False
        r.offset = off
        r.buf = self._view(off, r.n, r.shard_bytes)
        return True

    def _release(self, r: Request):
        self.arena.release(r.offset, r.n * r.shard_bytes)
        r.offset = -1

    def _plan(self, group: list, op: int, stream, f: "_Inflight") -> bool:
        """Launch `group` as one batch (a lone request as a single call);
        False if its memory does not fit."""
        if len(group) == 1:
            r, c = group[0], self.slot_ctx[f.slot]
            if op == lch.BATCH_ENCODE:
                c.rs_encode(r.n, r.k, r.field, r.buf, stream=stream)
            else:
                c.rs_decode(r.n, r.k, r.field, r.buf, r.mask, stream=stream)
            return True
        cws = [(r.n, r.k, r.field, r.buf, r.mask) for r in group]
        # size the plan from the admission estimate; plan exactly only if short
        nbytes = sum(_estimate(r) - r.n * r.shard_bytes for r in group)
        off = self.arena.alloc(nbytes)
        if off >= 0:
            try:
                b = self.ctx.batch(op, cws, mem=self.mem[off:off + nbytes], stream=stream)
            except lch.LchError as e:
                self.arena.release(off, nbytes)
                if e.status != lch.LCH_EINVAL:
                    raise
                b = None
        else:
            b = None
        if b is None:
            nbytes = self.ctx.batch_bytes(op, cws)
            off = self.arena.alloc(nbytes)
            if off < 0:
                return False
            b = self.ctx.batch(op, cws, mem=self.mem[off:off + nbytes], stream=stream)
        f.blocks.append((off, nbytes))
        b.run(stream)
        f.batches.append(b)
        return True

    def run(self, requests: list, clock=time.perf_counter, on_done=None) -> dict:
        """Serve `requests`; returns timing statistics.  on_done(r) is called
        when a request has completed, before its arena memory is reused."""
        torch = self.torch
        pending = deque(sorted(requests, key=lambda q: q.arrival))
        waiting: deque = deque()
        inflight: list = []
        direct: deque = deque()  # (event, request) of direct calls, in launch order
        free_slots = list(range(self.max_inflight))
        batches_launched = 0
        direct_launched = 0
        blocked = False  # admitted work did not fit: wait for a retirement
        t0 = clock()
        while pending or waiting or inflight or direct:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            # retire completed direct calls (one stream: in order)
            while direct and direct[0][0].query():
                _, r = direct.popleft()
                r.done = clock() - t0
                if on_done is not None:
                    on_done(r)
                self._release(r)
                blocked = False
            # launch waiting requests one by one while the direct stream has room
            while (waiting and len(direct) < self.max_direct and not blocked
                   and not (self.prefer_batch and len(waiting) >= self.min_batch and free_slots)):
                r = waiting[0]
                if _estimate(r) > self.arena.size - self.arena.used or not self._admit(r):
                    if not inflight and not direct and _estimate(r) > self.arena.size:
                        raise RuntimeError("a request does not fit in the serving memory budget")
                    break
                waiting.popleft()
                r.admitted = clock() - t0
                with torch.cuda.stream(self.direct_stream):
                    if r.payload is not None:
                        r.buf.copy_(r.payload, non_blocking=True)
                    if r.op == lch.BATCH_ENCODE:
                        self.direct_ctx.rs_encode(r.n, r.k, r.field, r.buf, stream=self.direct_stream)
                    else:
                        self.direct_ctx.rs_decode(r.n, r.k, r.field, r.buf, r.mask, stream=self.direct_stream)
                    ev = torch.cuda.Event()
                    ev.record(self.direct_stream)
                direct.append((ev, r))
                direct_launched += 1
            # retire completed batches
            still = []
            for f in inflight:
                if f.event.query():
                    t = clock() - t0
                    for b in f.batches:
                        b.status()
                        b.close()
                    for r in f.requests:
                        r.done = t
                        if on_done is not None:
                            on_done(r)
                        self._release(r)
                    for off, nb in f.blocks:
                        self.arena.release(off, nb)
                    free_slots.append(f.slot)
                    blocked = False
                else:
                    still.append(f)
            inflight = still
            # admit whatever fits and launch it as one batch per operation
            # a backlog goes out as a batch once the direct stream is full (or,
            # with prefer_batch, as soon as min_batch requests wait); fewer
            # than min_batch also go once no more requests arrive
            full = len(direct) >= self.max_direct
            if self.prefer_batch:
                enough = len(waiting) >= self.min_batch or (waiting and not pending and full)
            else:
                enough = full and (len(waiting) >= self.min_batch or (waiting and not pending))
            if enough and free_slots and not blocked:
                slot = free_slots[-1]
                stream = self.streams[slot]
                admitted = []
                room = self.arena.size - self.arena.used
                work = 0
                while waiting and len(admitted) < self.max_batch:
                    w = waiting[0].n * waiting[0].shard_bytes
                    if admitted and self.max_batch_bytes and work + w > self.max_batch_bytes:
                        break
                    need = _estimate(waiting[0])
                    if need > room or not self._admit(waiting[0]):
                        break
                    room -= need
                    work += w
                    admitted.append(waiting.popleft())
                if not admitted and waiting and not inflight and not direct and _estimate(waiting[0]) > self.arena.size:
                    raise RuntimeError("a request does not fit in the serving memory budget")
                if admitted:
                    f = _Inflight(event=torch.cuda.Event(), slot=slot, batches=[], requests=[])
                    with torch.cuda.stream(stream):
                        for r in admitted:
                            if r.payload is not None:
                                r.buf.copy_(r.payload, non_blocking=True)
                    back = []
                    for op in (lch.BATCH_ENCODE, lch.BATCH_DECODE):
                        group = [r for r in admitted if r.op == op]
                        if not group:
                            continue
                        while group:  # shrink the group from its tail until its plan fits
                            if self._plan(group, op, stream, f):
                                f.requests.extend(group)
                                batches_launched += 1
                                break
                            back.append(group.pop())
                    if back:
                        stream.synchronize()  # their payload copies must finish before reuse
                    for r in back:  # keep arrival order at the head of the queue
                        self._release(r)
                    for r in sorted(back, key=lambda q: q.arrival, reverse=True):
                        waiting.appendleft(r)
                    if back:
                        blocked = True
                        if not inflight and not direct and not f.requests:
                            raise RuntimeError("a request does not fit in the serving memory budget")
                    if f.requests:
                        for r in f.requests:
                            r.admitted = clock() - t0
                        free_slots.pop()
                        f.event.record(stream)
                        inflight.append(f)
                    continue
            if not inflight and not direct and not waiting and pending:
                # idle until the next arrival
                wait = pending[0].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        st = _stats(requests, batches_launched + direct_launched)
        st["batches"] = batches_launched
        st["direct_calls"] = direct_launched
        return st


def serve_plain(ctx: "lch.Context", requests: list, budget_bytes: int, clock=time.perf_counter, on_done=None) -> dict:
    """One rs_encode/rs_decode call per request on one stream, in arrival
    order, under the same memory budget (codeword buffers only)."""
    import torch

    arena = Arena(budget_bytes)
    mem = torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    pending = deque(sorted(requests, key=lambda q: q.arrival))
    waiting: deque = deque()
    inflight: deque = deque()
    t0 = clock()
    while pending or waiting or inflight:
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            waiting.append(pending.popleft())
        while inflight and inflight[0][0].query():
            ev, r = inflight.popleft()
            r.done = clock() - t0
            if on_done is not None:
                on_done(r)
            arena.release(r.offset, r.n * r.shard_bytes)
        while waiting:
            r = waiting[0]
            off = arena.alloc(r.n * r.shard_bytes)
            if off < 0:
                break
            waiting.popleft()
            r.offset = off
            r.buf = mem[off:off + r.n * r.shard_bytes].view(r.n, r.shard_bytes)
            r.admitted = clock() - t0
            with torch.cuda.stream(stream):
                if r.payload is not None:
                    r.buf.copy_(r.payload, non_blocking=True)
                if r.op == lch.BATCH_ENCODE:
                    ctx.rs_encode(r.n, r.k, r.field, r.buf, stream=stream)
                else:
                    ctx.rs_decode(r.n, r.k, r.field, r.buf, r.mask, stream=stream)
                ev = torch.cuda.Event()
                ev.record(stream)
            inflight.append((ev, r))
        if not inflight and not waiting and pending:
            wait = pending[0].arrival - (clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 1e-3))
    return _stats(requests, len(requests))


def _stats(requests: list, launches: int) -> dict:
    lat = np.array([r.done - r.arrival for r in requests])
    first = min(r.arrival for r in requests)
    last = max(r.done for r in requests)
    data = sum(r.shard_data for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "gbs": data / (last - first) / 1e9,
            "wall_s": last - first, "launch_groups": launches}
