"""Serving loop over device-resident compressed streams (continuous batching).

A logical stream is a list of shards, each an independent Sprintz stream held
in device memory (the first from the initial bulk compression, one more per
append). Requests:
  range   rows [a, b) of a stream -> decoded into a fresh device tensor; a
          range that spans shards becomes one batch item per shard, each
          writing its slice of the output;
  append  new rows -> compressed into a new shard at the stream's end.

The loop admits arrived requests while a device-memory budget allows and a
batch slot is free, groups them into one batched decode launch and one
batched encode launch on that slot's CUDA stream, and keeps several slots in
flight so their work overlaps on the GPU; requests arriving meanwhile join
the next batch. Completion is observed from each batch's CUDA event; latency
is completion minus arrival. All device work runs in the library's kernels
(sprintz_batch_plan / sprintz_batch_run); this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import sprintz as spz


@dataclass
class Shard:
    buf: object          # device uint8 tensor holding the stream
    size: int            # stream bytes
    info: spz.Info
    row0: int            # first row of the logical stream held here
    ptr: int = 0         # the stream's device address
    shape: tuple = ()    # (rows, D, w, Opts), as a batch item takes them

    def __post_init__(self):
        self.ptr = self.buf.data_ptr()
        self.shape = (self.info.rows, self.info.D, self.info.w, self.info.opts)


@dataclass
class Request:
    kind: str            # "range" or "append"
    sid: int
    t_arrival: float     # seconds from the start of the run
    a: int = 0           # range [a, b)
    b: int = 0
    rows: object = None  # append: device tensor (n, D)
    row0: int = 0        # append: first row of the new shard (reserved at admission)
    t_done: float = -1.0
    result: object = None
    mem: int = 0


@dataclass
class _Slot:
    codec: spz.Codec
    stream: object
    event: object = None
    reqs: list = field(default_factory=list)
    new_shards: list = field(default_factory=list)
    keep: list = field(default_factory=list)  # workspaces alive until completion


class ShardStore:
    """Device-resident compressed streams of one shape (D, w, options)."""

    def __init__(self, codec: spz.Codec, D: int, w: int, opts: spz.Opts):
        self.codec, self.D, self.w, self.opts = codec, D, w, opts
        self.streams: list[list[Shard]] = []
        self.reserved: list[int] = []  # rows of each stream including admitted appends

    def rows(self, sid: int) -> int:
        sh = self.streams[sid][-1]
        return sh.row0 + sh.info.rows

    def add_streams(self, xs: list, batch: int = 256) -> None:
        """Compress the initial contents of new streams (batched launches)."""
        for k in range(0, len(xs), batch):
            part = xs[k:k + batch]
            bufs, sizes, _ = self.codec.compress_batch(part, self.opts)
            self.codec.torch.cuda.synchronize()
            self.codec.check()
            sz = sizes.cpu().numpy()
            for buf, n in zip(bufs, sz):
                n = int(n)
                head = buf[:64].cpu().numpy().tobytes()
                info = spz.query(head)
                self.streams.append([Shard(buf[:n].clone(), n, info, 0)])
                self.reserved.append(info.rows)

    def pieces(self, sid: int, a: int, b: int):
        """Per-shard pieces (shard, local a, local b, output row offset) of
        rows [a, b) of a stream."""
        out = []
        for sh in self.streams[sid]:
            lo, hi = max(a, sh.row0), min(b, sh.row0 + sh.info.rows)
            if lo < hi:
                out.append((sh, lo - sh.row0, hi - sh.row0, lo - a))
        return out


class Server:
    """Continuous-batching request loop over a ShardStore."""

    def __init__(self, store: ShardStore, mem_budget: int = 2 << 30, max_batch: int = 256,
                 n_slots: int = 3):
        torch = store.codec.torch
        self.torch = torch
        self.store = store
        self.mem_budget = mem_budget
        self.max_batch = max_batch
        dev = store.codec.device
        self.slots = [_Slot(spz.Codec(dev), torch.cuda.Stream(device=dev)) for _ in range(n_slots)]
        self.mem_used = 0
        self.peak_mem = 0
        self.batches = 0
        self._caps = {}  # rows -> largest compressed size of an append of that many rows

    def _need(self, r: Request) -> int:
        rb = self.store.D * (self.store.w // 8)
        if r.kind == "range":
            # output + decoded covering chunks (at most one extra chunk each side)
            cr = self.store.opts.chunk_rows or 1 << 30
            return 2 * (r.b - r.a) * rb + 2 * cr * rb + 4096
        n = r.rows.shape[0]
        return spz.max_compressed_size(n, self.store.D, self.store.w, self.store.opts) + 4096

    def _cap(self, rows: int) -> int:
        c = self._caps.get(rows)
        if c is None:
            c = self._caps[rows] = spz.max_compressed_size(rows, self.store.D, self.store.w, self.store.opts)
        return c

    def _launch(self, slot: _Slot, reqs: list) -> None:
        torch = self.torch
        store = self.store
        codec = slot.codec
        dev = f"cuda:{codec.device}"
        rb = store.D * (store.w // 8)
        slot.reqs, slot.new_shards, slot.keep = reqs, [], []
        with torch.cuda.stream(slot.stream):
            ranges = [r for r in reqs if r.kind == "range"]
            if ranges:
                # one output tensor for the batch's ranges, a view per request;
                # the pieces go to the library as plain addresses
                dt = torch.uint8 if store.w == 8 else torch.int16
                out = torch.empty((sum(r.b - r.a for r in ranges), store.D), dtype=dt, device=dev)
                base = out.data_ptr()
                shapes, srcs, sizes, rng, dsts = [], [], [], [], []
                row = 0
                for r in ranges:
                    n = r.b - r.a
                    r.result = out[row:row + n]
                    for sh, la, lb, off in store.pieces(r.sid, r.a, r.b):
                        shapes.append(sh.shape)
                        srcs.append(sh.ptr)
                        sizes.append(sh.size)
                        rng.append((la, lb))
                        dsts.append((base + (row + off) * rb, (lb - la) * rb))
                    row += n
                if shapes:
                    slot.keep.append(codec.decompress_ranges_into(shapes, srcs, sizes, rng, dsts,
                                                                  stream=slot.stream))
            apps = [r for r in reqs if r.kind == "append"]
            if apps:
                # the batch's new shards share one buffer (256-byte aligned parts)
                caps = [self._cap(r.rows.shape[0]) for r in apps]
                offs, tot = [], 0
                for c in caps:
                    offs.append(tot)
                    tot += (c + 255) & ~255
                big = torch.empty(tot, dtype=torch.uint8, device=dev)
                bufs, sizes, ws = codec.compress_batch([r.rows for r in apps], store.opts, stream=slot.stream,
                                                       bufs=[big[o:o + c] for o, c in zip(offs, caps)])
                slot.keep += [ws, sizes]
                slot.new_shards = list(zip(apps, bufs, range(len(apps))))
                slot.sizes = sizes
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)
        self.batches += 1

    def _finish(self, slot: _Slot, now: float, keep_results: bool = True) -> None:
        store = self.store
        if slot.new_shards:
            sz = slot.sizes.cpu().numpy()
            # every new shard's header in one gather and one copy
            heads = self.torch.stack([buf[:64] for _, buf, _ in slot.new_shards]).cpu().numpy()
            for (r, buf, k), head in zip(slot.new_shards, heads):
                n = int(sz[k])
                info = spz.query(head.tobytes())
                sh = Shard(buf[:n], n, info, r.row0)
                store.streams[r.sid].append(sh)
                store.streams[r.sid].sort(key=lambda x: x.row0)
                r.result = sh
        rc = slot.codec.status(slot.stream)
        if rc != spz.OK:
            raise spz.SprintzError(rc, "serving batch")
        for r in slot.reqs:
            r.t_done = now
            self.mem_used -= r.mem
            if not keep_results and r.kind == "range":
                r.result = None  # the client has taken its rows: their memory goes back to the pool
        slot.reqs, slot.new_shards, slot.keep, slot.event = [], [], [], None

    def run(self, requests: list, realtime: bool = True, keep_results: bool = True) -> dict:
        """Serve `requests` (sorted by arrival). With realtime=False every
        request is taken as arrived at once (a closed-loop throughput run).
        keep_results=False drops each range request's rows once it has
        completed (a client that consumes them), so that a long run does not
        hold every result in device memory."""
        pending = collections.deque(requests)
        queue: collections.deque = collections.deque()
        t0 = time.perf_counter()
        while pending or queue or any(s.event is not None for s in self.slots):
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].t_arrival <= now):
                queue.append(pending.popleft())
            for s in self.slots:
                if s.event is not None and s.event.query():
                    self._finish(s, time.perf_counter() - t0, keep_results)
            free = [s for s in self.slots if s.event is None]
            if free and queue:
                batch = []
                while queue and len(batch) < self.max_batch:
                    r = queue[0]
                    need = self._need(r)
                    if self.mem_used + need > self.mem_budget and batch:
                        break
                    if self.mem_used + need > self.mem_budget and any(
                            s.event is not None for s in self.slots):
                        break  # wait for memory to free up
                    queue.popleft()
                    r.mem = need
                    self.mem_used += need
                    if r.kind == "append":
                        r.row0 = self.store.reserved[r.sid]
                        self.store.reserved[r.sid] += r.rows.shape[0]
                    batch.append(r)
                if batch:
                    self.peak_mem = max(self.peak_mem, self.mem_used)
                    self._launch(free[0], batch)
            elif not free or not queue:
                time.sleep(0)
        wall = time.perf_counter() - t0
        lat = np.array([r.t_done - r.t_arrival for r in requests]) if requests else np.zeros(1)
        rb = self.store.D * (self.store.w // 8)
        served = sum((r.b - r.a) * rb if r.kind == "range" else r.rows.shape[0] * rb for r in requests)
        return {"requests": len(requests), "wall_s": wall, "batches": self.batches,
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "gbs": served / wall / 1e9, "served_bytes": served, "peak_mem": self.peak_mem}


def poisson_requests(store: ShardStore, n: int, rate: float, seed: int, append_frac: float = 0.1,
                     append_rows: int = 8192, min_len: int = 1024, max_len: int = 65536,
                     append_source=None) -> list:
    """Poisson arrivals at `rate` per second: range requests of log-uniform
    length in [min_len, max_len] rows starting uniformly inside the stream's
    rows at generation time, and appends of `append_rows` rows (rows from
    append_source(sid, k), the k-th append of stream sid)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    n_app = collections.Counter()
    lens = {sid: store.rows(sid) for sid in range(len(store.streams))}
    for _ in range(n):
        t += rng.exponential(1.0 / rate)
        sid = int(rng.integers(0, len(store.streams)))
        if rng.random() < append_frac and append_source is not None:
            rows = append_source(sid, n_app[sid])
            n_app[sid] += 1
            out.append(Request("append", sid, t, rows=rows))
        else:
            ln = int(np.exp(rng.uniform(np.log(min_len), np.log(max_len))))
            ln = min(ln, lens[sid])
            a = int(rng.integers(0, lens[sid] - ln + 1))
            out.append(Request("range", sid, t, a=a, b=a + ln))
    return out
