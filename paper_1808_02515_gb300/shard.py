"""Sharding of the codec's independent units over GPUs (one process per GPU).

Streams are independent, and so are the chunks of one stream (the forecaster
restarts at every chunk), so work splits without any exchange of samples:

  partition_streams   a batch of streams split into contiguous ranges, one per
                      rank, balanced by uncompressed bytes; each rank encodes
                      and decodes its range with no collective on the data.
  chunk_split         one stream's chunks split into contiguous ranges (whole
                      chunks; the last range also holds the raw tail rows).
  place_parts         where each rank's compressed bodies go in the one stream
                      they form: an exclusive scan of one u64 per rank (the
                      bytes of its chunk bodies), gathered over the process
                      group when one is given.
  stitch_parts        the stream itself, from each rank's part (a stream of its
                      own rows, as the codec writes it): header fields of the
                      whole, the chunk tables concatenated with their body
                      offsets moved by the scan, the bodies, the tail.

This is host logic only: the byte layout is the container's (64-byte header,
16-byte chunk entries, chunk bodies, raw tail), and nothing here codes a
sample.
"""
from __future__ import annotations

import numpy as np

HDR = 64
ENTRY = 16


def partition_streams(nbytes, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges [lo, hi) of streams, one per rank, whose byte sums
    are as equal as a contiguous split allows: rank r ends where the running
    byte count first reaches (r + 1) / world of the total."""
    n = len(nbytes)
    if world < 1:
        raise ValueError("world must be >= 1")
    pre = np.concatenate([[0], np.cumsum(np.asarray(nbytes, dtype=np.float64))])
    total = pre[-1]
    cuts = [0]
    for r in range(1, world):
        k = int(np.searchsorted(pre, total * r / world, side="left"))
        cuts.append(min(max(k, cuts[-1]), n))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def chunk_split(n_chunks: int, world: int) -> list[tuple[int, int]]:
    """Contiguous chunk ranges [c0, c1), sizes differing by at most one."""
    base, extra = divmod(n_chunks, world)
    out, c = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((c, c + k))
        c += k
    return out


def exclusive_scan(values) -> list[int]:
    out, acc = [], 0
    for v in values:
        out.append(acc)
        acc += int(v)
    return out


def place_parts(my_body_bytes: int, dist=None, rank: int = 0, world: int = 1):
    """(offset of this rank's bodies from the data start, total body bytes):
    an all-gather of one u64 per rank, then an exclusive scan."""
    if dist is None or world == 1:
        return 0, int(my_body_bytes)
    import torch
    t = torch.tensor([int(my_body_bytes)], dtype=torch.int64)
    got = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(got, t)
    sizes = [int(g.item()) for g in got]
    return exclusive_scan(sizes)[rank], sum(sizes)


def _le(b: np.ndarray, off: int, n: int) -> int:
    return int.from_bytes(bytes(b[off:off + n]), "little")


def _put(b: np.ndarray, off: int, v: int, n: int) -> None:
    b[off:off + n] = np.frombuffer(int(v).to_bytes(n, "little"), dtype=np.uint8)


def part_fields(part: np.ndarray) -> dict:
    """The header fields of one part that stitching needs."""
    p = np.ascontiguousarray(part, dtype=np.uint8)
    if bytes(p[:4]) != b"SPZ1" or p[7] & 1:
        raise ValueError("not a Sprintz stream without Huffman coding")
    return dict(n_chunks=_le(p, 20, 4), rows=_le(p, 24, 8), tail_rows=_le(p, 32, 4),
                data_off=_le(p, 40, 8), tail_off=_le(p, 48, 8), total=_le(p, 56, 8),
                chunk_rows=_le(p, 12, 4), D=_le(p, 8, 2), w=int(p[5]))


def stitch_parts(parts, dist=None, rank: int = 0, world: int = 1) -> np.ndarray:
    """One stream from the parts of consecutive chunk ranges (all parts but
    the last hold whole chunks and no tail).  With a process group, `parts`
    is this rank's part alone: the body offset comes from place_parts and the
    parts are gathered to every rank before they are joined."""
    if dist is not None and world > 1:
        mine = np.ascontiguousarray(parts, dtype=np.uint8)
        f = part_fields(mine)
        place_parts(f["tail_off"] - f["data_off"], dist, rank, world)  # the one-u64 exchange
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        parts = gathered
    ps = [np.ascontiguousarray(p, dtype=np.uint8) for p in parts]
    fs = [part_fields(p) for p in ps]
    for f in fs[:-1]:
        if f["tail_rows"] or (f["chunk_rows"] and f["rows"] % f["chunk_rows"]):
            raise ValueError("every part but the last must hold whole chunks")
    n_chunks = sum(f["n_chunks"] for f in fs)
    rows = sum(f["rows"] for f in fs)
    body = [f["tail_off"] - f["data_off"] for f in fs]
    offs = exclusive_scan(body)
    data_off = HDR + ENTRY * n_chunks
    tail = ps[-1][fs[-1]["tail_off"]:fs[-1]["total"]]
    tail_off = data_off + sum(body)
    total = tail_off + tail.size
    out = np.zeros(total, dtype=np.uint8)
    out[:HDR] = ps[0][:HDR]
    _put(out, 20, n_chunks, 4)
    _put(out, 24, rows, 8)
    _put(out, 32, fs[-1]["tail_rows"], 4)
    _put(out, 40, data_off, 8)
    _put(out, 48, tail_off, 8)
    _put(out, 56, total, 8)
    c = 0
    for p, f, o in zip(ps, fs, offs):
        tab = p[HDR:HDR + ENTRY * f["n_chunks"]].reshape(-1, ENTRY).copy()
        body_off = tab[:, :8].copy().view("<u8")[:, 0] + np.uint64(o)
        tab[:, :8] = body_off.astype("<u8").view(np.uint8).reshape(-1, 8)
        out[HDR + ENTRY * c:HDR + ENTRY * (c + f["n_chunks"])] = tab.reshape(-1)
        out[data_off + o:data_off + o + (f["tail_off"] - f["data_off"])] = p[f["data_off"]:f["tail_off"]]
        c += f["n_chunks"]
    out[tail_off:] = tail
    return out
