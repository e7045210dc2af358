"""The N > 1 paths on the CPU: two gloo ranks (127.0.0.1).

- bench.py: the job's time is the slowest rank's, agreed on by every rank;
  the whole-job value counts every rank's bytes; the batch's streams split
  into contiguous, byte-balanced ranges that cover every stream once; the
  reference arm runs on rank 0 only.
- One stream split over ranks by chunk ranges: each rank encodes its range
  (here with the oracle, standing in for its GPU), the ranks exchange one
  u64 each (their body bytes) and place their bodies by an exclusive scan;
  the stitched stream equals the oracle's stream of the whole series."""
import argparse
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [3.0, 5.0][rank]
    got = bench.slowest_rank_ms(ms, dist, "cpu")
    q.put((rank, got, bench.job_gbs(2.0e8, world, got), bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [5.0, 5.0]
    # 2 ranks x 200 MB in 5 ms = 80 GB/s, on every rank
    assert all(abs(r[2] - 80.0) < 1e-9 for r in res)
    assert res[0][3] != res[1][3]


def test_one_rank_is_the_single_gpu_case():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(4.5, None, "cpu") == 4.5
    assert abs(bench.job_gbs(4.5e8, 1, 4.5) - 100.0) < 1e-9


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2, ref_every=1000)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, rank=0, world=2)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    import oracle
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == oracle.host_cores()
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"] > 0


def test_stream_partition_covers_every_stream_once():
    sys.path.insert(0, ROOT)
    import bench
    from paper_1808_02515_gb300 import shard
    got = []
    per_rank = []
    for r in range(4):
        ids, shapes, nbytes = bench.rank_streams(r, 4)
        got += ids
        per_rank.append(sum(nbytes[i] for i in ids))
    assert got == list(range(bench.N_STREAMS))
    total = sum(per_rank)
    # contiguous split: every rank within one stream's bytes of an equal share
    biggest = max(r * d * (w // 8) for r, d, w in shapes)
    assert all(abs(b - total / 4) <= biggest for b in per_rank)
    assert shard.partition_streams([3, 3, 3], 1) == [(0, 3)]
    assert shard.partition_streams([], 2) == [(0, 0), (0, 0)]


def _stitch_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1808_02515_gb300 import shard, synth
    o = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=512, huff_chunks=64)
    x = synth.sensor_u16(9 * 512 + 21, 6, seed=8)
    n_chunks = -(-(x.shape[0] - x.shape[0] % 8) // 512)
    c0, c1 = shard.chunk_split(n_chunks, world)[rank]
    r1 = c1 * 512 if rank < world - 1 else x.shape[0]
    part = oracle.compress(x[c0 * 512:r1], **o)
    f = shard.part_fields(part)
    off, total = shard.place_parts(f["tail_off"] - f["data_off"], dist, rank, world)
    stitched = shard.stitch_parts(part, dist, rank, world)
    whole = oracle.compress(x, **o)
    q.put((rank, off, total, bool(np.array_equal(stitched, whole))))
    dist.barrier()
    dist.destroy_process_group()


def test_chunk_range_split_over_two_gloo_ranks_equals_the_oracle_stream():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_stitch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == 0 and res[1][1] > 0 and res[0][2] == res[1][2]
    assert all(r[3] for r in res)
