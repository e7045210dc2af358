"""The N > 1 path of bench.py on the CPU: two gloo ranks (127.0.0.1). Each
rank encodes its own series (its own seed, no data crosses ranks); the job's
time is the slowest rank's, agreed on by every rank; the whole-job value
counts every rank's bytes. The reference arm runs on rank 0 only."""
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
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""
    bench.run_reference(args, rank=0, world=2)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"] > 0
