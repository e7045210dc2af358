"""Parity at the workloads' full sizes, in the launch configuration bench.py
times.

- The batch of 10,000 streams (rows log-uniform in [1e3, 1e6], D uniform in
  1..16, uint8 and uint16, about 18 GB, drawn with the numpy recipe as the
  benchmark draws it): one batched compress of every stream with the
  schedule the autotuner picks, for FIRE and for delta; every stream's bytes
  are compared with the CPU oracle's stream of the same samples (the oracle
  runs on all host cores, one stream per thread), and one batched
  decompress must give back every sample.
- The serving workload: 1,000 device-resident uint16 streams of 2^20 rows
  and 4 columns (8 GB), each compressed stream equal to the oracle's; then a
  Poisson mix of range reads and appends served with continuous batching,
  every range checked against the source rows, a sample of them also served
  alone, and every appended shard equal to the oracle's stream of its rows.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def spz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_02515_gb300 import _build
    _build.build()
    import paper_1808_02515_gb300.sprintz as spz
    return spz


def _host(t):
    a = t.cpu().numpy()
    return a.view(np.uint16) if a.dtype == np.int16 else a


def _check_slices(xh, bufs, sizes, opts, oracle_mod, step=250):
    """Every stream's bytes against the oracle's stream of the host samples
    xh, `step` streams at a time (bounded host memory); returns the indices
    that differ."""
    sz = sizes.cpu().numpy()
    bad = []
    for a in range(0, len(xh), step):
        part = range(a, min(len(xh), a + step))
        got = [bufs[k][:int(sz[k])].cpu().numpy() for k in part]
        ref = oracle_mod.compress_many([xh[k] for k in part], opts)
        bad += [k for k, g, r in zip(part, got, ref) if g.size != r.size or not np.array_equal(g, r)]
    return bad


def test_batch_of_10000_streams_full_size(spz, oracle_mod):
    from paper_1808_02515_gb300 import synth
    xh = oracle_mod.map_streams(synth.batch_stream, list(range(10_000)))
    assert sum(x.nbytes for x in xh) == 18_048_708_071
    xs = [torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).cuda() for x in xh]
    torch.cuda.synchronize()
    codec = spz.Codec(0)
    try:
        for fc in (1, 0):
            o = dict(forecaster=fc, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
            bufs, sizes, _ = codec.compress_batch(xs, spz.Opts(**o), autotune=(fc == 1))
            torch.cuda.synchronize()
            assert codec.status() == spz.OK
            bad = _check_slices(xh, bufs, sizes, o, oracle_mod)
            assert not bad, (fc, bad[:10], len(bad))
            sz = [int(v) for v in sizes.cpu().numpy()]
            infos = [spz.query(h.tobytes()) for h in torch.stack([b[:64] for b in bufs]).cpu().numpy()]
            outs, _ = codec.decompress_batch(bufs, infos, sz, autotune=(fc == 1))
            torch.cuda.synchronize()
            assert codec.status() == spz.OK
            wrong = [k for k, (x, y) in enumerate(zip(xs, outs)) if not torch.equal(x.view(-1), y.view(-1))]
            assert not wrong, (fc, wrong[:10])
            # the oracle decodes a sample of the GPU's streams to the same samples
            for k in range(0, 10_000, 500):
                got = oracle_mod.decompress(bufs[k][:sz[k]].cpu().numpy())
                assert np.array_equal(got.reshape(-1), xh[k].reshape(-1)), k
            del bufs, outs
    finally:
        codec.close()


def test_serving_workload_full_size(spz, oracle_mod):
    from paper_1808_02515_gb300 import serve, synth
    n_streams, rows, D = 1000, 1 << 20, 4
    xs = [synth.sensor_u16_torch(rows, D, seed=4000 + i, device="cuda") for i in range(n_streams)]
    torch.cuda.synchronize()
    opts = spz.Opts(forecaster=1)
    o = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
    codec = spz.Codec(0)
    try:
        store = serve.ShardStore(codec, D, 16, opts)
        store.add_streams(xs)
        # every resident stream equals the oracle's
        bad = []
        for a in range(0, n_streams, 100):
            part = range(a, a + 100)
            ref = oracle_mod.compress_many([_host(xs[k]) for k in part], o)
            for k, r in zip(part, ref):
                sh = store.streams[k][0]
                if sh.size != r.size or not np.array_equal(sh.buf[:sh.size].cpu().numpy(), r):
                    bad.append(k)
        assert not bad, bad[:10]
        pool = [synth.sensor_u16_torch(8192, D, seed=500000 + k, device="cuda") for k in range(64)]
        reqs = serve.poisson_requests(store, 20_000, rate=20_000.0, seed=4, append_frac=0.1, append_rows=8192,
                                      append_source=lambda sid, k: pool[(sid * 7 + k) % len(pool)])
        server = serve.Server(store, mem_budget=4 << 30, max_batch=512, n_slots=3)
        stats = server.run(reqs, realtime=True)
        torch.cuda.synchronize()
        assert stats["batches"] >= 2
        ranges = [r for r in reqs if r.kind == "range"]
        apps = [r for r in reqs if r.kind == "append"]
        assert len(ranges) > 1000 and len(apps) > 100
        wrong = [i for i, r in enumerate(ranges) if not torch.equal(r.result, xs[r.sid][r.a:r.b])]
        assert not wrong, wrong[:10]
        # a sample of the ranges served alone gives the same rows
        sample = ranges[::100]
        alone = [serve.Request("range", r.sid, 0.0, a=r.a, b=r.b) for r in sample]
        serve.Server(store, max_batch=1, n_slots=1).run(alone, realtime=False)
        torch.cuda.synchronize()
        assert all(torch.equal(p.result, q.result) for p, q in zip(sample, alone))
        # every appended shard is the oracle's stream of its rows
        uniq = {}
        for r in apps:
            uniq.setdefault(id(r.rows), r.rows)
        ref = {k: oracle_mod.compress(_host(v), **o) for k, v in uniq.items()}
        for r in apps:
            sh = r.result
            assert np.array_equal(sh.buf[:sh.size].cpu().numpy(), ref[id(r.rows)])
    finally:
        codec.close()
