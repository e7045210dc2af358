"""Serving: continuous batching over device-resident compressed shards.
Each request's result is checked against the source rows, against the same
request served alone, and (appends) against the oracle's stream."""
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


N_STREAMS, ROWS, D = 10, (1 << 14) + 5, 4


def _source(sid):
    from paper_1808_02515_gb300 import synth
    return synth.sensor_u16(ROWS, D, seed=4000 + sid)


def _append_rows(sid, k):
    from paper_1808_02515_gb300 import synth
    return synth.sensor_u16(2048, D, seed=90000 + 100 * sid + k)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.view(np.int16))).cuda()


def _serve(spz, realtime, max_batch, n_slots, seed=3):
    from paper_1808_02515_gb300 import serve
    codec = spz.Codec(0)
    store = serve.ShardStore(codec, D, 16, spz.Opts())
    store.add_streams([_dev(_source(s)) for s in range(N_STREAMS)])
    reqs = serve.poisson_requests(store, 160, rate=20000.0, seed=seed, append_frac=0.15,
                                  append_rows=2048, min_len=100, max_len=6000,
                                  append_source=lambda sid, k: _dev(_append_rows(sid, k)))
    server = serve.Server(store, mem_budget=64 << 20, max_batch=max_batch, n_slots=n_slots)
    stats = server.run(reqs, realtime=realtime)
    torch.cuda.synchronize()
    return store, reqs, stats


def test_serving_results_alone_and_mixed(spz, oracle_mod):
    store_m, mixed, stats = _serve(spz, realtime=True, max_batch=32, n_slots=3)
    assert stats["batches"] >= 2 and stats["p99_ms"] >= stats["p50_ms"] >= 0
    store_a, alone, _ = _serve(spz, realtime=False, max_batch=1, n_slots=1)
    src = [_source(s) for s in range(N_STREAMS)]
    n_app = {}
    for rm, ra in zip(mixed, alone):
        assert (rm.kind, rm.sid, rm.a, rm.b) == (ra.kind, ra.sid, ra.a, ra.b)
        if rm.kind == "range":
            got = rm.result.cpu().numpy().view(np.uint16)
            assert np.array_equal(got, src[rm.sid][rm.a:rm.b])
            assert torch.equal(rm.result, ra.result)
        else:
            k = n_app.get(rm.sid, 0)
            n_app[rm.sid] = k + 1
            ref = oracle_mod.compress(_append_rows(rm.sid, k), forecaster=1)
            for r in (rm, ra):
                got = r.result.buf[:r.result.size].cpu().numpy()
                assert np.array_equal(got, ref)
                assert r.result.row0 == ROWS + 2048 * k
    # the appended shards decode back to their rows through a range request
    from paper_1808_02515_gb300 import serve
    sid = next(s for s in range(N_STREAMS) if len(store_m.streams[s]) > 1)
    codec = store_m.codec
    total = store_m.rows(sid)
    req = serve.Request("range", sid, 0.0, a=ROWS - 100, b=total)
    serve.Server(store_m, n_slots=1).run([req], realtime=False)
    want = np.vstack([src[sid][ROWS - 100:]] + [_append_rows(sid, k) for k in range(n_app[sid])])
    assert np.array_equal(req.result.cpu().numpy().view(np.uint16), want)


def test_consumed_results_are_released(spz, oracle_mod):
    """keep_results=False: every request completes, range rows are dropped
    once served, appends still land as shards with the oracle's bytes."""
    from paper_1808_02515_gb300 import serve
    codec = spz.Codec(0)
    store = serve.ShardStore(codec, D, 16, spz.Opts())
    store.add_streams([_dev(_source(s)) for s in range(N_STREAMS)])
    reqs = serve.poisson_requests(store, 120, rate=20000.0, seed=7, append_frac=0.2, append_rows=2048,
                                  min_len=100, max_len=6000,
                                  append_source=lambda sid, k: _dev(_append_rows(sid, k)))
    stats = serve.Server(store, mem_budget=64 << 20, max_batch=16, n_slots=3).run(reqs, realtime=False,
                                                                                  keep_results=False)
    torch.cuda.synchronize()
    assert stats["requests"] == len(reqs) and all(r.t_done >= 0 for r in reqs)
    n_app = {}
    for r in reqs:
        if r.kind == "range":
            assert r.result is None
        else:
            k = n_app.get(r.sid, 0)
            n_app[r.sid] = k + 1
            got = r.result.buf[:r.result.size].cpu().numpy()
            assert np.array_equal(got, oracle_mod.compress(_append_rows(r.sid, k), forecaster=1))


def test_decompress_ranges_into_matches_tensor_form(spz):
    """The address form of range requests writes what the tensor form
    returns, into outputs placed anywhere in one buffer."""
    codec = spz.Codec(0)
    xs = [_dev(_source(s)) for s in range(3)]
    streams, infos, sizes = [], [], []
    for x in xs:
        buf, size = codec.compress(x, spz.Opts())
        torch.cuda.synchronize()
        n = int(size.item())
        streams.append(buf[:n])
        sizes.append(n)
        infos.append(spz.query(buf[:64].cpu().numpy().tobytes()))
    ranges = [(0, 1000), (1234, 9000), (ROWS - 77, ROWS)]
    want, _ = codec.decompress_ranges(streams, infos, sizes, ranges)
    torch.cuda.synchronize()
    rb = D * 2
    total = sum(b - a for a, b in ranges)
    out = torch.full((total + 3, D), -1, dtype=torch.int16, device="cuda")
    shapes = [(i.rows, i.D, i.w, i.opts) for i in infos]
    dsts, row = [], 1
    for a, b in ranges:
        dsts.append((out.data_ptr() + row * rb, (b - a) * rb))
        row += b - a
    ws = codec.decompress_ranges_into(shapes, [s.data_ptr() for s in streams], sizes, ranges, dsts)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    del ws
    row = 1
    for (a, b), w in zip(ranges, want):
        assert torch.equal(out[row:row + (b - a)], w)
        row += b - a
    assert torch.all(out[0] == -1) and torch.all(out[row:] == -1)
