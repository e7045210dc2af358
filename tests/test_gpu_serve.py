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
