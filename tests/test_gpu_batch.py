"""Batched launches: many independent streams of uneven length, width, D and
options encoded and decoded by one persistent kernel each. Every stream must
equal the oracle's stream for it byte for byte, and decode bit-exactly."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def codec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1808_02515_gb300 import _build
    _build.build()
    import paper_1808_02515_gb300.sprintz as spz
    c = spz.Codec(0)
    yield c
    c.close()


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x.view(np.int16) if x.dtype == np.uint16 else x)).cuda()


def _mixed_streams(n, seed):
    from paper_1808_02515_gb300 import synth
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = k % 5
        if kind == 0:
            x = synth.batch_stream(k, max_rows=12_000, min_rows=100)
        elif kind == 1:
            x = synth.uniform(int(rng.integers(0, 3000)), int(rng.integers(1, 17)),
                              int(rng.choice([8, 16])), seed=k)
        elif kind == 2:
            x = np.full((int(rng.integers(0, 40)), int(rng.integers(1, 9))), k, dtype=np.uint8)
        elif kind == 3:
            x = synth.sensor_u16(int(rng.integers(64, 9000)), int(rng.integers(1, 17)), seed=k)
        else:
            x = synth.random_walk_u8(int(rng.integers(8, 7000)), int(rng.integers(1, 17)),
                                     scale=1.3, const_frac=0.35, seed=k)
        o = dict(forecaster=int(rng.integers(0, 2)), huffman=0,
                 group_blocks=int(rng.choice([1, 2, 2, 3, 8])), learn_shift=int(rng.integers(0, 3)),
                 chunk_rows=int(rng.choice([8, 64, 1024, 1024, 0])), huff_chunks=64)
        out.append((x, o))
    return out


def test_batch_parity(codec, oracle_mod):
    import paper_1808_02515_gb300.sprintz as spz
    streams = _mixed_streams(40, seed=5)
    xs = [_dev(x) for x, _ in streams]
    opts = [spz.Opts(**o) for _, o in streams]
    for rep in range(2):  # a second plan + run on fresh buffers
        bufs, sizes, ws = codec.compress_batch(xs, opts)
        torch.cuda.synchronize()
        assert codec.status() == spz.OK
        sz = sizes.cpu().numpy()
        infos = []
        for k, (x, o) in enumerate(streams):
            ref = oracle_mod.compress(x, **o)
            got = bufs[k][:int(sz[k])].cpu().numpy()
            assert got.size == ref.size and np.array_equal(got, ref), (rep, k, x.shape, o)
            infos.append(spz.query(ref[:64].tobytes()))
        outs, _ = codec.decompress_batch(bufs, infos, [int(v) for v in sz])
        torch.cuda.synchronize()
        assert codec.status() == spz.OK
        for k, (x, _) in enumerate(streams):
            y = outs[k].cpu().numpy()
            if x.dtype == np.uint16:
                y = y.view(np.uint16)
            assert np.array_equal(y.reshape(x.shape), x), (rep, k)


def test_batch_run_repeats(codec, oracle_mod):
    """batch_run on the planned workspace again rewrites the same bytes."""
    import paper_1808_02515_gb300.sprintz as spz
    streams = _mixed_streams(12, seed=9)
    xs = [_dev(x) for x, _ in streams]
    bufs, sizes, ws = codec.compress_batch(xs, [spz.Opts(**o) for _, o in streams])
    torch.cuda.synchronize()
    first = [b.clone() for b in bufs]
    for b in bufs:
        b.fill_(0)
    codec.batch_run(ws)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    sz = sizes.cpu().numpy()
    for k in range(len(bufs)):
        n = int(sz[k])
        assert torch.equal(bufs[k][:n], first[k][:n]), k


def _class_streams():
    """One stream per (w, D) class for D = 1..16 and a few wider ones, with
    every forecaster, ragged lengths and several chunks each."""
    from paper_1808_02515_gb300 import synth
    rng = np.random.default_rng(77)
    out = []
    for D in list(range(1, 17)) + [20, 32]:
        for w in (8, 16):
            rows = int(rng.integers(2500, 9000)) + int(rng.integers(0, 8))
            seed = 1000 + 40 * D + w
            x = (synth.random_walk_u8(rows, D, scale=1.7, const_frac=0.25, seed=seed) if w == 8
                 else synth.sensor_u16(rows, D, seed=seed))
            o = dict(forecaster=(D + w) % 4, huffman=0, group_blocks=int(rng.choice([1, 2, 3, 4])),
                     learn_shift=1, chunk_rows=int(rng.choice([256, 1024])), huff_chunks=64)
            out.append((x, o))
    return out


SCHEDULES = [
    dict(),
    dict(ctas_per_sm=2, order=2, prefetch_bytes=1),
    dict(ctas_per_sm=5, order=3, prefetch_bytes=8192, ring_segments=4),
    dict(ctas_per_sm=1, order=1, prefetch_bytes=1024, ring_segments=2),
]


@pytest.mark.parametrize("sched", SCHEDULES)
def test_batch_every_class_every_schedule(codec, oracle_mod, sched):
    """Every (w, D) specialisation of the batched kernels under several
    schedules (grid size, work order, prefetch, ring depth) writes the
    oracle's bytes and decodes bit-exactly: a schedule changes speed only."""
    import paper_1808_02515_gb300.sprintz as spz
    streams = _class_streams()
    xs = [_dev(x) for x, _ in streams]
    opts = [spz.Opts(**o) for _, o in streams]
    sc = spz.Schedule(**sched)
    bufs, sizes, ws = codec.compress_batch(xs, opts, schedule=sc)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    sz = sizes.cpu().numpy()
    infos = []
    for k, (x, o) in enumerate(streams):
        ref = oracle_mod.compress(x, **o)
        got = bufs[k][:int(sz[k])].cpu().numpy()
        assert got.size == ref.size and np.array_equal(got, ref), (k, x.shape, x.dtype, o)
        infos.append(spz.query(ref[:64].tobytes()))
    outs, _ = codec.decompress_batch(bufs, infos, [int(v) for v in sz], schedule=sc)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    for k, (x, _) in enumerate(streams):
        y = outs[k].cpu().numpy()
        if x.dtype == np.uint16:
            y = y.view(np.uint16)
        assert np.array_equal(y.reshape(x.shape), x), k


def test_batch_autotune_keeps_bytes(codec, oracle_mod):
    """The autotuner runs the batch under its candidate schedules and leaves
    it planned with the fastest; the bytes are the oracle's whichever it
    chose, and the chosen schedule is what the plan reports."""
    import paper_1808_02515_gb300.sprintz as spz
    streams = _class_streams()[::3]
    xs = [_dev(x) for x, _ in streams]
    opts = [spz.Opts(**o) for _, o in streams]
    bufs, sizes, ws = codec.compress_batch(xs, opts, autotune=True)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    chosen, ms = codec.last_tune
    assert ms > 0 and chosen.ctas_per_sm >= 1 and chosen.order in (1, 2, 3)
    assert codec.batch_schedule() == chosen
    for b in bufs:
        b.fill_(0)
    codec.batch_run(ws)
    torch.cuda.synchronize()
    sz = sizes.cpu().numpy()
    infos = []
    for k, (x, o) in enumerate(streams):
        ref = oracle_mod.compress(x, **o)
        got = bufs[k][:int(sz[k])].cpu().numpy()
        assert np.array_equal(got, ref), k
        infos.append(spz.query(ref[:64].tobytes()))
    outs, _ = codec.decompress_batch(bufs, infos, [int(v) for v in sz], autotune=True)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    for k, (x, _) in enumerate(streams):
        y = outs[k].cpu().numpy()
        if x.dtype == np.uint16:
            y = y.view(np.uint16)
        assert np.array_equal(y.reshape(x.shape), x), k
