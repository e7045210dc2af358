"""GPU parity: the CUDA codec, called through the C ABI, writes byte-for-byte
the oracle's stream and decodes it bit-exactly (integer work: the bar is
exact equality), over shapes, options and data that span several chunks and
ragged tails, the degenerate cases, and the full-size workloads."""
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


def _spz():
    import paper_1808_02515_gb300.sprintz as spz
    return spz


def to_dev(x):
    if x.dtype == np.uint16:
        x = x.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def roundtrip(codec, oracle_mod, x, **opts):
    spz = _spz()
    full = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024,
                huff_chunks=64)
    full.update(opts)
    o = spz.Opts(**full)
    ref = oracle_mod.compress(x, **full)
    xt = to_dev(x)
    dst, size = codec.compress(xt, o)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    n = int(size.item())
    got = dst[:n].cpu().numpy()
    assert n == ref.size, (n, ref.size)
    if not np.array_equal(got, ref):
        bad = np.nonzero(got != ref)[0]
        raise AssertionError(f"stream differs at {bad[:10]} of {n} bytes")
    info = spz.query(ref[:64].tobytes())
    y = codec.decompress(dst, info, src_size=n)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    yv = y.cpu().numpy()
    if x.dtype == np.uint16:
        yv = yv.view(np.uint16)
    assert np.array_equal(yv.reshape(x.shape), x)
    return ref


def gen(kind, rows, D, w, seed):
    from paper_1808_02515_gb300 import synth
    rng = np.random.default_rng(seed)
    dt = np.uint8 if w == 8 else np.uint16
    if kind == "uniform":
        return synth.uniform(rows, D, w, seed)
    if kind == "const":
        return np.full((rows, D), rng.integers(0, 1 << w), dtype=dt)
    if kind == "walk":
        if w == 8:
            return synth.random_walk_u8(rows, D, scale=1.0 + seed % 3, const_frac=0.3, seed=seed)
        return (np.cumsum(rng.integers(-300, 301, (rows, D)), axis=0) % 65536).astype(dt)
    if kind == "sensor":
        if w == 16:
            return synth.sensor_u16(rows, D, seed=seed, flat_frac=0.2) if rows >= 64 else \
                rng.integers(0, 65536, (rows, D)).astype(dt)
        return synth.accel_u8(rows, D, seed=seed) if rows else np.zeros((0, D), dt)
    if kind == "sparse":
        x = np.zeros((rows, D), dtype=np.int64)
        m = rng.random((rows, D)) < 0.01
        x[m] = rng.integers(-5, 6, m.sum())
        return (np.cumsum(x, axis=0) % (1 << w)).astype(dt)
    raise ValueError(kind)


CASES = []
for w in (8, 16):
    for D in (1, 2, 3, 4, 5, 8, 16, 33):
        for fc in (0, 1):
            for kind in ("walk", "uniform", "sensor", "sparse"):
                CASES.append((kind, 3000 + 8 * D + 5, D, w, fc, 2, 1024))
CASES += [
    ("walk", 0, 1, 8, 0, 2, 1024), ("walk", 5, 3, 16, 1, 2, 1024), ("walk", 8, 1, 8, 1, 2, 1024),
    ("walk", 8 * 1024, 2, 8, 0, 2, 1024), ("walk", 8 * 1024 + 7, 2, 16, 1, 2, 1024),
    ("const", 5000, 4, 8, 0, 2, 1024), ("const", 5000, 4, 16, 1, 2, 1024),
    ("const", 1000, 1, 8, 1, 1, 0), ("walk", 20000, 3, 8, 1, 2, 0), ("sensor", 20000, 2, 16, 1, 2, 0),
    ("walk", 2000, 7, 8, 1, 1, 8), ("walk", 2000, 7, 16, 0, 8, 16), ("sparse", 4000, 5, 16, 1, 3, 64),
    ("uniform", 513, 100, 16, 1, 2, 1024), ("walk", 300, 1024, 16, 1, 2, 1024),
    ("walk", 300, 1024, 8, 0, 7, 64), ("sparse", 4000, 12, 8, 1, 4, 1024),
    ("sensor", 4096, 8, 16, 1, 2, 2048), ("walk", 3000, 3, 16, 1, 5, 3000 // 8 * 8),
]


@pytest.mark.parametrize("kind,rows,D,w,fc,G,cr", CASES)
def test_parity_small(codec, oracle_mod, kind, rows, D, w, fc, G, cr):
    x = gen(kind, rows, D, w, seed=rows + D + w)
    roundtrip(codec, oracle_mod, x, forecaster=fc, group_blocks=G, chunk_rows=cr)


@pytest.mark.parametrize("shift", [0, 1, 3, 7])
def test_parity_learn_shift(codec, oracle_mod, shift):
    x = gen("sensor", 8192 + 3, 4, 16, seed=shift)
    roundtrip(codec, oracle_mod, x, forecaster=1, learn_shift=shift)
    x8 = gen("walk", 8192, 3, 8, seed=shift)
    roundtrip(codec, oracle_mod, x8, forecaster=1, learn_shift=shift)


def test_parity_long_run_split(codec, oracle_mod):
    """A single chunk (chunk_rows = 0) with a zero run longer than 65535
    blocks: the run is cut into records of at most 65535 blocks."""
    x = np.full((8 * 70000 + 3, 1), 9, dtype=np.uint8)
    x[:8, 0] = np.arange(8)
    s = roundtrip(codec, oracle_mod, x, forecaster=0, chunk_rows=0)
    # block 0 (0..7), block 1 (7 -> 9), a run of 65535 blocks, a run of the rest
    assert int.from_bytes(s[64 + 8:64 + 12].tobytes(), "little") == 4


def test_parity_random_walk_100k(codec, oracle_mod):
    """The small single-stream workload: uint8, 1 column, 100,000 rows, delta
    coding, chunk_rows 1024 and a single chunk."""
    from paper_1808_02515_gb300 import synth
    x = synth.random_walk_u8(100_000, 1, scale=2.0, const_frac=0.2, seed=0)
    roundtrip(codec, oracle_mod, x, forecaster=0, chunk_rows=1024)
    roundtrip(codec, oracle_mod, x, forecaster=0, chunk_rows=0)


def test_parity_sensor_full_size(codec, oracle_mod):
    """The headline workload: uint16, 8 columns, 2^24 rows (256 MiB), FIRE,
    in the launch configuration the benchmark times; every byte compared."""
    from paper_1808_02515_gb300 import synth
    x = synth.sensor_u16(1 << 24, 8, seed=1)
    roundtrip(codec, oracle_mod, x, forecaster=1, chunk_rows=1024)


def test_repeat_calls_identical(codec, oracle_mod):
    """The encoder's look-back state is reset per call: two calls in a row
    give identical bytes."""
    spz = _spz()
    x = gen("sensor", 50_000, 8, 16, seed=3)
    xt = to_dev(x)
    d1, s1 = codec.compress(xt, spz.Opts())
    d2, s2 = codec.compress(xt, spz.Opts())
    torch.cuda.synchronize()
    n = int(s1.item())
    assert n == int(s2.item()) and torch.equal(d1[:n], d2[:n])


def _decode_rc(codec, s, src_size=None):
    spz = _spz()
    try:
        inf = spz.query(s[:64].tobytes())
    except spz.SprintzError as e:
        return e.code
    if inf.rows * inf.D > 10_000_000:
        return None
    st = torch.from_numpy(np.ascontiguousarray(s)).cuda()
    codec.decompress(st, inf, src_size=s.size if src_size is None else src_size)
    return codec.status()


@pytest.mark.parametrize("D,w", [(3, 16), (8, 16), (1, 8), (40, 8)])
def test_corrupt_streams_flag_errors(codec, oracle_mod, D, w):
    """Corrupted streams either decode or set ERR_CORRUPT in the device
    status, in agreement with the oracle; the decoder's bounds checks keep
    every access inside the stream. Covers random byte flips, chunk-table
    fields (offset, record count, packed size), zeroed run counts and group
    headers, and a truncated stream size."""
    import struct
    spz = _spz()
    rng = np.random.default_rng(7 + D)
    x = gen("sparse", 4000 + 3, D, w, seed=11)
    ref = oracle_mod.compress(x, forecaster=1, chunk_rows=256)
    info = spz.query(ref[:64].tobytes())
    assert _decode_rc(codec, ref) == spz.OK
    corrupt = 0
    for trial in range(48):
        s = ref.copy()
        kind = trial % 4
        c = int(rng.integers(0, info.n_chunks))
        e = 64 + 16 * c
        if kind == 0:  # random flips anywhere after the header
            for _ in range(int(rng.integers(1, 4))):
                pos = int(rng.integers(64, s.size))
                s[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        elif kind == 1:  # one chunk-table field
            field = int(rng.integers(0, 3))
            off = e + (0, 8, 12)[field]
            s[off + int(rng.integers(0, 2))] ^= np.uint8(1 << int(rng.integers(0, 8)))
        elif kind == 2:  # a chunk's first group header zeroed: records become runs
            body = info.data_off + struct.unpack_from("<Q", s, e)[0]
            hdr = (2 * D * (3 if w == 8 else 4) + 7) // 8
            s[body:body + hdr] = 0
        else:  # a stream shorter than its header says
            rc = _decode_rc(codec, s, src_size=int(rng.integers(info.data_off, s.size)))
            assert rc == spz.ERR_CORRUPT
            corrupt += 1
            continue
        rc = _decode_rc(codec, s)
        if rc is None:
            continue
        assert rc in (spz.OK, spz.ERR_CORRUPT)
        if oracle_mod.decompress_rc(s) == oracle_mod.ERR_CORRUPT:
            assert rc == spz.ERR_CORRUPT, (trial, kind)
        corrupt += rc == spz.ERR_CORRUPT
    assert corrupt >= 12
    assert _decode_rc(codec, ref) == spz.OK
