"""The Huffman stage (Sec. 4.4, our length-limited canonical code per segment
of chunks): GPU streams equal the oracle's byte for byte, including segments
stored raw, and decode bit-exactly; corrupt tables are flagged."""
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


def _rt(codec, oracle_mod, x, **o):
    import paper_1808_02515_gb300.sprintz as spz
    full = dict(forecaster=1, huffman=1, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
    full.update(o)
    ref = oracle_mod.compress(x, **full)
    xt = torch.from_numpy(np.ascontiguousarray(x.view(np.int16) if x.dtype == np.uint16 else x)).cuda()
    dst, size = codec.compress(xt, spz.Opts(**full))
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    n = int(size.item())
    got = dst[:n].cpu().numpy()
    assert n == ref.size, (n, ref.size)
    if not np.array_equal(got, ref):
        raise AssertionError(f"stream differs at {np.nonzero(got != ref)[0][:10]} of {n}")
    info = spz.query(ref[:64].tobytes())
    y = codec.decompress(dst, info, src_size=n)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    yv = y.cpu().numpy()
    if x.dtype == np.uint16:
        yv = yv.view(np.uint16)
    assert np.array_equal(yv.reshape(x.shape), x)
    return ref


@pytest.mark.parametrize("rows,hc,cr,fc,G", [(1 << 16, 64, 1024, 1, 2), ((1 << 16) + 5, 7, 1024, 1, 2),
                                              (20000, 1, 256, 0, 3), (3000, 3, 64, 1, 1),
                                              (4096, 64, 0, 1, 2), (5, 64, 1024, 1, 2)])
def test_huffman_accel(codec, oracle_mod, rows, hc, cr, fc, G):
    from paper_1808_02515_gb300 import synth
    x = synth.accel_u8(rows, 3, seed=rows % 97) if rows >= 8 else np.arange(15, dtype=np.uint8).reshape(5, 3)
    _rt(codec, oracle_mod, x, huff_chunks=hc, chunk_rows=cr, forecaster=fc, group_blocks=G)


def test_huffman_u16_and_wide(codec, oracle_mod):
    from paper_1808_02515_gb300 import synth
    _rt(codec, oracle_mod, synth.sensor_u16(30000 + 3, 8, seed=2), huff_chunks=5)
    _rt(codec, oracle_mod, synth.random_walk_u8(9000, 40, scale=1.0, seed=3), huff_chunks=4)


@pytest.mark.parametrize("w,D", [(8, 24), (8, 32), (16, 40), (16, 80), (16, 200)])
def test_huffman_large_chunk_bodies(codec, oracle_mod, w, D):
    """Wide rows: a chunk body of up to 400 KB is coded as up to 200
    sub-blocks of 2048 packed bytes behind its jump table."""
    from paper_1808_02515_gb300 import synth
    x = synth.uniform(2048 + 3, D, w, seed=D)
    _rt(codec, oracle_mod, x, huff_chunks=1)
    xs = synth.random_walk_u8(3000, D, scale=3.0, seed=D) if w == 8 else synth.sensor_u16(3000, D, seed=D)
    _rt(codec, oracle_mod, xs, huff_chunks=2)


def test_huffman_raw_segments(codec, oracle_mod):
    """Near-uniform packed bytes: the segments are stored raw (zero tables)."""
    from helpers import flat_bytes_u8
    x = flat_bytes_u8(4096, seed=1)
    ref = _rt(codec, oracle_mod, x, forecaster=0, huff_chunks=16)
    n_chunks = int.from_bytes(ref[20:24].tobytes(), "little")
    base = 64 + 16 * n_chunks
    assert not ref[base:base + 256].any()


def test_huffman_full_size_accel(codec, oracle_mod):
    """The Huffman workload: uint8, D = 3, 2^28 rows (768 MiB), FIRE + bit
    packing + runs + Huffman, every byte compared with the oracle."""
    from paper_1808_02515_gb300 import synth
    x = synth.accel_u8(1 << 28, 3, seed=3)
    _rt(codec, oracle_mod, x)


def test_huffman_corrupt_tables(codec, oracle_mod):
    """Bit flips in the Huffman tables and coded bodies either decode or set
    ERR_CORRUPT, in agreement with the oracle."""
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import synth
    x = synth.accel_u8(20000, 3, seed=8)
    ref = oracle_mod.compress(x, forecaster=1, huffman=1, huff_chunks=4)
    info = spz.query(ref[:64].tobytes())
    rng = np.random.default_rng(4)
    seen = 0
    for trial in range(40):
        s = ref.copy()
        lo = 64 + 16 * info.n_chunks
        pos = int(rng.integers(lo, s.size))
        s[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
        st = torch.from_numpy(s).cuda()
        codec.decompress(st, info, src_size=s.size)
        rc = codec.status()
        assert rc in (spz.OK, spz.ERR_CORRUPT)
        if oracle_mod.decompress_rc(s) == oracle_mod.ERR_CORRUPT:
            assert rc == spz.ERR_CORRUPT, trial
        seen += rc == spz.ERR_CORRUPT
    assert seen >= 5
