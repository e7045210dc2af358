"""Single-stream range decode (sprintz_decompress_rows) and append
(sprintz_append) through the C ABI.

- Any row range decodes to exactly those rows of the source (only the chunks
  that cover it are decoded; Huffman-coded streams are decoded whole first),
  including empty ranges, ranges inside one chunk, across chunks, inside the
  raw tail and across into it.
- Appending rows gives, byte for byte, the oracle's stream of the whole
  series: the old stream's complete chunks are kept, its last partial chunk
  and raw tail rows are decoded and encoded again with the new rows."""
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


def _host(t):
    a = t.cpu().numpy()
    return a.view(np.uint16) if a.dtype == np.int16 else a


def _series(kind, rows, D, seed):
    from paper_1808_02515_gb300 import synth
    if kind == "walk":
        return synth.random_walk_u8(rows, D, scale=1.8, const_frac=0.3, seed=seed)
    if kind == "sensor":
        return synth.sensor_u16(rows, D, seed=seed)
    return synth.uniform(rows, D, 8, seed=seed)


ROW_CASES = [
    ("walk", 9000 + 5, 1, dict(forecaster=0, chunk_rows=1024)),
    ("walk", 7000 + 3, 3, dict(forecaster=1, chunk_rows=64, group_blocks=3)),
    ("sensor", 6000 + 7, 8, dict(forecaster=1, chunk_rows=1024)),
    ("sensor", 5000 + 1, 16, dict(forecaster=3, chunk_rows=256)),
    ("walk", 3000 + 6, 40, dict(forecaster=2, chunk_rows=512)),
    ("sensor", 4000 + 2, 5, dict(forecaster=1, chunk_rows=0)),
    ("walk", 20000 + 4, 3, dict(forecaster=1, huffman=1, huff_chunks=4, chunk_rows=1024)),
    ("walk", 6, 2, dict(forecaster=1)),
]


@pytest.mark.parametrize("kind,rows,D,o", ROW_CASES)
def test_decompress_rows(codec, kind, rows, D, o):
    import paper_1808_02515_gb300.sprintz as spz
    x = _series(kind, rows, D, seed=rows + D)
    opts = spz.Opts(**o)
    dst, size = codec.compress(_dev(x), opts)
    n = int(size.item())
    info = spz.query(dst[:64].cpu().numpy().tobytes())
    cr = o.get("chunk_rows", 1024) or rows
    full = rows - rows % 8
    rng = np.random.default_rng(rows)
    ranges = [(0, rows), (0, 0), (rows, rows), (rows - 1, rows), (0, 1), (full, rows),
              (max(0, full - 3), rows), (min(cr, rows) - 1, min(cr + 9, rows)),
              (3, 3 + min(cr, rows - 3) // 2)]
    for _ in range(8):
        a = int(rng.integers(0, rows))
        b = int(rng.integers(a, rows + 1))
        ranges.append((a, b))
    for a, b in ranges:
        y = codec.decompress_rows(dst, info, a, b, src_size=n)
        torch.cuda.synchronize()
        assert codec.status() == spz.OK, (a, b)
        assert np.array_equal(_host(y).reshape(b - a, D), x[a:b]), (a, b)


def test_decompress_rows_rejects_bad_ranges(codec):
    import paper_1808_02515_gb300.sprintz as spz
    x = _series("walk", 1000, 2, seed=1)
    dst, size = codec.compress(_dev(x), spz.Opts())
    info = spz.query(dst[:64].cpu().numpy().tobytes())
    with pytest.raises(spz.SprintzError) as e:
        codec.decompress_rows(dst, info, 10, 1001)
    assert e.value.code == spz.ERR_INVALID_ARG


APPEND_CASES = [
    # kind, old rows, new rows, D, options
    ("sensor", 3 * 1024, 8192, 4, dict(forecaster=1)),            # old ends on a chunk boundary
    ("sensor", 3 * 1024 + 500, 8192 + 3, 4, dict(forecaster=1)),  # partial last chunk, ragged new rows
    ("walk", 2 * 1024 + 13, 5, 3, dict(forecaster=0)),            # old and new rows end in tails
    ("walk", 700, 900, 1, dict(forecaster=2, chunk_rows=256)),
    ("sensor", 1500 + 4, 2500 + 1, 16, dict(forecaster=3, chunk_rows=512, group_blocks=4)),
    ("walk", 2000 + 1, 3000 + 2, 40, dict(forecaster=1, chunk_rows=256)),  # the wide (D > 32) decoder
    ("sensor", 1000 + 3, 2000, 2, dict(forecaster=1, chunk_rows=0)),       # one chunk: all re-encoded
    ("walk", 0, 4096 + 7, 2, dict(forecaster=1)),                           # empty old stream
    ("walk", 5, 3, 2, dict(forecaster=1)),                                  # tails only
    ("sensor", 4096 + 9, 0, 8, dict(forecaster=1)),                         # nothing appended
]


@pytest.mark.parametrize("kind,old_rows,new_rows,D,o", APPEND_CASES)
def test_append_equals_oracle_of_the_whole(codec, oracle_mod, kind, old_rows, new_rows, D, o):
    import paper_1808_02515_gb300.sprintz as spz
    whole = _series(kind, old_rows + new_rows, D, seed=old_rows * 7 + new_rows)
    x, y = whole[:old_rows], whole[old_rows:]
    full = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
    full.update(o)
    opts = spz.Opts(**full)
    old = oracle_mod.compress(x, **full)
    src = torch.from_numpy(old).cuda()
    info = spz.query(old[:64].tobytes())
    dst, size = codec.append(src, info, _dev(y).view(-1, D) if new_rows else _dev(y).view(0, D))
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    n = int(size.item())
    ref = oracle_mod.compress(whole, **full)
    assert n == ref.size and np.array_equal(dst[:n].cpu().numpy(), ref)
    # and the result decodes back to the whole series
    info2 = spz.query(ref[:64].tobytes())
    back = codec.decompress(dst, info2, src_size=n)
    torch.cuda.synchronize()
    assert np.array_equal(_host(back).reshape(whole.shape), whole)
    assert opts.chunk_rows == full["chunk_rows"]


def test_append_chain_and_huffman_refused(codec, oracle_mod):
    """Three appends in a row equal the oracle's stream of everything; a
    Huffman-coded stream is refused."""
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import synth
    parts = [synth.sensor_u16(r, 4, seed=60 + k) for k, r in enumerate((2000 + 3, 1024, 777, 8192))]
    full = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
    s = torch.from_numpy(oracle_mod.compress(parts[0], **full)).cuda()
    n = s.numel()
    for k in range(1, len(parts)):
        info = spz.query(s[:64].cpu().numpy().tobytes())
        s, size = codec.append(s, info, _dev(parts[k]), src_size=n)
        torch.cuda.synchronize()
        assert codec.status() == spz.OK
        n = int(size.item())
        ref = oracle_mod.compress(np.vstack(parts[:k + 1]), **full)
        assert np.array_equal(s[:n].cpu().numpy(), ref), k
    h = oracle_mod.compress(parts[0], **{**full, "huffman": 1, "huff_chunks": 2})
    info = spz.query(h[:64].tobytes())
    with pytest.raises(spz.SprintzError) as e:
        codec.append(torch.from_numpy(h).cuda(), info, _dev(parts[1]))
    assert e.value.code == spz.ERR_UNSUPPORTED
