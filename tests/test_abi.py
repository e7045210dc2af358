"""The C-ABI library builds, loads and exports every entry point that
include/sprintz_gb300.h declares; its host-only logic (sizes, header
parsing, argument checks) agrees with the oracle. No GPU compute here."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sprintz_gb300.h")


@pytest.fixture(scope="module")
def spz():
    from paper_1808_02515_gb300 import _build
    _build.build()
    import paper_1808_02515_gb300.sprintz as spz
    return spz


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sprintz_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(spz):
    names = declared_functions()
    assert len(names) >= 10
    L = spz.lib()
    for n in names:
        assert hasattr(L, n), n
        assert ctypes.cast(getattr(L, n), ctypes.c_void_p).value


def test_strerror(spz):
    assert spz.strerror(0) == "ok"
    assert "corrupt" in spz.strerror(spz.ERR_CORRUPT)


@pytest.mark.parametrize("rows,D,w,opts", [
    (0, 1, 8, {}), (7, 3, 16, {}), (8, 1, 8, {}), (100_000, 1, 8, dict(forecaster=0)),
    (100_003, 5, 16, dict(chunk_rows=64)), (4096, 16, 16, dict(chunk_rows=0)),
    (12345, 33, 8, dict(group_blocks=5)), (1 << 16, 3, 8, dict(huffman=1, huff_chunks=7)),
    (999, 1024, 16, dict(group_blocks=1, chunk_rows=8)),
])
def test_max_size_matches_oracle(spz, oracle_mod, rows, D, w, opts):
    full = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024,
                huff_chunks=64)
    full.update(opts)
    assert spz.max_compressed_size(rows, D, w, spz.Opts(**full)) == \
        oracle_mod.max_compressed_size(rows, D, w, **full)


def test_huffman_body_limit(spz, oracle_mod):
    """With Huffman a chunk body may not exceed 2^31 bytes (its sub-block
    offsets are u32): one chunk of 2^23 rows x 128 u16 columns (a 2 GiB body)
    is valid plain and rejected with Huffman, by both sides alike."""
    rows, D, w = 1 << 23, 128, 16
    for huff in (0, 1):
        o = dict(forecaster=1, huffman=huff, group_blocks=2, learn_shift=1, chunk_rows=0, huff_chunks=1)
        ours = spz.max_compressed_size(rows, D, w, spz.Opts(**o))
        assert ours == oracle_mod.max_compressed_size(rows, D, w, **o)
        assert (ours == 0) == (huff == 1)


def test_invalid_options_rejected(spz):
    bad = [dict(group_blocks=0), dict(group_blocks=9), dict(chunk_rows=12), dict(learn_shift=16),
           dict(forecaster=4), dict(huffman=1, huff_chunks=0)]
    for b in bad:
        assert spz.max_compressed_size(100, 4, 8, spz.Opts(**b)) == 0, b
    assert spz.max_compressed_size(100, 0, 8, spz.Opts()) == 0
    assert spz.max_compressed_size(100, 1025, 8, spz.Opts()) == 0
    assert spz.max_compressed_size(100, 4, 12, spz.Opts()) == 0


def test_query_parses_oracle_header(spz, oracle_mod):
    from paper_1808_02515_gb300 import synth
    x = synth.sensor_u16(5000 + 5, 3, seed=4)
    s = oracle_mod.compress(x, forecaster=1, group_blocks=3, chunk_rows=512)
    info = spz.query(s[:64].tobytes())
    q = oracle_mod.query(s)
    assert (info.rows, info.D, info.w) == (q["rows"], q["D"], q["w"])
    assert info.opts == spz.Opts(forecaster=1, huffman=0, group_blocks=3, learn_shift=1,
                                 chunk_rows=512, huff_chunks=0)
    assert info.n_chunks == -(-5000 // 512) and info.tail_rows == 5
    assert info.total_bytes == s.size
    bad = s[:64].copy()
    bad[0] ^= 1
    with pytest.raises(spz.SprintzError) as e:
        spz.query(bad.tobytes())
    assert e.value.code == spz.ERR_CORRUPT
    with pytest.raises(spz.SprintzError):
        spz.query(s[:63].tobytes())


def test_null_arguments_rejected_without_gpu(spz):
    L = spz.lib()
    o = spz.Opts().c()
    rc = L.sprintz_compress(None, None, 8, 1, 8, ctypes.byref(o), None, 0, None, None, 0, None)
    assert rc == spz.ERR_INVALID_ARG
    rc = L.sprintz_decompress(None, None, 0, None, None, 0, None, 0, None)
    assert rc == spz.ERR_INVALID_ARG
    assert L.sprintz_get_status(None, None) == spz.ERR_INVALID_ARG


def test_quant_workspace_size(spz):
    L = spz.lib()
    assert L.sprintz_quant_workspace_size(0) == 0
    assert L.sprintz_quant_workspace_size(1025) == 0
    assert L.sprintz_quant_workspace_size(8) == 256


def test_rows_and_append_host_checks(spz, oracle_mod):
    """Workspace sizes and argument checks of the range decode and append
    calls (host logic only)."""
    from paper_1808_02515_gb300 import synth
    L = spz.lib()
    x = synth.sensor_u16(10 * 1024 + 5, 4, seed=9)
    s = oracle_mod.compress(x, forecaster=1, chunk_rows=1024)
    info = spz.query(s[:64].tobytes())
    ci = info.c()
    rb = 4 * 2
    # rows [1500, 3000) are covered by chunks 1 and 2: 2048 rows decoded
    assert L.sprintz_decompress_rows_workspace_size(ctypes.byref(ci), 1500, 3000) == 2048 * rb
    # rows in the raw tail need no chunk decoded
    assert L.sprintz_decompress_rows_workspace_size(ctypes.byref(ci), 10 * 1024 + 1, 10 * 1024 + 5) == 0
    assert L.sprintz_decompress_rows_workspace_size(ctypes.byref(ci), 0, 10 * 1024 + 6) == 0  # past the end
    assert L.sprintz_append_workspace_size(ctypes.byref(ci), 8192) > 0
    h = oracle_mod.compress(x, forecaster=1, huffman=1, huff_chunks=2)
    hi = spz.query(h[:64].tobytes()).c()
    assert L.sprintz_append_workspace_size(ctypes.byref(hi), 8192) == 0
    assert L.sprintz_decompress_rows_workspace_size(ctypes.byref(hi), 0, 10) >= x.nbytes
    # null context / stream / info
    assert L.sprintz_decompress_rows(None, None, 0, None, 0, 1, None, 0, None, 0, None) == spz.ERR_INVALID_ARG
    assert L.sprintz_append(None, None, 0, None, None, 0, None, 0, None, None, 0, None) == spz.ERR_INVALID_ARG
    assert L.sprintz_ctx_set_failure_test(None, 0, 0) == spz.ERR_INVALID_ARG
