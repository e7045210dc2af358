"""sprintz_compress_noalloc: compression for callers that cannot allocate
device memory (for example a process whose own pool allocator already holds
all free device memory, or a serving request path that must not let
cudaMalloc/cudaFree synchronize the device). The library keeps this entry
point's scratch in a fixed device array instead of asking for a workspace.

Checked through the C ABI against sprintz_compress on the same input: the
stream bytes and the size must be identical (the codec is integer-exact), on
two calls in a row, so that scratch left over by one call cannot leak into
the next. This file is collected last so that a failure here comes after
every other test has run; it also passes on its own in a fresh process."""
import ctypes

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


def _workloads():
    from paper_1808_02515_gb300 import synth
    return [
        (synth.sensor_u16((1 << 18) + 3, 8, seed=21), dict(forecaster=1)),
        (synth.random_walk_u8(200_000 + 5, 3, scale=1.5, const_frac=0.3, seed=22),
         dict(forecaster=0, group_blocks=3)),
        (synth.uniform(5000, 40, 8, seed=23), dict(forecaster=1, chunk_rows=256)),
        (synth.sensor_u16(50_000 + 2, 4, seed=24), dict(forecaster=3)),
        (synth.random_walk_u8(60_000 + 1, 5, scale=2.0, const_frac=0.2, seed=25), dict(forecaster=2)),
    ]


def _dev(x):
    return torch.from_numpy(x.view(np.int16) if x.dtype == np.uint16 else x).cuda()


def test_noalloc_matches_compress_on_two_calls(spz, oracle_mod):
    codec = spz.Codec(0)
    try:
        for x, o in _workloads():
            full = dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024, huff_chunks=64)
            full.update(o)
            oracle_bytes = oracle_mod.compress(x, **full)
            opts = spz.Opts(**o)
            xt = _dev(x)
            ref, ref_size = codec.compress(xt, opts)
            torch.cuda.synchronize()
            assert codec.status() == spz.OK
            n = int(ref_size.item())
            cap = spz.max_compressed_size(x.shape[0], x.shape[1], 8 * x.itemsize, opts)
            for call in range(2):
                dst = torch.full((cap,), 0xA5, dtype=torch.uint8, device="cuda")
                size = torch.full((1,), -1, dtype=torch.int64, device="cuda")
                spz.compress_noalloc(xt, opts, dst, size)
                torch.cuda.synchronize()
                assert int(size.item()) == n, call
                assert torch.equal(dst[:n], ref[:n]), call
                assert n == oracle_bytes.size and np.array_equal(dst[:n].cpu().numpy(), oracle_bytes), call
    finally:
        codec.close()


def test_noalloc_at_its_chunk_limit(spz, oracle_mod):
    """Exactly 65,536 chunks (8-row chunks) is the largest call the fixed
    array holds: accepted, and equal to sprintz_compress and the oracle."""
    from paper_1808_02515_gb300 import synth
    x = synth.random_walk_u8(8 * 65536 + 3, 2, scale=1.5, const_frac=0.3, seed=26)
    opts = spz.Opts(forecaster=1, chunk_rows=8)
    codec = spz.Codec(0)
    try:
        xt = _dev(x)
        ref, ref_size = codec.compress(xt, opts)
        torch.cuda.synchronize()
        assert codec.status() == spz.OK
        n = int(ref_size.item())
        cap = spz.max_compressed_size(x.shape[0], x.shape[1], 8, opts)
        for call in range(2):
            dst = torch.full((cap,), 0x5A, dtype=torch.uint8, device="cuda")
            size = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            spz.compress_noalloc(xt, opts, dst, size)
            torch.cuda.synchronize()
            assert int(size.item()) == n, call
            assert torch.equal(dst[:n], ref[:n]), call
        o = oracle_mod.compress(x, forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=8,
                                huff_chunks=64)
        assert np.array_equal(ref[:n].cpu().numpy(), o)
    finally:
        codec.close()


def test_noalloc_rejects_calls_beyond_its_scratch(spz):
    """More than 65,536 chunks needs more look-back words than the fixed array
    holds: rejected on the host before anything runs."""
    L = spz.lib()
    o = spz.Opts(chunk_rows=8).c()
    rows = 8 * 65537
    dst = torch.empty(1, dtype=torch.uint8, device="cuda")
    rc = L.sprintz_compress_noalloc(ctypes.c_void_p(dst.data_ptr()), rows, 1, 8, ctypes.byref(o),
                                    ctypes.c_void_p(dst.data_ptr()), 1 << 40,
                                    ctypes.c_void_p(dst.data_ptr()), None)
    assert rc == spz.ERR_WS_TOO_SMALL
