"""GPU parity of the double-delta forecaster (2) and FIRE per sample (3):
the lane kernels (D <= 32), the per-chunk kernels (D > 32), the batched
launches and the Huffman path all write the oracle's stream byte for byte and
decode it bit-exactly."""
import numpy as np
import pytest

from test_gpu_parity import gen, roundtrip

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


CASES = []
for fc in (2, 3):
    for w in (8, 16):
        for D in (1, 2, 3, 4, 8, 16, 33, 40):
            for kind in ("walk", "sensor", "sparse", "uniform"):
                CASES.append((kind, 2000 + 8 * D + 3, D, w, fc))
    CASES += [("const", 3000, 3, 8, fc), ("walk", 7, 2, 16, fc), ("walk", 0, 1, 8, fc)]


@pytest.mark.parametrize("kind,rows,D,w,fc", CASES)
def test_parity_new_forecasters(codec, oracle_mod, kind, rows, D, w, fc):
    x = gen(kind, rows, D, w, seed=rows + D + 10 * fc)
    roundtrip(codec, oracle_mod, x, forecaster=fc)


@pytest.mark.parametrize("fc", [2, 3])
@pytest.mark.parametrize("shift", [0, 1, 3, 7])
def test_learn_shift(codec, oracle_mod, fc, shift):
    x = gen("sensor", 4096, 4, 16, seed=shift)
    roundtrip(codec, oracle_mod, x, forecaster=fc, learn_shift=shift)


@pytest.mark.parametrize("fc", [2, 3])
def test_options(codec, oracle_mod, fc):
    x = gen("walk", 9000, 5, 8, seed=3)
    roundtrip(codec, oracle_mod, x, forecaster=fc, group_blocks=5, chunk_rows=256)
    roundtrip(codec, oracle_mod, x, forecaster=fc, chunk_rows=0)


@pytest.mark.parametrize("fc", [2, 3])
def test_huffman(codec, oracle_mod, fc):
    from paper_1808_02515_gb300 import synth
    x = synth.accel_u8(40_000, 3, seed=fc)
    roundtrip(codec, oracle_mod, x, forecaster=fc, huffman=1, huff_chunks=8)


@pytest.mark.parametrize("fc", [2, 3])
def test_batch(codec, oracle_mod, fc):
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import synth
    xs = [synth.batch_stream(k, max_rows=6000, min_rows=50) for k in range(24)]
    opts = spz.Opts(forecaster=fc)
    devs = [torch.from_numpy(np.ascontiguousarray(x.view(np.int16) if x.dtype == np.uint16 else x)).cuda()
            for x in xs]
    bufs, sizes, _ = codec.compress_batch(devs, opts)
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    sz = sizes.cpu().numpy()
    for x, buf, n in zip(xs, bufs, sz):
        ref = oracle_mod.compress(x, forecaster=fc)
        assert int(n) == ref.size
        assert np.array_equal(buf[:int(n)].cpu().numpy(), ref)
    infos = [spz.query(b[:64].cpu().numpy().tobytes()) for b in bufs]
    outs, _ = codec.decompress_batch(bufs, infos, [int(n) for n in sz])
    torch.cuda.synchronize()
    assert codec.status() == spz.OK
    for x, y in zip(xs, outs):
        yv = y.cpu().numpy()
        if x.dtype == np.uint16:
            yv = yv.view(np.uint16)
        assert np.array_equal(yv.reshape(x.shape), x)
