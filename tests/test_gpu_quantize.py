"""GPU parity of the float quantization of Sec. 5.8: column extremes, codes
and rebuilt floats equal the oracle's bit for bit (both sides compute in
double with every operation rounded on its own); the normalized errors agree
to a relative 1e-9 (their sums are taken in another order); quantized data
then round-trips through the codec."""
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


def _floats(rows, D, seed):
    rng = np.random.default_rng(seed)
    x = np.cumsum(rng.standard_normal((rows, D)), axis=0) * (10.0 ** rng.integers(-3, 4, D))
    x[:, 0] = np.sin(np.arange(rows) / 50.0) + 0.01 * rng.standard_normal(rows)
    if D > 2:
        x[:, 2] = 7.25  # a constant column
    return x.astype(np.float32)


@pytest.mark.parametrize("w", [8, 16])
@pytest.mark.parametrize("rows,D", [(1, 1), (1000, 3), (100_003, 8), (4096, 300), (777, 1024)])
def test_quantize_parity(codec, oracle_mod, w, rows, D):
    x = _floats(rows, D, seed=rows + D + w)
    q_ref, lh_ref = oracle_mod.quantize(x, w)
    q, lh = codec.quantize(torch.from_numpy(x).cuda(), w)
    torch.cuda.synchronize()
    assert np.array_equal(lh.cpu().numpy().reshape(-1), lh_ref)
    qh = q.cpu().numpy()
    if w == 16:
        qh = qh.view(np.uint16)
    assert np.array_equal(qh, q_ref)
    y = codec.dequantize(q, lh)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), oracle_mod.dequantize(q_ref, lh_ref))
    if rows > 1:
        nm = codec.quant_nmse(torch.from_numpy(x).cuda(), q, lh)
        torch.cuda.synchronize()
        assert np.allclose(nm.cpu().numpy(), oracle_mod.quant_nmse(x, q_ref, lh_ref), rtol=1e-9, atol=1e-300)


def test_quantized_data_round_trips_through_codec(codec):
    import paper_1808_02515_gb300.sprintz as spz
    x = torch.from_numpy(_floats(50_000, 4, seed=3)).cuda()
    q, lh = codec.quantize(x, 16)
    dst, size = codec.compress(q, spz.Opts(forecaster=1))
    info = spz.query(dst[:64].cpu().numpy().tobytes())
    y = codec.decompress(dst, info, src_size=int(size.item()))
    torch.cuda.synchronize()
    assert torch.equal(y.view(q.shape), q)
