"""GPU parity of the forecast step alone (sprintz_forecast, the subroutine of
the FIRE Speed experiment): errors and rebuilt samples equal the oracle's
chunk-by-chunk transform bit for bit, for every forecaster, over column
counts 1..80 and beyond, ragged tails, one-chunk streams and in-place calls."""
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


def _host(t, dtype):
    y = t.cpu().numpy()
    return y.view(np.uint16) if dtype == np.uint16 else y


def _data(rows, D, w, seed):
    from paper_1808_02515_gb300 import synth
    if seed % 2:
        return synth.uniform(rows, D, w, seed)
    rng = np.random.default_rng(seed)
    return (np.cumsum(rng.integers(-40, 41, (rows, D)), axis=0) % (1 << w)).astype(
        np.uint8 if w == 8 else np.uint16)


CASES = [(fc, w, D, rows, cr)
         for fc in (0, 1, 2, 3) for w in (8, 16)
         for D, rows, cr in ((1, 5000 + 3, 1024), (3, 2048, 256), (8, 4100, 1024), (17, 999, 64),
                             (40, 1600 + 7, 1024), (80, 1000, 512), (1024, 40, 16))]


@pytest.mark.parametrize("fc,w,D,rows,cr", CASES)
def test_forecast_transform_parity(codec, oracle_mod, fc, w, D, rows, cr):
    x = _data(rows, D, w, seed=fc * 100 + D + w)
    e_ref = oracle_mod.forecast_transform(x, fc, chunk_rows=cr)
    e = codec.forecast(_dev(x), forecaster=fc, chunk_rows=cr)
    torch.cuda.synchronize()
    assert np.array_equal(_host(e, x.dtype), e_ref)
    y = codec.forecast(_dev(e_ref), forecaster=fc, chunk_rows=cr, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(_host(y, x.dtype), x)


@pytest.mark.parametrize("fc", [1, 3])
def test_one_chunk_and_learn_shift(codec, oracle_mod, fc):
    x = _data(3000, 4, 16, seed=7)
    for shift, cr in ((1, 0), (3, 0), (0, 512)):
        e_ref = oracle_mod.forecast_transform(x, fc, learn_shift=shift, chunk_rows=cr)
        e = codec.forecast(_dev(x), forecaster=fc, learn_shift=shift, chunk_rows=cr)
        torch.cuda.synchronize()
        assert np.array_equal(_host(e, x.dtype), e_ref)


def test_in_place(codec, oracle_mod):
    x = _data(4096 + 5, 6, 8, seed=9)
    t = _dev(x)
    codec.forecast(t, forecaster=1, out=t)
    torch.cuda.synchronize()
    assert np.array_equal(_host(t, x.dtype), oracle_mod.forecast_transform(x, 1))
    codec.forecast(t, forecaster=1, inverse=True, out=t)
    torch.cuda.synchronize()
    assert np.array_equal(_host(t, x.dtype), x)


def test_full_size_sample(codec, oracle_mod):
    """100M u8 values as 8 columns (the paper's experiment size): the whole
    output round-trips on the GPU, and sampled chunks equal the oracle."""
    from paper_1808_02515_gb300 import synth
    rows = 100_000_000 // 8
    x = _dev(synth.uniform(rows, 8, 8, seed=5))
    e = codec.forecast(x, forecaster=1)
    y = codec.forecast(e, forecaster=1, inverse=True)
    torch.cuda.synchronize()
    assert torch.equal(x, y)
    xs = x.cpu().numpy()
    es = e.cpu().numpy()
    for c in (0, 77, rows // 1024 - 1):
        part = xs[c * 1024:(c + 1) * 1024]
        assert np.array_equal(es[c * 1024:(c + 1) * 1024], oracle_mod.forecast_transform(part, 1))
