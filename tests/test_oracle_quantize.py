"""Pins of the oracle's float quantization (Sec. 5.8): each column's minimum
and maximum map linearly to 0 and 2^w - 1 and the result is floored; the
inverse undoes the linear map; the error is reported as MSE over variance."""
import numpy as np
import pytest


@pytest.mark.parametrize("w", [8, 16])
def test_integer_grid_is_identity(oracle_mod, w):
    """Values 0 .. 2^w - 1 already span the code range: the scale is 1 and
    every code equals its value; the inverse returns the values."""
    x = np.arange(1 << w, dtype=np.float32)[::-1].reshape(-1, 1)
    q, lh = oracle_mod.quantize(x, w)
    assert np.array_equal(q[:, 0].astype(np.int64), x[:, 0].astype(np.int64))
    assert list(lh) == [0.0, float((1 << w) - 1)]
    assert np.array_equal(oracle_mod.dequantize(q, lh), x)


@pytest.mark.parametrize("w", [8, 16])
def test_binary_step_grid(oracle_mod, w):
    """x = -3 + k / 4, k = 0 .. 2^w - 1: the scale 4 is exact, so code = k."""
    k = np.arange(1 << w)
    x = (-3.0 + k / 4.0).astype(np.float32).reshape(-1, 1)
    q, lh = oracle_mod.quantize(x, w)
    assert np.array_equal(q[:, 0].astype(np.int64), k)


def test_constant_column(oracle_mod):
    x = np.full((100, 2), 2.5, dtype=np.float32)
    x[:, 1] = np.linspace(-1, 1, 100, dtype=np.float32)
    q, lh = oracle_mod.quantize(x, 8)
    assert not q[:, 0].any()
    assert np.array_equal(oracle_mod.dequantize(q, lh)[:, 0], x[:, 0])
    assert oracle_mod.quant_nmse(x, q, lh)[0] == 0.0


@pytest.mark.parametrize("w", [8, 16])
def test_extremes_monotone_and_error_bound(oracle_mod, w):
    """The minimum gets code 0, the maximum one of the top two codes (the
    scaled maximum may round just below 2^w - 1); codes never decrease as x
    grows; each reconstruction is within one quantization step below x."""
    rng = np.random.default_rng(w)
    x = (rng.standard_normal((5000, 3)) * [1.0, 1e3, 1e-3] + [0.0, 5.0, -2.0]).astype(np.float32)
    q, lh = oracle_mod.quantize(x, w)
    top = (1 << w) - 1
    for j in range(3):
        c = q[:, j].astype(np.int64)
        assert c[np.argmin(x[:, j])] == 0 and c[np.argmax(x[:, j])] >= top - 1
        order = np.argsort(x[:, j], kind="stable")
        assert np.all(np.diff(c[order]) >= 0)
        step = (float(lh[2 * j + 1]) - float(lh[2 * j])) / top
        xh = oracle_mod.dequantize(q, lh)[:, j].astype(np.float64)
        d = x[:, j].astype(np.float64) - xh
        tol = 1e-6 * step + 2.0 ** -23 * np.abs(x[:, j]).max()
        assert d.min() >= -tol and d.max() <= step + tol


def test_nmse_uniform_closed_form(oracle_mod):
    """Uniform data on [0, 1): the floor error is uniform on [0, h) with
    h = 1/255, so MSE ~ h^2 / 3 and the variance ~ 1/12: nmse ~ 4 h^2."""
    rng = np.random.default_rng(11)
    x = rng.random((400_000, 1)).astype(np.float32)
    q, lh = oracle_mod.quantize(x, 8)
    nmse = oracle_mod.quant_nmse(x, q, lh)[0]
    h = (float(lh[1]) - float(lh[0])) / 255
    assert nmse == pytest.approx(4 * h * h, rel=0.03)


def test_nmse_matches_numpy(oracle_mod):
    """The oracle's ratio equals numpy's mean squared error of its own
    reconstruction over numpy's population variance."""
    rng = np.random.default_rng(12)
    x = np.cumsum(rng.standard_normal((20_000, 4)), axis=0).astype(np.float32)
    for w in (8, 16):
        q, lh = oracle_mod.quantize(x, w)
        xh = oracle_mod.dequantize(q, lh).astype(np.float64)
        xd = x.astype(np.float64)
        ref = ((xd - xh) ** 2).mean(axis=0) / xd.var(axis=0)
        assert np.allclose(oracle_mod.quant_nmse(x, q, lh), ref, rtol=1e-9)
