"""Pins of the oracle's two further forecasters against facts fixed outside it.

Forecaster 2 is double-delta coding, the a = 2, b = -1 member of the
autoregressive family of Sec. 4.2.2 (predict x_{i-1} + delta_{i-1}).
Forecaster 3 is FIRE in its per-sample form (Algorithm 3 without the practical
changes of Sec. 4.2.2): alpha derived from the
accumulator and one gradient step at every sample, instead of the block form
(alpha per block, one averaged update from every other sample) that Sec. 4.2.2
says is used in practice and that forecaster 1 implements.
"""
import numpy as np
import pytest


def _wrap(v, w):
    return (v + (1 << (w - 1))) % (1 << w) - (1 << (w - 1))


def _dtype(w):
    return np.uint8 if w == 8 else np.uint16


# --------------------------------------------------------------------------
# Double delta
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", [8, 16])
def test_double_delta_is_second_difference(oracle_mod, w):
    """Errors are numpy's second difference of the series preceded by two
    zero samples, wrapped to w bits."""
    rng = np.random.default_rng(20 + w)
    x = rng.integers(0, 1 << w, (200, 3)).astype(_dtype(w))
    e = oracle_mod.forecast_errors(x, forecaster=2).astype(np.int64)
    xi = np.vstack([np.zeros((2, 3), np.int64), x.astype(np.int64)])
    d2 = _wrap(np.diff(xi, n=2, axis=0), w)
    assert np.array_equal(e, d2)


@pytest.mark.parametrize("w", [8, 16])
def test_double_delta_equals_fire_with_alpha_one(oracle_mod, w):
    """FIRE with alpha pinned to 2^w (1.0) predicts the same delta."""
    rng = np.random.default_rng(30 + w)
    x = rng.integers(0, 1 << w, (96, 2)).astype(_dtype(w))
    e2 = oracle_mod.forecast_errors(x, forecaster=2)
    e1 = oracle_mod.forecast_errors(x, forecaster=1, test_mode=2, pinned_alpha=1 << w)
    assert np.array_equal(e2, e1)


@pytest.mark.parametrize("w,slope", [(8, 7), (8, 200), (16, 12345)])
def test_double_delta_ramp(oracle_mod, w, slope):
    """A wrapping ramp x_t = c + s t: e_0 = c, e_1 = s - c, then zero."""
    c = 5
    t = np.arange(64, dtype=np.int64)
    x = ((c + slope * t) % (1 << w)).astype(_dtype(w))
    e = oracle_mod.forecast_errors(x, forecaster=2)[:, 0].astype(np.int64)
    assert e[0] == _wrap(c, w) and e[1] == _wrap(slope - c, w)
    assert not e[2:].any()


# --------------------------------------------------------------------------
# FIRE per sample (Algorithm 3's per-sample form)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", [8, 16])
def test_fire_sample_constant_series(oracle_mod, w):
    """A constant c: e_0 = c (the state starts at zero); the gradient of
    sample 0 uses delta_{-1} = 0, so alpha stays 0 and x_1 is predicted
    exactly; from then on every delta is 0, so every prediction is exact."""
    c = 77 if w == 8 else 40000
    x = np.full((160, 2), c, dtype=_dtype(w))
    e = oracle_mod.forecast_errors(x, forecaster=3).astype(np.int64)
    assert (e[0] == _wrap(c, w)).all()
    assert not e[1:].any()


@pytest.mark.parametrize("w", [8, 16])
def test_fire_sample_starts_as_delta(oracle_mod, w):
    """The first two errors are delta coding's: sample 0's gradient is
    -sign(e_0) * delta_{-1} = 0, so alpha is still 0 at sample 1."""
    rng = np.random.default_rng(40 + w)
    x = rng.integers(0, 1 << w, (64, 4)).astype(_dtype(w))
    e3 = oracle_mod.forecast_errors(x, forecaster=3)
    e0 = oracle_mod.forecast_errors(x, forecaster=0)
    assert np.array_equal(e3[:2], e0[:2])
    assert not np.array_equal(e3, e0)


@pytest.mark.parametrize("w,slope,shift", [(8, 3, 1), (8, 9, 1), (16, 100, 1), (16, 250, 1), (16, 40, 2)])
def test_fire_sample_ramp_closed_form(oracle_mod, w, slope, shift):
    """x_t = c + s t (mod 2^w) with small s > 0: every delta after the first
    is s whether or not x wraps. From the definitions:
    e_0 = c, delta_0 = c; e_1 = s (alpha 0) and the accumulator becomes
    sign(s) * c = c; from sample 2 on every delta is s, so with
    alpha_t = acc >> shift the error is s - floor(alpha_t s / 2^w) and the
    accumulator moves by sign(error) * s. Once alpha reaches the window
    [2^w, 2^w (1 + 1/s)) the error is 0, sign(0) = 0 stops the updates, and
    every later error stays 0 (the ramp is learned as double delta)."""
    c = 2
    rows = 8 * 1200
    x = ((c + slope * np.arange(rows)) % (1 << w)).astype(_dtype(w))
    e = oracle_mod.forecast_errors(x, forecaster=3, learn_shift=shift)[:, 0].astype(np.int64)
    expect = [c, slope]
    acc = c
    for _ in range(2, rows):
        alpha = acc >> shift
        err = slope - ((alpha * slope) >> w)
        expect.append(err)
        acc += (1 if err > 0 else (-1 if err < 0 else 0)) * slope
    assert list(e) == expect
    nz = np.nonzero(e)[0]
    assert nz[-1] < rows - 8


def test_fire_sample_columns_are_independent(oracle_mod):
    """Each column's errors depend on that column alone."""
    rng = np.random.default_rng(50)
    x = np.cumsum(rng.integers(-3, 4, (256, 3)), axis=0).astype(np.uint16)
    e = oracle_mod.forecast_errors(x, forecaster=3)
    for j in range(3):
        ej = oracle_mod.forecast_errors(np.ascontiguousarray(x[:, j:j + 1]), forecaster=3)
        assert np.array_equal(e[:, j:j + 1], ej)


def test_fire_sample_differs_from_block_form(oracle_mod):
    """On a noisy walk the per-sample updates give different errors than the
    block form (alpha per block, every-other-sample gradients)."""
    rng = np.random.default_rng(51)
    x = np.cumsum(rng.integers(-20, 21, (512, 1)), axis=0).astype(np.uint16)
    assert not np.array_equal(oracle_mod.forecast_errors(x, forecaster=3),
                              oracle_mod.forecast_errors(x, forecaster=1))


# --------------------------------------------------------------------------
# Whole streams
# --------------------------------------------------------------------------

@pytest.mark.parametrize("fc", [2, 3])
@pytest.mark.parametrize("D,w", [(1, 8), (3, 8), (8, 16), (2, 16), (12, 8)])
def test_round_trip_new_forecasters(oracle_mod, fc, D, w):
    from paper_1808_02515_gb300 import synth
    rows = 5000
    if w == 8:
        x = synth.random_walk_u8(rows, D, scale=2.0, const_frac=0.25, seed=D + fc)
    else:
        x = synth.sensor_u16(rows, D, seed=D + fc, flat_frac=0.2)
    s = oracle_mod.compress(x, forecaster=fc, chunk_rows=1024)
    assert np.array_equal(oracle_mod.decompress(s), x)
    assert oracle_mod.query(s)["forecaster"] == fc


def test_forecaster_out_of_range_rejected(oracle_mod):
    x = np.zeros((16, 1), np.uint8)
    with pytest.raises(Exception):
        oracle_mod.compress(x, forecaster=4)


# --------------------------------------------------------------------------
# The forecast step alone and its inverse (the FIRE Speed subroutines)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", [8, 16])
def test_reconstruct_delta_is_cumsum(oracle_mod, w):
    """Delta's inverse is numpy's cumulative sum mod 2^w."""
    rng = np.random.default_rng(60 + w)
    e = rng.integers(-(1 << (w - 1)), 1 << (w - 1), (96, 3))
    x = oracle_mod.forecast_reconstruct(e, w, forecaster=0)
    assert np.array_equal(x.astype(np.int64), np.cumsum(e, axis=0) % (1 << w))


@pytest.mark.parametrize("w", [8, 16])
def test_reconstruct_double_delta_is_double_cumsum(oracle_mod, w):
    rng = np.random.default_rng(70 + w)
    e = rng.integers(-(1 << (w - 1)), 1 << (w - 1), (96, 2))
    x = oracle_mod.forecast_reconstruct(e, w, forecaster=2)
    assert np.array_equal(x.astype(np.int64), np.cumsum(np.cumsum(e, axis=0), axis=0) % (1 << w))


@pytest.mark.parametrize("fc", [0, 1, 2, 3])
@pytest.mark.parametrize("w", [8, 16])
def test_transform_round_trip(oracle_mod, fc, w):
    """Chunked transform and inverse undo each other, tail rows included."""
    rng = np.random.default_rng(80 + fc + w)
    x = rng.integers(0, 1 << w, (1000 + 5, 3)).astype(_dtype(w))
    e = oracle_mod.forecast_transform(x, fc, chunk_rows=256)
    assert np.array_equal(e[1000:], x[1000:])
    assert not np.array_equal(e[:1000], x[:1000])
    assert np.array_equal(oracle_mod.forecast_transform(e, fc, chunk_rows=256, inverse=True), x)
