"""Pins of the CPU oracle against facts fixed outside it.

Each test checks one step of the oracle against the paper's worked values,
hand-derived fixtures (tests/golden/streams.json), closed forms, library
routines or brute force, so that a dropped term, a wrong sign or index, or a
transposed operand in the oracle fails at least one of them.
"""
import json
import math
import os
import struct

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "streams.json")


def golden():
    with open(GOLDEN) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# Zigzag (Sec. 4.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("w", [8, 16])
def test_zigzag_bitwise_definition_exhaustive(oracle_mod, w):
    """The oracle's arithmetic zigzag equals the textbook bitwise form
    (e << 1) ^ (e >> (w-1)) on every signed w-bit value, and is a bijection
    onto [0, 2^w)."""
    lo, hi = -(1 << (w - 1)), 1 << (w - 1)
    step = 1 if w == 8 else 37  # all 256 values; a dense stride through 2^16
    es = list(range(lo, hi, step)) + [lo, hi - 1, -1, 0, 1]
    mask = (1 << w) - 1
    for e in es:
        z = ((e << 1) ^ (e >> (w - 1))) & mask
        assert oracle_mod.zigzag(e, w) == z, e
        assert oracle_mod.unzigzag(z, w) == e
    if w == 8:
        zs = sorted(oracle_mod.zigzag(e, 8) for e in range(lo, hi))
        assert zs == list(range(256))


def test_zigzag_paper_statement(oracle_mod):
    """Sec. 4.3: twice |e| for nonnegative e, twice |e| minus one for negative."""
    assert [oracle_mod.zigzag(e, 8) for e in (0, -1, 1, -2, 2, -64, 63)] == [0, 1, 2, 3, 4, 127, 126]


# --------------------------------------------------------------------------
# Bit widths (Sec. 4.3)
# --------------------------------------------------------------------------

def test_bit_length_matches_python(oracle_mod):
    for v in list(range(0, 70000, 7)) + [0, 1, 2, 3, 255, 256, 65535, 1 << 31]:
        assert oracle_mod.bit_length(v) == int(v).bit_length()


def test_width_worked_example(oracle_mod):
    """Sec. 4.3 worked value: largest zigzagged value 16 = 00010000 has three
    leading zeros, so the column needs 8 - 3 = 5 bits."""
    assert oracle_mod.column_width([16, 3, 0, 7, 1, 0, 2, 5], 8) == 5


@pytest.mark.parametrize("w", [8, 16])
def test_width_promotion(oracle_mod, w):
    """Sec. 4.3: width w-1 is stored and decoded as w; every other width is
    the bit length of the OR of the column."""
    assert oracle_mod.column_width([(1 << (w - 1)) - 1] + [0] * 7, w) == w
    assert oracle_mod.column_width([1 << (w - 2)] + [0] * 7, w) == w
    assert oracle_mod.column_width([(1 << (w - 2)) - 1] + [0] * 7, w) == w - 2
    assert oracle_mod.column_width([(1 << w) - 1] + [0] * 7, w) == w
    assert oracle_mod.column_width([0] * 8, w) == 0
    rng = np.random.default_rng(5)
    for _ in range(200):
        z = rng.integers(0, 1 << rng.integers(1, w + 1), 8)
        n = int(np.bitwise_or.reduce(z)).bit_length()
        assert oracle_mod.column_width(z, w) == (w if n == w - 1 else n)


# --------------------------------------------------------------------------
# Delta coding (Sec. 4.2.1)
# --------------------------------------------------------------------------

def test_delta_paper_example(oracle_mod):
    """Sec. 5.7: delta coding {0, -1, 0, 0} gives {0, -1, 1, 0}."""
    x = np.array([0, 255, 0, 0, 0, 0, 0, 0], dtype=np.uint8)
    e = oracle_mod.forecast_errors(x, forecaster=0)[:, 0]
    assert list(e[:4]) == [0, -1, 1, 0]


@pytest.mark.parametrize("w", [8, 16])
def test_delta_is_numpy_diff(oracle_mod, w):
    """Delta errors equal numpy's first difference with x_0 = 0, wrapped to
    w bits; numpy's cumulative sum mod 2^w inverts them."""
    rng = np.random.default_rng(w)
    dt = np.uint8 if w == 8 else np.uint16
    x = rng.integers(0, 1 << w, (64, 5)).astype(dt)
    e = oracle_mod.forecast_errors(x, forecaster=0).astype(np.int64)
    d = np.diff(x.astype(np.int64), axis=0, prepend=0)
    wrapped = (d + (1 << (w - 1))) % (1 << w) - (1 << (w - 1))
    assert np.array_equal(e, wrapped)
    assert np.array_equal(np.cumsum(e, axis=0) % (1 << w), x.astype(np.int64))


# --------------------------------------------------------------------------
# FIRE (Sec. 4.2.2, Algorithm 3)
# --------------------------------------------------------------------------

def _wrap(v, w):
    return (v + (1 << (w - 1))) % (1 << w) - (1 << (w - 1))


@pytest.mark.parametrize("w", [8, 16])
def test_fire_without_learning_is_delta(oracle_mod, w):
    """alpha = 0 (learning disabled) predicts the previous sample: FIRE's
    errors equal delta coding's (Sec. 4.2.2: a = 1, b = 0 is delta coding)."""
    rng = np.random.default_rng(1)
    dt = np.uint8 if w == 8 else np.uint16
    x = rng.integers(0, 1 << w, (128, 3)).astype(dt)
    e_fire = oracle_mod.forecast_errors(x, forecaster=1, test_mode=1)
    e_delta = oracle_mod.forecast_errors(x, forecaster=0)
    assert np.array_equal(e_fire, e_delta)


@pytest.mark.parametrize("w", [8, 16])
def test_fire_alpha_one_is_double_delta(oracle_mod, w):
    """alpha = 2^w (1.0 in fixed point) predicts x_{i-1} + delta_{i-1}: the
    errors are second differences (Sec. 4.2.2: a = 2, b = -1)."""
    rng = np.random.default_rng(2)
    dt = np.uint8 if w == 8 else np.uint16
    x = rng.integers(0, 1 << w, (96, 4)).astype(dt)
    e = oracle_mod.forecast_errors(x, forecaster=1, test_mode=2, pinned_alpha=1 << w)
    xi = x.astype(np.int64)
    d1 = _wrap(np.diff(xi, axis=0, prepend=0), w)
    d2 = _wrap(np.diff(d1, axis=0, prepend=0), w)
    assert np.array_equal(e.astype(np.int64), d2)


@pytest.mark.parametrize("w", [8, 16])
def test_fire_alpha_minus_half_is_mean_of_two(oracle_mod, w):
    """alpha = -2^(w-1) (-1/2) predicts x_{i-1} - floor(delta_{i-1} / 2), i.e.
    the mean of the previous two samples (Sec. 4.2.2: a = b = 1/2)."""
    rng = np.random.default_rng(3)
    dt = np.uint8 if w == 8 else np.uint16
    x = rng.integers(0, 1 << w, (64, 2)).astype(dt)
    e = oracle_mod.forecast_errors(x, forecaster=1, test_mode=2, pinned_alpha=-(1 << (w - 1)))
    xi = x.astype(np.int64)
    prev = np.vstack([np.zeros((1, 2), np.int64), xi[:-1]])
    d1 = _wrap(np.diff(xi, axis=0, prepend=0), w)
    dprev = np.vstack([np.zeros((1, 2), np.int64), d1[:-1]])
    xhat = (prev + np.floor_divide(-dprev, 2)) % (1 << w)
    assert np.array_equal(e.astype(np.int64), _wrap(xi - xhat, w))


@pytest.mark.parametrize("trace", golden()["fire_traces"], ids=lambda t: t["name"])
def test_fire_hand_traces(oracle_mod, trace):
    """Hand-traced FIRE blocks (derivations in the golden file)."""
    w, rows = trace["w"], trace["rows"]
    t = np.arange(rows, dtype=np.int64)
    dt = np.uint8 if w == 8 else np.uint16
    x = ((trace["slope"] * (t + 1)) % (1 << w)).astype(dt)
    e = oracle_mod.forecast_errors(x, forecaster=1, learn_shift=trace["learn_shift"])[:, 0]
    expect = np.repeat(np.array(trace["block_errors"]), 8)
    assert np.array_equal(e, expect)
    alpha, acc = oracle_mod.fire_trace(x, learn_shift=trace["learn_shift"])
    assert list(alpha[:, 0]) == trace["block_alpha"]
    assert list(acc[:, 0]) == trace["acc_after"]


@pytest.mark.parametrize("w,slope", [(8, 3), (8, 1), (8, 20), (16, 100), (16, 300)])
def test_fire_linear_series_closed_form(oracle_mod, w, slope):
    """Linear series x_t = c + s t (s > 0, no wrap of the deltas), shift 1.
    From the definitions: while alpha < 2^w the predicted delta is below s, so
    every error is positive and each block adds floor(4s/4) = s to the
    accumulator (block 0 adds floor(3s/4): delta_{-1} = 0); once alpha
    reaches 2^w the error is 0 while alpha < 2^w (1 + 1/s), sign(0) = 0 stops
    learning, and every later error is zero. The trace is checked against
    this closed form, not assumed."""
    rows = 8 * 2400
    c = 11
    x = ((c + slope * np.arange(rows)) % (1 << w)).astype(np.uint8 if w == 8 else np.uint16)
    alpha, acc = oracle_mod.fire_trace(x, learn_shift=1)
    e = oracle_mod.forecast_errors(x, forecaster=1, learn_shift=1)[:, 0]
    a = 0
    expect_acc, expect_alpha = [], []
    for k in range(rows // 8):
        al = a >> 1
        expect_alpha.append(al)
        pred = (al * slope) >> w
        err = slope - pred
        if k == 0:
            g = 3 * slope * (1 if err > 0 else (-1 if err < 0 else 0))
        else:
            g = 4 * slope * (1 if err > 0 else (-1 if err < 0 else 0))
        a = a + (g >> 2)
        expect_acc.append(a)
    assert list(alpha[:, 0]) == expect_alpha
    assert list(acc[:, 0]) == expect_acc
    # errors become zero after a finite number of blocks and stay zero
    nz = np.nonzero(e[8:])[0]
    last = (nz[-1] + 8) // 8 if nz.size else 0
    assert last < rows // 8 - 1
    assert alpha[last + 1, 0] >= (1 << w)


@pytest.mark.parametrize("fc", [0, 1])
def test_constant_series_one_run_per_chunk(oracle_mod, fc):
    """Sec. 4.2.1: delta gives zero errors exactly when the data is constant;
    FIRE with alpha = 0 in the first block predicts the constant from row 1 on
    and never learns (sign(0) = 0). So each chunk is its first block plus one
    run record of the remaining blocks."""
    x = np.full((4096, 2), 77, dtype=np.uint8)
    s = oracle_mod.compress(x, forecaster=fc, chunk_rows=1024)
    n_chunks = 4
    for c in range(n_chunks):
        off, nrec, packed = struct.unpack_from("<QII", s, 64 + 16 * c)
        assert nrec == 2
        # header of the group: 2 slots x 2 columns x 3 bits -> 2 bytes;
        # block 0: zigzag(77) = 154 -> 8 bits per column -> 16 bytes; run: 2 bytes
        assert packed == 2 + 16 + 2
    assert np.array_equal(oracle_mod.decompress(s), x)


# --------------------------------------------------------------------------
# Whole streams, hand-derived (tests/golden/streams.json)
# --------------------------------------------------------------------------

HEADER_FMT = "<4sBBBBHBBIIIQIIQQQ"


@pytest.mark.parametrize("case", golden()["streams"], ids=lambda c: c["name"])
def test_golden_streams(oracle_mod, case):
    w, D, o, h = case["w"], case["D"], case["opts"], case["header"]
    x = np.array(case["x"], dtype=np.uint8 if w == 8 else np.uint16).reshape(-1, D)
    header = struct.pack(HEADER_FMT, b"SPZ1", 1, w, o["forecaster"], o["huffman"], D,
                         o["group_blocks"], o["learn_shift"], o["chunk_rows"],
                         h["huff_chunks_field"], h["n_chunks"], h["rows"], h["tail_rows"], 0,
                         h["data_off"], h["tail_off"], h["total"])
    assert len(header) == 64
    table = b"".join(struct.pack("<QII", *e) for e in case["chunks"])
    expect = header + table + bytes.fromhex(case["body_hex"]) + bytes.fromhex(case["tail_hex"])
    got = oracle_mod.compress(x, **o).tobytes()
    assert got.hex() == expect.hex()
    assert np.array_equal(oracle_mod.decompress(np.frombuffer(expect, np.uint8)), x)


# --------------------------------------------------------------------------
# Stream sizes from an independent size model (records, groups, layouts)
# --------------------------------------------------------------------------

def _size_model(err, D, w, G, chunk_rows):
    """Per chunk (n_records, packed_bytes) computed from the errors alone with
    numpy: zigzag by the bitwise form, widths by Python bit_length, runs of
    all-zero blocks, ceil(G*D*log2(w)/8)-byte group headers, column-major
    payload sum(n_j) bytes when D*w <= 32 else 8*ceil(sum(n_j)/8), 2 bytes per
    run record."""
    hb = 3 if w == 8 else 4
    hdr = -(-G * D * hb // 8)
    z = ((err.astype(np.int64) << 1) ^ (err.astype(np.int64) >> (w - 1))) & ((1 << w) - 1)
    rows = err.shape[0]
    out = []
    cr = chunk_rows or rows
    for c0 in range(0, rows, cr):
        blocks = z[c0:c0 + cr].reshape(-1, 8, D)
        ors = np.bitwise_or.reduce(blocks, axis=1)
        widths = np.array([[int(v).bit_length() for v in row] for row in ors])
        widths[widths == w - 1] = w
        recs = []
        run = 0
        for b in range(blocks.shape[0]):
            if widths[b].sum() == 0:
                run += 1
                if run == 65535:
                    recs.append(2)
                    run = 0
                continue
            if run:
                recs.append(2)
                run = 0
            s = int(widths[b].sum())
            recs.append(s if D * w <= 32 else 8 * (-(-s // 8)))
        if run:
            recs.append(2)
        n_groups = -(-len(recs) // G)
        out.append((len(recs), n_groups * hdr + sum(recs)))
    return out


@pytest.mark.parametrize("D,w,fc,G,cr", [(1, 8, 0, 2, 1024), (3, 8, 1, 2, 1024),
                                         (4, 8, 0, 3, 64), (5, 8, 1, 2, 256),
                                         (2, 16, 0, 2, 1024), (8, 16, 1, 2, 1024),
                                         (3, 16, 1, 8, 128), (16, 16, 0, 1, 0),
                                         (3, 8, 2, 2, 1024), (8, 16, 2, 4, 512),
                                         (4, 8, 3, 2, 256), (8, 16, 3, 2, 1024)])
def test_sizes_match_independent_model(oracle_mod, D, w, fc, G, cr):
    from paper_1808_02515_gb300 import synth
    rows = 4096
    if w == 8:
        x = synth.random_walk_u8(rows, D, scale=1.5, const_frac=0.3, seed=D)
    else:
        x = synth.sensor_u16(rows, D, seed=D, flat_frac=0.2)
    s = oracle_mod.compress(x, forecaster=fc, group_blocks=G, chunk_rows=cr)
    err_chunks = []
    crr = cr or rows
    for c0 in range(0, rows, crr):
        err_chunks.append(oracle_mod.forecast_errors(x[c0:c0 + crr], forecaster=fc))
    err = np.vstack(err_chunks)
    model = _size_model(err, D, w, G, cr)
    n_chunks = struct.unpack_from("<I", s, 20)[0]
    assert n_chunks == len(model)
    for c, (nrec, packed) in enumerate(model):
        _, got_nrec, got_packed = struct.unpack_from("<QII", s, 64 + 16 * c)
        assert (got_nrec, got_packed) == (nrec, packed), c
    assert s.size == 64 + 16 * n_chunks + sum(p for _, p in model)


def test_column_major_payload_is_sum_of_widths(oracle_mod):
    """Sec. 4.3: with column-major packing each column's 8 values fill
    exactly n_j bytes (no padding), for every width 0..w."""
    seen = set()
    for v in range(0, 256, 3):
        x = np.array([[0], [v], [0], [v], [0], [v], [0], [v]], dtype=np.uint8)
        s = oracle_mod.compress(x, forecaster=0)
        _, nrec, packed = struct.unpack_from("<QII", s, 64)
        err = oracle_mod.forecast_errors(x, forecaster=0)[:, 0]
        width = oracle_mod.column_width([oracle_mod.zigzag(int(e), 8) for e in err], 8)
        seen.add(width)
        assert nrec == 1
        assert packed == (1 + width if width else 1 + 2)
    assert seen == {0, 2, 3, 4, 5, 6, 8}
