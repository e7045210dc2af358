"""Property tests of the oracle: decode(encode(x)) == x over random options,
sizes and data, and corrupt streams that fail cleanly."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


@st.composite
def cases(draw):
    w = draw(st.sampled_from([8, 16]))
    D = draw(st.integers(1, 40))
    rows = draw(st.integers(0, 1500))
    kind = draw(st.sampled_from(["uniform", "walk", "const", "sparse"]))
    seed = draw(st.integers(0, 2**31 - 1))
    opts = dict(forecaster=draw(st.sampled_from([0, 1])),
                huffman=draw(st.sampled_from([0, 1])),
                group_blocks=draw(st.integers(1, 8)),
                learn_shift=draw(st.integers(0, 4)),
                chunk_rows=draw(st.sampled_from([0, 8, 16, 64, 1024])),
                huff_chunks=draw(st.integers(1, 8)))
    return w, D, rows, kind, seed, opts


def make(w, D, rows, kind, seed):
    rng = np.random.default_rng(seed)
    dt = np.uint8 if w == 8 else np.uint16
    if kind == "uniform":
        return rng.integers(0, 1 << w, (rows, D)).astype(dt)
    if kind == "const":
        return np.full((rows, D), rng.integers(0, 1 << w), dtype=dt)
    if kind == "sparse":
        x = np.zeros((rows, D), dtype=np.int64)
        m = rng.random((rows, D)) < 0.02
        x[m] = rng.integers(-3, 4, m.sum())
        return (np.cumsum(x, axis=0) % (1 << w)).astype(dt)
    steps = rng.integers(-5, 6, (rows, D))
    return (np.cumsum(steps, axis=0) % (1 << w)).astype(dt)


@settings(max_examples=300, deadline=None)
@given(cases())
def test_round_trip(oracle_mod, case):
    w, D, rows, kind, seed, opts = case
    x = make(w, D, rows, kind, seed)
    s = oracle_mod.compress(x, **opts)
    assert s.size <= oracle_mod.max_compressed_size(rows, D, w, **opts)
    y = oracle_mod.decompress(s)
    assert y.shape == x.shape and np.array_equal(y, x)


@settings(max_examples=200, deadline=None)
@given(cases(), st.integers(0, 2**31 - 1))
def test_corruption_fails_cleanly(oracle_mod, case, seed):
    """Bit flips and truncations either decode to something or return
    ERR_CORRUPT; they never crash the decoder."""
    w, D, rows, kind, s0, opts = case
    x = make(w, D, max(rows, 8), kind, s0)
    s = oracle_mod.compress(x, **opts).copy()
    rng = np.random.default_rng(seed)
    if rng.random() < 0.3:
        cut = int(rng.integers(0, s.size))
        rc = oracle_mod.decompress_rc(s[:cut])
        assert rc == oracle_mod.ERR_CORRUPT
        return
    for _ in range(int(rng.integers(1, 4))):
        pos = int(rng.integers(0, s.size))
        s[pos] ^= np.uint8(1 << int(rng.integers(0, 8)))
    assert oracle_mod.decompress_rc(s) in (oracle_mod.OK, oracle_mod.ERR_CORRUPT)
