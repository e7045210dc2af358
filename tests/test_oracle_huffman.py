"""Pins of the oracle's byte Huffman coder (Sec. 4.4; our own length-limited
canonical code in place of Huff0).

Code lengths: Kraft inequality, the length limit, optimality against brute
force over all length vectors on tiny alphabets, and equality with the cost
of an unrestricted Huffman code (heapq construction) when the limit does not
bind. Canonical codes: the worked example of RFC 1951 Sec. 3.2.2.
Container: each chunk's code is split into n = ceil(packed / 2048) sub-blocks
of ceil(packed / n) packed bytes behind a jump table of u32 offsets; a
sub-block decoded on its own, with a bit-by-bit canonical decoder written
here, must give its slice of the packed body and use exactly its bytes.
"""
import heapq
import itertools
import json
import os
import struct

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "streams.json")
SUB = 2048  # packed bytes per Huffman sub-block


def _n_sub(packed):
    return max(1, -(-packed // SUB))


def _sub_slices(body):
    """The n = ceil(len / 2048) equal slices (the last may be shorter)."""
    n = _n_sub(len(body))
    q = -(-len(body) // n)
    return [body[min(len(body), k * q):min(len(body), (k + 1) * q)] for k in range(n)]


def _chunk_coded(body, lengths):
    """Coded bytes of one chunk: the jump table plus each sub-block's bits
    rounded up to a byte."""
    subs = _sub_slices(body)
    return 4 * (len(subs) - 1) + sum(-(-sum(int(lengths[v]) for v in sb) // 8) for sb in subs)


def test_rfc1951_canonical_example(oracle_mod):
    with open(GOLDEN) as f:
        g = json.load(f)["huffman_rfc1951"]
    lengths = np.zeros(256, np.uint8)
    lengths[g["symbols"]] = g["lengths"]
    codes = oracle_mod.huff_canonical(lengths)
    for sym, ln, want in zip(g["symbols"], g["lengths"], g["codes"]):
        assert format(int(codes[sym]), f"0{ln}b") == want


def _cost(freq, lengths):
    return int(sum(int(f) * int(l) for f, l in zip(freq, lengths)))


def _kraft_ok(lengths, L):
    return sum(1 << (L - int(l)) for l in lengths if l) <= (1 << L)


def _huffman(freq):
    """Unrestricted optimal code (textbook heap construction): returns
    (cost, deepest code length)."""
    items = [(int(f), k, [k]) for k, f in enumerate(freq) if f]
    if len(items) == 1:
        return items[0][0], 1
    depth = {k: 0 for _, k, _ in items}
    heapq.heapify(items)
    cost = 0
    while len(items) > 1:
        a, b = heapq.heappop(items), heapq.heappop(items)
        cost += a[0] + b[0]
        for m in a[2] + b[2]:
            depth[m] += 1
        heapq.heappush(items, (a[0] + b[0], min(a[1], b[1]), a[2] + b[2]))
    return cost, max(depth.values())


def _huffman_cost(freq):
    return _huffman(freq)[0]


@pytest.mark.parametrize("seed", range(40))
def test_lengths_kraft_and_limit(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 257))
    freq = np.zeros(256, np.uint64)
    syms = rng.choice(256, n, replace=False)
    if seed % 3 == 0:  # Fibonacci-like weights force the length limit to bind
        n = min(n, 60)
        syms = syms[:n]
        fib = [1, 1]
        while len(fib) < n:
            fib.append(fib[-1] + fib[-2])
        freq[syms] = np.array(fib[:n], dtype=np.uint64)
    else:
        freq[syms] = rng.integers(1, 10_000, n).astype(np.uint64)
    L = 11
    lengths = oracle_mod.huff_code_lengths(freq, L)
    assert lengths.max() <= L
    assert (lengths[freq == 0] == 0).all()
    assert (lengths[freq > 0] > 0).all()
    assert _kraft_ok(lengths, L)
    if n >= 2:  # package-merge yields a complete code
        assert sum(1 << (L - int(l)) for l in lengths if l) == (1 << L)
    # never better than the unrestricted optimum, and equal to it whenever an
    # unrestricted optimal tree already fits the limit
    unrestricted, deepest = _huffman(freq)
    got = _cost(freq, lengths)
    assert got >= unrestricted
    if deepest <= L:
        assert got == unrestricted
    if seed % 3 == 0 and n > 12:
        assert deepest > L  # the limit binds for these weights


@pytest.mark.parametrize("seed", range(60))
def test_lengths_optimal_brute_force(oracle_mod, seed):
    """Minimum sum(f * len) over every length vector with max length L and
    Kraft sum <= 1, on alphabets of 2..6 symbols."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 7))
    L = int(rng.integers(max(1, (n - 1).bit_length()), 5))
    f = rng.integers(1, 50, n)
    if seed % 4 == 0:
        f = np.array([1, 1, 2, 3, 5, 8][:n]) * int(rng.integers(1, 4))
    freq = np.zeros(256, np.uint64)
    syms = rng.choice(256, n, replace=False)
    freq[syms] = f.astype(np.uint64)
    lengths = oracle_mod.huff_code_lengths(freq, L)
    best = min(sum(int(a) * b for a, b in zip(f, combo))
               for combo in itertools.product(range(1, L + 1), repeat=n)
               if sum(2.0 ** -b for b in combo) <= 1.0)
    assert _cost(freq, lengths) == best
    assert lengths.max() <= L


def test_unrestricted_equality_small(oracle_mod):
    freq = np.zeros(256, np.uint64)
    freq[[3, 9, 27, 81, 200]] = [5, 9, 12, 13, 16]
    assert _cost(freq, oracle_mod.huff_code_lengths(freq, 11)) == _huffman_cost(freq)


def test_degenerate_alphabets(oracle_mod):
    freq = np.zeros(256, np.uint64)
    assert oracle_mod.huff_code_lengths(freq, 11).sum() == 0
    freq[42] = 1000
    lengths = oracle_mod.huff_code_lengths(freq, 11)
    assert lengths[42] == 1 and lengths.sum() == 1


def _tables(s):
    n_chunks = struct.unpack_from("<I", s, 20)[0]
    hc = struct.unpack_from("<I", s, 16)[0]
    n_seg = -(-n_chunks // hc)
    base = 64 + 16 * n_chunks
    return [bytes(s[base + 128 * k: base + 128 * (k + 1)]) for k in range(n_seg)]


def test_huffman_stream_round_trip_and_gain(oracle_mod):
    from paper_1808_02515_gb300 import synth
    x = synth.accel_u8(1 << 17, seed=3)
    plain = oracle_mod.compress(x, forecaster=1, huffman=0)
    coded = oracle_mod.compress(x, forecaster=1, huffman=1, huff_chunks=16)
    assert np.array_equal(oracle_mod.decompress(coded), x)
    assert coded.size < plain.size
    tables = _tables(coded)
    assert any(any(t) for t in tables)
    # packed sizes in the chunk table are the Huffman-free body sizes
    n_chunks = struct.unpack_from("<I", plain, 20)[0]
    for c in range(n_chunks):
        assert (struct.unpack_from("<II", coded, 64 + 16 * c + 8) ==
                struct.unpack_from("<II", plain, 64 + 16 * c + 8))


def _bodies(plain):
    """Packed chunk bodies of a stream written without Huffman."""
    n_chunks = struct.unpack_from("<I", plain, 20)[0]
    data_off, tail_off = struct.unpack_from("<QQ", plain, 40)
    out = []
    for c in range(n_chunks):
        off, _, packed = struct.unpack_from("<QII", plain, 64 + 16 * c)
        out.append(bytes(plain[data_off + off: data_off + off + packed]))
    return out


def test_huffman_raw_segments(oracle_mod):
    """Near-uniform packed bytes: the optimal byte code is 8 bits for every
    symbol, so each segment is stored raw under an all-zero table."""
    from helpers import flat_bytes_u8
    x = flat_bytes_u8(4096, seed=1)  # 32 chunks -> 2 segments of 16
    coded = oracle_mod.compress(x, forecaster=0, huffman=1, huff_chunks=16)
    plain = oracle_mod.compress(x, forecaster=0, huffman=0)
    tables = _tables(coded)
    assert len(tables) == 2 and all(not any(t) for t in tables)
    assert coded.size == plain.size + 128 * len(tables)
    assert np.array_equal(oracle_mod.decompress(coded), x)


@pytest.mark.parametrize("kind,cr,hc", [("uniform", 1024, 4), ("uniform", 8, 1), ("flat", 1024, 2), ("flat", 1024, 16),
                                        ("sensor", 1024, 3), ("sensor", 8, 1),
                                        ("walk", 16, 2)])
def test_huffman_container_size_model(oracle_mod, kind, cr, hc):
    """From the Huffman-free stream: each segment's histogram -> code lengths
    -> coded bytes = sum over chunks of the jump table plus ceil(bits / 8) per
    sub-block; the segment is stored
    raw (all-zero table) iff that is not smaller than its packed bytes. The
    Huffman stream's size and tables must follow."""
    from paper_1808_02515_gb300 import synth
    if kind == "uniform":
        x = synth.uniform(2048, 4, 8, seed=9)
    elif kind == "sensor":
        x = synth.sensor_u16(2048, 2, seed=4)
    elif kind == "flat":
        from helpers import flat_bytes_u8
        x = flat_bytes_u8(2048, seed=1)
    else:
        x = synth.random_walk_u8(2048, 3, scale=0.7, const_frac=0.3, seed=6)
    plain = oracle_mod.compress(x, forecaster=1, huffman=0, chunk_rows=cr)
    coded = oracle_mod.compress(x, forecaster=1, huffman=1, chunk_rows=cr, huff_chunks=hc)
    assert np.array_equal(oracle_mod.decompress(coded), x)
    bodies = _bodies(plain)
    tables = _tables(coded)
    expect_data = 0
    for k, t in enumerate(tables):
        seg = bodies[k * hc:(k + 1) * hc]
        freq = np.zeros(256, np.uint64)
        for b in seg:
            for v in b:
                freq[v] += 1
        lengths = oracle_mod.huff_code_lengths(freq, 11)
        coded_bytes = sum(_chunk_coded(b, lengths) for b in seg)
        packed = sum(len(b) for b in seg)
        raw = packed == 0 or coded_bytes >= packed
        want = bytes(128) if raw else bytes(int(lengths[2 * i]) | (int(lengths[2 * i + 1]) << 4)
                                            for i in range(128))
        assert t == want, k
        expect_data += packed if raw else coded_bytes
    assert coded.size == plain.size + 128 * len(tables) + expect_data - sum(len(b) for b in bodies)


def _canonical_decoder(lengths, codes):
    """(length, code) -> symbol, for a decoder that reads one bit at a time,
    each code's most significant bit first."""
    return {(int(lengths[v]), int(codes[v])): v for v in range(256) if lengths[v]}


def _decode_sub(data, n_sym, table):
    out, bit, cur, ln = [], 0, 0, 0
    while len(out) < n_sym:
        assert bit < 8 * len(data), "sub-block code ran out"
        cur = (cur << 1) | ((data[bit >> 3] >> (bit & 7)) & 1)
        ln += 1
        bit += 1
        if (ln, cur) in table:
            out.append(table[(ln, cur)])
            cur = ln = 0
        assert ln <= 11
    return bytes(out), bit


@pytest.mark.parametrize("cols,hc", [(4, 2), (7, 3)])
def test_huffman_sub_blocks(oracle_mod, cols, hc):
    """Chunks of 1024 u16 rows pack to several 2048-byte sub-blocks: parse
    every coded body (jump table, then codes) and decode each sub-block alone."""
    from paper_1808_02515_gb300 import synth
    x = synth.sensor_u16(4096, cols, seed=5)
    plain = oracle_mod.compress(x, forecaster=1, huffman=0)
    coded = oracle_mod.compress(x, forecaster=1, huffman=1, huff_chunks=hc)
    assert np.array_equal(oracle_mod.decompress(coded), x)
    bodies = _bodies(plain)
    tables = _tables(coded)
    n_chunks = len(bodies)
    data_off, tail_off = struct.unpack_from("<QQ", coded, 40)
    multi = 0
    for c, body in enumerate(bodies):
        off = struct.unpack_from("<Q", coded, 64 + 16 * c)[0]
        end = struct.unpack_from("<Q", coded, 64 + 16 * (c + 1))[0] if c + 1 < n_chunks else tail_off - data_off
        chunk = bytes(coded[data_off + off: data_off + end])
        t = tables[c // hc]
        if not any(t):
            assert chunk == body
            continue
        lengths = np.zeros(256, np.uint8)
        for i in range(128):
            lengths[2 * i], lengths[2 * i + 1] = t[i] & 15, t[i] >> 4
        dec = _canonical_decoder(lengths, oracle_mod.huff_canonical(lengths))
        subs = _sub_slices(body)
        n = len(subs)
        assert max(len(sb) for sb in subs) - min(len(sb) for sb in subs) < n
        multi += n > 1
        starts = [0] + [struct.unpack_from("<I", chunk, 4 * k)[0] for k in range(n - 1)]
        span = len(chunk) - 4 * (n - 1)
        bounds = starts + [span]
        assert all(a <= b for a, b in zip(bounds, bounds[1:]))
        for k in range(n):
            sub = chunk[4 * (n - 1) + bounds[k]: 4 * (n - 1) + bounds[k + 1]]
            want = subs[k]
            got, bits = _decode_sub(sub, len(want), dec)
            assert got == want, (c, k)
            assert -(-bits // 8) == len(sub), (c, k)
    assert multi > 0
