"""Crafted test inputs (not workloads)."""
import numpy as np


def flat_bytes_u8(n_blocks: int, D: int = 4, seed: int = 0) -> np.ndarray:
    """uint8 series whose delta-coded, bit-packed bytes are close to uniform:
    each (block, column) draws a header code uniformly from 0..7 and its eight
    zigzagged errors uniformly within that code's width, so both header and
    payload bits are near-uniform and a byte Huffman code cannot shrink them.
    Column-major packing (D <= 4) adds no padding bits."""
    rng = np.random.default_rng(seed)
    widths = np.array([0, 1, 2, 3, 4, 5, 6, 8])
    z = np.zeros((n_blocks, 8, D), dtype=np.int64)
    for b in range(n_blocks):
        for j in range(D):
            n = int(widths[rng.integers(0, 8)])
            if n == 0:
                continue
            lo = 64 if n == 8 else 1 << (n - 1)
            while True:
                v = rng.integers(0, 1 << n, 8)
                if int(np.bitwise_or.reduce(v)) >= lo:
                    break
            z[b, :, j] = v
    z = z.reshape(-1, D)
    e = np.where(z & 1, -((z + 1) >> 1), z >> 1)
    return (np.cumsum(e, axis=0) % 256).astype(np.uint8)
