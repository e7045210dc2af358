"""Seeded synthetic workloads (numpy, PCG64).

These generators produce the integer time series that the CUDA codec and the
CPU oracle are both run on. They hold none of the codec's arithmetic: they only
draw samples. Each one stands in for a workload shape of the paper: the paper's
own datasets (UCR, PAMAP, MSRC-12, UCI Gas, AMPDs) are not available, and its
throughput experiment (Sec. 5.4) uses uniformly random values, which
``uniform`` reproduces.

Workloads:
  random_walk_u8   1 column, uint8, x_t = (x_{t-1} + s_t) mod 256 with s_t a
                   discrete Laplace step; a fraction of 8-row blocks repeat the
                   previous value (100,000 rows, scale 2, 20 %, seed 0 is the
                   small single-stream case).
  sensor_u16       D columns of uint16: per column two sinusoids plus Gaussian
                   noise around 32768, with flat stretches where every column
                   holds its value (2^24 rows x 8 columns, seed 1 is the
                   headline case).
  accel_u8         3-axis accelerometer-like uint8: reflected random walk + a
                   1-3 Hz sinusoid at 100 Hz sampling + Laplace noise.
  uniform          uniformly random values over the full range.
  batch_streams    many independent streams of uneven length, width and D.
"""
from __future__ import annotations

import math

import numpy as np

BLOCK_ROWS = 8


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _discrete_laplace(rng: np.random.Generator, scale: float, n: int) -> np.ndarray:
    """P(k) proportional to exp(-|k|/scale): difference of two geometrics."""
    p = 1.0 - math.exp(-1.0 / scale)
    return rng.geometric(p, n).astype(np.int64) - rng.geometric(p, n).astype(np.int64)


def random_walk_u8(rows: int = 100_000, cols: int = 1, scale: float = 2.0,
                   const_frac: float = 0.2, seed: int = 0,
                   rng: np.random.Generator | None = None) -> np.ndarray:
    """Random walk mod 256; blocks chosen i.i.d. with probability const_frac
    take no step (they repeat the previous value). The block choice is shared
    by all columns."""
    rng = rng or _rng(seed)
    n_blocks = (rows + BLOCK_ROWS - 1) // BLOCK_ROWS
    steps = _discrete_laplace(rng, scale, rows * cols).reshape(rows, cols)
    flat = rng.random(n_blocks) < const_frac
    steps[np.repeat(flat, BLOCK_ROWS)[:rows]] = 0
    return (np.cumsum(steps, axis=0) % 256).astype(np.uint8)


def _flat_stretches(rng: np.random.Generator, x: np.ndarray, frac: float,
                    lo: int = 16, hi: int = 8192) -> None:
    """Non-overlapping stretches of log-uniform(lo, hi) rows, in which every
    column holds its value from the stretch start, until `frac` of the rows
    are covered."""
    rows = x.shape[0]
    target = int(frac * rows)
    if rows < 2 * lo or target == 0:
        return
    covered = np.zeros(rows, dtype=bool)
    done = 0
    attempts = 0
    while done < target and attempts < 100_000:
        attempts += 1
        length = int(math.exp(rng.uniform(math.log(lo), math.log(hi))))
        length = min(length, rows - 1)
        start = int(rng.integers(0, rows - length + 1))
        if covered[start:start + length].any():
            continue
        covered[start:start + length] = True
        x[start:start + length, :] = x[start, :]
        done += length


def sensor_u16(rows: int = 1 << 24, cols: int = 8, seed: int = 1,
               flat_frac: float = 0.05,
               rng: np.random.Generator | None = None) -> np.ndarray:
    """Per column: sum of 2 sinusoids (periods U(50, 5000) rows, amplitudes
    U(0, 8000), phases U(0, 2 pi)) + N(0, 20^2), rounded, offset to 32768 and
    clipped to uint16; then flat stretches over 5 % of the rows."""
    rng = rng or _rng(seed)
    x = np.empty((rows, cols), dtype=np.uint16)
    t = np.arange(rows, dtype=np.float64)
    for j in range(cols):
        v = rng.normal(0.0, 20.0, rows)
        for _ in range(2):
            period = rng.uniform(50.0, 5000.0)
            amp = rng.uniform(0.0, 8000.0)
            phase = rng.uniform(0.0, 2.0 * math.pi)
            v += amp * np.sin(2.0 * math.pi * t / period + phase)
        x[:, j] = np.clip(np.rint(v) + 32768.0, 0, 65535).astype(np.uint16)
    _flat_stretches(rng, x, flat_frac)
    return x


def accel_u8(rows: int = 1 << 28, cols: int = 3, seed: int = 3,
             fs_hz: float = 100.0, chunk: int = 1 << 24) -> np.ndarray:
    """128 + reflected random walk (discrete Laplace steps, scale 0.25, folded
    into [-60, 60]) + A sin(2 pi f t / fs + phi) (A ~ U(10, 30), f ~ U(1, 3) Hz)
    + Laplace(0, 3) noise, rounded and clipped to uint8. Generated in row
    slices to bound host memory."""
    rng = _rng(seed)
    params = [(rng.uniform(10.0, 30.0), rng.uniform(1.0, 3.0), rng.uniform(0.0, 2.0 * math.pi))
              for _ in range(cols)]
    x = np.empty((rows, cols), dtype=np.uint8)
    level = np.zeros(cols, dtype=np.int64)
    for r0 in range(0, rows, chunk):
        r1 = min(rows, r0 + chunk)
        n = r1 - r0
        t = np.arange(r0, r1, dtype=np.float64)
        for j, (amp, freq, phase) in enumerate(params):
            walk = level[j] + np.cumsum(_discrete_laplace(rng, 0.25, n))
            level[j] = walk[-1]
            u = np.mod(walk + 60, 240)
            folded = np.where(u <= 120, u, 240 - u) - 60
            v = 128.0 + folded + amp * np.sin(2.0 * math.pi * freq * t / fs_hz + phase)
            v += np.rint(rng.laplace(0.0, 3.0, n))
            x[r0:r1, j] = np.clip(np.rint(v), 0, 255).astype(np.uint8)
    return x


def uniform(rows: int, cols: int, w: int, seed: int) -> np.ndarray:
    """Uniformly random w-bit values (the paper's throughput workload)."""
    rng = _rng(seed)
    hi = 1 << w
    dt = np.uint8 if w == 8 else np.uint16
    return rng.integers(0, hi, size=(rows, cols), dtype=np.uint32).astype(dt)


def batch_stream_shape(idx: int, max_rows: int = 1_000_000, min_rows: int = 1_000) -> tuple[int, int, int]:
    """(rows, D, w) of stream `idx` of the batched workload, from the same
    first draws as batch_stream, without generating it."""
    rng = _rng(2 + idx)
    rows = int(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows))))
    cols = int(rng.integers(1, 17))
    return rows, cols, 8 if idx % 2 == 0 else 16


def batch_stream(idx: int, max_rows: int = 1_000_000, min_rows: int = 1_000) -> np.ndarray:
    """Stream `idx` of the batched workload: rows log-U(min_rows, max_rows),
    D ~ U{1..16}, uint8 for even idx (random walk with scale U(0.5, 4) and
    constant-block fraction U(0, 0.4)), uint16 for odd idx (sensor generator
    with its own draws). Seed 2 + idx."""
    rng = _rng(2 + idx)
    rows = int(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows))))
    cols = int(rng.integers(1, 17))
    if idx % 2 == 0:
        return random_walk_u8(rows, cols, scale=rng.uniform(0.5, 4.0),
                              const_frac=rng.uniform(0.0, 0.4), rng=rng)
    return sensor_u16(rows, cols, rng=rng)


# Codec options of each workload (plain numbers; both implementations take them).
DELTA, FIRE = 0, 1
DEFAULT_OPTS = dict(forecaster=FIRE, huffman=0, group_blocks=2, learn_shift=1,
                    chunk_rows=1024, huff_chunks=64)


# ---------------------------------------------------------------------------
# The same recipes drawn on the GPU with torch (for the large benchmark
# workloads: tens of GB would take minutes in numpy). Scalar parameters come
# from numpy PCG64 with the same seeds; the bulk draws from a torch CUDA
# generator seeded alike, so these series follow the same distributions as
# the numpy ones above but are different samples.
# ---------------------------------------------------------------------------

def _tgen(seed: int, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def uniform_torch(rows: int, cols: int, w: int, seed: int, device="cuda"):
    """Uniformly random w-bit values drawn on the device (uint8, or int16
    holding the 16-bit patterns)."""
    import torch
    g = _tgen(seed, device)
    if w == 8:
        return torch.randint(0, 256, (rows, cols), generator=g, device=device, dtype=torch.int32).to(torch.uint8)
    return torch.randint(-32768, 32768, (rows, cols), generator=g, device=device, dtype=torch.int32).to(torch.int16)


def random_walk_u8_torch(rows: int, cols: int, scale: float, const_frac: float, seed: int,
                         device="cuda"):
    import torch
    g = _tgen(seed, device)
    p = 1.0 - math.exp(-1.0 / scale)
    s = (torch.empty((rows, cols), device=device).geometric_(p, generator=g)
         - torch.empty((rows, cols), device=device).geometric_(p, generator=g)).to(torch.int32)
    n_blocks = (rows + BLOCK_ROWS - 1) // BLOCK_ROWS
    flat = torch.rand(n_blocks, generator=g, device=device) < const_frac
    # no step in the chosen blocks (a masked fill: no host synchronisation)
    s.masked_fill_(flat.repeat_interleave(BLOCK_ROWS)[:rows, None], 0)
    return torch.remainder(torch.cumsum(s, 0, dtype=torch.int64), 256).to(torch.uint8)


def _stretch_map(rng: np.random.Generator, rows: int, frac: float, lo: int = 16, hi: int = 8192) -> np.ndarray:
    """Row index map of the flat stretches of `_flat_stretches` (same draws):
    row r takes the value of row map[r]."""
    m = np.arange(rows, dtype=np.int64)
    target = int(frac * rows)
    if rows < 2 * lo or target == 0:
        return m
    covered = np.zeros(rows, dtype=bool)
    done = attempts = 0
    while done < target and attempts < 100_000:
        attempts += 1
        length = min(int(math.exp(rng.uniform(math.log(lo), math.log(hi)))), rows - 1)
        start = int(rng.integers(0, rows - length + 1))
        if covered[start:start + length].any():
            continue
        covered[start:start + length] = True
        m[start:start + length] = start
        done += length
    return m


def sensor_u16_torch(rows: int, cols: int, seed: int, flat_frac: float = 0.05, device="cuda"):
    """uint16 samples as an int16 tensor (the same bits)."""
    import torch
    rng = _rng(seed)
    g = _tgen(seed, device)
    # per column: two (period, amplitude, phase) draws, in the numpy recipe's order
    par = np.array([[rng.uniform(50.0, 5000.0), rng.uniform(0.0, 8000.0), rng.uniform(0.0, 2 * math.pi)]
                    for _ in range(2 * cols)]).reshape(cols, 2, 3)
    t = torch.arange(rows, dtype=torch.float64, device=device)[:, None]
    v = torch.randn((rows, cols), generator=g, dtype=torch.float64, device=device) * 20.0
    for k in range(2):
        per = torch.from_numpy(par[:, k, 0]).to(device)
        amp = torch.from_numpy(par[:, k, 1]).to(device)
        ph = torch.from_numpy(par[:, k, 2]).to(device)
        v += amp * torch.sin(2.0 * math.pi * t / per + ph)
    x = torch.clamp(torch.round(v) + 32768.0, 0, 65535).to(torch.int32)
    if rows >= 32:
        m = torch.from_numpy(_stretch_map(rng, rows, flat_frac)).to(device)
        x = x.index_select(0, m)
    return (x - 65536 * (x >= 32768)).to(torch.int16)


def accel_u8_torch(rows: int, cols: int = 3, seed: int = 3, fs_hz: float = 100.0, device="cuda"):
    import torch
    rng = _rng(seed)
    g = _tgen(seed, device)
    p = 1.0 - math.exp(-1.0 / 0.25)
    x = torch.empty((rows, cols), dtype=torch.uint8, device=device)
    step = 1 << 24
    for j in range(cols):
        amp, freq, phase = rng.uniform(10.0, 30.0), rng.uniform(1.0, 3.0), rng.uniform(0.0, 2 * math.pi)
        level = 0
        for r0 in range(0, rows, step):
            n = min(step, rows - r0)
            s = (torch.empty(n, device=device).geometric_(p, generator=g)
                 - torch.empty(n, device=device).geometric_(p, generator=g)).to(torch.int64)
            walk = level + torch.cumsum(s, 0)
            level = int(walk[-1].item())
            u = torch.remainder(walk + 60, 240)
            folded = torch.where(u <= 120, u, 240 - u) - 60
            t = torch.arange(r0, r0 + n, dtype=torch.float64, device=device)
            v = 128.0 + folded + amp * torch.sin(2.0 * math.pi * freq * t / fs_hz + phase)
            # Laplace(0, 3): the difference of two exponentials of mean 3
            lap = (torch.empty(n, dtype=torch.float64, device=device).exponential_(1.0 / 3.0, generator=g)
                   - torch.empty(n, dtype=torch.float64, device=device).exponential_(1.0 / 3.0, generator=g))
            v += torch.round(lap)
            x[r0:r0 + n, j] = torch.clamp(torch.round(v), 0, 255).to(torch.uint8)
    return x


def batch_stream_torch(idx: int, max_rows: int = 1_000_000, min_rows: int = 1_000, device="cuda"):
    """Stream `idx` of the batched workload (same recipe as batch_stream)."""
    rng = _rng(2 + idx)
    rows = int(math.exp(rng.uniform(math.log(min_rows), math.log(max_rows))))
    cols = int(rng.integers(1, 17))
    if idx % 2 == 0:
        return random_walk_u8_torch(rows, cols, scale=rng.uniform(0.5, 4.0),
                                    const_frac=rng.uniform(0.0, 0.4), seed=2 + idx, device=device)
    return sensor_u16_torch(rows, cols, seed=2 + idx, device=device)
