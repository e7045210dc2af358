"""Python access to the Sprintz CPU oracle (``sprintz_oracle.c``).

TEST INFRASTRUCTURE. The oracle is the plain, slow, scalar C encoder/decoder
that the CUDA codec is checked against. Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg import this
module; the CUDA library and its Python binding never do.

Functions that have no independent pin in the tests are listed in the module
docstrings of those tests; the byte container (header, chunk table, Huffman
segment tables) is our own format, so its parity is pinned by round trips and
closed-form sizes, not by the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sprintz_oracle.c")
_HDR = os.path.join(_HERE, "sprintz_oracle.h")
_LIB = os.path.join(_HERE, "libsprintz_oracle.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_W = -2
ERR_DST_TOO_SMALL = -3
ERR_CORRUPT = -5


class _Opts(ctypes.Structure):
    _fields_ = [("forecaster", ctypes.c_int32), ("huffman", ctypes.c_int32),
                ("group_blocks", ctypes.c_int32), ("learn_shift", ctypes.c_int32),
                ("chunk_rows", ctypes.c_uint32), ("huff_chunks", ctypes.c_uint32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (C99, portable: no target-specific flags)."""
    stale = (not os.path.exists(_LIB) or
             os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
        os.close(fd)
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-Wall", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u64, u32, i32, i64, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                  ctypes.c_int64, ctypes.c_void_p)
        L.spo_max_compressed_size.restype = u64
        L.spo_max_compressed_size.argtypes = [u64, u32, u32, ctypes.POINTER(_Opts)]
        L.spo_compress.restype = i64
        L.spo_compress.argtypes = [vp, u64, u32, u32, ctypes.POINTER(_Opts), vp, u64]
        L.spo_decompress.restype = ctypes.c_int
        L.spo_decompress.argtypes = [vp, u64, vp, u64]
        L.spo_query.restype = ctypes.c_int
        L.spo_query.argtypes = [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u32),
                                ctypes.POINTER(u32), ctypes.POINTER(_Opts)]
        L.spo_zigzag.restype = u32
        L.spo_zigzag.argtypes = [i32, u32]
        L.spo_unzigzag.restype = i32
        L.spo_unzigzag.argtypes = [u32, u32]
        L.spo_bit_length.restype = u32
        L.spo_bit_length.argtypes = [u32]
        L.spo_column_width.restype = u32
        L.spo_column_width.argtypes = [vp, u32]
        L.spo_forecast_errors.restype = ctypes.c_int
        L.spo_forecast_errors.argtypes = [vp, u64, u32, u32, i32, i32, i32, i64, vp]
        L.spo_forecast_reconstruct.restype = ctypes.c_int
        L.spo_forecast_reconstruct.argtypes = [vp, u64, u32, u32, i32, i32, vp]
        L.spo_quantize.restype = ctypes.c_int
        L.spo_quantize.argtypes = [vp, u64, u32, u32, vp, vp]
        L.spo_dequantize.restype = ctypes.c_int
        L.spo_dequantize.argtypes = [vp, u64, u32, u32, vp, vp]
        L.spo_quant_nmse.restype = ctypes.c_int
        L.spo_quant_nmse.argtypes = [vp, vp, u64, u32, u32, vp, vp]
        L.spo_fire_trace.restype = ctypes.c_int
        L.spo_fire_trace.argtypes = [vp, u64, u32, u32, i32, vp, vp]
        L.spo_huff_code_lengths.restype = ctypes.c_int
        L.spo_huff_code_lengths.argtypes = [vp, u32, vp]
        L.spo_huff_canonical.restype = ctypes.c_int
        L.spo_huff_canonical.argtypes = [vp, vp]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


def _opts(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024,
          huff_chunks=64) -> _Opts:
    return _Opts(forecaster, huffman, group_blocks, learn_shift, chunk_rows, huff_chunks)


def _as_samples(x: np.ndarray) -> tuple[np.ndarray, int, int, int]:
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    if x.dtype not in (np.uint8, np.uint16):
        raise TypeError("samples must be uint8 or uint16")
    x = np.ascontiguousarray(x)
    if x.dtype == np.uint16 and x.dtype.byteorder == ">":
        x = x.astype("<u2")
    return x, x.shape[0], x.shape[1], 8 * x.dtype.itemsize


def max_compressed_size(rows: int, D: int, w: int, **opts) -> int:
    o = _opts(**opts)
    return int(lib().spo_max_compressed_size(rows, D, w, ctypes.byref(o)))


def compress(x: np.ndarray, **opts) -> np.ndarray:
    """Compress a (rows, D) uint8/uint16 array; returns the stream bytes."""
    x, rows, D, w = _as_samples(x)
    o = _opts(**opts)
    cap = int(lib().spo_max_compressed_size(rows, D, w, ctypes.byref(o)))
    if cap == 0:
        raise OracleError(ERR_INVALID_ARG, "compress")
    out = np.zeros(cap, dtype=np.uint8)
    n = lib().spo_compress(x.ctypes.data if x.size else None, rows, D, w, ctypes.byref(o),
                           out.ctypes.data, cap)
    if n < 0:
        raise OracleError(int(n), "compress")
    return out[:n].copy()


def query(stream: np.ndarray) -> dict:
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    rows, D, w, o = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), _Opts()
    rc = lib().spo_query(s.ctypes.data, s.size, ctypes.byref(rows), ctypes.byref(D),
                         ctypes.byref(w), ctypes.byref(o))
    if rc != OK:
        raise OracleError(rc, "query")
    return dict(rows=rows.value, D=D.value, w=w.value, forecaster=o.forecaster,
                huffman=o.huffman, group_blocks=o.group_blocks, learn_shift=o.learn_shift,
                chunk_rows=o.chunk_rows, huff_chunks=o.huff_chunks)


def decompress(stream: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    info = query(s)
    dt = np.uint8 if info["w"] == 8 else np.uint16
    out = np.zeros((info["rows"], info["D"]), dtype=dt)
    rc = lib().spo_decompress(s.ctypes.data, s.size, out.ctypes.data if out.size else None,
                              out.nbytes)
    if rc != OK:
        raise OracleError(rc, "decompress")
    return out


def decompress_rc(stream: np.ndarray) -> int:
    """Return code of decompressing a (possibly corrupt) stream."""
    s = np.ascontiguousarray(stream, dtype=np.uint8)
    try:
        info = query(s)
    except OracleError as e:
        return e.code
    dt = np.uint8 if info["w"] == 8 else np.uint16
    if info["rows"] * info["D"] > (1 << 31):
        return ERR_CORRUPT
    out = np.zeros((info["rows"], info["D"]), dtype=dt)
    return int(lib().spo_decompress(s.ctypes.data, s.size, out.ctypes.data if out.size else None,
                                    out.nbytes))


def zigzag(e: int, w: int) -> int:
    return int(lib().spo_zigzag(int(e), w))


def unzigzag(z: int, w: int) -> int:
    return int(lib().spo_unzigzag(int(z), w))


def bit_length(v: int) -> int:
    return int(lib().spo_bit_length(int(v)))


def column_width(z8, w: int) -> int:
    a = np.ascontiguousarray(np.asarray(z8, dtype=np.uint32))
    assert a.size == 8
    return int(lib().spo_column_width(a.ctypes.data, w))


def forecast_errors(x: np.ndarray, forecaster: int, learn_shift: int = 1, test_mode: int = 0,
                    pinned_alpha: int = 0) -> np.ndarray:
    """Errors (signed, w-bit, as int32) of the forecaster over all rows."""
    x, rows, D, w = _as_samples(x)
    out = np.zeros((rows, D), dtype=np.int32)
    rc = lib().spo_forecast_errors(x.ctypes.data, rows, D, w, forecaster, learn_shift,
                                   test_mode, pinned_alpha, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "forecast_errors")
    return out


def forecast_reconstruct(err: np.ndarray, w: int, forecaster: int, learn_shift: int = 1) -> np.ndarray:
    """Samples (uint8/uint16, rows x D) rebuilt from forecast errors."""
    e = np.ascontiguousarray(np.asarray(err, dtype=np.int32))
    if e.ndim == 1:
        e = e.reshape(-1, 1)
    rows, D = e.shape
    out = np.zeros((rows, D), dtype=np.uint8 if w == 8 else np.uint16)
    rc = lib().spo_forecast_reconstruct(e.ctypes.data, rows, D, w, forecaster, learn_shift, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "forecast_reconstruct")
    return out


def forecast_transform(x: np.ndarray, forecaster: int, learn_shift: int = 1, chunk_rows: int = 1024,
                       inverse: bool = False) -> np.ndarray:
    """The forecast step alone, chunk by chunk (the state restarts every
    chunk_rows rows; 0 = one chunk); whole 8-row blocks are transformed and the
    rows % 8 trailing rows copied. Errors are returned as w-bit two's
    complement in the samples' dtype, and inverse=True takes that form."""
    x = np.ascontiguousarray(x)
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    w = 8 * x.itemsize
    rows = x.shape[0]
    full = rows - rows % 8
    out = x.copy()
    cr = chunk_rows or max(full, 8)
    for r0 in range(0, full, cr):
        part = x[r0:min(full, r0 + cr)]
        if not inverse:
            e = forecast_errors(part, forecaster, learn_shift)
            out[r0:r0 + part.shape[0]] = (e.astype(np.int64) % (1 << w)).astype(x.dtype)
        else:
            sgn = part.astype(np.int64)
            sgn = np.where(sgn >= 1 << (w - 1), sgn - (1 << w), sgn)
            out[r0:r0 + part.shape[0]] = forecast_reconstruct(sgn, w, forecaster, learn_shift)
    return out


def quantize(x: np.ndarray, w: int) -> tuple[np.ndarray, np.ndarray]:
    """Sec. 5.8 quantization of float32 columns to w-bit codes; returns
    (codes, lo_hi) with lo_hi[2 j] = min, lo_hi[2 j + 1] = max of column j."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim == 1:
        x = x.reshape(-1, 1)
    rows, D = x.shape
    q = np.zeros((rows, D), dtype=np.uint8 if w == 8 else np.uint16)
    lh = np.zeros(2 * D, dtype=np.float64)
    rc = lib().spo_quantize(x.ctypes.data, rows, D, w, q.ctypes.data, lh.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "quantize")
    return q, lh


def dequantize(q: np.ndarray, lo_hi: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q)
    rows, D = q.shape
    w = 8 * q.itemsize
    lh = np.ascontiguousarray(lo_hi, dtype=np.float64)
    out = np.zeros((rows, D), dtype=np.float32)
    rc = lib().spo_dequantize(q.ctypes.data, rows, D, w, lh.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "dequantize")
    return out


def quant_nmse(x: np.ndarray, q: np.ndarray, lo_hi: np.ndarray) -> np.ndarray:
    """Per column: mean squared error of the reconstruction over the
    column's variance (0 for a constant column)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.ascontiguousarray(q)
    rows, D = x.shape
    w = 8 * q.itemsize
    lh = np.ascontiguousarray(lo_hi, dtype=np.float64)
    out = np.zeros(D, dtype=np.float64)
    rc = lib().spo_quant_nmse(x.ctypes.data, q.ctypes.data, rows, D, w, lh.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "quant_nmse")
    return out


def fire_trace(x: np.ndarray, learn_shift: int = 1) -> tuple[np.ndarray, np.ndarray]:
    x, rows, D, w = _as_samples(x)
    nb = rows // 8
    alpha = np.zeros((nb, D), dtype=np.int64)
    acc = np.zeros((nb, D), dtype=np.int64)
    rc = lib().spo_fire_trace(x.ctypes.data, rows, D, w, learn_shift, alpha.ctypes.data,
                              acc.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "fire_trace")
    return alpha, acc


def huff_code_lengths(freq, max_len: int = 11) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(freq, dtype=np.uint64))
    assert f.size == 256
    out = np.zeros(256, dtype=np.uint8)
    rc = lib().spo_huff_code_lengths(f.ctypes.data, max_len, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "huff_code_lengths")
    return out


def huff_canonical(lengths) -> np.ndarray:
    L = np.ascontiguousarray(np.asarray(lengths, dtype=np.uint8))
    out = np.zeros(256, dtype=np.uint32)
    rc = lib().spo_huff_canonical(L.ctypes.data, out.ctypes.data)
    if rc != OK:
        raise OracleError(rc, "huff_canonical")
    return out


# ---------------------------------------------------------------------------
# Many independent streams on all host cores.  Streams share nothing, so the
# plain per-stream oracle runs on a pool of host threads, one stream per task
# (ctypes releases the GIL for the duration of each C call).  This is the
# oracle as it stands, spread over cores; nothing in it is tuned.
# ---------------------------------------------------------------------------

def host_cores() -> int:
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


def map_streams(fn, items, threads: int | None = None) -> list:
    """fn(item) for every item on `threads` host threads (all cores by
    default), results in item order."""
    from concurrent.futures import ThreadPoolExecutor
    n = threads or host_cores()
    if n <= 1:
        return [fn(it) for it in items]
    with ThreadPoolExecutor(n) as ex:
        return list(ex.map(fn, items))


def compress_many(xs, opts, threads: int | None = None) -> list:
    """compress() of every array in xs (opts: one dict, or one per array)."""
    ol = list(opts) if isinstance(opts, (list, tuple)) else [opts] * len(xs)
    return map_streams(lambda a: compress(a[0], **a[1]), list(zip(xs, ol)), threads)


def decompress_many(streams, threads: int | None = None) -> list:
    return map_streams(decompress, list(streams), threads)
