"""Python binding of the CUDA Sprintz codec (libsprintz_gb300.so).

Argument marshalling only: every step of compression and decompression runs
in the library's CUDA kernels. PyTorch supplies device memory and streams.
If the library is missing the binding raises; there is no CPU fallback.

The entry points mirror the C ABI in include/sprintz_gb300.h:
    sprintz_compress / sprintz_decompress / sprintz_query /
    sprintz_max_compressed_size / sprintz_*_workspace_size /
    sprintz_get_status / sprintz_strerror
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsprintz_gb300.so")

OK = 0
ERR_INVALID_ARG = -1
ERR_UNSUPPORTED_W = -2
ERR_DST_TOO_SMALL = -3
ERR_WS_TOO_SMALL = -4
ERR_CORRUPT = -5
ERR_TIMEOUT = -6
ERR_CUDA = -7
ERR_UNSUPPORTED = -8

DELTA, FIRE, DDELTA, FIRE_SAMPLE = 0, 1, 2, 3


class _Opts(ctypes.Structure):
    _fields_ = [("forecaster", ctypes.c_uint8), ("huffman", ctypes.c_uint8),
                ("group_blocks", ctypes.c_uint8), ("learn_shift", ctypes.c_uint8),
                ("chunk_rows", ctypes.c_uint32), ("huff_chunks", ctypes.c_uint32)]


class _Info(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint64), ("D", ctypes.c_uint32), ("w", ctypes.c_uint32),
                ("opts", _Opts), ("n_chunks", ctypes.c_uint32), ("tail_rows", ctypes.c_uint32),
                ("data_off", ctypes.c_uint64), ("tail_off", ctypes.c_uint64),
                ("total_bytes", ctypes.c_uint64)]


class _BatchItem(ctypes.Structure):
    _fields_ = [("src", ctypes.c_void_p), ("src_bytes", ctypes.c_uint64), ("dst", ctypes.c_void_p),
                ("dst_cap", ctypes.c_uint64), ("out_size", ctypes.c_void_p), ("rows", ctypes.c_uint64),
                ("D", ctypes.c_uint32), ("w", ctypes.c_uint32), ("opts", _Opts),
                ("row_begin", ctypes.c_uint64), ("row_end", ctypes.c_uint64)]


class _Schedule(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_uint32), ("ring_segments", ctypes.c_uint32),
                ("prefetch_bytes", ctypes.c_uint32), ("order", ctypes.c_uint32)]


@dataclass(frozen=True)
class Schedule:
    """Launch schedule of a batched launch (sprintz_schedule); 0 = default."""
    ctas_per_sm: int = 0
    ring_segments: int = 0
    prefetch_bytes: int = 0
    order: int = 0

    def c(self) -> _Schedule:
        return _Schedule(self.ctas_per_sm, self.ring_segments, self.prefetch_bytes, self.order)

    @staticmethod
    def of(c: _Schedule) -> "Schedule":
        return Schedule(c.ctas_per_sm, c.ring_segments, c.prefetch_bytes, c.order)


def _item_dtype():
    """numpy layout of sprintz_batch_item, taken from the ctypes struct."""
    import numpy as np
    kinds = {ctypes.c_void_p: "<u8", ctypes.c_uint64: "<u8", ctypes.c_uint32: "<u4", ctypes.c_uint8: "u1"}
    names, formats, offsets = [], [], []
    for name, t in _BatchItem._fields_:
        off = getattr(_BatchItem, name).offset
        if t is _Opts:
            for on, ot in _Opts._fields_:
                names.append(on)
                formats.append(kinds[ot])
                offsets.append(off + getattr(_Opts, on).offset)
        else:
            names.append(name)
            formats.append(kinds[t])
            offsets.append(off)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets,
                     "itemsize": ctypes.sizeof(_BatchItem)})


@dataclass(frozen=True)
class Opts:
    forecaster: int = FIRE
    huffman: int = 0
    group_blocks: int = 2
    learn_shift: int = 1
    chunk_rows: int = 1024
    huff_chunks: int = 64

    def c(self) -> _Opts:
        return _Opts(self.forecaster, self.huffman, self.group_blocks, self.learn_shift,
                     self.chunk_rows, self.huff_chunks)


_ITEM_DTYPE = _item_dtype()


class SprintzError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        PO, PI = ctypes.POINTER(_Opts), ctypes.POINTER(_Info)
        L.sprintz_ctx_create.restype = i32
        L.sprintz_ctx_create.argtypes = [ctypes.POINTER(vp), i32]
        L.sprintz_ctx_destroy.restype = None
        L.sprintz_ctx_destroy.argtypes = [vp]
        L.sprintz_max_compressed_size.restype = u64
        L.sprintz_max_compressed_size.argtypes = [u64, u32, u32, PO]
        L.sprintz_compress_workspace_size.restype = u64
        L.sprintz_compress_workspace_size.argtypes = [u64, u32, u32, PO]
        L.sprintz_decompress_workspace_size.restype = u64
        L.sprintz_decompress_workspace_size.argtypes = [PI]
        L.sprintz_compress.restype = i32
        L.sprintz_compress.argtypes = [vp, vp, u64, u32, u32, PO, vp, u64, vp, vp, u64, vp]
        L.sprintz_decompress.restype = i32
        L.sprintz_decompress.argtypes = [vp, vp, u64, PI, vp, u64, vp, u64, vp]
        L.sprintz_decompress_rows_workspace_size.restype = u64
        L.sprintz_decompress_rows_workspace_size.argtypes = [PI, u64, u64]
        L.sprintz_decompress_rows.restype = i32
        L.sprintz_decompress_rows.argtypes = [vp, vp, u64, PI, u64, u64, vp, u64, vp, u64, vp]
        L.sprintz_append_workspace_size.restype = u64
        L.sprintz_append_workspace_size.argtypes = [PI, u64]
        L.sprintz_append.restype = i32
        L.sprintz_append.argtypes = [vp, vp, u64, PI, vp, u64, vp, u64, vp, vp, u64, vp]
        L.sprintz_pack.restype = i32
        L.sprintz_pack.argtypes = [vp, vp, vp, u32, vp, u64, vp, vp]
        L.sprintz_ctx_set_failure_test.restype = i32
        L.sprintz_ctx_set_failure_test.argtypes = [vp, u32, u32]
        L.sprintz_compress_noalloc.restype = i32
        L.sprintz_compress_noalloc.argtypes = [vp, u64, u32, u32, PO, vp, u64, vp, vp]
        PB = ctypes.POINTER(_BatchItem)
        L.sprintz_batch_workspace_size.restype = u64
        L.sprintz_batch_workspace_size.argtypes = [vp, PB, u32, i32]
        L.sprintz_batch_plan.restype = i32
        L.sprintz_batch_plan.argtypes = [vp, PB, u32, i32, vp, u64, vp]
        L.sprintz_batch_run.restype = i32
        L.sprintz_batch_run.argtypes = [vp, vp, u64, vp]
        PS = ctypes.POINTER(_Schedule)
        L.sprintz_batch_plan_schedule.restype = i32
        L.sprintz_batch_plan_schedule.argtypes = [vp, PB, u32, i32, PS, vp, u64, vp]
        L.sprintz_batch_schedule.restype = i32
        L.sprintz_batch_schedule.argtypes = [vp, PS]
        L.sprintz_batch_autotune.restype = i32
        L.sprintz_batch_autotune.argtypes = [vp, PB, u32, i32, vp, u64, vp, PS, ctypes.POINTER(ctypes.c_float)]
        L.sprintz_forecast.restype = i32
        L.sprintz_forecast.argtypes = [vp, vp, u64, u32, u32, u32, u32, u32, i32, vp, vp]
        L.sprintz_quant_workspace_size.restype = u64
        L.sprintz_quant_workspace_size.argtypes = [u32]
        L.sprintz_quantize.restype = i32
        L.sprintz_quantize.argtypes = [vp, vp, u64, u32, u32, vp, vp, vp, u64, vp]
        L.sprintz_dequantize.restype = i32
        L.sprintz_dequantize.argtypes = [vp, vp, u64, u32, u32, vp, vp, vp]
        L.sprintz_quant_nmse.restype = i32
        L.sprintz_quant_nmse.argtypes = [vp, vp, vp, u64, u32, u32, vp, vp, vp, u64, vp]
        L.sprintz_query.restype = i32
        L.sprintz_query.argtypes = [vp, u64, PI]
        L.sprintz_get_status.restype = i32
        L.sprintz_get_status.argtypes = [vp, vp]
        L.sprintz_strerror.restype = ctypes.c_char_p
        L.sprintz_strerror.argtypes = [i32]
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().sprintz_strerror(code).decode()


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise SprintzError(rc, what)


def max_compressed_size(rows: int, D: int, w: int, opts: Opts) -> int:
    o = opts.c()
    return int(lib().sprintz_max_compressed_size(rows, D, w, ctypes.byref(o)))


def compress_workspace_size(rows: int, D: int, w: int, opts: Opts) -> int:
    o = opts.c()
    return int(lib().sprintz_compress_workspace_size(rows, D, w, ctypes.byref(o)))


@dataclass(frozen=True)
class Info:
    rows: int
    D: int
    w: int
    opts: Opts
    n_chunks: int
    tail_rows: int
    data_off: int
    tail_off: int
    total_bytes: int

    def c(self) -> _Info:
        return _Info(self.rows, self.D, self.w, self.opts.c(), self.n_chunks, self.tail_rows,
                     self.data_off, self.tail_off, self.total_bytes)


def query(header: bytes) -> Info:
    """Parse a host copy of a stream's first 64 (or more) bytes."""
    buf = ctypes.create_string_buffer(bytes(header), len(header))
    info = _Info()
    _check(lib().sprintz_query(buf, len(header), ctypes.byref(info)), "sprintz_query")
    o = info.opts
    return Info(info.rows, info.D, info.w,
                Opts(o.forecaster, o.huffman, o.group_blocks, o.learn_shift, o.chunk_rows,
                     o.huff_chunks),
                info.n_chunks, info.tail_rows, info.data_off, info.tail_off, info.total_bytes)


def decompress_workspace_size(info: Info) -> int:
    ci = info.c()
    return int(lib().sprintz_decompress_workspace_size(ctypes.byref(ci)))


def compress_noalloc(x, opts: Opts, dst, out_size, stream=None) -> None:
    """sprintz_compress_noalloc: compress a (rows, D) device tensor into the
    caller's dst / out_size without any allocation by the library (its scratch
    is a fixed device array); runs on the current device and torch stream."""
    import torch
    if x.dim() == 1:
        x = x.view(-1, 1)
    rows, D = x.shape
    w = 8 if x.dtype == torch.uint8 else 16
    s = stream if stream is not None else torch.cuda.current_stream()
    o = opts.c()
    rc = lib().sprintz_compress_noalloc(ctypes.c_void_p(x.data_ptr() if rows else 0), rows, D, w,
                                        ctypes.byref(o), ctypes.c_void_p(dst.data_ptr()),
                                        dst.numel() * dst.element_size(),
                                        ctypes.c_void_p(out_size.data_ptr()),
                                        ctypes.c_void_p(s.cuda_stream))
    _check(rc, "sprintz_compress_noalloc")


class Codec:
    """A library context on one device plus the torch-side plumbing.

    compress()/decompress() take device tensors and enqueue the library's
    kernels on the current torch stream (or the stream given)."""

    def __init__(self, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        ctx = ctypes.c_void_p()
        _check(lib().sprintz_ctx_create(ctypes.byref(ctx), device), "sprintz_ctx_create")
        self.ctx = ctx

    def close(self) -> None:
        if self.ctx:
            lib().sprintz_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def compress_into(self, src, rows: int, D: int, w: int, opts: Opts, dst, out_size, ws,
                      stream=None) -> None:
        """Raw entry point: src/dst/out_size/ws are device tensors (or None
        for an empty workspace)."""
        o = opts.c()
        rc = lib().sprintz_compress(self.ctx, ctypes.c_void_p(src.data_ptr() if rows else 0),
                                    rows, D, w, ctypes.byref(o), ctypes.c_void_p(dst.data_ptr()),
                                    dst.numel() * dst.element_size(),
                                    ctypes.c_void_p(out_size.data_ptr()),
                                    ctypes.c_void_p(ws.data_ptr() if ws is not None else 0),
                                    ws.numel() if ws is not None else 0, self._stream(stream))
        _check(rc, "sprintz_compress")

    def forecast(self, x, forecaster: int = FIRE, learn_shift: int = 1, chunk_rows: int = 1024,
                 inverse: bool = False, out=None, stream=None):
        """The forecast step alone (sprintz_forecast): samples -> errors, or
        errors -> samples with inverse=True, on a (rows, D) uint8 / 16-bit
        CUDA tensor; the result has x's shape and dtype (out may be x)."""
        torch = self.torch
        if x.dim() == 1:
            x = x.view(-1, 1)
        if x.dtype not in (torch.uint8, torch.int16, torch.uint16):
            raise TypeError("samples must be uint8 or 16-bit")
        x = x.contiguous()
        rows, D = x.shape
        w = 8 if x.dtype == torch.uint8 else 16
        y = torch.empty_like(x) if out is None else out
        rc = lib().sprintz_forecast(self.ctx, ctypes.c_void_p(x.data_ptr() if rows else 0), rows, D, w,
                                    forecaster, learn_shift, chunk_rows, 1 if inverse else 0,
                                    ctypes.c_void_p(y.data_ptr() if rows else 0), self._stream(stream))
        _check(rc, "sprintz_forecast")
        return y

    def quantize(self, x, w: int = 16, stream=None):
        """Float quantization (sprintz_quantize) of a (rows, D) float32 CUDA
        tensor: returns (codes, lo_hi), codes uint8 (w = 8) or int16 holding
        the 16-bit codes, lo_hi a (D, 2) float64 tensor of column min/max."""
        torch = self.torch
        if x.dim() == 1:
            x = x.view(-1, 1)
        x = x.contiguous()
        if x.dtype != torch.float32:
            raise TypeError("float32 samples expected")
        rows, D = x.shape
        codes = torch.empty((rows, D), dtype=torch.uint8 if w == 8 else torch.int16, device=x.device)
        lo_hi = torch.empty((D, 2), dtype=torch.float64, device=x.device)
        wsn = int(lib().sprintz_quant_workspace_size(D))
        ws = torch.empty(max(wsn, 1), dtype=torch.uint8, device=x.device)
        rc = lib().sprintz_quantize(self.ctx, ctypes.c_void_p(x.data_ptr()), rows, D, w,
                                    ctypes.c_void_p(codes.data_ptr()), ctypes.c_void_p(lo_hi.data_ptr()),
                                    ctypes.c_void_p(ws.data_ptr()), wsn, self._stream(stream))
        _check(rc, "sprintz_quantize")
        self._keep = ws
        return codes, lo_hi

    def dequantize(self, codes, lo_hi, out=None, stream=None):
        torch = self.torch
        rows, D = codes.shape
        w = 8 if codes.dtype == torch.uint8 else 16
        y = torch.empty((rows, D), dtype=torch.float32, device=codes.device) if out is None else out
        rc = lib().sprintz_dequantize(self.ctx, ctypes.c_void_p(codes.data_ptr()), rows, D, w,
                                      ctypes.c_void_p(lo_hi.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                      self._stream(stream))
        _check(rc, "sprintz_dequantize")
        return y

    def quant_nmse(self, x, codes, lo_hi, stream=None):
        """Per column: reconstruction MSE over variance (a (D,) float64 tensor)."""
        torch = self.torch
        rows, D = codes.shape
        w = 8 if codes.dtype == torch.uint8 else 16
        out = torch.empty(D, dtype=torch.float64, device=codes.device)
        wsn = int(lib().sprintz_quant_workspace_size(D))
        ws = torch.empty(max(wsn, 1), dtype=torch.uint8, device=codes.device)
        rc = lib().sprintz_quant_nmse(self.ctx, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(codes.data_ptr()),
                                      rows, D, w, ctypes.c_void_p(lo_hi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(ws.data_ptr()), wsn, self._stream(stream))
        _check(rc, "sprintz_quant_nmse")
        self._keep = ws
        return out

    def compress(self, x, opts: Opts = Opts(), stream=None):
        """Compress a (rows, D) uint8 / uint16 (or int16) CUDA tensor.
        Returns (dst, size): the stream buffer and a device uint64 size."""
        torch = self.torch
        if x.dim() == 1:
            x = x.view(-1, 1)
        if x.dtype not in (torch.uint8, torch.int16, torch.uint16):
            raise TypeError("samples must be uint8 or 16-bit")
        x = x.contiguous()
        rows, D = x.shape
        w = 8 if x.dtype == torch.uint8 else 16
        cap = max_compressed_size(rows, D, w, opts)
        if cap == 0:
            raise SprintzError(ERR_INVALID_ARG, "sprintz_max_compressed_size")
        dst = torch.empty(cap, dtype=torch.uint8, device=x.device)
        size = torch.zeros(1, dtype=torch.int64, device=x.device)
        wsn = compress_workspace_size(rows, D, w, opts)
        ws = torch.empty(wsn, dtype=torch.uint8, device=x.device) if wsn else None
        self.compress_into(x, rows, D, w, opts, dst, size, ws, stream)
        return dst, size

    def decompress_into(self, src, src_size: int, info: Info, dst, ws, stream=None) -> None:
        ci = info.c()
        rc = lib().sprintz_decompress(self.ctx, ctypes.c_void_p(src.data_ptr()), src_size,
                                      ctypes.byref(ci),
                                      ctypes.c_void_p(dst.data_ptr() if dst.numel() else 0),
                                      dst.numel() * dst.element_size(),
                                      ctypes.c_void_p(ws.data_ptr() if ws is not None else 0),
                                      ws.numel() if ws is not None else 0, self._stream(stream))
        _check(rc, "sprintz_decompress")

    def decompress(self, src, info: Info, src_size: int | None = None, stream=None):
        """Decompress a device stream; `info` comes from query() on a host copy
        of its header. Returns a (rows, D) uint8 / int16 tensor."""
        torch = self.torch
        dt = torch.uint8 if info.w == 8 else torch.int16
        dst = torch.empty((info.rows, info.D), dtype=dt, device=src.device)
        wsn = decompress_workspace_size(info)
        ws = torch.empty(wsn, dtype=torch.uint8, device=src.device) if wsn else None
        n = src_size if src_size is not None else src.numel()
        self.decompress_into(src, n, info, dst, ws, stream)
        return dst

    def decompress_rows(self, src, info: Info, row_begin: int, row_end: int, src_size: int | None = None,
                        out=None, stream=None):
        """sprintz_decompress_rows: rows [row_begin, row_end) of a device
        stream as a (row_end - row_begin, D) tensor (only the covering chunks
        are decoded)."""
        torch = self.torch
        dt = torch.uint8 if info.w == 8 else torch.int16
        n = max(0, row_end - row_begin)
        y = out if out is not None else torch.empty((n, info.D), dtype=dt, device=src.device)
        ci = info.c()
        wsn = int(lib().sprintz_decompress_rows_workspace_size(ctypes.byref(ci), row_begin, row_end))
        ws = torch.empty(max(wsn, 1), dtype=torch.uint8, device=src.device)
        rc = lib().sprintz_decompress_rows(self.ctx, ctypes.c_void_p(src.data_ptr()),
                                           src_size if src_size is not None else src.numel(), ctypes.byref(ci),
                                           row_begin, row_end, ctypes.c_void_p(y.data_ptr() if n else 0),
                                           y.numel() * y.element_size(), ctypes.c_void_p(ws.data_ptr()), wsn,
                                           self._stream(stream))
        _check(rc, "sprintz_decompress_rows")
        self._keep = ws
        return y

    def append(self, src, info: Info, rows, src_size: int | None = None, stream=None):
        """sprintz_append: the stream of the old series followed by `rows`
        ((n, D) device tensor of the stream's w). Returns (dst, size)."""
        torch = self.torch
        if rows.dim() == 1:
            rows = rows.view(-1, 1)
        rows = rows.contiguous()
        n = rows.shape[0]
        ci = info.c()
        cap = max_compressed_size(info.rows + n, info.D, info.w, info.opts)
        dst = torch.empty(cap, dtype=torch.uint8, device=src.device)
        size = torch.zeros(1, dtype=torch.int64, device=src.device)
        wsn = int(lib().sprintz_append_workspace_size(ctypes.byref(ci), n))
        if wsn == 0:
            raise SprintzError(ERR_UNSUPPORTED if info.opts.huffman else ERR_INVALID_ARG,
                               "sprintz_append_workspace_size")
        ws = torch.empty(wsn, dtype=torch.uint8, device=src.device)
        rc = lib().sprintz_append(self.ctx, ctypes.c_void_p(src.data_ptr()),
                                  src_size if src_size is not None else src.numel(), ctypes.byref(ci),
                                  ctypes.c_void_p(rows.data_ptr() if n else 0), n, ctypes.c_void_p(dst.data_ptr()),
                                  cap, ctypes.c_void_p(size.data_ptr()), ctypes.c_void_p(ws.data_ptr()), wsn,
                                  self._stream(stream))
        _check(rc, "sprintz_append")
        self._keep = ws
        return dst, size

    def pack(self, src_ptrs, sizes, dst, offsets, stream=None) -> None:
        """sprintz_pack: the buffers at the device addresses src_ptrs (int64
        device tensor) of device sizes `sizes` (int64 tensor) back to back in
        dst; offsets (int64 tensor, n + 1) receives where each starts."""
        n = int(src_ptrs.numel())
        rc = lib().sprintz_pack(self.ctx, ctypes.c_void_p(src_ptrs.data_ptr()), ctypes.c_void_p(sizes.data_ptr()),
                                n, ctypes.c_void_p(dst.data_ptr()), dst.numel() * dst.element_size(),
                                ctypes.c_void_p(offsets.data_ptr()), self._stream(stream))
        _check(rc, "sprintz_pack")

    def set_failure_test(self, wait_limit: int = 0, skip_first_group: int = 0) -> None:
        """sprintz_ctx_set_failure_test (0, 0 = normal use)."""
        _check(lib().sprintz_ctx_set_failure_test(self.ctx, wait_limit, skip_first_group),
               "sprintz_ctx_set_failure_test")

    def status(self, stream=None) -> int:
        return int(lib().sprintz_get_status(self.ctx, self._stream(stream)))

    def check(self, stream=None) -> None:
        _check(self.status(stream), "device status")

    # ---- batches of independent streams -----------------------------------

    def _items(self, rows_d_w_opts, srcs, src_bytes, dsts, out_sizes, ranges=None):
        """The sprintz_batch_item array, filled column by column with numpy in
        a buffer that the ctypes array views (no per-item Python structs)."""
        import numpy as np
        n = len(rows_d_w_opts)
        buf = np.zeros(n, dtype=_ITEM_DTYPE)
        if n:
            buf["src"] = srcs
            buf["src_bytes"] = src_bytes
            buf["dst"] = [d[0] for d in dsts]
            buf["dst_cap"] = [d[1] for d in dsts]
            buf["out_size"] = out_sizes
            buf["rows"] = [t[0] for t in rows_d_w_opts]
            buf["D"] = [t[1] for t in rows_d_w_opts]
            buf["w"] = [t[2] for t in rows_d_w_opts]
            opts = [t[3] for t in rows_d_w_opts]
            first = opts[0]
            if all(o is first or o == first for o in opts):
                opts = [first] * n
            for name in ("forecaster", "huffman", "group_blocks", "learn_shift", "chunk_rows", "huff_chunks"):
                buf[name] = [getattr(o, name) for o in opts]
            if ranges:
                buf["row_begin"] = [r[0] for r in ranges]
                buf["row_end"] = [r[1] for r in ranges]
        arr = (_BatchItem * n).from_buffer(buf)
        arr._keep = buf  # the numpy buffer backs the ctypes array
        return arr

    def batch_plan_run(self, arr, compress: int, stream=None, schedule: "Schedule | None" = None,
                       autotune: bool = False, run: bool = True):
        """Size a workspace, plan the batch into it (with `schedule`, or the
        context's remembered/default one; autotune=True searches for the
        fastest schedule first, running the batch several times) and run it
        once; returns the workspace (keep it to call batch_run again)."""
        n = len(arr)
        wsn = int(lib().sprintz_batch_workspace_size(self.ctx, arr, n, compress))
        if wsn == 0:
            raise SprintzError(ERR_INVALID_ARG, "sprintz_batch_workspace_size")
        ws = self.torch.empty(wsn, dtype=self.torch.uint8, device=f"cuda:{self.device}")
        wp, st = ctypes.c_void_p(ws.data_ptr()), self._stream(stream)
        if autotune:
            chosen, ms = _Schedule(), ctypes.c_float()
            _check(lib().sprintz_batch_autotune(self.ctx, arr, n, compress, wp, wsn, st, ctypes.byref(chosen),
                                                ctypes.byref(ms)), "sprintz_batch_autotune")
            self.last_tune = (Schedule.of(chosen), float(ms.value))
        elif schedule is not None:
            sc = schedule.c()
            _check(lib().sprintz_batch_plan_schedule(self.ctx, arr, n, compress, ctypes.byref(sc), wp, wsn, st),
                   "sprintz_batch_plan_schedule")
        else:
            _check(lib().sprintz_batch_plan(self.ctx, arr, n, compress, wp, wsn, st), "sprintz_batch_plan")
        if run:
            self.batch_run(ws, stream)
        return ws

    def batch_schedule(self) -> Schedule:
        """The resolved schedule of the current plan."""
        c = _Schedule()
        _check(lib().sprintz_batch_schedule(self.ctx, ctypes.byref(c)), "sprintz_batch_schedule")
        return Schedule.of(c)

    def batch_run(self, ws, stream=None) -> None:
        _check(lib().sprintz_batch_run(self.ctx, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                       self._stream(stream)), "sprintz_batch_run")

    def compress_batch(self, xs, opts, stream=None, schedule=None, autotune=False, bufs=None, sizes=None):
        """Compress a list of (rows, D) uint8/16-bit device tensors in one
        batched launch; `opts` is one Opts or one per stream. Returns
        (streams, sizes, ws): stream buffers (`bufs` if given: uint8 tensors
        of at least max_compressed_size bytes each), a device int64 tensor of
        sizes (`sizes` if given), and the planned workspace."""
        torch = self.torch
        n = len(xs)
        ol = list(opts) if isinstance(opts, (list, tuple)) else [opts] * n
        shapes, srcs, dsts = [], [], []
        if sizes is None:
            sizes = torch.zeros(n, dtype=torch.int64, device=xs[0].device)
        given = bufs
        bufs = []
        for k, (x, o) in enumerate(zip(xs, ol)):
            x2 = x.view(-1, 1) if x.dim() == 1 else x
            rows, D = x2.shape
            w = 8 if x2.dtype == torch.uint8 else 16
            cap = max_compressed_size(rows, D, w, o)
            buf = given[k] if given is not None else torch.empty(cap, dtype=torch.uint8, device=x.device)
            cap = buf.numel()
            bufs.append(buf)
            shapes.append((rows, D, w, o))
            srcs.append(x2.data_ptr() if rows else 0)
            dsts.append((buf.data_ptr(), cap))
        arr = self._items(shapes, srcs, [0] * n, dsts,
                          [sizes.data_ptr() + 8 * k for k in range(n)])
        ws = self.batch_plan_run(arr, 1, stream, schedule=schedule, autotune=autotune)
        return bufs, sizes, ws

    def decompress_ranges(self, streams, infos, sizes, ranges, outs=None, stream=None):
        """Range requests: rows [a, b) of each device stream, decoded in one
        batched launch (only the covering chunks are decoded). Returns the
        output tensors and the planned workspace."""
        torch = self.torch
        res, shapes, srcs, dsts = [], [], [], []
        for k, (s, info, (a, b)) in enumerate(zip(streams, infos, ranges)):
            dt = torch.uint8 if info.w == 8 else torch.int16
            y = outs[k] if outs is not None else torch.empty((b - a, info.D), dtype=dt, device=s.device)
            res.append(y)
            shapes.append((info.rows, info.D, info.w, info.opts))
            srcs.append(s.data_ptr())
            dsts.append((y.data_ptr(), y.numel() * y.element_size()))
        return res, self.decompress_ranges_into(shapes, srcs, sizes, ranges, dsts, stream)

    def decompress_ranges_into(self, shapes, srcs, sizes, ranges, dsts, stream=None):
        """Range requests given as plain values: each stream's (rows, D, w,
        Opts), device address and byte size, its row range [a, b), and the
        (device address, capacity in bytes) its rows go to. One batched
        launch; returns the planned workspace (keep it until the launch has
        completed)."""
        arr = self._items(shapes, srcs, list(sizes), dsts, [0] * len(shapes), list(ranges))
        return self.batch_plan_run(arr, 0, stream)

    def decompress_batch(self, streams, infos, sizes, stream=None, schedule=None, autotune=False, outs=None):
        """Decompress device streams (with their host-parsed infos and byte
        sizes) in one batched launch into `outs` (or new tensors); returns
        the decoded tensors and the planned workspace."""
        torch = self.torch
        given = outs
        outs, shapes, srcs, dsts = [], [], [], []
        for k, (s, info, n) in enumerate(zip(streams, infos, sizes)):
            dt = torch.uint8 if info.w == 8 else torch.int16
            y = given[k] if given is not None else torch.empty((info.rows, info.D), dtype=dt, device=s.device)
            outs.append(y)
            shapes.append((info.rows, info.D, info.w, info.opts))
            srcs.append(s.data_ptr())
            dsts.append((y.data_ptr() if y.numel() else 0, y.numel() * y.element_size()))
        arr = self._items(shapes, srcs, list(sizes), dsts, [0] * len(streams))
        ws = self.batch_plan_run(arr, 0, stream, schedule=schedule, autotune=autotune)
        return outs, ws

