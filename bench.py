"""Benchmark of the CUDA Sprintz codec on its headline workload.

Workload (default): the batch of 10,000 independent streams, rows
log-uniform in [1e3, 1e6], D uniform in 1..16, even streams uint8 random
walks and odd streams uint16 sensor-like series (about 18 GB), FIRE
forecaster, bit packing + zero-block runs, chunk_rows 1024, G = 2.  One step
= one batched compress and one batched decompress of every stream (the hot
path in both directions, each one persistent launch with the schedule the
library's autotuner picked during warm-up), inputs resident in HBM.
`value` is uncompressed GB/s of the round trip over all ranks; per-direction
GB/s, the delta forecaster, per-stream launches of the same work, the HBM
roofline of both batched kernels, an end-to-end figure through host buffers
and the CPU oracle on the host's cores are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batch|sensor|walk|huffman|serve|...]

--gpus N > 1 starts N ranks (one per GPU) through torch.distributed.run
unless it already runs under it; the 10,000 streams are split into N
contiguous ranges of about equal bytes (no collective on the data path; the
total work is fixed: strong scaling), and the barrier-bracketed time is the
slowest rank's.  `--impl reference` times the CPU oracle (the plain scalar C
codec) on all host cores, on a bounded sample of the same streams.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "decompress and compress GB/s (uncompressed bytes) at 1 GB300 and % HBM roofline"
N_STREAMS = 10_000
WORKLOAD = "batch_10000_streams_rows_logU_1e3_1e6_D1-16_u8u16_FIRE"
SENSOR_WORKLOAD = "sensor_u16_D8_2^24rows_FIRE"
ROWS, COLS, SEED = 1 << 24, 8, 1
NOMINAL_HBM_GBS = 8000.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", type=int, default=ROWS, help="sensor: rows of the series")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="batch: default schedules, no autotuner")
    ap.add_argument("--no-per-stream", action="store_true", help="batch: skip the per-stream launches")
    ap.add_argument("--no-delta", action="store_true", help="batch: skip the delta forecaster")
    ap.add_argument("--no-sensor", action="store_true", help="batch: skip the single-stream sensor series")
    ap.add_argument("--no-graph", action="store_true", help="batch: skip the CUDA-graph replay of the step")
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "sensor", "walk", "huffman", "serve", "fire_speed", "dsweep", "gsweep",
                             "quantize"])
    ap.add_argument("--streams", type=int, default=N_STREAMS, help="batch: number of streams")
    ap.add_argument("--huff-rows", type=int, default=1 << 28, help="huffman: rows of the accel series")
    ap.add_argument("--e2e-lanes", type=int, default=4,
                    help="end to end of the single-stream workloads: CUDA streams taking steps in turn")
    ap.add_argument("--e2e-lag", type=int, default=2,
                    help="end to end: slices between a slice's samples going in and its packed bytes coming back")
    ap.add_argument("--e2e-slices", type=int, default=16, help="end to end: slices of the batch per step")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    return ap.parse_args(argv)


def opts_dict():
    return dict(forecaster=1, huffman=0, group_blocks=2, learn_shift=1, chunk_rows=1024,
                huff_chunks=64)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling (every 50 ms). Each sample is stamped
    on arrival; mark(start, end) keeps only the samples inside the timed
    region when it held any (else all samples are kept)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.window = None

    def _reader(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._reader, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def summary(self):
        rows = [(t, r.split(", ")) for t, r in self.lines if r.count(",") >= 8]
        inside = [r for t, r in rows if self.window and self.window[0] <= t <= self.window[1]]
        sel = inside if inside else [r for _, r in rows]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in sel if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in sel if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in sel for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(sel),
                "samples_in_timed_region": len(inside)}


def sources_sha256(files):
    """Hash of the named files of the CUDA sources (the set one kernel is built from)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1808_02515_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(files):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def traffic_bytes(kernel: str):
    """DRAM bytes per launch of `kernel` on this workload from the committed
    ncu summary (profiles/traffic.json), or None when the kernel's sources
    changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        k = rec["kernels"][kernel]
        if k.get("sources_sha256") != sources_sha256(k["sources"]):
            return None
        return k.get("dram_bytes_per_launch")
    except Exception:
        return None


def slowest_rank_ms(ms, dist, device):
    """The job's time: the largest of the ranks' times (all ranks get it)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(bytes_per_rank, world, ms):
    """Whole-job throughput when every rank moves the same bytes."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def total_gbs(total_bytes, ms):
    """Whole-job throughput: all ranks' bytes over the slowest rank's time."""
    return total_bytes / (ms * 1e-3) / 1e9


def rank_seed(rank):
    """Single-stream workload: each rank draws its own series."""
    return SEED + rank


def rank_streams(rank, world, n_streams=N_STREAMS):
    """This rank's contiguous range of the batch's stream ids (byte-balanced)."""
    from paper_1808_02515_gb300 import shard, synth
    shapes = [synth.batch_stream_shape(i) for i in range(n_streams)]
    nbytes = [r * d * (w // 8) for r, d, w in shapes]
    lo, hi = shard.partition_streams(nbytes, world)[rank]
    return list(range(lo, hi)), shapes, nbytes


def launch_ranks(args) -> bool:
    """--gpus N > 1 outside torch.distributed.run: start N ranks through it
    (this process waits and returns its exit code). False when nothing was
    started (one GPU, or already a rank)."""
    if args.gpus <= 1 or "RANK" in os.environ:
        return False
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__), *sys.argv[1:]]
    raise SystemExit(subprocess.call(cmd))


class Cudart:
    """cudaMemcpyAsync from the CUDA runtime torch loaded (one call per
    compressed stream in the end-to-end figure: torch's per-call overhead
    would dominate 20,000 small copies a step)."""

    H2D, D2H = 1, 2

    def __init__(self):
        import torch  # noqa: F401  (loads the runtime)
        lib = None
        for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise RuntimeError("CUDA runtime library not found")
        lib.cudaMemcpyAsync.restype = ctypes.c_int
        lib.cudaMemcpyAsync.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int,
                                        ctypes.c_void_p]
        self.lib = lib

    def copy(self, dst: int, src: int, n: int, kind: int, stream) -> None:
        rc = self.lib.cudaMemcpyAsync(dst, src, n, kind, stream)
        if rc != 0:
            raise RuntimeError(f"cudaMemcpyAsync failed ({rc})")


class PinnedBuffer:
    """Page-locked host memory of exactly `n` bytes (cudaHostAlloc), seen as
    a numpy uint8 array.  Pinned from the start: host buffers that the GPU
    first read as pageable memory copy far slower once registered later."""

    def __init__(self, n: int, cudart: "Cudart"):
        lib = cudart.lib
        lib.cudaHostAlloc.restype = ctypes.c_int
        lib.cudaHostAlloc.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_uint]
        lib.cudaFreeHost.restype = ctypes.c_int
        lib.cudaFreeHost.argtypes = [ctypes.c_void_p]
        self.lib, self.n, self.ptr = lib, max(int(n), 1), ctypes.c_void_p()
        if lib.cudaHostAlloc(ctypes.byref(self.ptr), self.n, 0) != 0:
            raise RuntimeError(f"cudaHostAlloc of {self.n} bytes failed")
        self.array = np.ctypeslib.as_array((ctypes.c_uint8 * self.n).from_address(self.ptr.value))

    def free(self) -> None:
        if self.ptr.value:
            self.array = None
            self.lib.cudaFreeHost(self.ptr)
            self.ptr = ctypes.c_void_p()


def oracle_sample(ids, every):
    """Every `every`-th of the given stream ids (at least one)."""
    s = ids[::max(1, every)]
    return s if s else ids[:1]


def run_reference(args, rank, world):
    """The oracle, timed on the host cores (all of them, one stream per
    thread) on a bounded sample of the workload's streams: each step
    compresses and decompresses every sampled stream (FIRE)."""
    if rank != 0:
        return
    import oracle
    from paper_1808_02515_gb300 import synth
    oracle.build()
    every = getattr(args, "ref_every", 200)
    ids = oracle_sample(list(range(N_STREAMS)), every)
    xs = oracle.map_streams(synth.batch_stream, ids)
    U = sum(x.nbytes for x in xs)
    o = opts_dict()
    cores = oracle.host_cores()

    def step():
        oracle.decompress_many(oracle.compress_many(xs, o, cores), cores)

    for _ in range(max(0, min(args.warmup, 1))):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = U / t / 1e9
    sample = (f"{len(ids)} of the {N_STREAMS} streams (every {every}th, {U / 1e6:.0f} MB), "
              f"compress + decompress per step, one stream per thread")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "u8/u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "compress + decompress round trip (FIRE)",
                       "sample_streams": len(ids), "sample_bytes": U},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(xs_host, every_one=10):
    """The oracle on the host cores: all cores over the given streams, one
    core over every `every_one`-th of them (compress + decompress, FIRE)."""
    import oracle
    oracle.build()
    o = opts_dict()
    cores = oracle.host_cores()
    res = {}
    for label, xs, threads in (("all", xs_host, cores), ("one", oracle_sample(xs_host, every_one), 1)):
        U = sum(x.nbytes for x in xs)
        t0 = time.perf_counter()
        oracle.decompress_many(oracle.compress_many(xs, o, threads), threads)
        t = time.perf_counter() - t0
        res[label] = (U / t / 1e9, len(xs), U, threads)
    v, n, U, c = res["all"]
    v1, n1, U1, _ = res["one"]
    return {"value": v, "unit": "GB/s", "cores": c, "kind": "oracle",
            "sample": f"{n} of the streams ({U / 1e6:.0f} MB), one compress + decompress each, "
                      "one stream per thread",
            "single_core": {"value": v1, "unit": "GB/s", "cores": 1,
                            "sample": f"{n1} streams ({U1 / 1e6:.0f} MB)"}}


def _aligned_offsets(sizes, align=256):
    offs, o = [], 0
    for n in sizes:
        offs.append(o)
        o += (int(n) + align - 1) // align * align
    return offs, max(o, align)


class BatchWorkload:
    """This rank's streams on the device, laid out in `n_slices` contiguous
    slices (each slice one buffer: inputs, outputs and stream buffers alike),
    so that a slice moves to or from the host in one copy.  The streams are
    drawn with the numpy recipe (synth.batch_stream) on all host cores, one
    stream per thread, straight into one pinned host buffer per slice with
    the device layout (`host`, kept: the end-to-end figure's host input)."""

    def __init__(self, ids, shapes, nbytes, n_slices, dev, spz, synth, torch):
        from concurrent.futures import ThreadPoolExecutor

        from paper_1808_02515_gb300 import shard
        self.ids = ids
        self.dev = dev
        n = len(ids)
        self.slices = [s for s in shard.partition_streams([nbytes[i] for i in ids], max(1, min(n_slices, n)))
                       if s[1] > s[0]]
        o = spz.Opts(**opts_dict())
        self.xs, self.outs, self.bufs = [None] * n, [None] * n, [None] * n
        self.in_bufs, self.out_bufs, self.st_bufs, self.host, self.pinned = [], [], [], [], []
        self.cudart = Cudart()
        t0 = time.perf_counter()
        plan = []
        for a, b in self.slices:
            sz = [nbytes[ids[k]] for k in range(a, b)]
            offs, tot = _aligned_offsets(sz)
            caps = [spz.max_compressed_size(*shapes[ids[k]], o) for k in range(a, b)]
            coffs, ctot = _aligned_offsets(caps)
            buf = PinnedBuffer(tot, self.cudart)
            buf.array[:] = 0
            self.pinned.append(buf)
            self.host.append(buf.array[:tot])
            plan.append((a, b, sz, offs, tot, caps, coffs, ctot))

        def draw(job):
            s_i, k, lo, nb = job
            x = synth.batch_stream(ids[k])
            self.host[s_i][lo:lo + nb] = x.reshape(-1).view(np.uint8)

        jobs = [(s_i, k, offs[k - a], sz[k - a]) for s_i, (a, b, sz, offs, *_) in enumerate(plan)
                for k in range(a, b)]
        with ThreadPoolExecutor(max(1, len(os.sched_getaffinity(0)))) as ex:
            list(ex.map(draw, jobs))
        for s_i, (a, b, sz, offs, tot, caps, coffs, ctot) in enumerate(plan):
            xin = torch.empty(tot, dtype=torch.uint8, device=dev)
            self.cudart.copy(xin.data_ptr(), self.host[s_i].ctypes.data, tot, Cudart.H2D,
                             torch.cuda.current_stream(dev).cuda_stream)
            xout = torch.zeros(tot, dtype=torch.uint8, device=dev)
            st = torch.empty(ctot, dtype=torch.uint8, device=dev)
            for k in range(a, b):
                rows, D, w = shapes[ids[k]]
                dt = torch.uint8 if w == 8 else torch.int16
                lo, nb = offs[k - a], sz[k - a]
                self.xs[k] = xin[lo:lo + nb].view(dt).view(rows, D)
                self.outs[k] = xout[lo:lo + nb].view(dt).view(rows, D)
                self.bufs[k] = st[coffs[k - a]:coffs[k - a] + caps[k - a]]
            self.in_bufs.append(xin)
            self.out_bufs.append(xout)
            self.st_bufs.append(st)
        torch.cuda.synchronize()
        self.gen_s = time.perf_counter() - t0
        self.U = sum(nbytes[i] for i in ids)
        self.chunks = sum(-(-(shapes[i][0] - shapes[i][0] % 8) // 1024) if shapes[i][0] >= 8 else 0 for i in ids)

    def free(self):
        for b in self.pinned:
            b.free()
        self.pinned, self.host = [], []

    def host_stream(self, k):
        """Host copy of stream k (a view of the slice's host buffer)."""
        for s_i, (a, b) in enumerate(self.slices):
            if a <= k < b:
                lo = self.xs[k].data_ptr() - self.in_bufs[s_i].data_ptr()
                x = self.host[s_i][lo:lo + self.xs[k].numel() * self.xs[k].element_size()]
                return x.view(np.uint8 if self.xs[k].element_size() == 1 else np.uint16).reshape(self.xs[k].shape)
        raise IndexError(k)

    def outputs_equal_inputs(self, torch):
        return all(torch.equal(a, b) for a, b in zip(self.in_bufs, self.out_bufs))


def sensor_extra(args, dev, local, spz, synth, torch, stream):
    """One compress and one decompress of the 2^24 x 8 uint16 sensor series
    (FIRE, chunk_rows 1024) per step, CUDA events, the lane kernels."""
    x = synth.sensor_u16_torch(ROWS, COLS, seed=SEED, device=dev)
    rows, D, w = ROWS, COLS, 16
    o = spz.Opts(**opts_dict())
    codec = spz.Codec(local)
    try:
        dst = torch.empty(spz.max_compressed_size(rows, D, w, o), dtype=torch.uint8, device=dev)
        size = torch.zeros(1, dtype=torch.int64, device=dev)
        ws_c = torch.empty(max(spz.compress_workspace_size(rows, D, w, o), 1), dtype=torch.uint8, device=dev)
        codec.compress_into(x, rows, D, w, o, dst, size, ws_c)
        torch.cuda.synchronize()
        C = int(size.item())
        info = spz.query(dst[:64].cpu().numpy().tobytes())
        ws_d = torch.empty(max(spz.decompress_workspace_size(info), 1), dtype=torch.uint8, device=dev)
        out = torch.empty_like(x)
        steps = max(3, args.steps)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps + 3)]
        for k in range(steps + 3):
            ev[k][0].record(stream)
            codec.compress_into(x, rows, D, w, o, dst, size, ws_c)
            ev[k][1].record(stream)
            codec.decompress_into(dst, C, info, out, ws_d)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
        codec.check()
        if not torch.equal(out, x):
            raise SystemExit("single-stream round trip mismatch")
        enc = statistics.mean(e[0].elapsed_time(e[1]) for e in ev[3:])
        dec = statistics.mean(e[1].elapsed_time(e[2]) for e in ev[3:])
        U = x.numel() * 2
        peak, _ = peaks()
        return {"workload": SENSOR_WORKLOAD, "uncompressed_bytes": U, "compressed_bytes": C, "ratio": U / C,
                "compress_gbs": U / (enc * 1e-3) / 1e9, "decompress_gbs": U / (dec * 1e-3) / 1e9,
                "compress_ms": enc, "decompress_ms": dec,
                "encode_frac": (U + C + 16 * info.n_chunks) / (enc * 1e-3) / 1e9 / peak,
                "decode_frac": (U + C) / (dec * 1e-3) / 1e9 / peak,
                "kernels": "k_encode_slots<16, 8>, k_decode_lanes<16, 8>", "steps": steps,
                "generator": "sensor_u16 recipe drawn on the GPU (torch)"}
    finally:
        codec.close()


def _headers(bufs, torch):
    """Host copies of every stream's 64-byte header (one gather, one copy)."""
    return torch.stack([b[:64] for b in bufs]).cpu().numpy()


def run_e2e(wl, F, args, dev, local, dist, spz, torch, U_total):
    """End to end through the public API with pinned host buffers.  Every
    step, per slice of the batch: one host-to-device copy of its samples, a
    batched compress, sprintz_pack of its compressed streams into one
    device buffer, one device-to-host copy of those bytes and one back (a
    store / load round trip through the host), a batched decompress reading
    the packed streams, and one device-to-host copy of the decoded samples
    into the host buffer the inputs came from (the round trip is lossless,
    so every step's input is again the workload).  The slices run as a
    pipeline over four CUDA streams, one per copy direction, one for the
    compressions (with their packs) and one for the decompressions, linked
    by an event per slice and stage, so that both copy engines stay busy
    while the kernels run between them: slice s's samples go in while slice
    s - lag's packed bytes come back."""
    cr = wl.cudart
    in_sizes = [t.numel() for t in wl.in_bufs]
    lag = max(1, args.e2e_lag)
    s_h2d, s_d2h, s_enc, s_dec = [torch.cuda.Stream(dev) for _ in range(4)]
    sc = spz.Schedule(**{k: v for k, v in F["sched"]["compress"].items() if k != "tune_ms"})
    sd = spz.Schedule(**{k: v for k, v in F["sched"]["decompress"].items() if k != "tune_ms"})
    sz = F["sz"]
    sl = []
    tot = [sum(sz[lo:hi]) for lo, hi in wl.slices]
    h_off, h_tot = _aligned_offsets(tot, 256)
    hc = PinnedBuffer(h_tot, cr)
    try:
        for s_i, (lo, hi) in enumerate(wl.slices):
            cc, cd = spz.Codec(local), spz.Codec(local)
            _, _, wsc = cc.compress_batch(wl.xs[lo:hi], F["o"], stream=s_enc, schedule=sc, bufs=wl.bufs[lo:hi],
                                          sizes=F["sizes"][lo:hi])
            ptrs = torch.tensor([b.data_ptr() for b in wl.bufs[lo:hi]], dtype=torch.int64, device=dev)
            offs = torch.zeros(hi - lo + 1, dtype=torch.int64, device=dev)
            pk = torch.empty(max(tot[s_i], 1), dtype=torch.uint8, device=dev)
            # the packed streams, where the warm-up sizes put them (the sizes are
            # the same every step: the inputs are)
            o_host = np.concatenate([[0], np.cumsum(sz[lo:hi])]).astype(np.int64)
            views = [pk[int(o_host[k]):int(o_host[k + 1])] for k in range(hi - lo)]
            cc.pack(ptrs, F["sizes"][lo:hi], pk, offs, stream=s_enc)  # the plan below runs once on them
            _, wsd = cd.decompress_batch(views, F["infos"][lo:hi], sz[lo:hi], stream=s_enc, schedule=sd,
                                         outs=wl.outs[lo:hi])
            sl.append((cc, cd, wsc, wsd, ptrs, offs, pk))
        torch.cuda.synchronize()
        in_ptr = [t.data_ptr() for t in wl.in_bufs]
        out_ptr = [t.data_ptr() for t in wl.out_bufs]
        hin_ptr = [h.ctypes.data for h in wl.host]
        hc_ptr = hc.ptr.value
        S = len(sl)
        ev = {k: [torch.cuda.Event() for _ in range(S)] for k in ("in", "enc", "pkd", "pkh", "dec", "out")}

        def stage_a(s):
            """Samples in, compress and pack, packed bytes out."""
            cc, _, wsc, _, ptrs, offs, pk = sl[s]
            lo, hi = wl.slices[s]
            cr.copy(in_ptr[s], hin_ptr[s], in_sizes[s], Cudart.H2D, s_h2d.cuda_stream)
            ev["in"][s].record(s_h2d)
            s_enc.wait_event(ev["in"][s])
            s_enc.wait_event(ev["dec"][s])  # the previous step's decompress has read pk
            cc.batch_run(wsc, stream=s_enc)
            cc.pack(ptrs, F["sizes"][lo:hi], pk, offs, stream=s_enc)
            ev["enc"][s].record(s_enc)
            s_d2h.wait_event(ev["enc"][s])
            cr.copy(hc_ptr + h_off[s], pk.data_ptr(), tot[s], Cudart.D2H, s_d2h.cuda_stream)
            ev["pkd"][s].record(s_d2h)

        def stage_b(s):
            """Packed bytes back in, decompress, samples out."""
            _, cd, _, wsd, _, _, pk = sl[s]
            s_h2d.wait_event(ev["pkd"][s])
            cr.copy(pk.data_ptr(), hc_ptr + h_off[s], tot[s], Cudart.H2D, s_h2d.cuda_stream)
            ev["pkh"][s].record(s_h2d)
            s_dec.wait_event(ev["pkh"][s])
            s_dec.wait_event(ev["out"][s])  # the previous step's samples have left
            cd.batch_run(wsd, stream=s_dec)
            ev["dec"][s].record(s_dec)
            s_d2h.wait_event(ev["dec"][s])
            cr.copy(hin_ptr[s], out_ptr[s], in_sizes[s], Cudart.D2H, s_d2h.cuda_stream)
            ev["out"][s].record(s_d2h)

        def step():
            for s in range(S + lag):
                if s < S:
                    stage_a(s)
                if 0 <= s - lag < S:
                    stage_b(s - lag)

        step()
        torch.cuda.synchronize()
        a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_e2e = 3
        a2.record(s_h2d)
        for st in (s_d2h, s_enc, s_dec):
            st.wait_event(a2)
        for _ in range(n_e2e):
            step()
        for st in (s_d2h, s_enc, s_dec):
            done = torch.cuda.Event()
            done.record(st)
            s_h2d.wait_event(done)
        b2.record(s_h2d)
        torch.cuda.synchronize()
        for cc, cd, *_ in sl:
            cc.check()
            cd.check()
        if not all(torch.equal(torch.from_numpy(h).to(dev), t) for h, t in zip(wl.host, wl.in_bufs)):
            raise SystemExit("end-to-end round trip mismatch")
        e2e_ms = slowest_rank_ms(a2.elapsed_time(b2) / n_e2e, dist, dev)
        C = sum(tot)
        return {"value": total_gbs(U_total, e2e_ms), "unit": "GB/s",
                "h2d_bytes_per_step": sum(in_sizes) + C, "d2h_bytes_per_step": C + sum(in_sizes),
                "ms_per_step": e2e_ms, "steps": n_e2e,
                "pipelining": f"{S} slices; one CUDA stream per copy direction, one for compress + pack, one "
                              f"for decompress, an event per slice and stage; slice s's samples go in while "
                              f"slice s - {lag}'s packed bytes come back; pinned host buffers (cudaHostAlloc); "
                              "per slice one copy of its samples each way and one of its packed compressed "
                              "streams each way (sprintz_pack); the decoded samples return into the host "
                              "buffer the inputs came from"}
    finally:
        for cc, cd, *_ in sl:
            cc.close()
            cd.close()
        hc.free()


def run_batch(args, rank, world, local):
    import torch
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import _build, synth

    if rank == 0:
        _build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        _build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)

    ids, shapes, nbytes = rank_streams(rank, world, args.streams)
    wl = BatchWorkload(ids, shapes, nbytes, args.e2e_slices, dev, spz, synth, torch)
    U_total = sum(nbytes[:args.streams])
    tune = not args.no_tune

    def plans(fc, label):
        o = spz.Opts(**{**opts_dict(), "forecaster": fc})
        cc, cd = spz.Codec(local), spz.Codec(local)
        sizes = torch.zeros(len(ids), dtype=torch.int64, device=dev)
        _, _, ws_c = cc.compress_batch(wl.xs, o, autotune=tune, bufs=wl.bufs, sizes=sizes)
        tc = cc.last_tune if tune else (cc.batch_schedule(), None)
        torch.cuda.synchronize()
        cc.check()
        sz = [int(v) for v in sizes.cpu().numpy()]
        infos = [spz.query(h.tobytes()) for h in _headers(wl.bufs, torch)]
        _, ws_d = cd.decompress_batch(wl.bufs, infos, sz, autotune=tune, outs=wl.outs)
        td = cd.last_tune if tune else (cd.batch_schedule(), None)
        torch.cuda.synchronize()
        cd.check()
        if not wl.outputs_equal_inputs(torch):
            raise SystemExit(f"batched round trip mismatch ({label})")
        sched = {"compress": {**vars(tc[0]), "tune_ms": tc[1]}, "decompress": {**vars(td[0]), "tune_ms": td[1]}}
        return dict(o=o, cc=cc, cd=cd, ws_c=ws_c, ws_d=ws_d, sizes=sizes, sz=sz, infos=infos, sched=sched,
                    C=sum(sz))

    step_ms = {}

    def timed(P, steps, keep=False):
        """Mean compress and decompress ms per step over `steps` steps (keep:
        also their best and median into step_ms)."""
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        for k in range(steps):
            ev[k][0].record(stream)
            P["cc"].batch_run(P["ws_c"])
            ev[k][1].record(stream)
            P["cd"].batch_run(P["ws_d"])
            ev[k][2].record(stream)
        torch.cuda.synchronize()
        enc = [e[0].elapsed_time(e[1]) for e in ev]
        dec = [e[1].elapsed_time(e[2]) for e in ev]
        if keep:
            step_ms.update({"compress_best": min(enc), "compress_median": statistics.median(enc),
                            "decompress_best": min(dec), "decompress_median": statistics.median(dec)})
        return statistics.mean(enc), statistics.mean(dec)

    F = plans(1, "FIRE")
    with ClockSampler(local) as clk:
        timed(F, max(1, args.warmup))
        t_w = time.monotonic()
        while not clk.lines and time.monotonic() - t_w < 2.0:
            timed(F, 1)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0 = time.monotonic()
        a.record(stream)
        enc_ms, dec_ms = timed(F, args.steps, keep=True)
        b.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.monotonic())
    if dist:
        dist.barrier()
    total_ms = slowest_rank_ms(a.elapsed_time(b), dist, dev)
    ms_step = total_ms / args.steps
    F["cc"].check()
    F["cd"].check()
    if not wl.outputs_equal_inputs(torch):
        raise SystemExit("batched round trip mismatch after the timed steps")
    res = {"enc_ms": enc_ms, "dec_ms": dec_ms}

    # the same step as one CUDA graph (both directions' memsets and kernels
    # captured once), replayed `steps` times; single-rank runs only, so that a
    # capture refused on one rank cannot leave the ranks' collectives apart
    graph = None
    if not args.no_graph and dist is None:
        try:
            side = torch.cuda.Stream(dev)
            side.wait_stream(stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=side):
                F["cc"].batch_run(F["ws_c"], stream=side)
                F["cd"].batch_run(F["ws_d"], stream=side)
            torch.cuda.synchronize()
            g.replay()
            torch.cuda.synchronize()
            ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            cur = torch.cuda.current_stream(dev)
            ga.record(cur)
            for _ in range(args.steps):
                g.replay()
            gb.record(cur)
            torch.cuda.synchronize()
            F["cc"].check()
            F["cd"].check()
            if not wl.outputs_equal_inputs(torch):
                raise SystemExit("batched round trip mismatch after the graph replays")
            g_ms = ga.elapsed_time(gb) / args.steps
            graph = {"ms_per_step": g_ms, "round_trip_gbs": total_gbs(U_total, g_ms),
                     "graph_launches_per_step": 1, "steps": args.steps}
            del g
        except SystemExit:
            raise
        except Exception as exc:  # capture unsupported here: say so, keep the line
            graph = {"error": f"{type(exc).__name__}: {exc}"[:200]}

    # per-stream launches of the same work (one context, one shared workspace)
    per_stream = None
    if not args.no_per_stream:
        o = F["o"]
        codec = spz.Codec(local)
        shp = [shapes[i] for i in ids]
        ws_e = torch.empty(max(max(spz.compress_workspace_size(r, d, w, o) for r, d, w in shp), 1),
                           dtype=torch.uint8, device=dev)
        ws_dd = torch.empty(max(max(spz.decompress_workspace_size(i) for i in F["infos"]), 1),
                            dtype=torch.uint8, device=dev)

        def per_enc():
            for k, x in enumerate(wl.xs):
                r, d, w = shp[k]
                codec.compress_into(x, r, d, w, o, wl.bufs[k], F["sizes"][k:k + 1], ws_e)

        def per_dec():
            for k in range(len(ids)):
                codec.decompress_into(wl.bufs[k], F["sz"][k], F["infos"][k], wl.outs[k], ws_dd)

        per_enc()
        per_dec()
        torch.cuda.synchronize()
        codec.check()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(stream)
        per_enc()
        ev[1].record(stream)
        per_dec()
        ev[2].record(stream)
        torch.cuda.synchronize()
        codec.check()
        if not wl.outputs_equal_inputs(torch):
            raise SystemExit("per-stream round trip mismatch")
        pe, pd = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
        per_stream = {"compress_gbs": wl.U / (pe * 1e-3) / 1e9, "decompress_gbs": wl.U / (pd * 1e-3) / 1e9,
                      "compress_ms": pe, "decompress_ms": pd,
                      "launches": "one sprintz_compress / sprintz_decompress call per stream, one CUDA stream"}
        codec.close()

    e2e = None if args.no_e2e else run_e2e(wl, F, args, dev, local, dist, spz, torch, U_total)

    # the delta forecaster (its own autotuned plans; overwrites the stream buffers)
    delta = None
    if not args.no_delta:
        Dl = plans(0, "delta")
        de, dd = timed(Dl, max(1, min(args.steps, 10)))
        delta = {"compress_gbs": wl.U / (de * 1e-3) / 1e9, "decompress_gbs": wl.U / (dd * 1e-3) / 1e9,
                 "compress_ms": de, "decompress_ms": dd, "compressed_bytes": Dl["C"], "ratio": wl.U / Dl["C"],
                 "schedules": Dl["sched"]}
        Dl["cc"].close()
        Dl["cd"].close()

    # the single-stream workload beside it: uint16, D = 8, 2^24 rows, FIRE
    sensor = None if args.no_sensor else sensor_extra(args, dev, local, spz, synth, torch, stream)

    C_total = F["C"]
    chunks_total = wl.chunks
    if dist:
        t = torch.tensor([F["C"], wl.chunks], dtype=torch.int64, device=dev)
        dist.all_reduce(t)
        C_total, chunks_total = int(t[0].item()), int(t[1].item())
    enc_max = slowest_rank_ms(enc_ms, dist, dev)
    dec_max = slowest_rank_ms(dec_ms, dist, dev)
    if rank != 0:
        F["cc"].close()
        F["cd"].close()
        wl.free()
        return
    peak, peak_kind = peaks()
    enc_bytes = U_total + C_total + 16 * chunks_total
    dec_bytes = U_total + C_total
    enc_ach = enc_bytes / (enc_max * 1e-3) / 1e9
    dec_ach = dec_bytes / (dec_max * 1e-3) / 1e9
    dom = "encode" if enc_max >= dec_max else "decode"
    kern = "k_encode_batch" if dom == "encode" else "k_decode_batch"
    ach = enc_ach if dom == "encode" else dec_ach
    line = {
        "metric": METRIC, "value": total_gbs(U_total, ms_step), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u8/u16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "streams": args.streams, **opts_dict(),
                   "step": "batched compress + batched decompress of every stream (FIRE)",
                   "uncompressed_bytes": U_total, "compressed_bytes": C_total, "ratio": U_total / C_total,
                   "chunks": chunks_total,
                   "generator": "synth.batch_stream (numpy PCG64, seed 2 + stream id) on all host cores",
                   "generator_s": wl.gen_s,
                   "l2": "inputs (18 GB) and streams far larger than the 129 MB L2",
                   "parallelism": f"{world} rank(s), each a contiguous byte-balanced range of the streams",
                   "schedules": F["sched"]},
        "compress_gbs": total_gbs(U_total, enc_max), "decompress_gbs": total_gbs(U_total, dec_max),
        "compress_ms": enc_max, "decompress_ms": dec_max, "step_ms": step_ms,
        "roofline": {"bound": "hbm", "kernel": kern, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": ach / peak, "frac_of_nominal_8tbs": ach / NOMINAL_HBM_GBS,
                     "traffic": traffic_bytes(kern),
                     "algorithmic_bytes_per_launch": enc_bytes if dom == "encode" else dec_bytes,
                     "timing": "CUDA events around each sprintz_batch_run (its memset, the header/tail "
                               "kernel and the batched kernel)",
                     "encode": {"kernel": "k_encode_batch", "achieved": enc_ach, "frac": enc_ach / peak,
                                "frac_of_nominal_8tbs": enc_ach / NOMINAL_HBM_GBS,
                                "algorithmic_bytes_per_launch": enc_bytes,
                                "traffic": traffic_bytes("k_encode_batch")},
                     "decode": {"kernel": "k_decode_batch", "achieved": dec_ach, "frac": dec_ach / peak,
                                "frac_of_nominal_8tbs": dec_ach / NOMINAL_HBM_GBS,
                                "algorithmic_bytes_per_launch": dec_bytes,
                                "traffic": traffic_bytes("k_decode_batch")},
                     "encode_frac": enc_ach / peak, "decode_frac": dec_ach / peak},
        "gpu_launches": 4 * args.steps,
        "clocks": clk.summary(),
    }
    if graph:
        line["cuda_graph"] = graph
    if per_stream:
        line["per_stream_launches"] = per_stream
    if sensor:
        line["single_stream_sensor"] = sensor
    if delta:
        line["delta"] = delta
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        sample = oracle_sample(list(range(len(ids))), 50)
        line["cpu_baseline"] = cpu_baseline([wl.host_stream(k).copy() for k in sample])
    print(json.dumps(line), flush=True)
    F["cc"].close()
    F["cd"].close()
    wl.free()


def main():
    args = parse()
    if launch_ranks(args):
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and args.impl == "ours":
        raise SystemExit(f"--gpus {args.gpus} but {world} rank(s) were started")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local)
        return
    from paper_1808_02515_gb300 import bench_workloads
    if args.workload == "sensor":
        bench_workloads.run_sensor(args, sys.modules[__name__], rank, world, local)
        return
    bench_workloads.run(args, METRIC, ClockSampler, peaks)


if __name__ == "__main__":
    main()
