"""Benchmark of the CUDA Sprintz codec on its headline workload.

Workload (default): uint16, D = 8 columns, 2^24 rows (256 MiB) of the seeded
sensor-like generator (two sinusoids + Gaussian noise + 5 % flat stretches),
FIRE forecaster, bit packing + zero-block runs, chunk_rows 1024, G = 2.
One step = one compress and one decompress of the whole series (the hot path
in both directions), inputs resident in HBM. `value` is uncompressed GB/s of
the round trip; per-direction GB/s and the dominant kernel's HBM roofline
are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU, each rank on its own copy of
the workload (independent streams: weak scaling, no collective on the data
path); the barrier-bracketed time is the max over ranks.
`--impl reference` times the CPU oracle (the plain scalar C codec) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
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
WORKLOAD = "sensor_u16_D8_2^24rows_FIRE"
ROWS, COLS, SEED = 1 << 24, 8, 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", type=int, default=ROWS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--workload", default="sensor",
                    choices=["sensor", "walk", "batch", "huffman", "serve", "fire_speed", "dsweep", "gsweep",
                             "quantize"])
    ap.add_argument("--streams", type=int, default=10_000, help="batch: number of streams")
    ap.add_argument("--huff-rows", type=int, default=1 << 28, help="huffman: rows of the accel series")
    ap.add_argument("--e2e-lanes", type=int, default=4, help="end to end: steps in flight (streams)")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    return ap.parse_args()


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


def traffic_bytes(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary
    (profiles/traffic.json), or None when the kernel sources changed since
    the counters were taken."""
    import hashlib
    root = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(root, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    csrc = os.path.join(root, "paper_1808_02515_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    if rec.get("sources_sha256") != h.hexdigest():
        return None
    k = rec.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


def slowest_rank_ms(ms, dist, device):
    """The job's time: the largest of the ranks' times (all ranks get it)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(bytes_per_rank, world, ms):
    """Whole-job throughput: every rank's units over the slowest rank's time
    (weak scaling: each rank encodes and decodes its own series)."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def rank_seed(rank):
    """Each rank draws its own series (no data crosses ranks)."""
    return SEED + rank


def run_reference(args, rank, world):
    """The oracle timed on the host cores on a bounded sample of the workload."""
    if rank != 0:
        return
    import oracle
    from paper_1808_02515_gb300 import synth
    oracle.build()
    sample_rows = 1 << 20
    x = synth.sensor_u16(sample_rows, COLS, seed=SEED)
    o = opts_dict()
    for _ in range(max(0, min(args.warmup, 1))):
        oracle.decompress(oracle.compress(x, **o))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        s = oracle.compress(x, **o)
        oracle.decompress(s)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = x.nbytes / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "compress+decompress round trip",
                       "sample_rows": sample_rows},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {sample_rows} rows of the workload, single thread"},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "sensor":
        from paper_1808_02515_gb300 import bench_workloads
        bench_workloads.run(args, METRIC, ClockSampler, peaks)
        return

    import torch
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import _build, synth

    if rank == 0 or world == 1:
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

    x = synth.sensor_u16(args.rows, COLS, seed=rank_seed(rank))
    U = x.nbytes
    xd = torch.from_numpy(x.view(np.int16)).to(dev)
    codec = spz.Codec(local)
    o = spz.Opts(**opts_dict())
    rows, D, w = args.rows, COLS, 16
    cap = spz.max_compressed_size(rows, D, w, o)
    dst = torch.empty(cap, dtype=torch.uint8, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    wsc = spz.compress_workspace_size(rows, D, w, o)
    ws_c = torch.empty(max(wsc, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # one call to learn the stream's header and size
    codec.compress_into(xd, rows, D, w, o, dst, size, ws_c)
    torch.cuda.synchronize()
    codec.check()
    C = int(size.item())
    info = spz.query(dst[:64].cpu().numpy().tobytes())
    wsd = spz.decompress_workspace_size(info)
    ws_d = torch.empty(max(wsd, 1), dtype=torch.uint8, device=dev)
    out = torch.empty((rows, D), dtype=torch.int16, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        codec.compress_into(xd, rows, D, w, o, dst, size, ws_c)
        if ev is not None:
            ev[1].record(stream)
        codec.decompress_into(dst, C, info, out, ws_d)
        if ev is not None:
            ev[2].record(stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        # keep the GPU busy until the clock sampler delivers (at most 2 s)
        t_w = time.monotonic()
        while not clk.lines and time.monotonic() - t_w < 2.0:
            step()
            torch.cuda.synchronize()
        codec.check()
        if not torch.equal(out, xd):
            raise SystemExit("round trip mismatch")
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        h0 = time.monotonic()
        t_start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        t_end.record(stream)
        torch.cuda.synchronize()
        clk.mark(h0, time.monotonic())
    if dist:
        dist.barrier()
    enc_ms = [e[0].elapsed_time(e[1]) for e in evs]
    dec_ms = [e[1].elapsed_time(e[2]) for e in evs]
    total_ms = slowest_rank_ms(t_start.elapsed_time(t_end), dist, dev)
    ms_step = total_ms / args.steps

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        # End to end through the C ABI with pinned host buffers: every step
        # copies its input samples in, compresses, copies the stream out and
        # back in (a store/load round trip through the host), decompresses and
        # copies the samples out.  Several lanes (each its own CUDA stream and
        # buffers) take steps in turn, so one step's copies overlap the
        # others' kernels and the two copy directions overlap each other.
        nl = max(1, args.e2e_lanes)
        lanes = []
        for _ in range(nl):
            lanes.append({
                "s": torch.cuda.Stream(dev),
                "xh": torch.from_numpy(x.view(np.int16)).pin_memory(),
                "sh": torch.empty(cap, dtype=torch.uint8).pin_memory(),
                "yh": torch.empty((rows, D), dtype=torch.int16).pin_memory(),
                "xin": torch.empty_like(xd),
                "dst": torch.empty(cap, dtype=torch.uint8, device=dev),
                "size": torch.zeros(1, dtype=torch.int64, device=dev),
                "wsc": torch.empty(max(wsc, 1), dtype=torch.uint8, device=dev),
                "wsd": torch.empty(max(wsd, 1), dtype=torch.uint8, device=dev),
                "out": torch.empty((rows, D), dtype=torch.int16, device=dev),
            })

        def e2e_step(L):
            with torch.cuda.stream(L["s"]):
                L["xin"].copy_(L["xh"], non_blocking=True)
                codec.compress_into(L["xin"], rows, D, w, o, L["dst"], L["size"], L["wsc"], stream=L["s"])
                L["sh"][:C].copy_(L["dst"][:C], non_blocking=True)
                L["dst"][:C].copy_(L["sh"][:C], non_blocking=True)
                codec.decompress_into(L["dst"], C, info, L["out"], L["wsd"], stream=L["s"])
                L["yh"].copy_(L["out"], non_blocking=True)

        for k in range(2 * nl):
            e2e_step(lanes[k % nl])
        torch.cuda.synchronize()
        codec.check()
        if not torch.equal(lanes[0]["yh"], lanes[0]["xh"]):
            raise SystemExit("end-to-end round trip mismatch")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n_e2e = max(2 * nl, min(40, args.steps // 10)) // nl * nl
        a.record(lanes[0]["s"])
        for L in lanes[1:]:
            L["s"].wait_event(a)
        for k in range(n_e2e):
            e2e_step(lanes[k % nl])
        for L in lanes[1:]:
            done = torch.cuda.Event()
            done.record(L["s"])
            lanes[0]["s"].wait_event(done)
        b.record(lanes[0]["s"])
        torch.cuda.synchronize()
        e2e_ms = a.elapsed_time(b) / n_e2e
        e2e_ms = slowest_rank_ms(e2e_ms, dist, dev)
        e2e = {"value": job_gbs(U, world, e2e_ms), "unit": "GB/s",
               "h2d_bytes_per_step": U + C, "d2h_bytes_per_step": C + U,
               "ms_per_step": e2e_ms, "steps": n_e2e,
               "pipelining": f"{nl} lanes (streams) take steps in turn"}

    if rank != 0:
        return
    enc_avg, dec_avg = statistics.mean(enc_ms), statistics.mean(dec_ms)
    peak, peak_kind = peaks()
    table = 16 * info.n_chunks
    enc_bytes, dec_bytes = U + C + table, C + U
    dom = "decode" if dec_avg >= enc_avg else "encode"
    dom_kernel = "k_decode_lanes" if dom == "decode" else "k_encode_slots"
    dom_ms = dec_avg if dom == "decode" else enc_avg
    dom_bytes = dec_bytes if dom == "decode" else enc_bytes
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": job_gbs(U, world, ms_step), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "rows": rows, "D": D, "w": w, **opts_dict(),
                   "step": "compress+decompress round trip", "uncompressed_bytes": U,
                   "compressed_bytes": C, "ratio": U / C,
                   "l2": "inputs (256 MiB raw, compressed stream) larger than the 129 MB L2",
                   "parallelism": f"{world} independent streams (one per GPU)"},
        "decompress_gbs": U / (dec_avg * 1e-3) / 1e9,
        "compress_gbs": U / (enc_avg * 1e-3) / 1e9,
        "decompress_ms": dec_avg, "compress_ms": enc_avg,
        "roofline": {"bound": "hbm", "kernel": dom_kernel,
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_bytes(dom_kernel),
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "decode_frac": dec_bytes / (dec_avg * 1e-3) / 1e9 / peak,
                     "encode_frac": enc_bytes / (enc_avg * 1e-3) / 1e9 / peak},
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
    }
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        import oracle
        oracle.build()
        n_s = 1 << 22
        xs = x[:n_s]
        t0 = time.perf_counter()
        s = oracle.compress(xs, **opts_dict())
        oracle.decompress(s)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": xs.nbytes / tc / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {n_s} of {rows} rows, one compress+decompress, "
                                          "single thread"}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
