"""Benchmark runners of the workloads other than the headline one (selected
with bench.py --workload): the small single stream, the batch of 10,000
streams (batched launch vs per-stream launches), the Huffman workload,
the serving loop, and the paper's speed sweeps (the forecast step alone over
forecasters and column counts, the codec over column counts, header groups
G and chunk lengths). Each prints one JSON line like bench.py's."""
from __future__ import annotations

import json
import statistics
import time

import numpy as np


def _events(n):
    import torch
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def _time(fn, steps, stream):
    import torch
    a, b = _events(2)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def run(args, metric, ClockSampler, peaks):
    import torch
    import paper_1808_02515_gb300.sprintz as spz
    from paper_1808_02515_gb300 import _build, synth
    _build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    codec = spz.Codec(0)
    stream = torch.cuda.current_stream(dev)
    peak, peak_kind = peaks()
    line = {"metric": metric, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "impl": "ours", "workload_kind": args.workload}

    def single(x, opts, label, w):
        rows, D = x.shape
        cap = spz.max_compressed_size(rows, D, w, opts)
        dst = torch.empty(cap, dtype=torch.uint8, device=dev)
        size = torch.zeros(1, dtype=torch.int64, device=dev)
        wsn = spz.compress_workspace_size(rows, D, w, opts)
        ws = torch.empty(max(wsn, 1), dtype=torch.uint8, device=dev)
        codec.compress_into(x, rows, D, w, opts, dst, size, ws)
        torch.cuda.synchronize()
        codec.check()
        C = int(size.item())
        info = spz.query(dst[:64].cpu().numpy().tobytes())
        wsd = spz.decompress_workspace_size(info)
        ws_d = torch.empty(max(wsd, 1), dtype=torch.uint8, device=dev)
        out = torch.empty_like(x)
        for _ in range(args.warmup):
            codec.compress_into(x, rows, D, w, opts, dst, size, ws)
            codec.decompress_into(dst, C, info, out, ws_d)
        torch.cuda.synchronize()
        codec.check()
        assert torch.equal(out, x), "round trip mismatch"
        with ClockSampler(0) as clk:
            enc = _time(lambda: codec.compress_into(x, rows, D, w, opts, dst, size, ws), args.steps, stream)
            dec = _time(lambda: codec.decompress_into(dst, C, info, out, ws_d), args.steps, stream)
        U = x.numel() * x.element_size()
        extra = 16 * info.n_chunks
        line.update({
            "value": U / ((enc + dec) * 1e-3) / 1e9, "ms_per_step": enc + dec,
            "compress_ms": enc, "decompress_ms": dec,
            "compress_gbs": U / (enc * 1e-3) / 1e9, "decompress_gbs": U / (dec * 1e-3) / 1e9,
            "dtype": "u8" if w == 8 else "u16",
            "config": {"workload": label, "rows": rows, "D": D, "w": w, "forecaster": opts.forecaster,
                       "huffman": opts.huffman, "chunk_rows": opts.chunk_rows, "group_blocks": opts.group_blocks,
                       "huff_chunks": opts.huff_chunks, "uncompressed_bytes": U, "compressed_bytes": C,
                       "ratio": U / C, "step": "compress + decompress round trip"},
            "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                         "decode_frac": (U + C) / (dec * 1e-3) / 1e9 / peak,
                         "encode_frac": (U + C + extra) / (enc * 1e-3) / 1e9 / peak,
                         "traffic": None},
            "clocks": clk.summary()})

    if args.workload == "walk":
        x = torch.from_numpy(synth.random_walk_u8(100_000, 1, seed=0)).to(dev)
        single(x, spz.Opts(forecaster=0), "random_walk_u8_D1_100000rows_delta", 8)
        line["config"]["note"] = "100 KB: launch-latency bound; roofline not meaningful"
    elif args.workload == "huffman":
        rows = args.huff_rows
        x = synth.accel_u8_torch(rows, 3, seed=3, device=dev)
        label = "accel_u8_D3_2^28rows_FIRE_huffman" if rows == 1 << 28 else f"accel_u8_D3_{rows}rows_FIRE_huffman"
        single(x, spz.Opts(forecaster=1, huffman=1, huff_chunks=64), label, 8)
        line["config"]["generator"] = "accel_u8 recipe drawn on the GPU (torch)"
    elif args.workload == "batch":
        run_batch(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz)
    elif args.workload == "serve":
        run_serve(args, codec, dev, line, synth, spz)
    elif args.workload == "fire_speed":
        run_fire_speed(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz)
    elif args.workload == "dsweep":
        run_dsweep(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz)
    elif args.workload == "quantize":
        run_quantize(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz)
    elif args.workload == "gsweep":
        run_gsweep(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz)
    codec.close()
    print(json.dumps(line), flush=True)


def run_batch(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz):
    import torch
    t0 = time.perf_counter()
    xs = [synth.batch_stream_torch(i, device=dev) for i in range(args.streams)]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    U = sum(x.numel() * x.element_size() for x in xs)
    res = {}
    sched = {}
    for fc_name, fc in (("delta", 0), ("fire", 1)):
        opts = spz.Opts(forecaster=fc)
        bufs, sizes, ws_c = codec.compress_batch(xs, opts, autotune=True)
        enc_sched = codec.last_tune
        torch.cuda.synchronize()
        codec.check()
        sz = [int(v) for v in sizes.cpu().numpy()]
        C = sum(sz)
        infos = [spz.query(b[:64].cpu().numpy().tobytes()) for b in bufs]
        outs, ws_d = codec.decompress_batch(bufs, infos, sz, autotune=True)
        dec_sched = codec.last_tune
        torch.cuda.synchronize()
        codec.check()
        for x, y in zip(xs, outs):
            assert torch.equal(x, y), "batched round trip mismatch"
        sched[fc_name] = {"compress": vars(enc_sched[0]) | {"tune_ms": enc_sched[1]},
                          "decompress": vars(dec_sched[0]) | {"tune_ms": dec_sched[1]}}
        # the batched form: one plan, then batch_run per step
        dec_b = _time(lambda: codec.batch_run(ws_d), args.steps, stream)
        _, _, ws_c = codec.compress_batch(xs, opts)
        enc_b = _time(lambda: codec.batch_run(ws_c), args.steps, stream)
        # per-stream launches of the same work (one shared workspace: the
        # launches run one after another on the same CUDA stream)
        shapes = [((x.view(-1, 1) if x.dim() == 1 else x).shape, 8 if x.dtype == torch.uint8 else 16)
                  for x in xs]
        ws_e = torch.empty(max(spz.compress_workspace_size(r, d, w, opts) for (r, d), w in shapes),
                           dtype=torch.uint8, device=dev)
        ws_dd = torch.empty(max(max(spz.decompress_workspace_size(i) for i in infos), 1),
                            dtype=torch.uint8, device=dev)

        def per_stream_enc():
            for k, (x, b) in enumerate(zip(xs, bufs)):
                (rows, D), w = shapes[k]
                codec.compress_into(x, rows, D, w, opts, b, sizes[k:k + 1], ws_e)

        def per_stream_dec():
            for b, info, n, y in zip(bufs, infos, sz, outs):
                codec.decompress_into(b, n, info, y, ws_dd)
        per_stream_enc()
        per_stream_dec()
        torch.cuda.synchronize()
        enc_s = _time(per_stream_enc, max(1, args.steps // 5), stream)
        dec_s = _time(per_stream_dec, max(1, args.steps // 5), stream)
        res[fc_name] = dict(C=C, enc_b=enc_b, dec_b=dec_b, enc_s=enc_s, dec_s=dec_s)
    f = res["fire"]
    line.update({
        "value": U / ((f["enc_b"] + f["dec_b"]) * 1e-3) / 1e9, "ms_per_step": f["enc_b"] + f["dec_b"],
        "dtype": "u8/u16",
        "config": {"workload": f"batch_{args.streams}_streams_log_uniform_1e3_1e6_rows_D1-16_u8u16",
                   "streams": args.streams, "uncompressed_bytes": U, "generator_s": gen_s,
                   "generator": "batch_stream recipe drawn on the GPU (torch)",
                   "step": "batched compress + batched decompress (FIRE)"},
        "batched": {k: {"compress_gbs": U / (v["enc_b"] * 1e-3) / 1e9,
                        "decompress_gbs": U / (v["dec_b"] * 1e-3) / 1e9,
                        "compressed_bytes": v["C"], "ratio": U / v["C"],
                        "decode_frac": (U + v["C"]) / (v["dec_b"] * 1e-3) / 1e9 / peak,
                        "encode_frac": (U + v["C"]) / (v["enc_b"] * 1e-3) / 1e9 / peak}
                    for k, v in res.items()},
        "per_stream_launches": {k: {"compress_gbs": U / (v["enc_s"] * 1e-3) / 1e9,
                                    "decompress_gbs": U / (v["dec_s"] * 1e-3) / 1e9}
                                for k, v in res.items()},
        "schedules": sched,
        "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "traffic": None}})


def run_serve(args, codec, dev, line, synth, spz):
    import torch
    from paper_1808_02515_gb300 import serve
    n_streams, rows, D = 1000, 1 << 20, 4
    t0 = time.perf_counter()
    xs = [synth.sensor_u16_torch(rows, D, seed=4000 + i, device=dev) for i in range(n_streams)]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    opts = spz.Opts(forecaster=1)
    store = serve.ShardStore(codec, D, 16, opts)
    store.add_streams(xs)
    del xs
    torch.cuda.synchronize()
    pool = [synth.sensor_u16_torch(8192, D, seed=500000 + k, device=dev) for k in range(64)]
    rate = 20000.0
    n_req = int(rate * (args.serve_seconds + 1.0))
    reqs = serve.poisson_requests(store, n_req, rate=rate, seed=4, append_frac=0.1, append_rows=8192,
                                  append_source=lambda sid, k: pool[(sid * 7 + k) % len(pool)])
    server = serve.Server(store, mem_budget=4 << 30, max_batch=512, n_slots=3)
    stats = server.run(reqs, realtime=True, keep_results=False)
    warm = [r for r in reqs if r.t_arrival >= 1.0]
    lat = np.array([r.t_done - r.t_arrival for r in warm])
    rb = D * 2
    served = sum((r.b - r.a) * rb if r.kind == "range" else r.rows.shape[0] * rb for r in warm)
    span = max(r.t_done for r in warm) - min(r.t_arrival for r in warm)
    # capacity: the same mix, every request arrived at once (closed loop)
    reqs2 = serve.poisson_requests(store, n_req, rate=rate, seed=5, append_frac=0.1, append_rows=8192,
                                   append_source=lambda sid, k: pool[(sid * 7 + k) % len(pool)])
    b0 = server.batches
    cap = server.run(reqs2, realtime=False, keep_results=False)
    line.update({
        "value": served / span / 1e9, "ms_per_step": None, "dtype": "u16",
        "config": {"workload": "serve_1000_streams_u16_D4_2^20rows_poisson_20k_req_s",
                   "rate_req_s": rate, "requests": len(reqs), "measured_requests": len(warm),
                   "mix": "90% range 1K-64K rows (log-uniform, uniform start), 10% append 8192 rows",
                   "generator_s": gen_s, "mem_budget": 4 << 30, "slots": 3, "max_batch": 512,
                   "results": "each range's rows released once it completes (a consuming client)"},
        "serving": {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                    "gbs": served / span / 1e9, "batches": stats["batches"], "peak_mem": stats["peak_mem"],
                    "wall_s": stats["wall_s"],
                    "closed_loop": {"requests": len(reqs2), "req_s": len(reqs2) / cap["wall_s"],
                                    "gbs": cap["gbs"], "batches": cap["batches"] - b0}}})


SWEEP_D = (1, 2, 3, 4, 5, 6, 8, 12, 16, 24, 32, 40, 48, 64, 80)
SWEEP_VALUES = 100_000_000  # the paper's 100M uniformly random values


def run_fire_speed(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz):
    """The FIRE Speed experiment (Sec. 5.6): the forecast step alone
    (samples -> errors and back, no packing) on 100M uniform values viewed as
    D columns, for delta, FIRE, double delta and FIRE per sample. GB/s count
    the samples' bytes; the kernel moves twice that (read + write)."""
    import torch
    names = {0: "delta", 1: "fire", 2: "double_delta", 3: "fire_per_sample"}
    table = []
    with ClockSampler(0) as clk:
        for w in (8, 16):
            base = synth.uniform_torch(SWEEP_VALUES, 1, w, seed=6, device=dev).view(-1)
            for D in SWEEP_D:
                rows = SWEEP_VALUES // D
                x = base[:rows * D].view(rows, D)
                U = x.numel() * x.element_size()
                e = torch.empty_like(x)
                y = torch.empty_like(x)
                for fc in (0, 1, 2, 3):
                    for _ in range(args.warmup):
                        codec.forecast(x, forecaster=fc, out=e)
                        codec.forecast(e, forecaster=fc, inverse=True, out=y)
                    torch.cuda.synchronize()
                    assert torch.equal(y, x), ("forecast round trip", w, D, fc)
                    enc = _time(lambda: codec.forecast(x, forecaster=fc, out=e), args.steps, stream)
                    dec = _time(lambda: codec.forecast(e, forecaster=fc, inverse=True, out=y), args.steps, stream)
                    table.append({"w": w, "D": D, "forecaster": names[fc], "encode_gbs": U / (enc * 1e-3) / 1e9,
                                  "decode_gbs": U / (dec * 1e-3) / 1e9, "encode_ms": enc, "decode_ms": dec,
                                  "hbm_frac_encode": 2 * U / (enc * 1e-3) / 1e9 / peak,
                                  "hbm_frac_decode": 2 * U / (dec * 1e-3) / 1e9 / peak})
            del base
    fire = [r for r in table if r["forecaster"] == "fire"]
    best = max(fire, key=lambda r: r["decode_gbs"])
    line.update({"metric": "forecast-only (FIRE Speed) encode/decode GB/s over column counts",
                 "value": best["decode_gbs"], "dtype": "u8/u16",
                 "config": {"workload": "uniform_100M_values_D1-80_forecast_only", "values": SWEEP_VALUES,
                            "chunk_rows": 1024, "learn_shift": 1, "D": list(SWEEP_D),
                            "value_is": f"best FIRE decode GB/s (w={best['w']}, D={best['D']})"},
                 "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                              "kernel": "k_forecast", "bytes_per_launch": "2 x samples (read + write)",
                              "frac": max(r["hbm_frac_decode"] for r in fire), "traffic": None},
                 "table": table, "clocks": clk.summary()})


def run_dsweep(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz):
    """The codec over column counts (Sec. 5.4 / 5.5): 100M uniform values as
    D columns (rows % 8 stored raw), SprintzDelta, SprintzFIRE and
    SprintzFIRE+Huf, compress and decompress GB/s of the samples' bytes."""
    import torch
    variants = (("delta", spz.Opts(forecaster=0)), ("fire", spz.Opts(forecaster=1)),
                ("fire_huf", spz.Opts(forecaster=1, huffman=1)))
    table = []
    with ClockSampler(0) as clk:
        for w in (8, 16):
            base = synth.uniform_torch(SWEEP_VALUES, 1, w, seed=7, device=dev).view(-1)
            for D in SWEEP_D:
                rows = SWEEP_VALUES // D
                x = base[:rows * D].view(rows, D)
                U = x.numel() * x.element_size()
                out = torch.empty_like(x)
                for name, o in variants:
                    cap = spz.max_compressed_size(rows, D, w, o)
                    dst = torch.empty(cap, dtype=torch.uint8, device=dev)
                    size = torch.zeros(1, dtype=torch.int64, device=dev)
                    wsn = spz.compress_workspace_size(rows, D, w, o)
                    ws = torch.empty(max(wsn, 1), dtype=torch.uint8, device=dev)
                    codec.compress_into(x, rows, D, w, o, dst, size, ws)
                    torch.cuda.synchronize()
                    codec.check()
                    C = int(size.item())
                    info = spz.query(dst[:64].cpu().numpy().tobytes())
                    ws_d = torch.empty(max(spz.decompress_workspace_size(info), 1), dtype=torch.uint8, device=dev)
                    for _ in range(args.warmup):
                        codec.compress_into(x, rows, D, w, o, dst, size, ws)
                        codec.decompress_into(dst, C, info, out, ws_d)
                    torch.cuda.synchronize()
                    codec.check()
                    assert torch.equal(out, x), ("round trip", w, D, name)
                    enc = _time(lambda: codec.compress_into(x, rows, D, w, o, dst, size, ws), args.steps, stream)
                    dec = _time(lambda: codec.decompress_into(dst, C, info, out, ws_d), args.steps, stream)
                    table.append({"w": w, "D": D, "variant": name, "ratio": U / C,
                                  "compress_gbs": U / (enc * 1e-3) / 1e9, "decompress_gbs": U / (dec * 1e-3) / 1e9,
                                  "compress_ms": enc, "decompress_ms": dec,
                                  "hbm_frac_decode": (U + C) / (dec * 1e-3) / 1e9 / peak,
                                  "hbm_frac_encode": (U + C) / (enc * 1e-3) / 1e9 / peak})
                    del dst, ws, ws_d
            del base
    fire = [r for r in table if r["variant"] == "fire"]
    best = max(fire, key=lambda r: r["decompress_gbs"])
    line.update({"metric": "decompress and compress GB/s over column counts (uniform data)",
                 "value": best["decompress_gbs"], "dtype": "u8/u16",
                 "config": {"workload": "uniform_100M_values_D1-80_codec", "values": SWEEP_VALUES,
                            "chunk_rows": 1024, "D": list(SWEEP_D),
                            "value_is": f"best SprintzFIRE decompress GB/s (w={best['w']}, D={best['D']})"},
                 "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                              "frac": best["hbm_frac_decode"], "traffic": None},
                 "table": table, "clocks": clk.summary()})


def run_gsweep(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz):
    """Header groups G and chunk lengths on the 2^24-row sensor workload
    (FIRE): ratio and compress / decompress GB/s (Sec. 4.3 states the paper's
    G = 2; larger G amortizes header reads)."""
    import torch
    x = synth.sensor_u16_torch(1 << 24, 8, seed=1, device=dev)
    rows, D, w = x.shape[0], 8, 16
    U = x.numel() * x.element_size()
    out = torch.empty_like(x)
    table = []
    with ClockSampler(0) as clk:
        for G in (1, 2, 4, 8):
            for cr in (256, 1024, 4096, 16384):
                o = spz.Opts(forecaster=1, group_blocks=G, chunk_rows=cr)
                cap = spz.max_compressed_size(rows, D, w, o)
                dst = torch.empty(cap, dtype=torch.uint8, device=dev)
                size = torch.zeros(1, dtype=torch.int64, device=dev)
                ws = torch.empty(max(spz.compress_workspace_size(rows, D, w, o), 1), dtype=torch.uint8, device=dev)
                codec.compress_into(x, rows, D, w, o, dst, size, ws)
                torch.cuda.synchronize()
                codec.check()
                C = int(size.item())
                info = spz.query(dst[:64].cpu().numpy().tobytes())
                ws_d = torch.empty(max(spz.decompress_workspace_size(info), 1), dtype=torch.uint8, device=dev)
                for _ in range(args.warmup):
                    codec.compress_into(x, rows, D, w, o, dst, size, ws)
                    codec.decompress_into(dst, C, info, out, ws_d)
                torch.cuda.synchronize()
                codec.check()
                assert torch.equal(out, x), ("round trip", G, cr)
                enc = _time(lambda: codec.compress_into(x, rows, D, w, o, dst, size, ws), args.steps, stream)
                dec = _time(lambda: codec.decompress_into(dst, C, info, out, ws_d), args.steps, stream)
                table.append({"G": G, "chunk_rows": cr, "ratio": U / C,
                              "compress_gbs": U / (enc * 1e-3) / 1e9, "decompress_gbs": U / (dec * 1e-3) / 1e9,
                              "hbm_frac_decode": (U + C) / (dec * 1e-3) / 1e9 / peak,
                              "hbm_frac_encode": (U + C) / (enc * 1e-3) / 1e9 / peak})
                del dst, ws, ws_d
    ref = next(r for r in table if r["G"] == 2 and r["chunk_rows"] == 1024)
    line.update({"metric": "decompress and compress GB/s and ratio over header groups and chunk lengths",
                 "value": ref["decompress_gbs"], "dtype": "u16",
                 "config": {"workload": "sensor_u16_D8_2^24rows_FIRE_G_CR_sweep", "G": [1, 2, 4, 8],
                            "chunk_rows": [256, 1024, 4096, 16384], "value_is": "decompress GB/s at G=2, CR=1024"},
                 "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                              "frac": ref["hbm_frac_decode"], "traffic": None},
                 "table": table, "clocks": clk.summary()})


def run_quantize(args, codec, dev, stream, line, peak, peak_kind, ClockSampler, synth, spz):
    """Float data (Sec. 5.8): 2^24 x 8 float32 samples (the sensor recipe's
    sinusoids plus noise, as floats) quantized to 8 and 16 bits, compressed
    with FIRE, decompressed and mapped back. GB/s count the float bytes;
    the normalized errors are the paper's quality measure."""
    import torch
    rows, D = 1 << 24, 8
    x = (synth.sensor_u16_torch(rows, D, seed=1, device=dev).to(torch.int32) & 0xFFFF).to(torch.float32)
    x = (x - 32768.0) / 8000.0 + 0.001 * torch.randn((rows, D), device=dev, generator=synth._tgen(9, dev))
    F = x.numel() * 4
    table = []
    with ClockSampler(0) as clk:
        for w in (8, 16):
            q, lh = codec.quantize(x, w)
            o = spz.Opts(forecaster=1)
            dst, size = codec.compress(q, o)
            torch.cuda.synchronize()
            C = int(size.item())
            info = spz.query(dst[:64].cpu().numpy().tobytes())
            y = codec.decompress(dst, info, src_size=C).view(q.shape)
            xr = codec.dequantize(y, lh)
            nm = codec.quant_nmse(x, q, lh).cpu().numpy()
            torch.cuda.synchronize()
            tq = _time(lambda: codec.quantize(x, w), args.steps, stream)
            td = _time(lambda: codec.dequantize(q, lh, out=xr), args.steps, stream)
            table.append({"w": w, "quantize_gbs": F / (tq * 1e-3) / 1e9, "dequantize_gbs": F / (td * 1e-3) / 1e9,
                          "quantize_ms": tq, "dequantize_ms": td, "ratio_vs_float": F / C,
                          "nmse_max": float(nm.max()), "nmse_min": float(nm.min())})
    r16 = table[1]
    line.update({"metric": "float quantization GB/s (float bytes) and normalized MSE",
                 "value": r16["quantize_gbs"], "dtype": "f32->u16",
                 "config": {"workload": "float32_sensor_D8_2^24rows_quantize", "rows": rows, "D": D,
                            "value_is": "quantize GB/s at w = 16"},
                 "roofline": {"bound": "hbm", "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                              "frac": (F + F / 2) / (r16["quantize_ms"] * 1e-3) / 1e9 / peak,
                              "bytes_per_launch": "float reads (twice: extremes, codes) + code writes",
                              "traffic": None},
                 "table": table, "clocks": clk.summary()})


def run_sensor(args, B, rank, world, local):
    """The single-stream workload: uint16, D = 8, 2^24 rows (256 MiB) of the
    sensor recipe, FIRE, chunk_rows 1024; one step = one compress and one
    decompress of the whole series. N > 1: each rank its own series."""
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

    x = synth.sensor_u16(args.rows, B.COLS, seed=B.rank_seed(rank))
    U = x.nbytes
    xd = torch.from_numpy(x.view(np.int16)).to(dev)
    codec = spz.Codec(local)
    o = spz.Opts(**B.opts_dict())
    rows, D, w = args.rows, B.COLS, 16
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
    with B.ClockSampler(local) as clk:
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
    total_ms = B.slowest_rank_ms(t_start.elapsed_time(t_end), dist, dev)
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
        e2e_ms = B.slowest_rank_ms(e2e_ms, dist, dev)
        e2e = {"value": B.job_gbs(U, world, e2e_ms), "unit": "GB/s",
               "h2d_bytes_per_step": U + C, "d2h_bytes_per_step": C + U,
               "ms_per_step": e2e_ms, "steps": n_e2e,
               "pipelining": f"{nl} lanes (streams) take steps in turn"}

    if rank != 0:
        return
    enc_avg, dec_avg = statistics.mean(enc_ms), statistics.mean(dec_ms)
    peak, peak_kind = B.peaks()
    table = 16 * info.n_chunks
    enc_bytes, dec_bytes = U + C + table, C + U
    dom = "decode" if dec_avg >= enc_avg else "encode"
    dom_kernel = "k_decode_lanes" if dom == "decode" else "k_encode_slots"
    dom_ms = dec_avg if dom == "decode" else enc_avg
    dom_bytes = dec_bytes if dom == "decode" else enc_bytes
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    line = {
        "metric": B.METRIC, "value": B.job_gbs(U, world, ms_step), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
        "data": "synthetic",
        "config": {"workload": B.SENSOR_WORKLOAD, "rows": rows, "D": D, "w": w, **B.opts_dict(),
                   "step": "compress+decompress round trip", "uncompressed_bytes": U,
                   "compressed_bytes": C, "ratio": U / C,
                   "l2": "inputs (256 MiB raw, compressed stream) larger than the 129 MB L2",
                   "parallelism": f"{world} independent streams (one per GPU)"},
        "decompress_gbs": U / (dec_avg * 1e-3) / 1e9,
        "compress_gbs": U / (enc_avg * 1e-3) / 1e9,
        "decompress_ms": dec_avg, "compress_ms": enc_avg,
        "roofline": {"bound": "hbm", "kernel": dom_kernel,
                     "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": B.traffic_bytes(dom_kernel),
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
        s = oracle.compress(xs, **B.opts_dict())
        oracle.decompress(s)
        tc = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": xs.nbytes / tc / 1e9, "unit": "GB/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"first {n_s} of {rows} rows, one compress+decompress, "
                                          "single thread"}
    print(json.dumps(line), flush=True)

