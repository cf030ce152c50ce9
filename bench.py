#!/usr/bin/env python3
"""Decode throughput of the icx GPU library on the paper's long-array workload.

One step = one pass of the whole decoding path over the synthetic workload:
the 2^26-integer sorted uniform array and the clustered array (1,024 clusters,
56.3 M integers after deduplication), each decoded as SIMD-BP128* (stride-4
deltas), SIMD-BP128 (stride 1), W32* / W32 (the 32-lane layout) and
SIMD-FastPFOR / SIMD-FastPFOR* -- twelve decodes.  Inputs (compressed
streams + indexes, produced by the library's GPU encoders) are resident in
HBM before timing.  Between decodes L2 is flushed by reading a buffer twice
its size (untimed), so every decode starts cold and pays for its own
write-backs; CUDA events bracket each decode on its stream.

Prints one JSON line (see the keys below).  `--impl reference` times the
scalar CPU oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "decoded G ints/s"
UNIT = "Gints/s"

# (codec, delta, fmt, label) per array; a step decodes all of them on both arrays
COMBOS = [
    ("bp128", 4, 0, "SIMD-BP128*"),
    ("bp128", 1, 0, "SIMD-BP128"),
    ("bp128", 4, 1, "W32*"),
    ("bp128", 1, 1, "W32"),
    ("fastpfor", 1, 0, "SIMD-FastPFOR"),
    ("fastpfor", 4, 0, "SIMD-FastPFOR*"),
]
def kernel_name(codec: str, delta: int, fmt: int = 0) -> str:
    if codec == "bp128":
        return "bp128_blocklane_kernel" if fmt == 0 and delta else "bp128_decode_kernel"
    if delta:  # one decode call launches four kernels
        return "fastpfor_meta_kernel + fastpfor_prep_kernel + fastpfor_tile_scan_kernel + fastpfor_stream_kernel"
    return "fastpfor_decode_kernel"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_arrays(n=None):
    from paper_1209_2137_gb300 import workloads as W
    t = time.time()
    if n:  # reduced workload (profiling): the uniform array alone
        arrays = {"uniform": W.uniform_sorted(n, 29, W.SEED_BASE + 2)}
    else:
        arrays = {"uniform": W.workload_uniform_long(), "clustered": W.workload_clustered_long()}
    log(f"[bench] generated workload in {time.time() - t:.1f}s: "
        + ", ".join(f"{k} n={v.size}" for k, v in arrays.items()))
    return arrays


# ------------------------------------------------------------------ clocks --

class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            if ts < t0 or ts > t1:
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------- distributed --

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_rate(ints_per_rank: int, slowest_ms: float, world: int) -> float:
    """Whole-job G ints/s: every rank decodes ints_per_rank integers (weak
    scaling, replicas) and the job takes as long as its slowest rank."""
    return world * ints_per_rank / (slowest_ms / 1e3) / 1e9


def max_over_ranks(value: float, world: int) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- traffic --

def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1209_2137_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(label: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if len(parts) >= 4 and parts[0] == label and parts[1] == src:
                return float(parts[2]) * float(parts[3])  # bytes at capture size x scale to full size
    return None


# --------------------------------------------------------------- GPU arm --

def run_gpu(args, world, rank, local):
    import torch

    import paper_1209_2137_gb300 as icx

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    icx.lib()  # fails loudly if the CUDA library is missing
    if args.bp128_warps:
        icx.set_tuning("bp128.warps_per_cta", args.bp128_warps)
    if args.bp128_l2_prefetch >= 0:
        icx.set_tuning("bp128.l2_prefetch", args.bp128_l2_prefetch)
    if args.fastpfor_warps:
        icx.set_tuning("fastpfor.warps_per_cta", args.fastpfor_warps)
    for kv in args.tune:
        key, _, val = kv.partition("=")
        icx.set_tuning(key, int(val))

    arrays = workload_arrays(args.n)
    stream = torch.cuda.current_stream()

    # encode on the GPU (untimed) and verify one decode of each stream
    streams = []
    for name, x in arrays.items():
        xt = torch.from_numpy(x).to(dev)
        combos = COMBOS + ([("bp128", 0, 0, "SIMD-BP128 (no delta)"), ("bp128", 0, 1, "W32 (no delta)")]
                           if args.extra_none else [])
        for codec, delta, fmt, label in combos:
            if codec == "fastpfor" and args.skip_fastpfor:
                continue
            enc = icx.bp128_encode(xt, delta, fmt) if codec == "bp128" else icx.fastpfor_encode(xt, delta)
            streams.append(dict(array=name, codec=codec, delta=delta, fmt=fmt, label=label, enc=enc, n=x.size,
                                x=xt))
    nmax = max(s["n"] for s in streams)
    out = torch.empty(nmax, dtype=torch.uint32, device=dev)
    ws = icx.Workspace(nmax)
    for s in streams:
        o = out[: s["n"]]
        icx.decode(s["enc"], out=o, workspace=ws)
        ws.raise_status("verify decode")
        if not torch.equal(o, s["x"]):
            raise SystemExit(f"verification failed for {s['array']} {s['label']}")
        s["bits_per_int"] = 8.0 * s["enc"].nbytes / s["n"]
        s["alg_bytes"] = s["enc"].nbytes + 8 * s["enc"].index.numel() + 4 * s["n"]
    log(f"[bench] {len(streams)} streams encoded on the GPU and verified")
    for s in streams:
        del s["x"]
    torch.cuda.empty_cache()

    props = torch.cuda.get_device_properties(dev)
    l2 = getattr(props, "L2_cache_size", 132 * 1024 * 1024)
    flush = torch.empty(2 * l2 // 4 + 1024, dtype=torch.int32, device=dev)
    flush.fill_(1)

    def flush_l2():
        flush.sum(dtype=torch.int64)  # reads 2x L2 of clean lines

    def decode(s):
        icx.decode(s["enc"], out=out[: s["n"]], workspace=ws)

    # warm-up
    for _ in range(args.warmup):
        for s in streams:
            flush_l2()
            decode(s)
    torch.cuda.synchronize()

    # timed: events bracket each decode only
    K = args.steps
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in streams]
          for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        t0 = time.time()
        for k in range(K):
            for i, s in enumerate(streams):
                flush_l2()
                ev[k][i][0].record(stream)
                decode(s)
                ev[k][i][1].record(stream)
        torch.cuda.synchronize()
        t1 = time.time()
    barrier(world)
    per = np.array([[a.elapsed_time(b) for (a, b) in row] for row in ev])  # ms, [K, streams]
    step_ms = per.sum(axis=1)
    ms_per_step = float(np.mean(step_ms))
    total_ms = max_over_ranks(float(step_ms.sum()), world)
    ints_per_step = sum(s["n"] for s in streams)
    value = aggregate_rate(ints_per_step * K, total_ms, world)
    # SIMD-BP128: one kernel; SIMD-FastPFOR with a stride: page parse, prepare, tile scan and stream
    launches_per_step = sum(1 if s["codec"] == "bp128" else 4 if s["delta"] else 2 for s in streams)
    ws.raise_status("timed decodes")

    # roofline per stream and for the dominant one
    peak, peak_kind = peaks()
    kern = []
    for i, s in enumerate(streams):
        ms = float(np.mean(per[:, i]))
        gbs = s["alg_bytes"] / (ms / 1e3) / 1e9
        kern.append(dict(array=s["array"], codec=s["label"], n=s["n"], bits_per_int=round(s["bits_per_int"], 3),
                         ms=round(ms, 4), gints_s=round(s["n"] / (ms / 1e3) / 1e9, 1), achieved_gbs=round(gbs, 1),
                         frac=round(gbs / peak, 4)))
    dom = max(range(len(streams)), key=lambda i: float(np.sum(per[:, i])))
    ds = streams[dom]
    dom_ms = float(np.mean(per[:, dom]))
    achieved = ds["alg_bytes"] / (dom_ms / 1e3) / 1e9
    # recorded at the default sizes only
    traffic = None if args.n else recorded_traffic(f"{ds['array']}:{ds['label']}")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "kernel": f"{kernel_name(ds['codec'], ds['delta'], ds['fmt'])} ({ds['label']}, {ds['array']})",
                "alg_bytes_per_launch": ds["alg_bytes"], "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})"}
    headline = next(i for i, s in enumerate(streams) if s["label"] == "SIMD-BP128*" and s["array"] == "uniform")

    e2e = run_e2e(args, streams, out, ws, dev, world)
    exceptions = None if args.skip_exceptions else run_exceptions(args, out, ws, flush_l2, world)
    intersect = None if args.skip_intersect else run_intersect(args, streams, arrays, out, ws, flush_l2, world)
    bp32 = None if args.skip_bp32 else run_bp32(args, arrays, out, ws, flush_l2, world)
    encode = None if args.skip_encode else run_encode(args, arrays, dev, flush_l2, world)
    aux = None if args.skip_aux else run_aux(args, streams, arrays, dev, ws, flush_l2, world)
    batched = serving = None
    if not args.skip_batch:
        del out
        torch.cuda.empty_cache()
        batched, serving = run_batched(args, dev, flush_l2, world)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(arrays, args)

    clk = clocks.summary(t0, t1)
    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded SplitMix64)",
        "config": {
            "workload": workload_label(arrays, streams),
            "ints_per_step": ints_per_step, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "l2": "flushed between decodes (untimed read of 2x L2), events bracket each decode",
            "streams": kern,
        },
        "roofline": roofline,
        "headline_kernel": kern[headline],
        "e2e": e2e,
        "exceptions": exceptions,
        "intersect": intersect,
        "bp32": bp32,
        "encode": encode,
        "aux": aux,
        "batched": batched,
        "serving": serving,
        "gpu_launches": launches_per_step * K,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(result), flush=True)


def workload_label(arrays, streams):
    parts = []
    for name, x in arrays.items():
        parts.append(f"{name} n={x.size}" + (" (2^26 in [0,2^29))" if name == "uniform" and x.size == 1 << 26
                                               else " (1024 clusters, 2^18 windows)" if name == "clustered" else ""))
    order = [c[3] for c in COMBOS]
    labels = sorted({s["label"] for s in streams}, key=lambda l: order.index(l) if l in order else len(order))
    return (f"long sorted uint32 arrays, {len(streams)} decodes per step: {{" + "; ".join(parts) + "} x {"
            + ", ".join(labels) + "}")


def run_e2e(args, streams, out, ws, dev, world):
    """Same metric through the public API with host buffers: every step copies
    each stream and its index from pinned host memory, decodes, and copies the
    integers back to pinned host memory.  The decodes of a step rotate over
    `--e2e-streams` CUDA streams (each with its own buffers and workspace), so
    one decode's copies overlap another's kernels on the two copy engines."""
    import torch

    import paper_1209_2137_gb300 as icx

    steps = max(3, min(args.steps, args.e2e_steps))
    lanes = max(1, args.e2e_streams)
    host = []
    for s in streams:
        hd = torch.empty(s["enc"].nbytes, dtype=torch.uint8, pin_memory=True)
        hd.copy_(s["enc"].data)
        hi = torch.empty(s["enc"].index.numel(), dtype=torch.uint64, pin_memory=True)
        hi.copy_(s["enc"].index)
        dd = torch.empty_like(s["enc"].data)
        di = torch.empty_like(s["enc"].index)
        host.append((hd, hi, dd, di))
    nmax = out.numel()
    cuda = [torch.cuda.Stream(device=dev) for _ in range(lanes)]
    outs = [out] + [torch.empty(nmax, dtype=torch.uint32, device=dev) for _ in range(lanes - 1)]
    wss = [ws] + [icx.Workspace(nmax, device=dev) for _ in range(lanes - 1)]
    houts = [torch.empty(nmax, dtype=torch.uint32, pin_memory=True) for _ in range(lanes)]
    h2d = sum(h[0].numel() + 8 * h[1].numel() for h in host)
    d2h = sum(4 * s["n"] for s in streams)
    main = torch.cuda.current_stream()

    def step():
        start = torch.cuda.Event()
        start.record(main)
        for i, (s, (hd, hi, dd, di)) in enumerate(zip(streams, host)):
            k = i % lanes
            cs, o, w, ho = cuda[k], outs[k][: s["n"]], wss[k], houts[k][: s["n"]]
            cs.wait_event(start)
            with torch.cuda.stream(cs):
                dd.copy_(hd, non_blocking=True)
                di.copy_(hi, non_blocking=True)
                enc = icx.Encoded(dd, di, s["n"], s["codec"], s["delta"], s["fmt"])
                icx.decode(enc, out=o, workspace=w, stream=cs)
                ho.copy_(o, non_blocking=True)
        for cs in cuda:
            main.wait_stream(cs)

    step()
    torch.cuda.synchronize()
    for k in range(lanes):
        wss[k].raise_status("e2e decode", cuda[k])
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(main)
    for _ in range(steps):
        step()
    b.record(main)
    torch.cuda.synchronize()
    ms = max_over_ranks(a.elapsed_time(b), world)
    for k in range(lanes):
        wss[k].raise_status("e2e decode", cuda[k])
    ints = sum(s["n"] for s in streams) * steps * world
    return {"value": round(ints / (ms / 1e3) / 1e9, 2), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "cuda_streams": lanes,
            "host_link_gbs": round((h2d + d2h) * steps * world / (ms / 1e3) / 1e9, 1)}


# ------------------------------------------------- exception-heavy data --

def run_exceptions(args, out, ws, flush_l2, world):
    """2^26 unsorted integers, 90 % geometric (mean 8), 10 % uniform in
    [2^20, 2^28): SIMD-FastPFOR without differential decoding (unpack plus
    exception patch), and SIMD-BP128 on the same data for contrast."""
    import torch

    import paper_1209_2137_gb300 as icx
    from paper_1209_2137_gb300 import workloads as W

    x = W.workload_exceptions(args.exceptions_n) if args.exceptions_n else W.workload_exceptions()
    xt = torch.from_numpy(x).to(out.device)
    if out.numel() < x.size or ws.n < x.size:  # a reduced main workload: buffers of this size
        out = torch.empty(x.size, dtype=torch.uint32, device=out.device)
        ws = icx.Workspace(x.size, device=out.device)
    o = out[: x.size]
    peak, _ = peaks()
    res = {"workload": f"{x.size} unsorted uint32: 90 % geometric (mean 8), 10 % uniform in [2^20, 2^28)"}
    for codec, label in (("fastpfor", "SIMD-FastPFOR"), ("bp128", "SIMD-BP128")):
        enc = icx.fastpfor_encode(xt, icx.DELTA_NONE) if codec == "fastpfor" else icx.bp128_encode(xt, icx.DELTA_NONE)
        icx.decode(enc, out=o, workspace=ws)
        ws.raise_status("exception-heavy decode")
        if not torch.equal(o, xt):
            raise SystemExit(f"exception-heavy {label}: verification failed")
        for _ in range(args.warmup):
            flush_l2()
            icx.decode(enc, out=o, workspace=ws)
        steps = max(3, min(args.steps, 50))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush_l2()
            a.record()
            icx.decode(enc, out=o, workspace=ws)
            b.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world)
        alg = enc.nbytes + 8 * enc.index.numel() + 4 * x.size
        res[label] = {"bits_per_int": round(8.0 * enc.nbytes / x.size, 3), "ms": round(ms, 4),
                      "gints_s": round(x.size / (ms / 1e3) / 1e9, 1),
                      "achieved_gbs": round(alg / (ms / 1e3) / 1e9, 1), "frac": round(alg / (ms / 1e3) / 1e9 / peak, 4)}
    res["note"] = "the GPU encoders write the oracle's bytes (tests), so bits_per_int is the oracle's"
    log(f"[bench] exception-heavy: SIMD-FastPFOR {res['SIMD-FastPFOR']}, SIMD-BP128 {res['SIMD-BP128']}")
    return res


# ------------------------------------------------------------------ aux --

def run_aux(args, streams, arrays, dev, ws, flush_l2, world):
    """The remaining calls of the boundary on the uniform array: differential
    decoding alone (Sec. 3: prefix sums with stride 1 and 4 over 4-byte
    differences; roofline bytes 8 per integer), differential encoding, and
    the index walks over a SIMD-BP128 and a SIMD-FastPFOR stream (serial
    walks over the metablock / page headers)."""
    import torch

    import paper_1209_2137_gb300 as icx

    peak, _ = peaks()
    x = arrays["uniform"]
    n = x.size
    xt = torch.from_numpy(x).to(dev)
    res = {"workload": f"uniform n={n}"}

    def timed(fn, alg):
        for _ in range(args.warmup):
            flush_l2()
            fn()
        steps = max(3, min(args.steps, 20))
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush_l2()
            a.record()
            fn()
            b.record()
        torch.cuda.synchronize()
        ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world)
        r = {"ms": round(ms, 4), "gints_s": round(n / (ms / 1e3) / 1e9, 1)}
        if alg:
            r["achieved_gbs"] = round(alg / (ms / 1e3) / 1e9, 1)
            r["frac"] = round(alg / (ms / 1e3) / 1e9 / peak, 4)
        return r

    out = torch.empty_like(xt)
    for delta in (1, 4):
        d = icx.delta_encode(xt, delta)
        icx.delta_decode(d, delta, out=out, workspace=ws)
        ws.raise_status("delta decode")
        if not torch.equal(out, xt):
            raise SystemExit("delta decode: verification failed")
        res[f"delta_decode_d{delta}"] = timed(lambda: icx.delta_decode(d, delta, out=out, workspace=ws), 8 * n)
        res[f"delta_encode_d{delta}"] = timed(lambda: icx.delta_encode(xt, delta, out=out), 8 * n)
        del d
    for s in streams:
        if s["array"] != "uniform" or s["delta"] != 1 or s["fmt"] != 0:
            continue
        enc = s["enc"]
        ix = torch.empty_like(enc.index)
        if s["codec"] == "bp128":
            fn = lambda: icx.bp128_index(enc.data, enc.n, 0, index=ix, workspace=ws)
        else:
            fn = lambda: icx.fastpfor_index(enc.data, enc.n, index=ix, workspace=ws)
        fn()
        ws.raise_status("index walk")
        if not torch.equal(ix, enc.index):
            raise SystemExit(f"{s['label']} index walk: verification failed")
        r = timed(fn, None)
        r["entries"] = int(enc.index.numel())
        res[f"index_{s['codec']}"] = r
    del xt, out
    torch.cuda.empty_cache()
    log("[bench] aux: " + ", ".join(f"{k} {v['ms']} ms" for k, v in res.items() if isinstance(v, dict)))
    return res


# ---------------------------------------------------------------- encode --

ENCODE_COMBOS = [("bp128", 1, 0, "SIMD-BP128"), ("bp128", 4, 0, "SIMD-BP128*"),
                 ("fastpfor", 1, 0, "SIMD-FastPFOR"), ("fastpfor", 4, 0, "SIMD-FastPFOR*")]


def run_encode(args, arrays, dev, flush_l2, world):
    """Coding speed (the paper reports it beside decoding speed, Sec. 6.4 and
    6.5): the GPU encoders on the long sorted arrays, inputs resident, events
    around each call; roofline bytes = 4 B per integer read + the stream and
    index written.  Beside them, the oracle's encoder (one host thread) on a
    2^22-integer prefix."""
    import torch

    import oracle
    import paper_1209_2137_gb300 as icx

    peak, _ = peaks()
    L = icx.lib()
    stream = torch.cuda.current_stream()
    sp = ctypes.c_void_p(stream.cuda_stream)
    res = {"workload": "the long sorted arrays of the main step, encoded on the GPU (bytes identical to the "
                       "oracle's, tests)", "streams": []}
    for name, x in arrays.items():
        xt = torch.from_numpy(x).to(dev)
        n = x.size
        for codec, delta, fmt, label in ENCODE_COMBOS:
            if codec == "bp128":
                cap, ilen = icx.bp128_max_bytes(n, fmt), icx.bp128_index_len(n)
            else:
                cap, ilen = icx.fastpfor_max_bytes(n), icx.fastpfor_index_len(n)
            buf = torch.empty(cap, dtype=torch.uint8, device=dev)
            index = torch.empty(ilen, dtype=torch.uint64, device=dev)
            total = torch.zeros(1, dtype=torch.uint64, device=dev)
            ews = icx.Workspace(n, device=dev, encode=True)
            fn = L.bp128_encode if codec == "bp128" else L.fastpfor_encode

            def call():
                code = fn(icx._ptr(xt), n, delta, fmt, icx._ptr(buf), cap, icx._ptr(index), icx._ptr(total),
                          ews.ptr(), ews.bytes, sp)
                if code != 0:
                    raise SystemExit(f"{label} encode failed ({code})")

            for _ in range(args.warmup):
                flush_l2()
                call()
            torch.cuda.synchronize()
            ews.raise_status(f"{label} encode")
            steps = max(3, min(args.steps, 20))
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, b in ev:
                flush_l2()
                a.record(stream)
                call()
                b.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in ev])), world)
            nbytes = int(total.cpu().view(torch.int64).item())
            alg = 4 * n + nbytes + 8 * ilen
            xs = x[: 1 << 22]
            t = time.perf_counter()
            oracle.encode(codec, xs, delta, fmt)
            cpu_s = time.perf_counter() - t
            res["streams"].append({"array": name, "codec": label, "n": int(n), "bits_per_int": round(8.0 * nbytes / n, 3),
                                   "ms": round(ms, 4), "gints_s": round(n / (ms / 1e3) / 1e9, 1),
                                   "achieved_gbs": round(alg / (ms / 1e3) / 1e9, 1),
                                   "frac": round(alg / (ms / 1e3) / 1e9 / peak, 4),
                                   "oracle_gints_s": round(xs.size / cpu_s / 1e9, 4)})
            del buf, index, total, ews
        del xt
        torch.cuda.empty_cache()
    log("[bench] encode: " + ", ".join(f"{r['array']} {r['codec']} {r['ms']} ms ({r['frac']})" for r in res["streams"]))
    return res


# ------------------------------------------------------------------ BP32 --

def run_bp32(args, arrays, out, ws, flush_l2, world):
    """The paper's scalar formats on the long sorted arrays: BP32 (Sec. 6.2:
    binary packing of 32-integer blocks, 4 per 128-integer metablock),
    FastPFOR (Sec. 5: SIMD-FastPFOR's pages with one-lane packing) and
    SimplePFOR (its exception high parts as one Simple-8b stream per page),
    stride 1 and stride 4."""
    import torch

    import paper_1209_2137_gb300 as icx

    peak, _ = peaks()
    res = {"workload": "the long sorted arrays of the main step, BP32, FastPFOR and SimplePFOR streams encoded on "
                       "the GPU",
           "streams": []}
    steps = max(3, min(args.steps, 50))
    for name, x in arrays.items():
        xt = torch.from_numpy(x).to(out.device)
        o = out[: x.size]
        for codec, delta, label in (("bp128", icx.DELTA_1, "BP32"), ("bp128", icx.DELTA_4, "BP32*"),
                                    ("fastpfor", icx.DELTA_1, "FastPFOR"), ("fastpfor", icx.DELTA_4, "FastPFOR*"),
                                    ("simple", icx.DELTA_1, "SimplePFOR"), ("simple", icx.DELTA_4, "SimplePFOR*")):
            if codec == "bp128":
                e = icx.bp128_encode(xt, delta, icx.FMT_BP32)
            elif codec == "fastpfor":
                e = icx.fastpfor_encode(xt, delta, fmt=icx.FMT_SCALAR)
            else:
                e = icx.fastpfor_encode(xt, delta, fmt=icx.FMT_SIMPLE8B)
            icx.decode(e, out=o, workspace=ws)
            ws.raise_status("BP32 decode")
            if not torch.equal(o, xt):
                raise SystemExit(f"{label} {name}: verification failed")
            for _ in range(args.warmup):
                flush_l2()
                icx.decode(e, out=o, workspace=ws)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, z in ev:
                flush_l2()
                a.record()
                icx.decode(e, out=o, workspace=ws)
                z.record()
            torch.cuda.synchronize()
            ms = max_over_ranks(float(np.mean([a.elapsed_time(z) for a, z in ev])), world)
            alg = e.nbytes + 8 * e.index.numel() + 4 * x.size
            res["streams"].append({"array": name, "codec": label, "n": int(x.size),
                                   "bits_per_int": round(8.0 * e.nbytes / x.size, 3), "ms": round(ms, 4),
                                   "gints_s": round(x.size / (ms / 1e3) / 1e9, 1),
                                   "achieved_gbs": round(alg / (ms / 1e3) / 1e9, 1),
                                   "frac": round(alg / (ms / 1e3) / 1e9 / peak, 4)})
            del e
        del xt
    log(f"[bench] scalar layouts: {res['streams']}")
    return res


# ------------------------------------------------- decode into a consumer --

def run_intersect(args, streams, arrays, out, ws, flush_l2, world):
    """Decoding fused into a consumer (Sec. 7): membership of a sorted query
    list of ~2^22 integers (half drawn from the list) in the 2^26-integer
    uniform list, from its SIMD-BP128* and SIMD-BP128 streams.  Fused: one
    bp128_intersect call (the decoded integers are never written); unfused:
    bp128_decode into HBM, then sorted_intersect over the decoded list."""
    import torch

    import paper_1209_2137_gb300 as icx
    from paper_1209_2137_gb300 import workloads as W

    x = arrays.get("uniform")
    if x is None:
        return None
    q = W.query_list(x, 1 << 22, 29, W.SEED_BASE + 6)
    pos = np.minimum(np.searchsorted(x, q), x.size - 1)
    hits = int(np.count_nonzero(x[pos] == q))
    b = torch.from_numpy(q).to(out.device)
    bits = torch.empty((q.size + 31) // 32, dtype=torch.uint32, device=out.device)
    bits2 = torch.empty_like(bits)
    cnt = torch.empty(1, dtype=torch.uint64, device=out.device)
    cnt2 = torch.empty_like(cnt)
    o = out[: x.size]
    peak, _ = peaks()
    res = {"workload": f"sorted query list of {q.size} distinct integers (half drawn from the list, half uniform "
                       f"in [0, 2^29)) against the uniform list of {x.size}", "n": int(x.size), "nb": int(q.size),
           "hits": hits, "streams": []}
    steps = max(3, min(args.steps, 50))
    for st in streams:
        if st["array"] != "uniform" or st["codec"] != "bp128" or st["fmt"] != icx.FMT_PAPER:
            continue
        e = st["enc"]

        def fused():
            icx.bp128_intersect(e.data, e.n, b, e.delta, e.fmt, index=e.index, bits=bits, count=cnt, workspace=ws)

        def unfused():
            icx.bp128_decode(e.data, e.n, e.delta, e.fmt, index=e.index, out=o, workspace=ws)
            icx.sorted_intersect(o, b, bits=bits2, count=cnt2)

        fused()
        unfused()
        ws.raise_status("intersect")
        c1, c2 = int(cnt.cpu().view(torch.int64)[0]), int(cnt2.cpu().view(torch.int64)[0])
        if c1 != hits or c2 != hits or not torch.equal(bits, bits2):
            raise SystemExit(f"intersect {st['label']}: verification failed ({c1}, {c2}, want {hits})")
        times = {}
        for name, fn in (("fused", fused), ("unfused", unfused)):
            for _ in range(args.warmup):
                flush_l2()
                fn()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for a, z in ev:
                flush_l2()
                a.record()
                fn()
                z.record()
            torch.cuda.synchronize()
            times[name] = max_over_ranks(float(np.mean([a.elapsed_time(z) for a, z in ev])), world)
        ws.raise_status("intersect")
        stream_b = e.nbytes + 8 * e.index.numel()
        alg = stream_b + 4 * q.size + 4 * bits.numel()  # stream + query list + bitmap
        res["streams"].append({
            "codec": st["label"], "fused_ms": round(times["fused"], 4), "unfused_ms": round(times["unfused"], 4),
            "speedup": round(times["unfused"] / times["fused"], 3),
            "fused_gints_s": round(x.size / (times["fused"] / 1e3) / 1e9, 1),
            "fused_achieved_gbs": round(alg / (times["fused"] / 1e3) / 1e9, 1),
            "fused_frac": round(alg / (times["fused"] / 1e3) / 1e9 / peak, 4)})
    log(f"[bench] intersect: {res['streams']}")
    return res


# ------------------------------------------------------- batched decode --

def run_batched(args, dev, flush_l2, world):
    """Posting-list batch: Zipf(1.1) list lengths over [128, 2^22] scaled to
    about 2^28 integers in total (reading A), SIMD-BP128* or SIMD-FastPFOR
    per list; one graph launch of the plan (tuned on this batch) against one
    single-array call per list (the same kernels, captured in one graph)."""
    import torch

    import paper_1209_2137_gb300 as icx
    from paper_1209_2137_gb300 import workloads as W

    t0 = time.time()
    L, offsets, values, bp = W.posting_lists(nlists=args.batch_lists, total=args.batch_total)
    codecs = np.where(bp, icx.CODEC_BP128, icx.CODEC_FASTPFOR)
    deltas = np.where(bp, icx.DELTA_4, icx.DELTA_1)
    pool = icx.ListPool(values, offsets, codecs, deltas, device=dev)
    del values
    out_off, total = pool.output_offsets()
    out = torch.empty(total, dtype=torch.int32, device=dev).view(torch.uint32)
    t1 = time.time()
    plan = icx.Plan(pool.descs(out, out_off), None)  # tune every field on this batch
    tune = plan.tuning()
    t2 = time.time()
    ints = int(L.sum())

    def timed(launch, steps):
        for _ in range(args.warmup):
            flush_l2()
            launch()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for a, b in ev:
            flush_l2()
            a.record()
            launch()
            b.record()
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
        return max_over_ranks(ms, world)

    def verify(what):
        # every list position written and equal; padding is outside any list
        outi = out.view(torch.int32)
        outi[pool.padding] = 0
        if plan.status() != icx.OK or not torch.equal(out, pool.x):
            raise SystemExit(f"{what}: verification failed")
        outi.fill_(-1)

    out.view(torch.int32).fill_(-1)
    ms_plan = timed(plan.launch, args.batch_steps)
    verify("batched decode")
    plan.launch_per_list()  # captures the per-list graph
    torch.cuda.synchronize()
    t3 = time.time()
    ms_each = timed(plan.launch_per_list, max(3, args.batch_steps // 4))
    verify("per-list decode")
    comp = pool.nbytes
    alg = comp + 8 * int(sum(icx.bp128_index_len(int(n)) if c == 0 else icx.fastpfor_index_len(int(n))
                             for n, c in zip(L, codecs))) + 4 * ints
    peak, _ = peaks()
    res = {
        "workload": f"{len(L)} posting lists, Zipf(1.1) lengths over [128, 2^22] scaled to {ints} ints (reading A), "
                    f"{int(bp.sum())} SIMD-BP128* (stride 4) / {int((~bp).sum())} SIMD-FastPFOR (stride 1)",
        "ints": ints, "lists": int(len(L)), "bits_per_int": round(8.0 * comp / ints, 3),
        "value": round(world * ints / (ms_plan / 1e3) / 1e9, 2), "unit": UNIT, "ms": round(ms_plan, 4),
        "per_list_value": round(world * ints / (ms_each / 1e3) / 1e9, 2), "per_list_ms": round(ms_each, 4),
        "ratio_vs_per_list": round(ms_each / ms_plan, 2),
        "roofline_frac": round(alg / (ms_plan / 1e3) / 1e9 / peak, 4),
        "tuning": tune, "graph_launches": {"batched": 1, "per_list": int(len(L) + (~bp & (L >= 128)).sum())},
        "setup_s": {"generate_encode": round(t1 - t0, 1), "plan_tune": round(t2 - t1, 1),
                    "per_list_capture": round(t3 - t2, 1)},
    }
    plan.close()
    log(f"[bench] batched: {res['value']} Gints/s vs per-list {res['per_list_value']} ({res['ratio_vs_per_list']}x)")
    serving = None
    if not args.skip_serve:
        del out
        torch.cuda.empty_cache()
        serving = run_serving(args, pool, L)
    return res, serving


def run_serving(args, pool, L):
    """Serving loop over the batch's pool, resident in HBM: Poisson arrivals
    at each rate for args.serve_seconds; per request k ~ U{2..8} lists drawn
    with weight rank^-1.1 (rank 1 = longest list); 16 GB of decode buffers;
    latency = scheduled arrival -> completion event observed on the host."""
    import torch

    import paper_1209_2137_gb300 as icx
    from paper_1209_2137_gb300 import workloads as W

    dummy = torch.empty(16, dtype=torch.int32, device=pool.x.device)
    descs = pool.descs(dummy, np.zeros(len(L), dtype=np.int64))
    sv = icx.Server(descs, budget_bytes=args.serve_budget, streams=args.serve_streams)
    by_rank = np.argsort(-L, kind="stable")
    w = np.arange(1, len(L) + 1, dtype=np.float64) ** -1.1
    cum = np.cumsum(w) / w.sum()
    rows = []
    for i, rate in enumerate(list(args.serve_rates) + [0]):
        nreq = int(rate * args.serve_seconds) if rate > 0 else args.serve_saturation
        z = W.splitmix64(W.SEED_BASE + 5, 100 * i, 3 * nreq)
        u = ((z[:nreq] >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
        if rate > 0:
            arrival = np.cumsum(-np.log(u) / rate * 1e9).astype(np.uint64)
        else:  # closed loop at saturation: every request waiting at the start
            arrival = np.zeros(nreq, dtype=np.uint64)
        k = 2 + (z[nreq:2 * nreq] % np.uint64(7)).astype(np.int64)
        offs = np.zeros(nreq + 1, dtype=np.int64)
        np.cumsum(k, out=offs[1:])
        zz = W.splitmix64(W.SEED_BASE + 6, 100 * i, int(offs[-1]))
        uu = ((zz >> np.uint64(11)).astype(np.float64) + 0.5) / float(1 << 53)
        ids = by_rank[np.minimum(np.searchsorted(cum, uu), len(L) - 1)].astype(np.uint32)
        lat, st, _ = sv.run(arrival, offs, ids)
        ms = lat.astype(np.float64) / 1e6
        span = float(arrival[-1]) / 1e9 if nreq else 0.0
        nb = max(1, int(st["batches"]))
        rows.append({"rate_req_s": rate if rate > 0 else "saturation", "requests": nreq, "seconds": round(span, 2),
                     "gpu_busy": round(st["gpu_s"] / max(st["wall_s"], 1e-9), 3),
                     "mean_queue_ms": round(1e3 * st["queue_s"] / max(1, nreq), 4),
                     "mean_batch_service_ms": round(1e3 * st["service_s"] / nb, 4),
                     "mean_batch_gpu_ms": round(1e3 * st["gpu_s"] / nb, 4),
                     "p50_ms": round(float(np.percentile(ms, 50)), 3), "p99_ms": round(float(np.percentile(ms, 99)), 3),
                     "max_ms": round(float(ms.max()), 3),
                     "gints_s": round(st["ints"] / max(st["wall_s"], 1e-9) / 1e9, 3),
                     "ints_per_request": round(st["ints"] / max(1, nreq)), "batches": int(st["batches"]),
                     "mean_batch": round(nreq / max(1, st["batches"]), 2), "max_batch": int(st["max_batch"]),
                     "max_queue": int(st["max_queue"]), "peak_buffer_gb": round(st["peak_bytes"] / 2**30, 3)})
        log(f"[bench] serve {rows[-1]['rate_req_s']} req/s: p50 {rows[-1]['p50_ms']} ms p99 {rows[-1]['p99_ms']} ms, "
            f"{rows[-1]['gints_s']} Gints/s, {rows[-1]['mean_batch']} req/batch")
    sv.close()
    return {"workload": "the batch's pool resident in HBM; Poisson arrivals; k ~ U{2..8} lists per request, "
                        "weight rank^-1.1 by length; FCFS admission", "budget_bytes": args.serve_budget,
            "streams": args.serve_streams, "latency": "scheduled arrival -> completion event observed (host)",
            "breakdown": "a request's latency = queue (arrival to its batch's issue) + batch service (issue to "
                         "completion seen by the host) = queue + batch GPU time (copies + kernel) + host loop",
            "rates": rows}


# --------------------------------------------------------- CPU baseline --

def oracle_streams(arrays, prefix):
    import oracle
    out = []
    for name, x in arrays.items():
        xs = x[:prefix]
        for codec, delta, fmt, label in COMBOS:
            out.append((codec, delta, fmt, label, oracle.encode(codec, xs, delta, fmt), xs.size))
    return out


def cpu_baseline(arrays, args):
    """The oracle decoder as it stands on a bounded sample: on every host core
    (unit ranges on threads, plus the differential carry per range) and, for
    comparison, on one thread."""
    import concurrent.futures as cf

    import oracle
    from oracle import parallel
    prefix = args.cpu_prefix
    enc = oracle_streams(arrays, prefix)
    idx = [oracle.index(codec, data, n, fmt) for codec, delta, fmt, label, data, n in enc]
    t = time.perf_counter()
    ints = 0
    for codec, delta, fmt, label, data, n in enc:
        oracle.decode(codec, data, n, delta, fmt)
        ints += n
    dt1 = time.perf_counter() - t
    cores = parallel.host_cores()
    with cf.ThreadPoolExecutor(max_workers=cores) as pool:
        for (codec, delta, fmt, label, data, n), ix in zip(enc[:1], idx[:1]):  # warm the pool
            parallel.decode_parallel(codec, data, n, delta, fmt, threads=cores, pool=pool, idx=ix)
        t = time.perf_counter()
        for (codec, delta, fmt, label, data, n), ix in zip(enc, idx):
            parallel.decode_parallel(codec, data, n, delta, fmt, threads=cores, pool=pool, idx=ix)
        dtn = time.perf_counter() - t
    sample = f"first {prefix} integers of each array, all 12 decodes ({ints} ints)"
    return {"value": round(ints / dtn / 1e9, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample + f", {dtn:.2f} s on {cores} threads (unit ranges, carry added per range)",
            "single_thread": {"value": round(ints / dt1 / 1e9, 4), "cores": 1, "seconds": round(dt1, 2)}}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle on every host core, each step a bounded
    sample."""
    if rank != 0:
        return
    import concurrent.futures as cf

    import oracle
    from oracle import parallel
    arrays = workload_arrays(args.n)
    cores = parallel.host_cores()
    pool = cf.ThreadPoolExecutor(max_workers=cores)

    def run(enc, idx):
        for (codec, delta, fmt, label, data, n), ix in zip(enc, idx):
            parallel.decode_parallel(codec, data, n, delta, fmt, threads=cores, pool=pool, idx=ix)

    def indexed(enc):
        return [oracle.index(codec, data, n, fmt) for codec, delta, fmt, label, data, n in enc]

    # size the per-step sample so the whole run stays within ~2 minutes
    calib = oracle_streams({k: v[: 1 << 20] for k, v in arrays.items()}, 1 << 20)
    cidx = indexed(calib)
    run(calib, cidx)
    t = time.perf_counter()
    run(calib, cidx)
    rate = sum(c[-1] for c in calib) / (time.perf_counter() - t)
    budget = 100.0 / max(1, args.steps + args.warmup)
    prefix = int(min(1 << 26, max(65536, rate * budget / len(calib)))) // 65536 * 65536
    enc = oracle_streams(arrays, prefix)
    idx = indexed(enc)
    for _ in range(args.warmup):
        run(enc, idx)
    t = time.perf_counter()
    for _ in range(args.steps):
        run(enc, idx)
    dt = time.perf_counter() - t
    pool.shutdown()
    ints = sum(e[-1] for e in enc) * args.steps
    value = ints / dt / 1e9
    sample = (f"first {prefix} integers of each array per step, all 12 decodes, on {cores} threads "
              "(unit ranges, carry added per range)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": workload_label(arrays, [{"label": c[3]} for c in COMBOS for _ in arrays]),
                   "parallelism": f"{cores} CPU threads", "sample_per_step": sample},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["icx", "reference"], default="icx")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-prefix", type=int, default=1 << 24)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-fastpfor", action="store_true")
    ap.add_argument("--skip-encode", action="store_true")
    ap.add_argument("--skip-aux", action="store_true", help="skip the prefix-sum and index-walk timings")
    ap.add_argument("--e2e-streams", type=int, default=3, help="CUDA streams the end-to-end decodes rotate over")
    ap.add_argument("--extra-none", action="store_true", help="also time decodes without differential decoding")
    ap.add_argument("--n", type=int, default=0, help="reduced workload: uniform array of n integers only")
    ap.add_argument("--bp128-warps", type=int, default=0, help="warps per CTA of the SIMD-BP128 decoder")
    ap.add_argument("--bp128-l2-prefetch", type=int, default=-1, help="1/0: L2 prefetch of the metablocks one grid ahead")
    ap.add_argument("--fastpfor-warps", type=int, default=0, help="warps per CTA of the SIMD-FastPFOR decoder")
    ap.add_argument("--tune", action="append", default=[], metavar="KEY=VALUE",
                    help="library tuning key (icx_set_tuning), repeatable")
    ap.add_argument("--skip-exceptions", action="store_true", help="skip the exception-heavy decode")
    ap.add_argument("--exceptions-n", type=int, default=0, help="integers of the exception-heavy array (0: 2^26)")
    ap.add_argument("--skip-intersect", action="store_true", help="skip the decode-into-intersection leg")
    ap.add_argument("--skip-bp32", action="store_true", help="skip the scalar-layout (BP32, FastPFOR) decodes")
    ap.add_argument("--skip-batch", action="store_true", help="skip the batched posting-list decode")
    ap.add_argument("--batch-lists", type=int, default=65536)
    ap.add_argument("--batch-total", type=int, default=1 << 28)
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--skip-serve", action="store_true", help="skip the serving loop")
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[10000, 100000, 300000, 1000000])
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--serve-saturation", type=int, default=300000,
                    help="requests of the closed-loop run (all waiting at the start)")
    ap.add_argument("--serve-budget", type=int, default=16 << 30)
    ap.add_argument("--serve-streams", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
