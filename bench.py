#!/usr/bin/env python
"""Benchmark of the balanced k-means partitioner on GB300.

One step = one gk_partition call on the device-resident workload: Hilbert bootstrap
(bounding box, keys, radix sort, gather, initial centers), the balanced k-means loop
(assignment passes with influence updates, center movement, erosion) and the scatter of
block ids to input order.  Default workload: 3D Gaussian mixture, n = 1e7, k = 1024,
eps = 0.03, FP64 points and FP64 assignment.

Prints one JSON line (rank 0):
  value      points processed per second by the balanced k-means iterations of the whole
             job: sum over steps of n * (assignment passes) / sum of step times (bootstrap
             and movement time included in the denominator)
  e2e        the same through the C ABI with pinned host buffers (copies in the region)
  roofline   the assignment kernel: algorithmic bytes per launch / mean launch time
  cpu_baseline  the FP64 oracle's balance pass on a bounded sample, host cores

--impl reference times the oracle (the slow FP64 CPU restatement) on the same metric.
--gpus N > 1 runs N independent replicas (one per rank, weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "points/s per balanced k-means iter and partition time (s), FP32 vs FP64, 1 GB300"
UNIT = "points/s"
DEFAULT_WORKLOAD = "gmm3d_1e7_k1024_f64"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gk", choices=["gk", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="override the number of points")
    ap.add_argument("--assign", default=None, choices=["f32", "f64"],
                    help="override the workload's assignment precision")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-fp32-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sampled", action="store_true",
                    help="skip the partition with random initialization (Section 4.5)")
    ap.add_argument("--no-quality", action="store_true",
                    help="skip the edge cut / communication volume comparison on a mesh")
    ap.add_argument("--no-bounds", action="store_true",
                    help="skip the partition with per-point bounds (gk_options.bounds = 1)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=float(np.median(sm)), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


# --------------------------------------------------------------------------------------
# CPU baseline: the oracle's balance pass (assign + block weights + influence update)
# --------------------------------------------------------------------------------------
def replica_points(spec, rank: int):
    """Points of rank's independent replica of a workload (rank 0: the workload itself)."""
    from paper_1805_01208_gb300 import synth
    return synth.make_points(spec["shape"], spec["n"], spec["d"], spec["seed"] + 1000 * rank,
                             spec["dtype"])


def reduce_over_ranks(total_ms: float, work: float, dist, device):
    """Whole-job figures of N replicas: the slowest rank's time, the sum of their work."""
    import torch
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([work], device=device, dtype=torch.float64)
    dist.all_reduce(w)
    return float(t.item()), float(w.item())


def cpu_baseline(x, w, spec, seconds: float):
    import oracle
    cores = len(os.sched_getaffinity(0))
    k = spec["k"]
    m = int(min(len(x), max(4 * k, 2_000_000_000 // (k * 150))))
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(len(x), m, replace=False))
    xs = np.ascontiguousarray(x[idx], dtype=np.float64)
    ws = None if w is None else np.ascontiguousarray(w[idx], dtype=np.float64)
    xs = xs[oracle.sort_keys(oracle.hilbert_keys(xs))]
    C = oracle.sfc_centers(xs, k)
    I = np.ones(k)
    times = []
    t_end = time.perf_counter() + seconds
    while True:
        t0 = time.perf_counter()
        A, _, _ = oracle.assign(xs, C, I, threads=cores)
        S, W = oracle.block_weights(A, ws, k)
        bal, I, _ = oracle.balance_update(S, W, k, spec["d"], spec["eps"], I)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end and len(times) >= 2:
            break
    t = float(np.mean(times))
    return {"value": m / t, "unit": UNIT, "cores": cores, "kind": "oracle", "ms_per_pass": 1e3 * t,
            "sample": (f"{m} of the workload's points (uniform sample, curve-sorted), k={k}: "
                       f"one FP64 balance pass (brute-force assignment over all k with "
                       f"{cores} OpenMP threads, block weights, influence update), "
                       f"mean of {len(times)} passes")}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1805_01208_gb300 import synth
    x, w, spec = synth.workload(args.workload, n=args.n)
    cores = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        cpu_baseline(x, w, spec, 0.0)
    per_step = max(1.0, min(20.0, 120.0 / max(1, args.steps)))
    vals = [cpu_baseline(x, w, spec, per_step) for _ in range(args.steps)]
    value = float(np.mean([v["value"] for v in vals]))
    ms = float(np.mean([v["ms_per_pass"] for v in vals]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": _config(spec, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _config(spec, args):
    return {"workload": args.workload, "n": spec["n"], "d": spec["d"], "k": spec["k"],
            "eps": spec["eps"], "points": spec["dtype"], "assign": spec["assign"],
            "weights": "uniform[1,10]" if spec["weighted"] else "unit",
            "l2": "inputs larger than L2 and a 512 MB write between timed steps",
            "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single"}


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------
BATCHED_WORKLOAD = "batched64_f32"


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == BATCHED_WORKLOAD:
        return run_batched(args)
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1805_01208_gb300 as gk
    gk.build()
    from paper_1805_01208_gb300 import synth

    x, w, spec = synth.workload(args.workload, n=args.n)
    if args.assign:
        spec["assign"] = args.assign
    if world > 1 and rank > 0:  # replicas: an independent instance per rank
        x = replica_points(spec, rank)
    n, d, k, eps = len(x), spec["d"], spec["k"], spec["eps"]
    xt = torch.from_numpy(x).to(dev)
    wt = None if w is None else torch.from_numpy(w).to(dev)
    opts = gk.default_options(assign_dtype=spec["assign"])
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def step(options):
        return gk.partition(xt, k, eps, weights=wt, options=options)

    for _ in range(args.warmup):
        step(opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    times, results = [], []
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, _, res = step(opts)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        results.append(res)
    clk = clocks.stop()
    torch.cuda.synchronize()
    total_ms = float(sum(times))
    points_passes = float(sum(n * r["balance_passes"] for r in results))
    if dist:
        total_ms, points_passes = reduce_over_ranks(total_ms, points_passes, dist, dev)
    value = points_passes / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    launches = int(sum(r["kernel_launches"] for r in results))

    # ---- end to end through the C ABI with pinned host buffers -------------------------
    e2e = _e2e(gk, x, w, spec, opts, stream, max(1, min(3, args.steps)))

    # ---- roofline of the assignment kernel ---------------------------------------------
    live_ms = sum(r["assign_live_ms"] for r in results)
    live_n = sum(r["assign_live_launches"] for r in results)
    timed = gk.default_options(assign_dtype=spec["assign"], use_graph=0, timing=1)
    _, _, _, tres = step(timed)
    ev_avg = tres["time_assign_ms"] / max(1, tres["assign_launches"])
    es = 8 if spec["dtype"] == "f64" else 4
    sw = es if spec["weighted"] else 0
    # algorithmic bytes of one balance pass: every point's coordinates (and weight) read
    # once; writing the block ids is not counted (only the last pass of a loop needs it)
    bytes_per_launch = n * (d * es + sw)
    # what this assignment kernel itself streams: FP32 frame coordinates, block ids (16
    # bits when k <= 65535)
    kernel_bytes = n * (d * 4 + (2 if k <= 65535 else 4) + sw)
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch / (ev_avg * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "kernel": "assign_kernel",
            "bytes_per_launch": bytes_per_launch, "kernel_stream_bytes_per_launch": kernel_bytes,
            "kernel_stream_frac": kernel_bytes / (ev_avg * 1e-3) / 1e9 / peak,
            "launch_ms_events": ev_avg,
            "launch_ms_live_graph": live_ms / max(1, live_n), "peak_source": peak_kind,
            "other_kernels_ms_per_pass": {
                "filter": tres["time_filter_ms"] / max(1, tres["filter_launches"]),
                "balance": tres["time_balance_ms"] / max(1, tres["balance_launches"]),
                "move_per_phase": tres["time_move_ms"] / max(1, tres["move_launches"])}}
    _attach_traffic(roof, args.workload)

    # ---- FP32 form on the same data ------------------------------------------------------
    fp32 = None
    if not args.no_fp32_compare and spec["assign"] == "f64":
        o32 = gk.default_options(assign_dtype="f32")
        step(o32)
        t32, r32 = [], []
        for _ in range(max(1, min(2, args.steps))):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, _, _, res = step(o32)
            e1.record(stream)
            torch.cuda.synchronize()
            t32.append(e0.elapsed_time(e1))
            r32.append(res)
        v32 = sum(n * r["balance_passes"] for r in r32) / (sum(t32) * 1e-3)
        fp64_pass = live_ms / max(1, live_n)
        fp32_pass = sum(r["assign_live_ms"] for r in r32) / max(1, sum(r["assign_live_launches"] for r in r32))
        fp32 = {"value": v32, "ms_per_step": float(np.mean(t32)),
                "balance_passes": r32[-1]["balance_passes"], "balanced": r32[-1]["balanced"],
                "assign_ms_per_pass": fp32_pass, "speedup_per_pass_vs_fp64": fp64_pass / fp32_pass,
                "speedup_partition_vs_fp64": ms_per_step / float(np.mean(t32))}

    # ---- random initialization (Section 4.5) on the same data -----------------------------
    sampled = None
    if not args.no_sampled:
        sampled = _sampled_init(gk, xt, wt, spec, opts, stream, flush, synth, ms_per_step,
                                max(1, min(3, args.steps)))

    # ---- per-point bounds (Section 4.3 in spirit; gk_options.bounds) ---------------------
    bounds = None
    if not args.no_bounds:
        bounds = _bounds_leg(gk, xt, wt, spec, stream, flush, ms_per_step, max(1, min(3, args.steps)))

    # ---- partition quality (Section 5 measures) on a mesh of the same scale ---------------
    quality = None
    if not args.no_quality and rank == 0:
        quality = _quality(gk, synth, spec, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x, w, spec, args.cpu_seconds)

    last = results[-1]
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": spec["assign"], "data": "synthetic", "config": _config(spec, args),
                "partition_time_s": ms_per_step / 1e3,
                "balance_passes_per_step": last["balance_passes"],
                "iterations_per_step": last["iterations"], "balanced": last["balanced"],
                "max_imbalance": last["max_imbalance"], "avg_candidates": last["avg_candidates"],
                "rechecked_points_per_step": last["rechecked_points"],
                "bootstrap_ms": last["time_bootstrap_ms"], "kmeans_loop_ms": last["time_kmeans_ms"],
                "gpu_launches": launches, "clocks": clk, "e2e": e2e, "roofline": roof,
                "fp32_form": fp32, "sampled_init": sampled, "bounds": bounds, "quality": quality,
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """64 instances of mixed n, d, k with weights, FP32 form, one gk_partition_batched
    call per step (one graph launch for all k-means loops)."""
    import torch
    import paper_1805_01208_gb300 as gk
    from paper_1805_01208_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gk.build()
    specs = synth.batched_instances(64, seed=4 + 1000 * rank)
    host = [synth.instance_data(sp) for sp in specs]
    xs = [torch.from_numpy(x).to(dev) for x, _ in host]
    ws = [torch.from_numpy(w).to(dev) if w is not None else None for _, w in host]
    probs = [(xs[i], sp["k"], sp["eps"], ws[i]) for i, sp in enumerate(specs)]
    opts = gk.default_options(assign_dtype="f32")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        gk.partition_batched(probs, options=opts)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    times, pp = [], 0.0
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        outs, st = gk.partition_batched(probs, options=opts)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        pp += sum(sp["n"] * r["balance_passes"] for sp, (_, _, _, r) in zip(specs, outs))
    clk = clocks.stop()
    total_ms = float(sum(times))
    if dist:
        total_ms, pp = reduce_over_ranks(total_ms, pp, dist, dev)
    res = [r for _, _, _, r in outs]
    # end to end: inputs from pinned host memory, block ids back, inside the timed region
    hx = [torch.from_numpy(x).pin_memory() for x, _ in host]
    hw = [torch.from_numpy(w).pin_memory() if w is not None else None for _, w in host]
    hb = [torch.empty(sp["n"], dtype=torch.int32).pin_memory() for sp in specs]
    e2e_ms, e2e_pp = 0.0, 0.0
    for _ in range(max(1, min(3, args.steps))):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(len(specs)):
            xs[i].copy_(hx[i], non_blocking=True)
            if ws[i] is not None:
                ws[i].copy_(hw[i], non_blocking=True)
        outs, st = gk.partition_batched(probs, options=opts)
        for i, (b, _, _, _) in enumerate(outs):
            hb[i].copy_(b, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_pp += sum(sp["n"] * r["balance_passes"] for sp, (_, _, _, r) in zip(specs, outs))
    h2d = sum(x.nbytes + (0 if w is None else w.nbytes) for x, w in host)
    if rank == 0:
        ntot = sum(sp["n"] for sp in specs)
        line = {"metric": METRIC, "value": pp / (total_ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": BATCHED_WORKLOAD, "instances": len(specs), "points": ntot,
                           "n_range": [min(sp["n"] for sp in specs), max(sp["n"] for sp in specs)],
                           "k_range": [min(sp["k"] for sp in specs), max(sp["k"] for sp in specs)],
                           "weights": "uniform[1,10]", "assign": "f32",
                           "l2": "a 512 MB write between timed steps", "parallelism": "single"},
                "partition_time_s": total_ms / args.steps / 1e3,
                "balance_passes_total": int(sum(r["balance_passes"] for r in res)),
                "balance_passes_max": int(max(r["balance_passes"] for r in res)),
                "balanced": int(sum(r["balanced"] for r in res)),
                "bootstrap_ms": res[0]["time_bootstrap_ms"], "kmeans_loop_ms": res[0]["time_kmeans_ms"],
                "gpu_launches": int(sum(r["kernel_launches"] for r in res)) * args.steps,
                "clocks": clk, "roofline": None, "cpu_baseline": None,
                "e2e": {"value": e2e_pp / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": 4 * ntot, "ms_per_step": e2e_ms / max(1, min(3, args.steps))}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _e2e(gk, x, w, spec, opts, stream, steps):
    """Same metric through gk_partition with pinned host input and output buffers."""
    import torch
    n, d, k = len(x), spec["d"], spec["k"]
    xh = torch.from_numpy(x).pin_memory()
    wh = None if w is None else torch.from_numpy(w).pin_memory()
    bh = torch.empty(n, dtype=torch.int32).pin_memory()
    ch = torch.empty((k, d), dtype=torch.float64).pin_memory()
    ih = torch.empty(k, dtype=torch.float64).pin_memory()
    code = gk.GK_F64 if spec["dtype"] == "f64" else gk.GK_F32
    L = gk.lib()
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def call():
        res = gk.Result()
        st = L.gk_partition(ctypes.c_void_p(xh.data_ptr()), code,
                            None if wh is None else ctypes.c_void_p(wh.data_ptr()), n, d, k,
                            spec["eps"], ctypes.byref(opts), ctypes.c_void_p(bh.data_ptr()),
                            ctypes.c_void_p(ch.data_ptr()), ctypes.c_void_p(ih.data_ptr()),
                            ctypes.byref(res), sptr)
        assert st in (gk.GK_OK, gk.GK_ERR_NOT_BALANCED), gk.status_string(st)
        return res

    call()
    torch.cuda.synchronize()
    tot, pp = 0.0, 0.0
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = call()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
        pp += n * res.balance_passes
    es = 8 if spec["dtype"] == "f64" else 4
    h2d = n * d * es + (n * es if w is not None else 0)
    d2h = n * 4 + k * d * 8 + k * 8
    return {"value": pp / (tot * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": tot / steps}


def _sampled_init(gk, xt, wt, spec, opts, stream, flush, synth, plain_ms, steps):
    """gk_partition_sampled on the device-resident workload with a seeded random order:
    the sample rounds on doubling samples (first sample 100 k points), then the k-means
    loop on all points.  Partition time against the plain gk_partition step."""
    import torch
    n, k, eps = int(xt.shape[0]), spec["k"], spec["eps"]
    order = torch.from_numpy(synth.random_order(n, spec["seed"])).to(xt.device)
    m0 = min(n, max(100 * k, k))
    rounds = min(max(0, math.ceil(math.log2(n / m0) - 1e-12)) if n > m0 else 0,
                 opts.max_iter - 1)

    def call():
        return gk.partition_sampled(xt, k, eps, order, 0, weights=wt, options=opts)

    call()
    torch.cuda.synchronize()
    times, res = [], None
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, _, res = call()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    return {"ms_per_step": ms, "partition_time_s": ms / 1e3, "first_sample": m0,
            "sample_rounds": rounds, "iterations": res["iterations"],
            "balance_passes": res["balance_passes"], "balanced": res["balanced"],
            "max_imbalance": res["max_imbalance"], "speedup_vs_plain": plain_ms / ms,
            "order": "seeded uniform permutation (host-generated, device-resident)"}


def _bounds_leg(gk, xt, wt, spec, stream, flush, plain_ms, steps):
    """The same partition with per-point bounds: identical results, the fraction of point
    evaluations that remain, and the time against the plain step."""
    import torch
    n, k, eps = int(xt.shape[0]), spec["k"], spec["eps"]
    o = gk.default_options(assign_dtype=spec["assign"], bounds=1)
    gk.partition(xt, k, eps, weights=wt, options=o)
    torch.cuda.synchronize()
    times, res = [], None
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, _, _, res = gk.partition(xt, k, eps, weights=wt, options=o)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.mean(times))
    return {"ms_per_step": ms, "balance_passes": res["balance_passes"],
            "evaluated_fraction": res["evaluated_points"] / (n * res["balance_passes"]),
            "assign_ms_per_pass": res["assign_live_ms"] / max(1, res["assign_live_launches"]),
            "speedup_vs_plain": plain_ms / ms}


def _quality(gk, synth, spec, stream):
    """Edge cut and communication volume (gk_partition_quality) and block diameter bounds
    (gk_block_diameter, three sweeps) of balanced k-means and of the plain curve split (the i-th n/k points on the Hilbert curve form block i) on a
    graded 3-D lattice mesh with as many vertices as the workload has points (at most
    200^3), the workload's k and eps."""
    import torch
    side = int(round(min(spec["n"], 200 ** 3) ** (1.0 / 3.0)))
    x, rp, col = synth.lattice_mesh((side, side, side), spec["seed"])
    n, k = len(x), spec["k"]
    xt = torch.from_numpy(x).cuda()
    rpt, colt = torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda()
    block, _, _, res = gk.partition(xt, k, spec["eps"])
    perm, _ = gk.sfc_init(xt, k)
    sfc = torch.empty(n, dtype=torch.int32, device=xt.device)
    sfc[perm] = (torch.arange(n, device=xt.device, dtype=torch.int64) * k // n).to(torch.int32)
    torch.cuda.synchronize()
    qs, _, _ = gk.partition_quality(rpt, colt, sfc, k)  # also loads the kernels
    reps = 5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        qk, _, _ = gk.partition_quality(rpt, colt, block, k)
    e1.record(stream)
    torch.cuda.synchronize()
    qms = e0.elapsed_time(e1) / reps
    qbytes = 8 * (n + 1) + 4 * int(rp[-1]) + 4 * n
    peak, peak_src = _peaks()
    ds, _ = gk.block_diameter(rpt, colt, sfc, k, 3)  # also loads the kernels
    t0 = time.perf_counter()
    dk, _ = gk.block_diameter(rpt, colt, block, k, 3)  # waits for its own work
    diam_ms = (time.perf_counter() - t0) * 1e3
    return {"mesh": f"graded 3-D lattice {side}^3 (6-neighbour), random vertex order",
            "vertices": n, "edges": int(rp[-1]) // 2, "k": k, "kmeans": qk, "sfc_split": qs,
            "kmeans_balanced": res["balanced"], "kmeans_partition_ms": res["time_total_ms"],
            "quality_ms": qms,
            "quality_roofline": {"bound": "hbm", "bytes": qbytes, "achieved": qbytes / qms / 1e6,
                                 "peak": peak, "unit": "GB/s", "frac": qbytes / qms / 1e6 / peak,
                                 "peak_source": peak_src,
                                 "what": "one gk_partition_quality call, mean of 5 after a "
                                         "first call (row offsets, neighbour ids and block "
                                         "ids read once)"},
            "cut_ratio_kmeans_over_sfc": qk["edge_cut"] / max(1, qs["edge_cut"]),
            "max_comm_ratio_kmeans_over_sfc": qk["max_comm_volume"] / max(1, qs["max_comm_volume"]),
            "diameter_sweeps": 3, "diameter_kmeans": dk, "diameter_sfc_split": ds,
            "diameter_ms": diam_ms}


def _attach_traffic(roof, workload):
    """DRAM traffic per launch from the committed ncu summary of this kernel, if any."""
    path = os.path.join(ROOT, "profiles", f"assign_kernel_{workload}.md")
    try:
        with open(path) as f:
            for line in f:
                if line.strip().startswith("dram_bytes_per_launch:"):
                    val = line.split(":", 1)[1].strip().split()[0]
                    roof["traffic"] = None if val == "null" else float(val)
                    roof["traffic_source"] = os.path.relpath(path, ROOT)
    except OSError:
        pass


if __name__ == "__main__":
    sys.exit(main())
