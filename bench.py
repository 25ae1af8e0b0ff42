#!/usr/bin/env python
"""Benchmark of the balanced k-means partitioner on GB300.

One step = one gk_partition call on the device-resident workload: Hilbert bootstrap
(bounding box, keys, radix sort, gather, initial centers), the balanced k-means loop
(assignment passes with influence updates, center movement, erosion) and the scatter of
block ids to input order.  Default workload (the largest one-GPU configuration): 2D,
n = 1e9, uniform background plus 256 Gaussian refinement spots, FP32 coordinates,
unit weights, k = 16384, eps = 0.03, FP32 assignment with FP64 block weights, centroids
and influence.

Prints one JSON line (rank 0):
  value        points processed per second by the balanced k-means iterations of the
               whole job: sum over steps of n * (assignment passes) / sum of step times
               (bootstrap and movement time included in the denominator)
  e2e          the same through the C ABI with pinned host buffers (copies in the region)
  roofline     the assignment pass (filter, assignment and balance kernels, which together
               assign every point once): algorithmic bytes per pass / mean pass time
  fp32_form    the FP32 form's statistics: fraction of points assigned differently from
               the FP64 argmin under the returned centers and influence (all points), the
               largest error of the centroid step against FP64 means, the exact imbalance
               (block sizes counted on the host)
  fp64_form    the FP64 argmin (certified FP32 search + FP64 re-decision) on the same
               points, and the FP32 form's speedup over it
  legs         the other workloads (3D mixture n = 1e7 k = 1024 FP64; 2D radial n = 1e8
               k = 4096 FP32; 64 batched instances), each with its own roofline
  cpu_baseline the FP64 oracle's balance pass on a uniform sample, host cores

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
DEFAULT_WORKLOAD = "spots2d_1e9_k16384_f32"
BATCHED_WORKLOAD = "batched64_f32"
EXTRA_LEGS = ("gmm3d_1e7_k1024_f64", "radial2d_1e8_k4096_f32", BATCHED_WORKLOAD)
FLUSH_BYTES = 512 << 20  # written between timed steps: evicts the 129 MB L2
FIXED_SHAPES: dict = {}  # --shapes: fixed launch shapes (with --no-legs: the headline's calls)


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gk", choices=["gk", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--n", type=int, default=None, help="override the number of points")
    ap.add_argument("--shapes", default=None,
                    help="fix the launch shapes as 'supertile_tiles,hypertiles,ctas_per_sm' for the "
                         "headline workload's partitions and its roofline run (for profiles: the "
                         "tuner's choice can differ under a profiler)")
    ap.add_argument("--k", type=int, default=None,
                    help="override the number of blocks (profiling a smaller n at the "
                         "workload's points per block)")
    ap.add_argument("--assign", default=None, choices=["f32", "f64"],
                    help="override the workload's assignment precision")
    ap.add_argument("--cpu-seconds", type=float, default=20.0,
                    help="CPU time budget of one oracle pass of the cpu_baseline")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the other workloads (3D mixture, 2D radial, batched)")
    ap.add_argument("--no-fp64-compare", action="store_true")
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
# replicas (N > 1) and the CPU baseline
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


def _oracle_pass(xs, ws, C, I, spec, cores):
    """One FP64 balance pass of the oracle (brute-force assignment over all k centers with
    OpenMP on `cores` threads, block weights, influence update); returns its time in s."""
    import oracle
    t0 = time.perf_counter()
    A, _, _ = oracle.assign(xs, C, I, threads=cores)
    S, W = oracle.block_weights(A, ws, spec["k"])
    oracle.balance_update(S, W, spec["k"], spec["d"], spec["eps"], I)
    return time.perf_counter() - t0


def _oracle_sample(x, w, m, seed=12345):
    """A uniform sample of m of the points, curve-sorted, with its curve centers."""
    import oracle
    rng = np.random.default_rng(seed)
    n = len(x)
    idx = np.sort(rng.choice(n, m, replace=False)) if m < n else np.arange(n)
    xs = np.ascontiguousarray(x[idx], dtype=np.float64)
    ws = None if w is None else np.ascontiguousarray(w[idx], dtype=np.float64)
    order = oracle.sort_keys(oracle.hilbert_keys(xs))
    xs = xs[order]
    ws = None if ws is None else ws[order]
    return xs, ws


def _sample_size(x, w, spec, seconds, cores):
    """Points of the sample whose oracle pass takes about `seconds` (calibrated on a small
    sample; the pass is O(points x k)), at most 1% of the workload above 1e8 points and
    all of a smaller one."""
    import oracle
    n, k = len(x), spec["k"]
    cap = n // 100 if n >= 100_000_000 else n
    mc = int(min(cap, max(4 * k, 2_000_000_000 // (k * 400))))
    xs, ws = _oracle_sample(x, w, mc, seed=777)
    C = oracle.sfc_centers(xs, k)
    t = _oracle_pass(xs, ws, C, np.ones(k), spec, cores)
    per_point = t / mc
    return int(max(min(cap, seconds / per_point), min(cap, 4 * k)))


def cpu_baseline(x, w, spec, seconds: float, m: int | None = None, passes: int = 1):
    """The oracle's FP64 balance pass on a uniform sample of the workload, sized to about
    `seconds` per pass (1% of the points for the 1e9-point workload when that fits);
    reported per point, with the full pass extrapolated from it."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    n, k = len(x), spec["k"]
    if m is None:
        m = _sample_size(x, w, spec, seconds, cores)
    xs, ws = _oracle_sample(x, w, m)
    C = oracle.sfc_centers(xs, k)
    I = np.ones(k)
    times = [_oracle_pass(xs, ws, C, I, spec, cores) for _ in range(passes)]
    t = float(np.mean(times))
    frac = m / n
    return {"value": m / t, "unit": UNIT, "cores": cores, "kind": "oracle", "ms_per_pass": 1e3 * t,
            "sample_points": m, "sample_fraction": frac,
            "full_pass_s_extrapolated": t * n / m,
            "sample": (f"{m} of the workload's {n} points ({100 * frac:.3g}%, uniform sample, "
                       f"curve-sorted), k={k}: one FP64 balance pass (brute-force assignment over "
                       f"all k with {cores} OpenMP threads, block weights, influence update), "
                       f"mean of {len(times)} pass(es); a full pass extrapolated x{n / m:.4g} "
                       f"(extrapolated, not measured): {t * n / m:.1f} s")}


def run_reference(args):
    """The oracle on the headline workload's metric: every step one FP64 balance pass on
    a bounded uniform sample of the workload's distribution (the generator's first points:
    independent draws of the same distribution), sized so the whole run takes about two
    minutes on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1805_01208_gb300 import synth
    spec0 = dict(synth.WORKLOADS[args.workload]) if args.workload in synth.WORKLOADS else None
    if spec0 is None:  # the batched workload: its largest instance stands in
        return _reference_unavailable(args, "the batched workload has no single-config oracle arm")
    n_full = args.n or spec0["n"]
    cores = len(os.sched_getaffinity(0))
    probe_n = int(min(n_full, 4_000_000))
    x, w, spec = synth.workload(args.workload, n=probe_n)
    if args.k:
        spec["k"] = args.k
    budget = max(1.0, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    m = min(probe_n, _sample_size(x, w, spec, budget, cores))
    for _ in range(args.warmup):
        cpu_baseline(x, w, spec, 0.0, m=max(spec["k"], m // 10))
    vals = [cpu_baseline(x, w, spec, 0.0, m=m) for _ in range(args.steps)]
    value = float(np.mean([v["value"] for v in vals]))
    ms = float(np.mean([v["ms_per_pass"] for v in vals]))
    spec["n"] = n_full
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": _config(spec, args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": (f"{m} points drawn from the workload's distribution "
                                        f"(the generator's first points) per step, k="
                                        f"{spec['k']}: one FP64 balance pass (brute-force "
                                        f"assignment with {cores} OpenMP threads, block "
                                        f"weights, influence update)")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _reference_unavailable(args, why):
    print(json.dumps({"impl": "reference", "unavailable": why}), flush=True)
    return 0


def _config(spec, args):
    return {"workload": args.workload, "n": spec["n"], "d": spec["d"], "k": spec["k"],
            "eps": spec["eps"], "points": spec["dtype"], "assign": spec["assign"],
            "reductions": "f64", "weights": "uniform[1,10]" if spec["weighted"] else "unit",
            "l2": "inputs larger than L2 and a 512 MB write between timed steps",
            "parallelism": f"replicas{args.gpus}" if args.gpus > 1 else "single"}


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------
def _timed(stream, flush, fn, steps):
    """(times in ms, results) of `steps` calls of fn, each bracketed by CUDA events on the
    library's stream, the L2 flushed before each (outside the events)."""
    import torch
    times, outs = [], []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        outs.append(out)
    return times, outs


def _roofline(gk, xt, wt, spec, workload):
    """The HBM roofline of the assignment pass, the unit that assigns every point once:
    the filter kernels (which also finish the tiles with a single candidate), the
    assignment kernel (the tiles of the filter's work list) and the balance kernel.
    achieved = algorithmic bytes of one pass (every point's coordinates and weight read
    once) over the mean CUDA-event duration of those launches per pass, in a host-driven
    run of the same partition (events on the library's stream)."""
    n, d, k = int(xt.shape[0]), spec["d"], spec["k"]
    timed = gk.default_options(assign_dtype=spec["assign"], use_graph=0, timing=1, **FIXED_SHAPES)
    _, _, _, tres = gk.partition(xt, k, spec["eps"], weights=wt, options=timed)
    npass = max(1, tres["assign_launches"])
    ev_assign = tres["time_assign_ms"] / npass
    ev_filter = tres["time_filter_ms"] / max(1, tres["filter_launches"])
    ev_balance = tres["time_balance_ms"] / max(1, tres["balance_launches"])
    pass_ms = (tres["time_assign_ms"] + tres["time_filter_ms"] + tres["time_balance_ms"]) / npass
    es = 8 if spec["dtype"] == "f64" else 4
    sw = es if spec["weighted"] else 0
    bytes_per_pass = n * (d * es + sw)
    peak, peak_kind = _peaks()
    achieved = bytes_per_pass / (pass_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "kernel": "assignment pass (filter_kernel + filter_big_kernel [+ hyper_kernel] "
                      "[+ filter_tile_kernel] + assign_kernel + balance_kernel)",
            "note": "achieved counts every point's coordinates once (the algorithmic bytes); "
                    "by design the pass reads fewer: the filter finishes the tiles whose "
                    "candidate list holds one center without reading their points, so frac "
                    "can exceed 1",
            "bytes_per_launch": bytes_per_pass, "launch_ms_events": pass_ms,
            "peak_source": peak_kind,
            "kernels_ms_per_pass": {"filter": ev_filter, "assign": ev_assign, "balance": ev_balance},
            "shapes": {"supertile_tiles": tres["supertile_tiles"], "hypertiles": tres["hypertiles"],
                       "assign_ctas_per_sm": tres["assign_ctas_per_sm"]},
            "move_ms_per_phase": tres["time_move_ms"] / max(1, tres["move_launches"])}
    _attach_traffic(roof, workload)
    return roof


def _exact_imbalance(block_host, w_host, k, eps):
    """Block sizes counted on the host from the returned block ids (exact integers for
    unit weights), the largest over ceil(W/k) minus 1, and whether it meets eps."""
    import torch
    if w_host is None:
        S = torch.bincount(torch.from_numpy(block_host), minlength=k).numpy()
        W = float(len(block_host))
    else:
        S = np.bincount(block_host, weights=w_host.astype(np.float64), minlength=k)
        W = float(w_host.astype(np.float64).sum())
    ceil_avg = math.ceil(W / k)
    return {"max_block": float(S.max()), "ceil_avg": ceil_avg,
            "max_imbalance": float(S.max()) / ceil_avg - 1.0,
            "meets_eps": bool(S.max() <= (1 + eps) * ceil_avg * (1 + 1e-15)),
            "counted": "on the host from the returned block ids"}


def _fp32_stats(gk, xt, wt, spec, block, C, I, block_host, w_host):
    """The FP32 form's stated figures under the returned centers and influence.
    disagreement: fraction of all points whose block differs from the FP64 argmin of the
      effective distance (the library's certified FP64 assignment, parity-tested against
      the oracle), on the curve-sorted points;
    center_error: largest |centroid step - FP64 weighted mean| over the blocks of the
      returned assignment (library: exact fixed-point sums; reference: plain FP64 sums with
      torch), relative to the bounding-box extent;
    imbalance: block sizes counted on the host."""
    import torch
    n, d, k = int(xt.shape[0]), spec["d"], spec["k"]
    perm, _ = gk.sfc_init(xt, k)
    As = block.index_select(0, perm)
    xs = xt.index_select(0, perm)
    A64, _ = gk.assign(xs, C, I, assign_dtype="f64")
    differ = int((As != A64).sum().item())
    del xs, As, A64, perm
    ext = float((xt.amax(0).double() - xt.amin(0).double()).max().item())
    Cm, _, _ = gk.move_centers(xt, block, C, weights=wt)
    sums = torch.zeros((k, d), dtype=torch.float64, device=xt.device)
    cnt = torch.zeros(k, dtype=torch.float64, device=xt.device)
    chunk = 1 << 26
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        b = block[s:e].long()
        wv = torch.ones(e - s, dtype=torch.float64, device=xt.device) if wt is None else wt[s:e].double()
        sums.index_add_(0, b, xt[s:e].double() * wv[:, None])
        cnt.index_add_(0, b, wv)
    ne = cnt > 0
    mean = sums[ne] / cnt[ne][:, None]
    cerr = float((Cm[ne] - mean).abs().max().item()) / ext
    # a second reference on the host: FP64 brute force over all k centers (numpy) for a
    # uniform sample of the points
    m = min(n, 10_000)
    rng = np.random.default_rng(2024)
    idx = np.sort(rng.choice(n, m, replace=False)) if m < n else np.arange(n)
    it = torch.from_numpy(idx).to(xt.device)
    xs_h = xt.index_select(0, it).double().cpu().numpy()
    bs_h = block.index_select(0, it).cpu().numpy()
    Ch, gh = C.double().cpu().numpy(), 1.0 / I.double().cpu().numpy() ** 2
    ref = np.empty(m, dtype=np.int64)
    for s0 in range(0, m, 512):  # the squared distance axis by axis, then times 1/I^2
        xc = xs_h[s0:s0 + 512]
        d2 = (xc[:, 0, None] - Ch[None, :, 0]) ** 2
        for j in range(1, d):
            d2 += (xc[:, j, None] - Ch[None, :, j]) ** 2
        d2 *= gh[None, :]
        ref[s0:s0 + 512] = np.argmin(d2, axis=1)
    host_differ = int((ref != bs_h).sum())
    out = {"disagreement": differ / n, "disagreeing_points": differ, "points_checked": n,
           "disagreement_host_sample": host_differ / m, "host_sample_points": m,
           "host_sample_reference": "FP64 brute force over all k centers on the host (numpy), "
                                    "uniform sample",
           "disagreement_reference": "FP64 argmin under the returned centers and influence "
                                     "(gk_assign in FP64 mode), every point",
           "center_error": cerr,
           "center_error_reference": "FP64 weighted means of the returned assignment (torch "
                                     "FP64 sums), relative to the bounding-box extent"}
    out.update(_exact_imbalance(block_host, w_host, k, spec["eps"]))
    return out


def _config_leg(gk, name, stream, flush, steps, x=None, w=None, spec=None):
    """One workload as a leg of the line: partition time and points/s over `steps` timed
    calls, its assignment pass's roofline and, for the FP32 form, its statistics."""
    import torch
    from paper_1805_01208_gb300 import synth
    if name == BATCHED_WORKLOAD:
        return _batched_leg(gk, stream, flush, steps)
    if x is None:
        x, w, spec = synth.workload(name)
    dev = torch.device("cuda", torch.cuda.current_device())
    xt = torch.from_numpy(x).to(dev)
    wt = None if w is None else torch.from_numpy(w).to(dev)
    n, k, eps = len(x), spec["k"], spec["eps"]
    opts = gk.default_options(assign_dtype=spec["assign"])

    def step():
        return gk.partition(xt, k, eps, weights=wt, options=opts)

    step()
    torch.cuda.synchronize()
    times, outs = _timed(stream, flush, step, steps)
    res = outs[-1][3]
    leg = {"workload": name, "n": n, "d": spec["d"], "k": k, "points": spec["dtype"],
           "assign": spec["assign"], "weights": "uniform[1,10]" if spec["weighted"] else "unit",
           "value": sum(n * o[3]["balance_passes"] for o in outs) / (sum(times) * 1e-3),
           "unit": UNIT, "ms_per_step": float(np.mean(times)), "steps": steps,
           "balance_passes": res["balance_passes"], "iterations": res["iterations"],
           "balanced": res["balanced"], "max_imbalance": res["max_imbalance"],
           "bootstrap_ms": res["time_bootstrap_ms"], "avg_candidates": res["avg_candidates"],
           "assign_ms_per_pass_live": res["assign_live_ms"] / max(1, res["assign_live_launches"]),
           "launch_shapes": {"supertile_tiles": res["supertile_tiles"], "hypertiles": res["hypertiles"],
                             "assign_ctas_per_sm": res["assign_ctas_per_sm"]},
           "roofline": _roofline(gk, xt, wt, spec, name)}
    if spec["assign"] == "f32":
        block, C, I, _ = outs[-1]
        leg["fp32_form"] = _fp32_stats(gk, xt, wt, spec, block, C, I, block.cpu().numpy(), w)
    del xt, wt, outs
    gk.release()
    torch.cuda.empty_cache()
    return leg


def _batched_leg(gk, stream, flush, steps, rank=0):
    """64 instances of mixed n, d, k with weights, FP32 form, one gk_partition_batched call
    per step (one graph launch for all k-means loops); per instance the FP32-form
    disagreement (all points) and the exact imbalance."""
    import torch
    from paper_1805_01208_gb300 import synth
    dev = torch.device("cuda", torch.cuda.current_device())
    specs = synth.batched_instances(64, seed=4 + 1000 * rank)
    host = [synth.instance_data(sp) for sp in specs]
    xs = [torch.from_numpy(x).to(dev) for x, _ in host]
    ws = [torch.from_numpy(w).to(dev) if w is not None else None for _, w in host]
    probs = [(xs[i], sp["k"], sp["eps"], ws[i]) for i, sp in enumerate(specs)]
    opts = gk.default_options(assign_dtype="f32")
    gk.partition_batched(probs, options=opts)
    torch.cuda.synchronize()
    times, outs = _timed(stream, flush, lambda: gk.partition_batched(probs, options=opts)[0], steps)
    last = outs[-1]
    res = [r for _, _, _, r in last]
    pp = sum(sum(sp["n"] * r["balance_passes"] for sp, (_, _, _, r) in zip(specs, o)) for o in outs)
    ntot = sum(sp["n"] for sp in specs)
    dis, imb, meets = [], [], 0
    for i, (sp, (b, C, I, r)) in enumerate(zip(specs, last)):
        perm, _ = gk.sfc_init(xs[i], sp["k"])
        A64, _ = gk.assign(xs[i].index_select(0, perm), C, I, assign_dtype="f64")
        dis.append(int((b.index_select(0, perm) != A64).sum().item()) / sp["n"])
        e = _exact_imbalance(b.cpu().numpy(), host[i][1], sp["k"], sp["eps"])
        imb.append(e["max_imbalance"])
        meets += int(e["meets_eps"])
    leg = {"workload": BATCHED_WORKLOAD, "instances": len(specs), "points": ntot,
           "n_range": [min(sp["n"] for sp in specs), max(sp["n"] for sp in specs)],
           "k_range": [min(sp["k"] for sp in specs), max(sp["k"] for sp in specs)],
           "weights": "uniform[1,10]", "assign": "f32",
           "value": pp / (sum(times) * 1e-3), "unit": UNIT, "ms_per_step": float(np.mean(times)),
           "steps": steps, "balance_passes_total": int(sum(r["balance_passes"] for r in res)),
           "balance_passes_max": int(max(r["balance_passes"] for r in res)),
           "balanced_instances": int(sum(r["balanced"] for r in res)),
           "bootstrap_ms": res[0]["time_bootstrap_ms"],
           "kernel_launches_per_step": int(sum(r["kernel_launches"] for r in res)),
           "fp32_form": {"disagreement_max": max(dis), "disagreement_mean": float(np.mean(dis)),
                         "disagreement_reference": "FP64 argmin under each instance's returned "
                                                   "state (gk_assign FP64), every point",
                         "max_imbalance_per_instance": imb,
                         "instances_meeting_eps": meets,
                         "counted": "block weights summed on the host from the returned ids"}}
    del xs, ws, probs, outs, last
    gk.release()
    torch.cuda.empty_cache()
    return leg, host, specs


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
    if args.k:
        spec["k"] = args.k
    if world > 1 and rank > 0:  # replicas: an independent instance per rank
        x = replica_points(spec, rank)
    n, d, k, eps = len(x), spec["d"], spec["k"], spec["eps"]
    xt = torch.from_numpy(x).to(dev)
    wt = None if w is None else torch.from_numpy(w).to(dev)
    if args.shapes:
        stl, hy, ct = (int(v) for v in args.shapes.split(","))
        FIXED_SHAPES.update(supertile_tiles=stl, hypertiles=hy, assign_ctas_per_sm=ct)
    opts = gk.default_options(assign_dtype=spec["assign"], **FIXED_SHAPES)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(options=opts):
        return gk.partition(xt, k, eps, weights=wt, options=options)

    warm = [step()[3] for _ in range(args.warmup)]
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    times, outs = _timed(stream, flush, step, args.steps)
    clk = clocks.stop()
    results = [o[3] for o in outs]
    torch.cuda.synchronize()
    total_ms = float(sum(times))
    points_passes = float(sum(n * r["balance_passes"] for r in results))
    if dist:
        total_ms, points_passes = reduce_over_ranks(total_ms, points_passes, dist, dev)
    value = points_passes / (total_ms * 1e-3)
    ms_per_step = total_ms / args.steps
    launches = int(sum(r["kernel_launches"] for r in results))
    block, C, I, last = outs[-1]
    block_host = block.cpu().numpy()
    del outs

    # ---- end to end through the C ABI with pinned host buffers -------------------------
    e2e = _e2e(gk, x, w, spec, opts, stream, max(1, min(3, args.steps)))

    # ---- roofline of the assignment pass -----------------------------------------------
    roof = _roofline(gk, xt, wt, spec, args.workload)
    live_ms = sum(r["assign_live_ms"] for r in results)
    live_n = sum(r["assign_live_launches"] for r in results)
    roof["assign_kernel_ms_live_graph"] = live_ms / max(1, live_n)

    # ---- FP32-form statistics under the returned state ----------------------------------
    fp32 = None
    if spec["assign"] == "f32":
        fp32 = _fp32_stats(gk, xt, wt, spec, block, C, I, block_host, w)

    # ---- FP64 argmin on the same points --------------------------------------------------
    fp64 = None
    if not args.no_fp64_compare and spec["assign"] == "f32":
        o64 = gk.default_options(assign_dtype="f64")
        step(o64)
        t64, o64s = _timed(stream, flush, lambda: step(o64), max(1, min(2, args.steps)))
        r64 = o64s[-1][3]
        b64, C64, I64 = o64s[-1][:3]
        pass32 = live_ms / max(1, live_n)
        pass64 = sum(o[3]["assign_live_ms"] for o in o64s) / max(1, sum(o[3]["assign_live_launches"] for o in o64s))
        ext = float((xt.amax(0).double() - xt.amin(0).double()).max().item())
        fp64 = {"value": sum(n * o[3]["balance_passes"] for o in o64s) / (sum(t64) * 1e-3),
                "ms_per_step": float(np.mean(t64)), "balance_passes": r64["balance_passes"],
                "iterations": r64["iterations"], "balanced": r64["balanced"],
                "max_imbalance": r64["max_imbalance"],
                "rechecked_points_per_step": r64["rechecked_points"],
                "assign_ms_per_pass_live": pass64,
                "fp32_speedup_per_pass": pass64 / pass32,
                "fp32_speedup_per_partition": float(np.mean(t64)) / ms_per_step,
                "partitions_differ_fraction": float((b64 != block).double().mean().item()),
                "center_diff_vs_fp32_form": float((C64 - C).abs().max().item()) / ext}
        del o64s, b64, C64, I64

    # ---- launch shapes: the tuned ones against the fixed defaults of the kernels -----------
    shapes = {"supertile_tiles": last["supertile_tiles"], "assign_ctas_per_sm": last["assign_ctas_per_sm"],
              "hypertiles": last["hypertiles"],
              "tune_ms_first_call": warm[0]["tune_ms"] if warm else None}
    ofix = gk.default_options(assign_dtype=spec["assign"], supertile_tiles=16, hypertiles=1,
                              assign_ctas_per_sm=64)
    step(ofix)
    tfix, rfix = _timed(stream, flush, lambda: step(ofix), max(1, min(2, args.steps)))
    shapes["fixed"] = {"supertile_tiles": 16, "hypertiles": 1,
                       "assign_ctas_per_sm": rfix[-1][3]["assign_ctas_per_sm"],
                       "ms_per_step": float(np.mean(tfix))}
    shapes["tuned_speedup_vs_fixed"] = float(np.mean(tfix)) / ms_per_step
    del rfix

    # ---- random initialization (Section 4.5) on the same data -----------------------------
    sampled = None
    if not args.no_sampled:
        sampled = _sampled_init(gk, xt, wt, spec, opts, stream, flush, synth, ms_per_step, 1)

    # ---- per-point bounds (Section 4.3 in spirit; gk_options.bounds) ---------------------
    bounds = None
    if not args.no_bounds:
        bounds = _bounds_leg(gk, xt, wt, spec, stream, flush, ms_per_step, 1)

    del xt, wt, block, C, I
    gk.release()
    torch.cuda.empty_cache()

    # ---- the other workloads -------------------------------------------------------------
    legs = {}
    if not args.no_legs and rank == 0:
        for name in EXTRA_LEGS:
            if name == args.workload:
                continue
            if name == BATCHED_WORKLOAD:
                legs[name] = _batched_leg(gk, stream, flush, 2)[0]
            else:
                legs[name] = _config_leg(gk, name, stream, flush, 3)

    # ---- partition quality (Section 5 measures) on a mesh --------------------------------
    quality = None
    if not args.no_quality and rank == 0:
        quality = _quality(gk, synth, spec, stream)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(x, w, spec, args.cpu_seconds)

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
                "launch_shapes": shapes,
                "fp32_form": fp32, "fp64_form": fp64, "legs": legs, "sampled_init": sampled,
                "bounds": bounds, "quality": quality, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batched(args):
    """The batched workload as the line's own workload (--workload batched64_f32)."""
    import torch
    import paper_1805_01208_gb300 as gk
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
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # warm-up calls inside the leg (one), then the timed steps
    for _ in range(max(0, args.warmup - 1)):
        _batched_leg(gk, stream, flush, 1, rank)
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    leg, host, specs = _batched_leg(gk, stream, flush, args.steps, rank)
    clk = clocks.stop()
    total_ms = leg["ms_per_step"] * args.steps
    pp = leg["value"] * total_ms * 1e-3
    if dist:
        total_ms, pp = reduce_over_ranks(total_ms, pp, dist, dev)
    # end to end: inputs from pinned host memory, block ids back, inside the timed region
    xs = [torch.empty(x.shape, dtype=torch.from_numpy(x).dtype, device=dev) for x, _ in host]
    ws = [None if w is None else torch.empty(w.shape, dtype=torch.from_numpy(w).dtype, device=dev)
          for _, w in host]
    probs = [(xs[i], sp["k"], sp["eps"], ws[i]) for i, sp in enumerate(specs)]
    hx = [torch.from_numpy(x).pin_memory() for x, _ in host]
    hw = [torch.from_numpy(w).pin_memory() if w is not None else None for _, w in host]
    hb = [torch.empty(sp["n"], dtype=torch.int32).pin_memory() for sp in specs]
    opts = gk.default_options(assign_dtype="f32")
    e2e_ms, e2e_pp, reps = 0.0, 0.0, max(1, min(3, args.steps))
    for _ in range(reps):
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
        line = {"metric": METRIC, "value": pp / (total_ms * 1e-3), "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": BATCHED_WORKLOAD, "instances": leg["instances"],
                           "points": leg["points"], "n_range": leg["n_range"],
                           "k_range": leg["k_range"], "weights": "uniform[1,10]", "assign": "f32",
                           "reductions": "f64", "l2": "a 512 MB write between timed steps",
                           "parallelism": "single"},
                "partition_time_s": total_ms / args.steps / 1e3,
                "gpu_launches": leg["kernel_launches_per_step"] * args.steps,
                "clocks": clk, "roofline": None, "cpu_baseline": None, "batched": leg,
                "e2e": {"value": e2e_pp / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": 4 * leg["points"], "ms_per_step": e2e_ms / reps}}
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
    del xh, wh, bh
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
    times, outs = _timed(stream, flush, call, steps)
    res = outs[-1][3]
    del outs, order
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
    times, outs = _timed(stream, flush, lambda: gk.partition(xt, k, eps, weights=wt, options=o),
                         steps)
    res = outs[-1][3]
    del outs
    ms = float(np.mean(times))
    return {"ms_per_step": ms, "balance_passes": res["balance_passes"],
            "evaluated_fraction": res["evaluated_points"] / (n * res["balance_passes"]),
            "assign_ms_per_pass": res["assign_live_ms"] / max(1, res["assign_live_launches"]),
            "speedup_vs_plain": plain_ms / ms}


def _quality(gk, synth, spec, stream, k=1024, seed=2):
    """Edge cut and communication volume (gk_partition_quality) and block diameter bounds
    (gk_block_diameter, three sweeps) of balanced k-means and of the plain curve split (the
    i-th n/k points on the Hilbert curve form block i) on a graded 3-D lattice mesh of
    200^3 vertices (at most as many as the workload has points), k = 1024, the workload's
    eps."""
    import torch
    side = int(round(min(spec["n"], 200 ** 3) ** (1.0 / 3.0)))
    x, rp, col = synth.lattice_mesh((side, side, side), seed)
    n = len(x)
    k = min(k, n)
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
    """DRAM traffic of one assignment pass from the committed ncu summary, if any."""
    path = os.path.join(ROOT, "profiles", f"assignment_pass_{workload}.md")
    try:
        with open(path) as f:
            for line in f:
                if line.strip().startswith("dram_bytes_per_pass:"):
                    val = line.split(":", 1)[1].strip().split()[0]
                    roof["traffic"] = None if val == "null" else float(val)
                    roof["traffic_source"] = os.path.relpath(path, ROOT)
    except OSError:
        pass


if __name__ == "__main__":
    sys.exit(main())
