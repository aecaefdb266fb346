#!/usr/bin/env python
"""Lloyd k-means benchmark: prints ONE JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

A step is one ``kmeans_run`` call: every Lloyd iteration of the workload (20 for
the default 4,194,304 x 128 x 1024 precision workload) as one graph-captured
sequence of the library's kernels, on inputs already resident in HBM. The
headline is the BF16 distance contraction with the FP32 near-tie re-check;
``value`` is Lloyd iterations per second over all ranks and the distance
TFLOP/s (2nkd per iteration) is reported beside it. ``e2e`` times the same runs
through ``kmeans_run_host`` from pinned host buffers, copies included.

On one GPU the default run also measures, on the same data, the metric's
comparison arms (plain FP32, E4M3 + re-check, two-part BF16 + re-check), the
other workloads (8M x 256 x 8192 E4M3, the 512-instance batch, 10k x 16 x 8),
and the FP32 FFMA and FP8 tensor peaks that their roofline fractions use.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step), the one other place this script
runs oracle code; so does the ``cpu_baseline`` leg of the default arm.

Multi-GPU (torchrun, one rank per GPU): the single-instance workloads run as one
sharded problem (strong scaling): every rank holds a contiguous shard of the
points and all centroids, and each Lloyd iteration is kmeans_step_partial on the
shard, one NCCL sum all-reduce of the k*d + k + 2 partials, and
kmeans_apply_partials (paper_1109_0778_b300.sharded); value = the problem's
iterations / the slowest rank's time. The training and SPADE workloads run
independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from synth import SPADE_WORKLOADS, WORKLOADS  # noqa: E402

METRIC = "Lloyd iter/s + distance TFLOP/s: FP32 vs BF16/FP8+recheck, exact assignments"
DEFAULT_WORKLOAD = "prec_n4M_d128_k1024"
# precision of a workload's headline line (else the workload's first)
HEADLINE_PRECISION = {"prec_n4M_d128_k1024": "bf16", "large_n8M_d256_k8192": "fp8"}
DTYPE_NAMES = {"fp32": "f32", "bf16": "bf16", "fp8": "e4m3", "bf16x3": "bf16x3"}
STAGE_KERNELS = ("prep", "assign", "recheck", "count", "scan", "scatter", "segsum", "divide")
# Source file of each stage's kernel (a change to it voids a stored ncu traffic figure).
KERNEL_SOURCES = {"assign": {"fp32": "km_assign_simt.cu", "bf16": "km_assign_tc.cu", "fp8": "km_assign_tc.cu",
                             "bf16x3": "km_assign_tc.cu"},
                  "spade_pairs": {"f32": "km_spade.cu"}}


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + sorted(TRAIN_WORKLOADS) + sorted(SPADE_WORKLOADS))
    ap.add_argument("--precision", default=None,
                    help="fp32 | bf16 | fp8 | bf16x3 (default: bf16 on the precision workload, else the workload's first)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="target CPU time of the oracle sample")
    ap.add_argument("--rows", type=int, default=0, help="use only the first ROWS points (profiling cases)")
    ap.add_argument("--instances", type=int, default=0,
                    help="batched workload: use only the first INSTANCES instances (profiling cases)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="headline only: skip the precision arms, the other workloads and the peak measurements")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def dist_init(world, backend):
    import torch.distributed as dist

    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def max_over_ranks(dist, value: float, device=None) -> float:
    if dist is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


def aggregate_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job rate of weak-scaling replicas: all ranks' units over the slowest rank's time."""
    return units_per_rank * world / t_max


# ----------------------------------------------------------------------------- clocks

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs (read-only)."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- peaks / profiles

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


def fp32_simt_peak_tflops(sm_count: int, mhz: float) -> float:
    """FFMA peak: SMs x 128 FP32 lanes x 2 flops x clock."""
    return sm_count * 128 * 2 * mhz * 1e6 / 1e12


def kernel_source_sha(stage: str, precision: str) -> str | None:
    src = KERNEL_SOURCES.get(stage, {}).get(precision)
    if not src:
        return None
    with open(os.path.join(ROOT, "paper_1109_0778_b300", "csrc", src), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def stored_traffic(stage: str, precision: str, workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current source."""
    path = os.path.join(ROOT, "profiles", f"{stage}_{precision}_{workload}.txt")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"^traffic_bytes_per_launch:\s*([0-9.eE+]+)", text, re.M)
    s = re.search(r"^source_sha256_16:\s*([0-9a-f]+)", text, re.M)
    if not m or not s or s.group(1) != kernel_source_sha(stage, precision):
        return None
    return float(m.group(1))


# ----------------------------------------------------------------------------- CPU oracle timing

def oracle_sample_rate(w, target_s: float, X=None):
    """Lloyd iterations/s of the FP64 oracle on the host cores, extrapolated linearly in n from a
    bounded row sample (full centroid set)."""
    import oracle

    orc = oracle.oracle()
    cores = orc.set_threads(0)
    rows = min(w.n, 1 << 18)
    if X is None:
        X, C0 = synth.workload_data(w, rows=max(rows, w.k))
        X = X[:rows]
    else:
        X, C0 = X[:rows], X[: w.k].copy()
    C = C0.astype(np.float64)
    t0 = time.perf_counter()
    orc.step(X[: min(rows, 4096)], C)  # calibrate on a few rows
    t_small = time.perf_counter() - t0
    per_row = max(t_small / min(rows, 4096), 1e-9)
    rows = int(min(rows, max(4096, target_s / per_row)))
    Xs = np.ascontiguousarray(X[:rows])
    steps, t0 = 0, time.perf_counter()
    while True:
        orc.step(Xs, C)
        steps += 1
        el = time.perf_counter() - t0
        if el >= target_s or steps >= 50:
            break
    rate = steps / el * rows / w.n
    return rate, cores, (f"{steps} oracle Lloyd steps on the first {rows} of {w.n} points with the full "
                         f"k={w.k} centroid set, {el:.1f} s; iter/s extrapolated linearly in n")


# ----------------------------------------------------------------------------- arms

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    import oracle

    orc = oracle.oracle()
    cores = orc.set_threads(0)
    rows = min(w.n, 1 << 16)
    X, C0 = synth.workload_data(w, rows=max(rows, w.k))
    Xs = np.ascontiguousarray(X[:rows])
    C = C0.astype(np.float64)
    for _ in range(args.warmup):
        orc.step(Xs, C)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(Xs, C)
    el = time.perf_counter() - t0
    value = args.steps * rows / w.n / el
    sample = (f"each step: one oracle Lloyd step on the first {rows} of {w.n} points with the full k={w.k} "
              f"centroid set; iter/s extrapolated linearly in n")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(w, "f64-oracle"), step=sample),
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(w, precision):
    return {"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "iters_per_step": w.iters, "precision": precision,
            "mixture": {"m": w.m, "R": w.R, "sigma": w.sigma, "seed": hex(w.seed)}, "init": "first k points",
            "l2": f"inputs larger than L2 (X = {w.n * w.d * 4 / 1e6:.0f} MB > 126 MB)",
            "step": f"one kmeans_run call = {w.iters} graph-captured Lloyd iterations"}


def batched_problems(torch, dev, w, limit=0):
    """Device tensors of the batched workload's instances (seeded mixtures, C0 = first k points)."""
    from synth import batched_instances

    inst = batched_instances(w)
    if limit:
        inst = inst[:limit]
    probs, flops, xbytes = [], 0.0, 0
    # every instance's C is a view of one flat buffer, so a step resets all of them with one copy
    kd = [iw.k * iw.d for iw in inst]
    c_flat = torch.empty(sum(kd), dtype=torch.float32, device=dev)
    c0_flat = torch.empty_like(c_flat)
    at = 0
    for iw, m in zip(inst, kd):
        X = synth.mixture(iw.seed, iw.n, iw.d, iw.m, iw.R, iw.sigma)
        Xd = torch.from_numpy(X).to(dev)
        c0_flat[at:at + m].copy_(torch.from_numpy(X[: iw.k].reshape(-1)))
        probs.append((Xd, c_flat[at:at + m].view(iw.k, iw.d)))
        at += m
        flops += 2.0 * iw.n * iw.k * iw.d
        xbytes += 4 * iw.n * iw.d
    c_flat.copy_(c0_flat)
    return inst, probs, flops, xbytes, (c_flat, c0_flat)


def run_batched(args, torch, dev, dist, rank, world, local, emit=True):
    from paper_1109_0778_b300 import kmeans as km

    w = WORKLOADS["batched_512"]
    prec = args.precision or w.precision[0]
    inst, probs, flops_iter, xbytes, (c_flat, c0_flat) = batched_problems(torch, dev, w, args.instances)
    work = []
    for Xd, C in probs:
        a, s, c = km.alloc_outputs(Xd, C)
        work.append((Xd, C, a, s, c))
    batch = km.Batch(work)  # checked and marshalled once; the tensors' contents change per step
    stream = torch.cuda.current_stream(dev)

    def one_step():
        c_flat.copy_(c0_flat)
        return batch.run(w.iters, precision=prec, stream=stream, profile=True)

    for _ in range(max(args.warmup, 0)):
        one_step()
    torch.cuda.synchronize(dev)
    barrier(dist)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    call_ms = 0.0
    launches_tot = 0
    stage_tot = {k: 0.0 for k in ("xnorm",) + STAGE_KERNELS}
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            st = one_step()
            call_ms += float(st["ms"][0])
            for si, kname in enumerate(km.STAGES):
                stage_tot[kname] += float(st["stage_ms"][0][si])
            flagged = (int(st["n_flagged"].sum()), int(st["n_full"].sum()))
            shape = int(st["batch_shape"][0])
            launches_tot += int(st["launches"][0])
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    clocks = clk.summary()
    t = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, dev)
    value = aggregate_rate(args.steps * w.iters, world, t)
    peaks, peak_src = measured_peaks()
    ms_iter = call_ms / args.steps / w.iters
    achieved = xbytes / (ms_iter / 1e3) / 1e9
    if rank == 0:
        ns = [iw.n for iw in inst]
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": w.name, "instances": len(inst), "total_points": int(sum(ns)),
                       "iters_per_step": w.iters, "precision": prec,
                       "step": f"one kmeans_run_batched call = {w.iters} graph-captured Lloyd iterations of all "
                               f"{len(inst)} instances; value counts iterations of the whole batch",
                       "l2": f"inputs larger than L2 (X = {xbytes / 1e9:.2f} GB)",
                       "autotuned_shape": {"chunk_width": shape % 1000, "instance_order": ["as given", "by work"][
                           (shape // 1000) % 10], "row_order": ["order of X", "cluster-sorted for multi-chunk k"][shape // 10000]}},
            "distance_tflops": value * flops_iter / 1e12,
            "stage_ms_per_iter": {k: v / args.steps / w.iters for k, v in stage_tot.items()},
            "flagged_last_iter": {"flagged": flagged[0], "full_recheck": flagged[1],
                                  "note": "summed over instances, each at its last iteration"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "kernel": "whole batched step",
                         "note": "algorithmic bytes = one FP32 read of every X per iteration", "traffic": None},
            "gpu_launches": launches_tot,
            "clocks": clocks, "e2e": None, "cpu_baseline": None, "peaks_source": peak_src,
        }
        if not emit:
            return {k: line[k] for k in ("value", "unit", "ms_per_step", "config", "distance_tflops",
                                          "stage_ms_per_iter", "flagged_last_iter", "roofline", "gpu_launches",
                                          "clocks")} | {"ms_per_iter": ms_iter, "steps": args.steps}
        print(json.dumps(line), flush=True)
    return 0


# Keyed-reduce training workloads (GDA: labelled Gaussian mixture; NB: Poisson feature counts).
TRAIN_WORKLOADS = {
    "gda_n1M_d64_c16": {"kind": "gda", "n": 1 << 20, "d": 64, "ncls": 16, "seed": 0x5EED0100},
    "nb_n1M_d256_c20": {"kind": "nb", "n": 1 << 20, "d": 256, "ncls": 20, "seed": 0x5EED0101},
}


def training_data(tw):
    if tw["kind"] == "gda":
        X, y = synth.mixture(tw["seed"], tw["n"], tw["d"], tw["ncls"], 6.0, 1.5, with_comp=True)
        return X, y.astype(np.int32)
    rng = np.random.default_rng(tw["seed"])
    y = rng.integers(0, tw["ncls"], tw["n"]).astype(np.int32)
    X = rng.poisson(rng.uniform(0.2, 3.0, (tw["ncls"], tw["d"]))[y]).astype(np.float32)
    return X, y


def run_training(args, torch, dev, dist, rank, world, local):
    """One step = one training call (kmeans_gda_train / kmeans_nb_train) on HBM-resident inputs."""
    from paper_1109_0778_b300 import kmeans as km

    tw = TRAIN_WORKLOADS[args.workload]
    X, y = training_data(tw)
    n, d, ncls = tw["n"], tw["d"], tw["ncls"]
    Xd, yd = torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev)
    stream = torch.cuda.current_stream(dev)
    train = km.gda_train if tw["kind"] == "gda" else km.nb_train
    for _ in range(max(args.warmup, 0)):
        train(Xd, yd, ncls, stream=stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            train(Xd, yd, ncls, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    t = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, dev)
    value = aggregate_rate(args.steps, world, t)
    peaks, peak_src = measured_peaks()
    # algorithmic bytes: X once for the class sums (+ once more for the covariance), labels twice
    passes = 2 if tw["kind"] == "gda" else 1
    algo = passes * 4.0 * n * d + 8.0 * n
    achieved = algo / (t / args.steps) / 1e9
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        orc = oracle.oracle()
        cores = orc.set_threads(0)
        rows = 1 << 16
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < min(args.cpu_seconds, 10.0) or reps == 0:
            (orc.gda if tw["kind"] == "gda" else orc.nb)(X[:rows], y[:rows], ncls)
            reps += 1
        el = time.perf_counter() - t0
        cpu = {"value": reps * rows / n / el, "unit": "trainings/s", "cores": cores, "kind": "oracle",
               "sample": f"{reps} oracle trainings on the first {rows} of {n} rows, {el:.1f} s; "
                         f"trainings/s extrapolated linearly in n"}
    if rank == 0:
        line = {
            "metric": f"{tw['kind'].upper()} trainings/s (keyed reduce by class)", "value": value,
            "unit": "trainings/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "d": d, "ncls": ncls, "seed": hex(tw["seed"]),
                       "l2": f"inputs larger than L2 (X = {4 * n * d / 1e6:.0f} MB)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "kernel": "whole training call",
                         "note": f"algorithmic bytes = {passes} FP32 read(s) of X + labels", "traffic": None},
            # per call: label check, count, scan, scatter, segmented sum (+ means, covariance tiles and
            # their reduction for GDA; the smoothed distributions for NB)
            "gpu_launches": args.steps * (8 if tw["kind"] == "gda" else 6),
            "clocks": clk.summary(), "e2e": None, "cpu_baseline": cpu, "peaks_source": peak_src,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_spade(args, torch, dev, dist, rank, world, local):
    """One step = one kmeans_spade_densities call (policy last: the generated code's bulk update)
    on an HBM-resident X. Roofline: the tile passes are FP32 ALU work, one subtract and one add of
    the absolute value per (row, row, column) element; the algorithmic elements of a pass are
    n_evaluated x n x d (the rows the loop evaluates), timed by the library's CUDA events around
    each tile pass."""
    from paper_1109_0778_b300 import kmeans as km

    sw = SPADE_WORKLOADS[args.workload]
    X = synth.spade_data(sw)
    n, d = X.shape
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 0)):
        km.spade_densities(Xd, sw.apprx, sw.kernel, stream=stream)
    torch.cuda.synchronize(dev)
    barrier(dist)
    # X (15 MB) fits in L2: every step starts from a flushed L2 (a 256 MB write outside the timed spans)
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    pairs_ms, stats = 0.0, None
    with ClockSampler(local) as clk:
        for e0, e1 in evs:
            flush.fill_(1.0)
            e0.record(stream)
            _, _, _, stats = km.spade_densities(Xd, sw.apprx, sw.kernel, stream=stream)
            e1.record(stream)
            pairs_ms += stats["ms_pairs"]
        torch.cuda.synchronize(dev)
        barrier(dist)
    clocks = clk.summary()
    t = max_over_ranks(dist, sum(e0.elapsed_time(e1) for e0, e1 in evs) / 1e3, dev)
    value = aggregate_rate(args.steps, world, t)
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = peaks.get("sm_max_mhz", 2032.0)
    peak = sms * 128 * mhz * 1e6 / 2 / 1e12  # element-pairs/s: 2 FP32 lane ops each
    algo = float(stats["n_evaluated"]) * n * d
    issued = float(stats["n_computed"]) * n * d
    achieved = algo / (pairs_ms / args.steps / 1e3) / 1e12
    batches = stats["batches"]
    launched = ((batches + 1 + 3) // 4) * 4  # batches run in groups of four until one finds no candidate
    launches = args.steps * (6 * launched + 2)

    # e2e: the same call with X copied in from pinned host memory and the densities read back
    Xh = torch.from_numpy(X).pin_memory()
    dens_h = torch.empty(n, dtype=torch.int32).pin_memory()
    Xe = torch.empty_like(Xd)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        Xe.copy_(Xh, non_blocking=True)
        dens, _, _, _ = km.spade_densities(Xe, sw.apprx, sw.kernel, stream=stream)
        dens_h.copy_(dens, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    te = max_over_ranks(dist, e0.elapsed_time(e1) / 1e3, dev)
    e2e = {"value": aggregate_rate(args.steps, world, te), "unit": "pass/s", "h2d_bytes_per_step": 4 * n * d,
           "d2h_bytes_per_step": 4 * n}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        orc = oracle.oracle()
        cores = orc.set_threads(0)
        rows = n // 2
        t0 = time.perf_counter()
        _, _, proc = orc.spade(X[:rows], sw.apprx, sw.kernel, 0)
        el = time.perf_counter() - t0
        rate = float(proc.sum()) * rows * d / el  # oracle element-pairs/s on the sample
        cpu = {"value": rate / algo, "unit": "pass/s", "cores": cores, "kind": "oracle",
               "sample": f"the oracle's loop on the first {rows} of {n} rows ({int(proc.sum())} evaluated), "
                         f"{el:.1f} s; pass/s = its element-pair rate over the full pass's {algo:.3g} elements"}
    if rank == 0:
        line = {
            "metric": "SPADE downsampling passes/s (fused L1 find + count, Sec. 4.1)", "value": value,
            "unit": "pass/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": sw.name, "n": n, "d": d, "mixture": {"m": sw.m, "R": sw.R, "sigma": sw.sigma,
                                                                         "seed": hex(sw.seed)},
                       "apprx_width": sw.apprx, "kernel_width": sw.kernel, "policy": "last",
                       "l2": f"L2 flushed before every step (256 MB write outside the timed spans); X = {4 * n * d / 1e6:.0f} MB"},
            "stats_last_step": stats,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Telem/s",
                         "frac": achieved / peak, "kernel": "spade_pairs (tile passes)",
                         "peak_source": f"{sms} SMs x 128 lanes x {mhz:.0f} MHz / 2 FP32 ops per element",
                         "issued_frac": (issued / (pairs_ms / args.steps / 1e3) / 1e12) / peak,
                         "note": "algorithmic elements = evaluated rows x n x d; issued adds speculative rows",
                         "traffic": stored_traffic("spade_pairs", "f32", sw.name)},
            "gpu_launches": launches, "clocks": clocks, "e2e": e2e, "cpu_baseline": cpu, "peaks_source": peak_src,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def single_problem(torch, dev, w, pinned=True):
    """Host (pinned) and device copies of a single-instance workload: X, C0."""
    if pinned:
        Xh = torch.empty((w.n, w.d), dtype=torch.float32, pin_memory=True)
        synth.mixture(w.seed, w.n, w.d, w.m, w.R, w.sigma, out=Xh.numpy())
    else:
        Xh = torch.from_numpy(synth.mixture(w.seed, w.n, w.d, w.m, w.R, w.sigma))
    C0h = Xh[: w.k].clone()
    if pinned:
        C0h = C0h.pin_memory()
    return Xh, C0h, Xh.to(dev), C0h.to(dev)


def time_runs(torch, km, dev, local, dist, Xd, C0d, w, prec, steps, warmup, profile=True):
    """Device-timed kmeans_run calls (each = w.iters graph-captured Lloyd iterations from C0).

    ``warmup`` untimed calls, then ``steps`` calls between two CUDA events on the launching
    stream, bracketed by a synchronize (and a barrier under torchrun); clocks sampled meanwhile.
    Returns the slowest rank's time, per-stage device times (CUDA events recorded between the
    stages inside the captured graph) and the last call's statistics."""
    stream = torch.cuda.current_stream(dev)
    Cd = C0d.clone()
    a, s, c = km.alloc_outputs(Xd, Cd)

    def one():
        Cd.copy_(C0d)
        return km.run(Xd, Cd, w.iters, assign=a, sums=s, counts=c, precision=prec, profile=profile, stream=stream)

    for _ in range(max(warmup, 0)):
        one()
    torch.cuda.synchronize(dev)
    barrier(dist)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage_tot = {k: 0.0 for k in ("xnorm",) + STAGE_KERNELS}
    launches = 0
    call_ms = 0.0
    out = None
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        barrier(dist)
        ev0.record(stream)
        for _ in range(steps):
            out = one()
            for kname, v in out.stats["stage_ms"].items():
                stage_tot[kname] += v
            launches += out.stats["launches"]
            call_ms += out.stats["ms"]
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    t = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, dev)
    st = out.stats
    return {"t": t, "iter_s": steps * w.iters / t, "ms_per_step": t * 1e3 / steps,
            "stage_ms_per_iter": {k: v / steps / w.iters for k, v in stage_tot.items()},
            "assign_ms": stage_tot["assign"] / (steps * w.iters), "launches": launches, "clocks": clk.summary(),
            "call_ms_per_iter": call_ms / (steps * w.iters),
            "last": {"objective": st["objective"], "n_flagged": st["n_flagged"], "n_full": st["n_full"],
                     "n_queued": st["n_queued"], "iters_bf16": st["iters_bf16"], "n_empty": st["n_empty"]}}


def time_e2e(torch, km, dist, dev, Xh, C0h, w, prec, reps):
    """The same runs through kmeans_run_host from pinned host buffers: the copy of X and C in and
    of C, assign, sums and counts out are inside the timed region."""
    Ch = C0h.clone().pin_memory()
    ah = torch.empty(w.n, dtype=torch.int32, pin_memory=True)
    sh = torch.empty((w.k, w.d), dtype=torch.float32, pin_memory=True)
    ch = torch.empty(w.k, dtype=torch.int32, pin_memory=True)
    km.run_host(Xh, Ch, w.iters, 0.0, ah, sh, ch, precision=prec)  # warm-up (staging buffers, graph)
    barrier(dist)
    t0 = time.perf_counter()
    for _ in range(reps):
        Ch.copy_(C0h)
        km.run_host(Xh, Ch, w.iters, 0.0, ah, sh, ch, precision=prec)
    te = max_over_ranks(dist, time.perf_counter() - t0, dev)
    _, world, _ = dist_env()
    return {"value": aggregate_rate(reps * w.iters, world, te), "unit": "iter/s",
            "h2d_bytes_per_step": 4 * w.n * w.d + 4 * w.k * w.d,
            "d2h_bytes_per_step": 4 * w.k * w.d * 2 + 4 * w.n + 4 * w.k, "reps": reps,
            "api": "kmeans_run_host (pinned host buffers)"}


def measure_peaks(torch, km, dev):
    """FP32 SIMT and FP8 tensor peaks measured on this GPU now (best of several, CUDA events).

    FFMA: the library's probe kernel (independent FMA chains, 8 CTAs x 256 threads per SM,
    scalar FFMA and packed FFMA2; the faster counts). FP8: torch._scaled_mm (cuBLASLt) E4M3 x
    E4M3 -> BF16 on 8192^3 with unit scales, 2 x 8192^3 flop."""
    res = {}
    for packed in (False, True):
        km.probe_ffma(1 << 12, packed=packed)
        best = 0.0
        for _ in range(3):
            fl, ms = km.probe_ffma(1 << 16, packed=packed)
            best = max(best, fl / (ms / 1e3) / 1e12)
        res["ffma2_tflops" if packed else "ffma_tflops"] = best
    res["fp32_simt_tflops"] = max(res["ffma_tflops"], res["ffma2_tflops"])
    try:
        N = 8192
        g = torch.Generator(device=dev).manual_seed(0)
        a = torch.randn(N, N, device=dev, generator=g).to(torch.float8_e4m3fn)
        b = torch.randn(N, N, device=dev, generator=g).to(torch.float8_e4m3fn).t()
        one = torch.tensor(1.0, device=dev)
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        best = 0.0
        for _ in range(10):
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize(dev)
            best = max(best, 2.0 * N ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12)
        res["fp8_tflops"] = best
        del a, b
    except Exception as exc:  # noqa: BLE001 -- reported, the nominal ratio then stands in
        res["fp8_tflops"] = None
        res["fp8_error"] = f"{type(exc).__name__}: {exc}"[:200]
    res["how"] = ("FFMA: kmeans_probe_ffma, 2 x FMAs / CUDA-event time of one launch, best of 3, max of scalar "
                  "and packed; FP8: torch._scaled_mm E4M3 8192^3 -> BF16, best of 10 after 3 warm-ups")
    torch.cuda.empty_cache()
    return res


def tensor_peak(prec, peaks, live, burst):
    """(peak TFLOP/s, source) of the tensor-core arithmetic a precision runs on."""
    key = "bf16_tflops" if burst else "bf16_tflops_sustained"
    if prec == "fp8":
        if live and live.get("fp8_tflops"):
            if burst:
                return live["fp8_tflops"], "FP8 E4M3 measured now (torch._scaled_mm 8192^3, burst)"
            ratio = peaks["bf16_tflops_sustained"] / peaks["bf16_tflops"]
            return live["fp8_tflops"] * ratio, "FP8 measured now x (BF16 sustained / burst)"
        return 2.0 * peaks[key], f"2 x BF16 {'burst' if burst else 'sustained'} (nominal FP8/BF16 ratio)"
    return peaks[key], f"BF16 {'burst' if burst else 'sustained'} ({'MEASURED_PEAKS.json'})"


def assign_roofline(prec, w, r, peaks, peak_src, live, sms):
    """Roofline of the dominant kernel (the fused assignment): 2nkd algorithmic flop per launch
    (3 x for the two-part BF16 products) over the launch's mean CUDA-event time. A timed region
    under 1.5 s is compared with the burst peak, a longer one with the sustained peak."""
    burst = r["t"] < 1.5
    products = 3 if prec == "bf16x3" else 1
    achieved = products * w.flops_per_iter / (r["assign_ms"] / 1e3) / 1e12
    if prec == "fp32":
        if live and live.get("fp32_simt_tflops"):
            peak, src = live["fp32_simt_tflops"], "FP32 FFMA measured now (kmeans_probe_ffma)"
        else:
            peak = fp32_simt_peak_tflops(sms, peaks.get("sm_max_mhz", 2032.0))
            src = f"nominal FFMA: {sms} SMs x 128 lanes x 2 flop x {peaks.get('sm_max_mhz', 2032.0):.0f} MHz"
        bound, kern = "alu", "assign_simt (FP32 FFMA)"
    else:
        peak, src = tensor_peak(prec, peaks, live, burst)
        bound, kern = "tensor", f"assign_tc ({prec})"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"{src}; {peak_src}", "peak_kind": "burst" if burst else "sustained",
            "kernel": kern, "launch_ms": r["assign_ms"],
            "algorithmic": f"{products} x 2 n k d = {products * w.flops_per_iter:.4g} flop per launch",
            "traffic": stored_traffic("assign", prec, w.name)}


def arm_summary(prec, w, r, roof, e2e=None):
    d = {"iter_s": r["iter_s"], "ms_per_step": r["ms_per_step"], "distance_tflops": r["iter_s"] * w.flops_per_iter / 1e12,
         "assign_ms_per_iter": r["assign_ms"], "roofline": roof, "stage_ms_per_iter": r["stage_ms_per_iter"],
         "last_iter": r["last"], "clocks": r["clocks"], "gpu_launches": r["launches"], "e2e": e2e}
    if prec == "fp8":
        d["arithmetic"] = (f"{r['last']['iters_bf16']} of {w.iters} steps per call with BF16 codes (cold start), "
                           f"the rest E4M3; queued points re-scored with BF16 codes "
                           f"({r['last']['n_queued']} in the last step)")
    return d


def run_large(torch, km, dev, local, args, peaks, peak_src, live, sms):
    """8M x 256 x 8192 E4M3 + re-check, 10 iterations per call (the largest single-GPU workload)."""
    w = WORKLOADS["large_n8M_d256_k8192"]
    _, _, Xd, C0d = single_problem(torch, dev, w, pinned=False)
    reps = max(5, min(args.steps, 8))
    r = time_runs(torch, km, dev, local, None, Xd, C0d, w, "fp8", reps, 1)
    roof = assign_roofline("fp8", w, r, peaks, peak_src, live, sms)
    out = arm_summary("fp8", w, r, roof)
    out.update({"workload": w.name, "n": w.n, "d": w.d, "k": w.k, "iters_per_step": w.iters, "steps": reps,
                "near_ties": {"flagged_last_iter": r["last"]["n_flagged"], "full_recheck_last_iter": r["last"]["n_full"],
                              "note": "points whose low-precision top-2 margin fell under the rigorous bound and "
                                      "were re-checked in FP32 (the library's near-tie set)"}})
    del Xd, C0d
    torch.cuda.empty_cache()
    return out


def run_plain(torch, km, dev, local, args):
    """10,000 x 16 x 8 FP32, 10 iterations per call: microseconds per iteration, from the events
    around the calls (host work of each call included) and from the library's own events around
    each call's device work. The library runs such small FP32 problems as one cooperative kernel
    per call; the staged path (one launch per stage, graph-captured) is timed beside it."""
    w = WORKLOADS["plain_n10k_d16_k8"]
    _, _, Xd, C0d = single_problem(torch, dev, w, pinned=False)
    reps = max(400, args.steps)  # ~0.1 s of calls, so one slow call does not set the mean
    r = time_runs(torch, km, dev, local, None, Xd, C0d, w, "fp32", reps, 3, profile=False)
    rs = time_runs(torch, km, dev, local, None, Xd, C0d, w, "fp32", reps, 3, profile=True)
    return {"workload": w.name, "us_per_iter": 1e6 / r["iter_s"], "iter_s": r["iter_s"], "steps": reps,
            "device_us_per_iter": 1e3 * r["call_ms_per_iter"],
            "kernel_launches_per_call": r["launches"] // reps,
            "staged_path": {"us_per_iter": 1e6 / rs["iter_s"], "device_us_per_iter": 1e3 * rs["call_ms_per_iter"],
                            "kernel_launches_per_call": rs["launches"] // reps,
                            "note": "the same call with opts.profile (per-stage events force the staged path)"},
            "note": "one kmeans_run call = one cooperative kernel for all 10 iterations; us_per_iter includes "
                    "each call's host work (argument checks, copies of the statistics, a synchronize)",
            "clocks": r["clocks"]}


def run_sharded(args, torch, dev, dist, rank, world, local):
    """The single-instance workload as one problem sharded over the ranks (strong scaling)."""
    from paper_1109_0778_b300 import kmeans as km
    from paper_1109_0778_b300.sharded import ShardedLloyd, shard_bounds

    w = WORKLOADS[args.workload]
    prec = args.precision or HEADLINE_PRECISION.get(w.name, w.precision[0])
    lo, hi = shard_bounds(w.n, rank, world)
    Xh = torch.empty((hi - lo, w.d), dtype=torch.float32, pin_memory=True)
    synth.mixture(w.seed, hi - lo, w.d, w.m, w.R, w.sigma, row0=lo, out=Xh.numpy())
    C0h = torch.from_numpy(synth.mixture(w.seed, w.k, w.d, w.m, w.R, w.sigma))  # the first k points of the data set
    Xd, C0d = Xh.to(dev), C0h.to(dev)
    Cd = C0d.clone()
    stream = torch.cuda.current_stream(dev)

    def one_run(Xsrc=None):
        Cd.copy_(C0d)
        sl = ShardedLloyd(Xd, Cd, precision=prec, stream=stream)
        if Xsrc is not None:
            Xd.copy_(Xsrc, non_blocking=True)
        st = sl.run(w.iters)
        return sl, st

    # kernels per Lloyd step of this shard: the kernel nodes of a captured kmeans_run graph of the
    # same shard (one per-call point pass + iters steps); a sharded step launches the same stages
    # (the partials finish in place of the divide) plus the two kernels of kmeans_apply_partials
    probe = km.run(Xd, C0d.clone(), w.iters, precision=prec)
    per_step = (probe.stats["launches"] - 1) // w.iters
    launches_per_run = 1 + w.iters * (per_step + 2)
    for _ in range(max(args.warmup, 0)):
        one_run()
    torch.cuda.synchronize(dev)
    barrier(dist)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize(dev)
        barrier(dist)
        ev0.record(stream)
        for _ in range(args.steps):
            _, st = one_run()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier(dist)
    t = max_over_ranks(dist, ev0.elapsed_time(ev1) / 1e3, dev)
    value = args.steps * w.iters / t
    # end to end: every step copies the shard in from pinned host memory and reads C and the labels back
    e2e = None
    if not args.no_e2e:
        ah = torch.empty(hi - lo, dtype=torch.int32, pin_memory=True)
        Ch = torch.empty((w.k, w.d), dtype=torch.float32, pin_memory=True)
        barrier(dist)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sl, _ = one_run(Xh)
            ah.copy_(sl.assign)
            Ch.copy_(Cd)
        te = max_over_ranks(dist, time.perf_counter() - t0, dev)
        e2e = {"value": args.steps * w.iters / te, "unit": "iter/s", "h2d_bytes_per_step": 4 * (hi - lo) * w.d,
               "d2h_bytes_per_step": 4 * (hi - lo) + 4 * w.k * w.d,
               "api": "ShardedLloyd over kmeans_step_partial / kmeans_apply_partials, per rank"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": DTYPE_NAMES.get(prec, prec), "data": "synthetic",
            "config": dict(workload_config(w, prec), parallelism=f"points sharded over {world} GPUs; one NCCL "
                                                                 f"all-reduce of k*d + k + 2 FP64 partials per iteration"),
            "distance_tflops": value * w.flops_per_iter / 1e12,
            "last_iter": {"objective": st["objective"], "n_changed": st["n_changed"],
                          "n_flagged_rank0": st["n_flagged_shard"]},
            "clocks": clk.summary(), "e2e": e2e,
            "gpu_launches": args.steps * launches_per_run, "cpu_baseline": None, "peaks_source": measured_peaks()[1],
            "note": "each iteration: kmeans_step_partial + all-reduce + kmeans_apply_partials (host-sequenced)",
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = dist_init(world, "nccl")
    from paper_1109_0778_b300 import kmeans as km

    if args.workload in TRAIN_WORKLOADS:
        return run_training(args, torch, dev, dist, rank, world, local)
    if args.workload in SPADE_WORKLOADS:
        return run_spade(args, torch, dev, dist, rank, world, local)
    if args.workload == "batched_512":
        return run_batched(args, torch, dev, dist, rank, world, local)
    if world > 1:
        return run_sharded(args, torch, dev, dist, rank, world, local)
    w = WORKLOADS[args.workload]
    if args.rows:
        import dataclasses

        w = dataclasses.replace(w, n=min(w.n, args.rows), name=f"{w.name}[:{min(w.n, args.rows)}]")
    prec = args.precision or HEADLINE_PRECISION.get(w.name, w.precision[0])
    full = rank == 0 and world == 1 and not args.no_variants and w.name == DEFAULT_WORKLOAD
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    live = measure_peaks(torch, km, dev) if full else None

    Xh, C0h, Xd, C0d = single_problem(torch, dev, w)
    r = time_runs(torch, km, dev, local, dist, Xd, C0d, w, prec, args.steps, args.warmup)
    value = aggregate_rate(args.steps * w.iters, world, r["t"])
    roof = assign_roofline(prec, w, r, peaks, peak_src, live, sms)
    e2e = None if args.no_e2e else time_e2e(torch, km, dist, dev, Xh, C0h, w, prec, args.steps)

    arms = None
    if full:  # the metric's comparison on the same data: FP32, E4M3 and two-part BF16, each + re-check
        arms = {}
        reps = max(5, min(args.steps, 10))
        for p2 in ("fp32", "fp8", "bf16x3"):
            ra = time_runs(torch, km, dev, local, None, Xd, C0d, w, p2, reps, 1)
            e2 = None if (args.no_e2e or p2 == "bf16x3") else time_e2e(torch, km, None, dev, Xh, C0h, w, p2,
                                                                       min(reps, 5))
            arms[p2] = arm_summary(p2, w, ra, assign_roofline(p2, w, ra, peaks, peak_src, live, sms), e2)
            arms[p2]["steps"] = reps
        for p2 in ("bf16", "fp8", "bf16x3"):
            base = arms["fp32"]["iter_s"]
            if p2 == "bf16":
                arms.setdefault("speedup_vs_fp32", {})["bf16"] = value / base
            else:
                arms["speedup_vs_fp32"][p2] = arms[p2]["iter_s"] / base
    del Xd, C0d
    torch.cuda.empty_cache()

    others = None
    if full:
        others = {"large_n8M_d256_k8192": run_large(torch, km, dev, local, args, peaks, peak_src, live, sms)}
        bargs = argparse.Namespace(**vars(args))
        bargs.steps, bargs.warmup, bargs.precision, bargs.instances = max(5, min(args.steps, 10)), 2, None, 0
        others["batched_512"] = run_batched(bargs, torch, dev, None, 0, 1, local, emit=False)
        others["plain_n10k_d16_k8"] = run_plain(torch, km, dev, local, args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample_rate(w, args.cpu_seconds, X=Xh.numpy())
        cpu = {"value": rate, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["t"] * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAMES.get(prec, prec),
            "data": "synthetic", "config": workload_config(w, prec),
            "distance_tflops": value * w.flops_per_iter / 1e12,
            "roofline": roof, "stage_ms_per_iter": r["stage_ms_per_iter"], "last_iter": r["last"],
            "clocks": r["clocks"], "e2e": e2e, "gpu_launches": r["launches"],
            "precision_arms": arms, "other_configs": others, "peaks_live": live,
            "cpu_baseline": cpu, "peaks_source": peak_src,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
