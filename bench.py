#!/usr/bin/env python
"""Benchmark: chi2 + gradient bin-evaluations per second on one GB300.

Workload (the gradient configuration): 32 detector histograms x 131072 bins
of 0.09765625 ns (12.8 us), theory = exponentially damped line +
Gaussian-damped line (B1 + dB) + static Gaussian Kubo-Toyabe, 104 parameters
(72 free), Poisson counts.  One step is one evaluation of chi2 and its
gradient over every bin (objective kernel in adjoint mode) for a fresh
parameter vector.  The steps cycle through 16 independent runs of the
workload (268 MB of counts, larger than L2) so every step reads its counts
from HBM; they are launched back to back between two CUDA events.  The same
evaluation timed one launch at a time with L2 flushed before each is reported
beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs an independent replica (the path has no
exchange step); value = all ranks' bin-evaluations / max-over-ranks time.
Prints one JSON line on rank 0 (details of the extra measurements go to
stderr as one JSON line before it).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "chi2+grad bin-evals/s"
UNIT = "bin-evals/s"
WORKLOAD = "32 hist x 131072 bins, 2 lines + static GKT, 104 params (72 free), chi2 + gradient"

# Algorithmic work per bin of chi2 + gradient for this theory (the scope
# table's count, independent of how the kernel schedules it): the model needs
# 4 exponentials (lifetime, two line envelopes, Kubo-Toyabe), 2 cosines and,
# for the chi2 weight, 1 reciprocal on the SFU, and ~25 FMA; the adjoint adds
# ~10 partials x ~3 FMA; the counts are read once (4 B, FP32).
ALG_FP32_FLOP_PER_BIN = 2 * (25 + 30)
ALG_SFU_PER_BIN = {"ex2": 4, "cos": 2, "rcp": 1}
ALG_BYTES_PER_BIN = 4
# FP32 FLOPs per bin the kernel executes for the same work (ncu instruction
# counts of the batched adjoint kernel over 67,108,864 bins, where per-launch
# costs vanish; FMA = 2); reported beside the algorithmic count
EXEC_FP32_FLOP_PER_BIN = 83.5
# DRAM bytes (read + write) of one eval_kernel<1,1,0,1,kGrad> launch of this
# workload from an ncu capture of the current kernel (16,926,720 B read, 0
# written; algorithmic 16,777,216 B)
TRAFFIC_BYTES_GRAD_LAUNCH = 16926720
# FP32-pipe FLOPs per bin-evaluation the value-only batched kernel executes on
# the 64-run workload (batch_kernel<1,1,0,1>, ncu instruction counts over
# 2,720,958,581 bin-evaluations)
FLOPS_PER_BINEVAL_VALUE_BATCH = 57.1
# algorithmic work per bin-evaluation of the value-only objective: the model's
# SFU operations and FMAs, no partials
ALG_FP32_FLOP_PER_BINEVAL_VALUE = 2 * 25
HBM_FALLBACK_GBS = 6800.0


def measured_peaks():
    """Denominators of the roofline: the device's measured pipe rates (library
    probe) and the measured HBM copy bandwidth of the GB300s."""
    from paper_1604_02334_gb300 import pipe_rates
    r = pipe_rates()
    hbm, src = HBM_FALLBACK_GBS, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm, src = float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        pass
    fp32 = 2.0 * max(r["ffma"], r["ffma2"])
    return {"rates": r, "fp32_flops": fp32, "hbm_bytes": hbm * 1e9, "hbm_src": src}


def roofline(bins, seconds, peaks, flop_per_bin, sfu_per_bin, bytes_per_bin, traffic=None, kernel=""):
    """Fractions of the FP32, SFU and HBM rooflines for `bins` bins in
    `seconds` (one launch), by algorithmic counts; the binding one is reported."""
    r = peaks["rates"]
    sfu_s_per_bin = sum(n / r[op] for op, n in sfu_per_bin.items())
    n_sfu = sum(sfu_per_bin.values())
    fr = {"fp32": flop_per_bin * bins / seconds / peaks["fp32_flops"],
          "sfu": sfu_s_per_bin * bins / seconds,
          "hbm": bytes_per_bin * bins / seconds / peaks["hbm_bytes"]}
    pipe = max(fr, key=fr.get)
    if pipe == "fp32":
        a, p, u = flop_per_bin * bins / seconds / 1e12, peaks["fp32_flops"] / 1e12, "TFLOP/s"
    elif pipe == "sfu":
        a, p, u = n_sfu * bins / seconds / 1e12, n_sfu / sfu_s_per_bin / 1e12, "T SFU-op/s"
    else:
        a, p, u = bytes_per_bin * bins / seconds / 1e9, peaks["hbm_bytes"] / 1e9, "GB/s"
    return {"bound": "hbm" if pipe == "hbm" else "alu", "pipe": pipe, "achieved": _r(a), "peak": _r(p),
            "unit": u, "frac": _r(a / p), "traffic": traffic, "fracs": {k: _r(v) for k, v in fr.items()},
            "kernel": kernel}


def _r(x, n=4):
    """Round to n significant digits (keeps the JSON line short)."""
    if x is None or not isinstance(x, float) or x == 0.0 or not math.isfinite(x):
        return x
    return float(f"{x:.{n}g}")


def _short(obj):
    if isinstance(obj, dict):
        return {k: _short(v) for k, v in obj.items()}
    if isinstance(obj, (list, tuple)):
        return [_short(v) for v in obj]
    return _r(obj) if isinstance(obj, float) else obj


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed setup (replicas only)
# --------------------------------------------------------------------------
def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        if torch.cuda.is_available():
            torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over all ranks (every rank gets it); NCCL on GPUs, gloo on CPU."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, seconds_per_rank, world):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / max_over_ranks(seconds_per_rank, world)


# --------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample
# --------------------------------------------------------------------------
SAMPLE_BINS = 8192  # leading bins of each histogram
N_RUNS = 16          # independent runs cycled by the timed steps


def cpu_sample(lay, data):
    offs = np.r_[0, np.cumsum(lay.n_bins)]
    sub = W.multi_detector_layout(lay.n_hist, SAMPLE_BINS, window_us=lay.dt_us * SAMPLE_BINS)
    sub.dt_us = lay.dt_us
    d = np.concatenate([data[offs[k]:offs[k] + SAMPLE_BINS] for k in range(lay.n_hist)])
    return sub, d


def cpu_baseline(lay, data, thetas, seconds=12.0):
    """The FP64 oracle on the host cores, all of them and 8 threads (the
    paper's CPU baseline used 8 threads), on a bounded sample of the workload:
    the median rate of 5 consecutive timing windows."""
    import oracle
    sub, d = cpu_sample(lay, data)
    all_threads = oracle.num_threads()
    k = [0]

    def window(secs):
        n = 0
        t0 = time.perf_counter()
        while True:
            oracle.gradient(sub, d, thetas[k[0] % len(thetas)], oracle.CHI2, with_gn=False)
            k[0] += 1
            n += 1
            el = time.perf_counter() - t0
            if el >= secs and n >= 2:
                return sub.total_bins * n / el, n, el

    def rate(secs):
        w = [window(secs / 5) for _ in range(5)]
        return float(np.median([x[0] for x in w])), sum(x[1] for x in w), sum(x[2] for x in w)

    v, n, el = rate(seconds)
    oracle.set_num_threads(8)
    v8, _, _ = rate(seconds / 3)
    oracle.set_num_threads(all_threads)
    return {"value": v, "unit": UNIT, "cores": all_threads, "kind": "oracle",
            "sample": f"{sub.n_hist} hist x {SAMPLE_BINS} leading bins of the workload, "
                      f"{n} chi2+gradient evaluations in {el:.1f} s, median of 5 windows",
            "value_8_threads": v8}


# --------------------------------------------------------------------------
def make_workload():
    lay, theta, seed = W.config_gradient()
    return lay, theta, seed


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    lay, theta, seed = make_workload()
    # Poisson data drawn from the oracle's own model (reference arm only)
    data = W.poisson_counts(oracle.model(lay, theta), seed)
    sub, d = cpu_sample(lay, data)
    g = W.rng(seed + 11)
    thetas = [W.perturb(theta, lay.free, 0.01, g) for _ in range(args.steps + args.warmup)]
    for i in range(args.warmup):
        oracle.gradient(sub, d, thetas[i], oracle.CHI2, with_gn=False)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.gradient(sub, d, thetas[args.warmup + i], oracle.CHI2, with_gn=False)
    el = time.perf_counter() - t0
    value = sub.total_bins * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_bins_per_step": sub.total_bins},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"{sub.n_hist} hist x {SAMPLE_BINS} leading bins per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_throughput(dev, rank, peaks, reps=5):
    """Value-only bin-evaluations per second of the batched persistent kernel on
    64 uneven runs x (P+1) Jacobian vectors, device-resident (L2 flushed)."""
    import torch
    from paper_1604_02334_gb300 import Batch, Run
    runs = W.config_batched()
    gruns, vecs = [], []
    for br in runs:
        with Run(br.layout) as m:
            mean = m.model(br.theta).astype(np.float64)
        d = W.poisson_counts(mean, br.seed + rank).astype(np.float32)
        gruns.append(Run(br.layout, torch.tensor(d, device=dev)))
        vecs.append(W.jacobian_vectors(br.theta, br.layout.free, 1e-6))
    mv = [v.shape[0] for v in vecs]
    flat = np.concatenate([v.ravel() for v in vecs])
    b = Batch(gruns, mv)
    th = torch.tensor(flat, device=dev)
    out = torch.empty(b.n_values, dtype=torch.float64, device=dev)
    b.eval_device(th, out)  # autotunes on first use
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    ms = []
    for i in range(reps):
        flush.fill_(i & 255)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.eval_device(th, out)
        torch.cuda.synchronize()
        ms.append(1e3 * (time.perf_counter() - t0))
    binevals = sum(br.layout.total_bins * m for br, m in zip(runs, mv))
    med = float(np.median(ms))
    b.close()
    for g in gruns:
        g.close()
    rl = roofline(binevals, med * 1e-3, peaks, ALG_FP32_FLOP_PER_BINEVAL_VALUE, {"ex2": 4, "cos": 2, "rcp": 1},
                  0.0, kernel="batch_kernel<1,1,0,1>")
    rl["exec_fp32_frac"] = _r(FLOPS_PER_BINEVAL_VALUE_BATCH * binevals / (med * 1e-3) / peaks["fp32_flops"])
    return {"workload": "64 runs, K~U{1..32} x M~U[2^14,2^17] bins, P+1 vectors each",
            "bins": int(sum(br.layout.total_bins for br in runs)), "bin_evals": int(binevals),
            "ms": med, "value": binevals / (med * 1e-3), "unit": "bin-evals/s (chi2, value only)",
            "roofline": rl, "note": "host-timed (includes the launch), L2 flushed before each"}


def _device_rate(run, theta, obj, mode, reps=50):
    """Device-entry evaluations replayed from a captured CUDA graph of `reps`
    launches (no host dispatch between them; inputs L2-resident):
    (microseconds per evaluation, bin-evaluations per second)."""
    import torch
    P = theta.shape[0]
    th = torch.tensor(theta, dtype=torch.float64, device="cuda")
    out = torch.empty(1 + P, dtype=torch.float64, device="cuda")
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        for _ in range(3):
            run.chi2_grad_device(th, out, obj, mode, stream=cap.cuda_stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        for _ in range(reps):
            run.chi2_grad_device(th, out, obj, mode, stream=cap.cuda_stream)
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    graph.replay()
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / reps
    del graph
    return us, run.total_bins / (us * 1e-6)


def _fit_rate(run, starts, obj, free, method):
    from paper_1604_02334_gb300 import MUSR_FIT_LM  # noqa: F401
    t0 = time.perf_counter()
    iters, evals, vals = [], [], []
    for st in starts:
        _, info, _ = run.fit(st, obj, free=free, method=method)
        iters.append(info["iters"])
        evals.append(info["evals"])
        vals.append(info["value"] / info["ndf"])
    dt = time.perf_counter() - t0
    return {"fits_per_s": len(starts) / dt, "ms_per_fit": 1e3 * dt / len(starts),
            "mean_iters": float(np.mean(iters)), "mean_evals": float(np.mean(evals)),
            "chi2_ndf": float(np.median(vals))}


def _flushed_us(run, thetas_t, out, obj, mode, flush, stream, steps=20):
    """Median microseconds of one device-entry evaluation, L2 flushed before
    each, CUDA events on the launching stream around the launch alone."""
    import torch
    ms = []
    n = thetas_t.shape[0]
    for j in range(steps + 3):
        flush.fill_(j & 255)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run.chi2_grad_device(thetas_t[j % n], out, obj, mode, stream=stream.cuda_stream)
        e1.record(stream)
        if j >= 3:
            ms.append((e0, e1))
    torch.cuda.synchronize()
    return 1e3 * float(np.median([x.elapsed_time(y) for x, y in ms]))


def _b2b_us(run, thetas_t, out, obj, mode, stream, steps=50):
    """Microseconds per device-entry evaluation launched back to back (no
    flush; the inputs stay in L2), CUDA events around all of them."""
    import torch
    n = thetas_t.shape[0]
    for j in range(5):
        run.chi2_grad_device(thetas_t[j % n], out, obj, mode, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(steps):
        run.chi2_grad_device(thetas_t[j % n], out, obj, mode, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / steps


def _queued_us(run, thetas, out, obj, mode, stream, steps=50):
    """Microseconds per evaluation queued back to back through the host-theta
    entry (theta by value: each evaluation's bin loop may overlap the previous
    one's reduction), CUDA events around all of them."""
    import torch
    rows = [np.ascontiguousarray(t) for t in thetas]
    n = len(rows)
    for j in range(5):
        run.chi2_grad_async(rows[j % n], out, obj, mode, stream=stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for j in range(steps):
        run.chi2_grad_async(rows[j % n], out, obj, mode, stream=stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return 1e3 * e0.elapsed_time(e1) / steps


def other_configs(rank, peaks, flush, stream):
    """The remaining workloads of the measurement plan, each a small extra:
    the 16 x 65536 workload (chi2 + gradient, Gauss-Newton, value, deviance;
    L2 flushed), the Gauss-Newton mode on the headline shape, the single
    histogram (fits/s, latency), the stretched-line variant, the paper's
    Table 1 shapes, fits on the headline shape (adjoint LM / BFGS, central
    differences) and the user-theory kernels."""
    import torch
    from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD, MUSR_FIT_LM, MUSR_POISSON,
                                        MUSR_VALUE, MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN, Run)
    res = {}
    dev = torch.device("cuda", torch.cuda.current_device())
    # 16 x 65536, 40 free: every mode, L2 flushed, events around the launch
    lay, theta, seed = W.config_multi_detector()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    g = W.rng(seed + 11 + rank)
    ths = torch.tensor(np.stack([W.perturb(theta, lay.free, 0.01, g) for _ in range(8)]), device=dev)
    P = lay.n_params
    out = torch.empty(1 + P + P * P, dtype=torch.float64, device=dev)
    with Run(lay, torch.tensor(W.poisson_counts(mean, seed + rank), dtype=torch.float32, device=dev)) as run:
        t_grad = _flushed_us(run, ths, out, MUSR_CHI2, MUSR_VALUE_GRAD, flush, stream)
        t_gn = _flushed_us(run, ths, out, MUSR_CHI2, MUSR_VALUE_GRAD_GN, flush, stream)
        t_val = _flushed_us(run, ths, out, MUSR_CHI2, MUSR_VALUE, flush, stream)
        t_dev = _flushed_us(run, ths, out, MUSR_POISSON, MUSR_VALUE_GRAD, flush, stream)
        t_b2b = _b2b_us(run, ths, out, MUSR_CHI2, MUSR_VALUE_GRAD, stream)
        t_b2b_gn = _b2b_us(run, ths, out, MUSR_CHI2, MUSR_VALUE_GRAD_GN, stream)
        t_q = _queued_us(run, ths.cpu().numpy(), out, MUSR_CHI2, MUSR_VALUE_GRAD, stream)
        t_q_gn = _queued_us(run, ths.cpu().numpy(), out, MUSR_CHI2, MUSR_VALUE_GRAD_GN, stream)
    rl = roofline(lay.total_bins, t_grad * 1e-6, peaks, ALG_FP32_FLOP_PER_BIN, ALG_SFU_PER_BIN, ALG_BYTES_PER_BIN)
    res["cfg_16x65536"] = {"chi2_grad_us": t_grad, "bin_evals_per_s": lay.total_bins / (t_grad * 1e-6),
                           "frac": rl["frac"], "pipe": rl["pipe"], "gn_us": t_gn, "value_us": t_val,
                           "deviance_grad_us": t_dev, "chi2_grad_us_b2b_l2": t_b2b, "gn_us_b2b_l2": t_b2b_gn,
                           "chi2_grad_us_queued_l2": t_q, "gn_us_queued_l2": t_q_gn}
    # Gauss-Newton mode on the headline shape (what every LM iteration evaluates)
    lay, theta, seed = W.config_gradient()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    g = W.rng(seed + 31 + rank)
    P = lay.n_params
    ths = torch.tensor(np.stack([W.perturb(theta, lay.free, 0.01, g) for _ in range(8)]), device=dev)
    out = torch.empty(1 + P + P * P, dtype=torch.float64, device=dev)
    data = W.poisson_counts(mean, seed + rank)
    with Run(lay, torch.tensor(data, dtype=torch.float32, device=dev)) as run:
        res["cfg_32x131072_gn_us"] = _flushed_us(run, ths, out, MUSR_CHI2, MUSR_VALUE_GRAD_GN, flush, stream)
        res["cfg_32x131072_gn_us_queued_l2"] = _queued_us(run, ths.cpu().numpy(), out, MUSR_CHI2,
                                                          MUSR_VALUE_GRAD_GN, stream)
        starts = [W.perturb(theta, lay.free, 0.01, g) for _ in range(5)]
        res["cfg_32x131072_fits"] = {
            "lm_adjoint_gn": _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_LM),
            "bfgs_adjoint": _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_BFGS),
            "bfgs_central_differences": _fit_rate(run, starts[:2], MUSR_CHI2, lay.free, MUSR_FIT_BFGS_FD)}
    # single histogram, 8192 bins, FP64 data, 6 free: LM fits from 5 % perturbed starts
    lay, theta, seed = W.config_single()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        g = W.rng(seed + 21 + rank)
        starts = [W.perturb(theta, lay.free, 0.05, g) for _ in range(200)]
        fit = _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_LM)
        t0 = time.perf_counter()
        for i in range(500):
            run.chi2(starts[i % 200], MUSR_CHI2)
        host_us = 1e6 * (time.perf_counter() - t0) / 500
        dev_us, _ = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
    res["single_8192"] = {"fit_lm": fit, "host_chi2_us": host_us, "device_chi2_us": dev_us}
    # same shape as 16 x 65536 with the second line a stretched exponential, 41 free
    lay, theta, seed = W.config_stretched()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        us, rate = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE_GRAD)
        us_v, rate_v = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
    res["stretched_16x65536"] = {"chi2_grad_us": us, "chi2_value_us": us_v}
    # the paper's Table 1 shapes: chi2 value per evaluation (its Table 1 times one chi2 per "Iter.")
    sweep = []
    for M in W.SWEEP_BINS:
        lay, theta, seed = W.config_sweep(M)
        with Run(lay) as m:
            mean = m.model(theta).astype(np.float64)
        with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
            us, rate = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
            us_g, rate_g = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE_GRAD)
        sweep.append({"bins": f"16x{M}", "chi2_us": us, "chi2_grad_us": us_g})
    res["table1_shapes_graph_replay"] = sweep
    # the 16 x 65536 theory as a user expression compiled at run time (FP64 and FP32 kernels)
    from paper_1604_02334_gb300 import UserTheory
    lay, theta, seed = W.config_multi_detector()
    t0 = time.perf_counter()
    th = UserTheory(W.MD_USER_EXPR)
    compile_s = time.perf_counter() - t0
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    nvec = 64
    thetas = np.repeat(theta[None, :], nvec, axis=0)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        th.eval(run, thetas, MUSR_CHI2)
        t0 = time.perf_counter()
        for _ in range(5):
            th.eval(run, thetas, MUSR_CHI2)
        us64 = 1e6 * (time.perf_counter() - t0) / 5
        th.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=0.0)
        t0 = time.perf_counter()
        th.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=0.0)
        fwd_ms = 1e3 * (time.perf_counter() - t0)
    th.close()
    th32 = UserTheory(W.MD_USER_EXPR, fp32=True)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        th32.eval(run, thetas, MUSR_CHI2)
        t0 = time.perf_counter()
        for _ in range(5):
            th32.eval(run, thetas, MUSR_CHI2)
        us64_32 = 1e6 * (time.perf_counter() - t0) / 5
        th32.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=0.0)
        t0 = time.perf_counter()
        th32.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=0.0)
        fwd32_ms = 1e3 * (time.perf_counter() - t0)
    th32.close()
    res["user_theory_16x65536"] = {
        "compile_s": compile_s,
        "fp64_bin_evals_per_s_64_vectors": 64 * lay.total_bins / (us64 * 1e-6),
        "fp64_forward_mode_gradient_ms": fwd_ms,
        "fp32_bin_evals_per_s_64_vectors": 64 * lay.total_bins / (us64_32 * 1e-6),
        "fp32_forward_mode_gradient_ms": fwd32_ms}
    return res


def batched_grad_throughput(dev, rank, peaks, n_runs=64, reps=5):
    """chi2 + gradient of 64 runs of the benchmark workload (16 x 65536 bins
    each, own parameters and counts) in one launch of the batched adjoint
    kernel: device-resident inputs (268 MB, larger than L2), CUDA events."""
    import torch
    from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_VALUE_GRAD, GBatch, Run
    lay = W.multi_detector_layout(16, 65536, 12.8)
    g = W.rng(W.BASE_SEED + 3005 + rank)
    thetas = np.stack([W.multi_detector_theta(lay, g) for _ in range(n_runs)])
    with Run(lay) as layout:
        data = torch.empty((n_runs, lay.total_bins), dtype=torch.float32, device=dev)
        layout.generate(torch.tensor(thetas, device=dev), 1, W.BASE_SEED + 3006 + rank, data)
        torch.cuda.synchronize()
    runs = [Run(lay, data[i].contiguous()) for i in range(n_runs)]
    del data
    b = GBatch(runs, with_gn=False)
    th = torch.tensor(np.concatenate([W.perturb(t, lay.free, 0.01, g) for t in thetas]), device=dev)
    out = torch.empty(int(np.sum(b.out_sizes(MUSR_VALUE_GRAD))), dtype=torch.float64, device=dev)
    b.eval_device(th, out, MUSR_CHI2, MUSR_VALUE_GRAD)  # tunes on first use
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.eval_device(th, out, MUSR_CHI2, MUSR_VALUE_GRAD)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    med = float(np.median(ms))
    bins = n_runs * lay.total_bins
    b.close()
    for r in runs:
        r.close()
    rl = roofline(bins, med * 1e-3, peaks, ALG_FP32_FLOP_PER_BIN, ALG_SFU_PER_BIN, ALG_BYTES_PER_BIN,
                  kernel="gbatch_kernel<1,1,0,1,kGrad>")
    rl["exec_fp32_frac"] = _r(EXEC_FP32_FLOP_PER_BIN * bins / (med * 1e-3) / peaks["fp32_flops"])
    return {"workload": f"{n_runs} runs x 16 hist x 65536 bins, chi2 + gradient, one launch", "bin_evals": bins,
            "ms": med, "value": bins / (med * 1e-3), "unit": "bin-evals/s", "roofline": rl}


def learned_start_ab(dev, rank, train_steps, n_runs=64):
    """Fits/s and success of the learned-start fit against the plain fit.

    The proposer trains on device-generated histograms (16 x 65536 bins,
    parameters uniform in the prior box); then n_runs held-out runs (numpy
    draws of the parameters, device Poisson counts) are fitted (chi2, LM,
    40 free) three ways: from the truth (the reference minimum), learned start
    (proposal + fit, plain fit as fallback when chi2/ndf > 1.2), and plain
    (range centre with a 10-point B1 grid, best of 10).  A fit succeeds when
    its chi2 is within 1e-6 relative of the truth-start fit's."""
    import torch
    from paper_1604_02334_gb300 import MUSR_CHI2, GBatch, Proposer, Run, fit_multistart_batch
    lay = W.multi_detector_layout(16, 65536, 12.8)
    lo, hi = W.multi_detector_box(lay)
    layout = Run(lay)
    prop = Proposer(layout, lo, hi, seed=W.BASE_SEED + 5 + 100 * rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = prop.train(train_steps, 1e-3, 3e-5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    g = W.rng(W.BASE_SEED + 2005 + rank)
    thetas = np.stack([W.multi_detector_theta(lay, g) for _ in range(n_runs)])
    data = torch.empty((n_runs, lay.total_bins), dtype=torch.float32, device=dev)
    layout.generate(torch.tensor(thetas, device=dev), 1, W.BASE_SEED + 2006 + rank, data)
    torch.cuda.synchronize()
    runs = [Run(lay, data[i].contiguous()) for i in range(n_runs)]
    free = lay.free
    starts = W.default_starts(lay)
    gb = GBatch(runs)
    ref = [x["value"] for x in gb.fit(list(thetas), MUSR_CHI2, free=[free] * n_runs)[1]]
    res = {}
    # batched arms: every run's learned start fitted in lockstep (fallback batched
    # too); every (run, start) pair of the plain grid fitted in lockstep
    from paper_1604_02334_gb300 import MUSR_FIT_BFGS, MUSR_FIT_LM
    arms = []
    for tag, method in (("", MUSR_FIT_LM), ("_bfgs", MUSR_FIT_BFGS)):
        t0 = time.perf_counter()
        _, il = prop.fit_batch(gb, MUSR_CHI2, free=[free] * n_runs, chi2ndf_max=1.2,
                               fallback_starts=[starts] * n_runs, method=method)
        t1 = time.perf_counter()
        _, ip = fit_multistart_batch(runs, [starts] * n_runs, MUSR_CHI2, free=[free] * n_runs, method=method)
        t2 = time.perf_counter()
        arms += [("learned_batched" + tag, il, t1 - t0), ("plain_batched" + tag, ip, t2 - t1)]
    for name, infos, dt in arms:
        ok = [abs(x["value"] - r) <= 1e-6 * r for x, r in zip(infos, ref)]
        res[name] = {"fits_per_s": n_runs / dt, "success": float(np.mean(ok)),
                     "mean_iters": float(np.mean([x["iters"] for x in infos])), "ms_per_fit": 1e3 * dt / n_runs}
        if name.startswith("learned"):
            res[name]["fallbacks"] = int(sum(x["fallback"] for x in infos))
    gb.close()
    for name in ("learned", "plain"):
        ok, iters, fallback = [], [], 0
        t0 = time.perf_counter()
        for i, r in enumerate(runs):
            if name == "learned":
                _, info, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=1.2, fallback_starts=starts)
                fallback += int(info["fallback"])
            else:
                _, info, _ = r.fit_multistart(starts, MUSR_CHI2, free=free)
            ok.append(abs(info["value"] - ref[i]) <= 1e-6 * ref[i])
            iters.append(info["iters"])
        dt = time.perf_counter() - t0
        res[name] = {"fits_per_s": n_runs / dt, "success": float(np.mean(ok)), "mean_iters": float(np.mean(iters)),
                     "ms_per_fit": 1e3 * dt / n_runs}
        if name == "learned":
            res[name]["fallbacks"] = fallback
    for r in runs:
        r.close()
    prop.close()
    layout.close()
    return {"workload": "16 hist x 65536 bins, 40 free, chi2 LM fits of held-out runs from the prior box",
            "n_runs": n_runs, "train_steps": train_steps, "train_samples": train_steps * 512,
            "train_s": t_train, "train_samples_per_s": train_steps * 512 / t_train,
            "final_loss": float(np.mean(losses[-100:])), **res,
            "speedup_fits_per_s": res["learned"]["fits_per_s"] / res["plain"]["fits_per_s"],
            "speedup_fits_per_s_batched": res["learned_batched"]["fits_per_s"] / res["plain_batched"]["fits_per_s"],
            "speedup_fits_per_s_batched_bfgs":
                res["learned_batched_bfgs"]["fits_per_s"] / res["plain_batched_bfgs"]["fits_per_s"]}


def learned_summary(ls):
    """The learned-start A/B in a few keys: fits/s of both arms, success, fallbacks."""
    if not ls:
        return None
    out = {"speedup_batched_lm": ls["speedup_fits_per_s_batched"],
           "speedup_batched_bfgs": ls["speedup_fits_per_s_batched_bfgs"],
           "speedup_sequential": ls["speedup_fits_per_s"]}
    for k in ("learned_batched", "plain_batched", "learned_batched_bfgs", "plain_batched_bfgs", "learned", "plain"):
        x = ls[k]
        out[k] = {"fits_per_s": x["fits_per_s"], "success": x["success"], "iters": x["mean_iters"]}
        if "fallbacks" in x:
            out[k]["fallbacks"] = x["fallbacks"]
    out["n_runs"] = ls["n_runs"]
    out["train_samples"] = ls["train_samples"]
    return out


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args.gpus)
    from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_VALUE_GRAD, Run

    dev = torch.device("cuda", torch.cuda.current_device())
    peaks = measured_peaks()
    lay, theta, seed = make_workload()
    P = lay.n_params
    # N_RUNS independent runs of the workload (own Poisson counts each), cycled
    # step by step: together larger than L2, so each step reads its counts
    # from HBM without a flush between launches
    with Run(lay) as mrun:
        mean = mrun.model(theta).astype(np.float64)
    datas = [W.poisson_counts(mean, seed + rank + 1000 * r) for r in range(N_RUNS)]
    data = datas[0]
    runs = [Run(lay, torch.tensor(d, dtype=torch.float32, device=dev)) for d in datas]
    run = runs[0]
    g = W.rng(seed + 11 + rank)
    n_vec = args.steps + args.warmup
    thetas = np.stack([W.perturb(theta, lay.free, 0.01, g) for _ in range(n_vec)])
    thetas_t = torch.tensor(thetas, dtype=torch.float64, device=dev)
    outs = torch.empty((n_vec, 1 + P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # one explicit (non-default) stream carries the events and the kernels
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream

    # a step: one chi2 + gradient evaluation queued with its theta by value
    # (the library's queued entry), results into device memory; the rows are
    # sliced beforehand so that the host keeps ahead of the GPU
    th_rows = [np.ascontiguousarray(t) for t in thetas]
    th_rows_t = [thetas_t[i] for i in range(n_vec)]
    out_rows = [outs[i] for i in range(n_vec)]

    def step(i):
        runs[i % N_RUNS].chi2_grad_async(th_rows[i], out_rows[i], MUSR_CHI2, MUSR_VALUE_GRAD, stream=sptr)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    # untimed soak (the same steps) so the clock samples see the GPU under load
    t_soak = time.perf_counter()
    while time.perf_counter() - t_soak < 0.4:
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e_start, e_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wall0 = time.perf_counter()
    e_start.record(stream)
    for j in range(args.steps):
        step(args.warmup + j)
    enqueue = time.perf_counter() - wall0
    e_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    t_timed = e_start.elapsed_time(e_end) / 1e3
    t_total = max_over_ranks(t_timed, world)
    value = job_value(lay.total_bins * args.steps, t_timed, world)
    mean_ms = 1e3 * t_total / args.steps
    # the same evaluation one launch at a time, L2 flushed before each, events around the launch alone
    flushed_us = _flushed_us(run, thetas_t, outs[0], MUSR_CHI2, MUSR_VALUE_GRAD, flush, stream)
    # the same steps through the device-theta entry (theta read from device
    # memory after the previous kernel completes: no overlap between steps)
    def step_dev(i):
        runs[i % N_RUNS].chi2_grad_device(th_rows_t[i], out_rows[i], MUSR_CHI2, MUSR_VALUE_GRAD, stream=sptr)

    for i in range(args.warmup):
        step_dev(i)
    torch.cuda.synchronize()
    e_start.record(stream)
    for j in range(args.steps):
        step_dev(args.warmup + j)
    e_end.record(stream)
    torch.cuda.synchronize()
    device_theta_us = 1e3 * e_start.elapsed_time(e_end) / args.steps

    # end to end through the C ABI with host buffers: per step, upload the
    # histograms from pinned memory, evaluate chi2 + gradient, read them back
    host_data = torch.tensor(data, dtype=torch.float32).pin_memory()
    host_np = host_data.numpy()
    e2e_steps = max(10, min(args.steps, 100))
    run_h = Run(lay, host_np)
    for i in range(3):
        run_h.set_data(host_np)
        run_h.chi2_grad(thetas[i], MUSR_CHI2)
    barrier(world)
    t0 = time.perf_counter()
    for j in range(e2e_steps):
        run_h.set_data(host_np)
        run_h.chi2_grad(thetas[j % n_vec], MUSR_CHI2)
    e2e_t = max_over_ranks(time.perf_counter() - t0, world)
    run_h.close()
    e2e = {"value": world * lay.total_bins * e2e_steps / e2e_t, "unit": UNIT,
           "h2d_bytes_per_step": lay.total_bins * 4 + P * 8, "d2h_bytes_per_step": (1 + P) * 8 + 4,
           "steps": e2e_steps}

    # sanity: results are finite
    assert torch.isfinite(outs[args.warmup:]).all().item()
    for r in runs[1:]:
        r.close()
    others = None if args.no_other_configs else other_configs(rank, peaks, flush, stream)
    # the batched legs record their events on the current (explicit) stream and
    # launch on it: a NULL stream would send the library's work to its own
    batched = None if args.no_batched else batched_throughput(dev, rank, peaks)
    batched_grad = None if args.no_batched else batched_grad_throughput(dev, rank, peaks)
    learned = None if args.learned_steps <= 0 else learned_start_ab(dev, rank, args.learned_steps)

    if rank != 0:
        run.close()
        return
    rl = roofline(lay.total_bins, mean_ms * 1e-3, peaks, ALG_FP32_FLOP_PER_BIN, ALG_SFU_PER_BIN,
                  ALG_BYTES_PER_BIN, traffic=TRAFFIC_BYTES_GRAD_LAUNCH, kernel="eval_kernel<1,1,0,1,kGrad>")
    rl["exec_fp32_frac"] = _r(EXEC_FP32_FLOP_PER_BIN * lay.total_bins / (mean_ms * 1e-3) / peaks["fp32_flops"])
    rl["peak_src"] = ("measured: musr_pipe_rates probe (FP32 FMA, SFU ex2/cos/rcp); HBM from the pool's "
                      f"copy bandwidth ({peaks['hbm_src']})")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 eval (packed pairs), f32 warp sums, exact 126-bit fixed-point block and final sums, f64 out",
        "data": "synthetic (Poisson counts of the model, numpy PCG64)",
        "config": {"workload": WORKLOAD, "bins": lay.total_bins, "params": P,
                   "l2": f"inputs larger than L2: {N_RUNS} independent runs of the workload "
                         f"({N_RUNS * lay.total_bins * 4 / 1e6:.0f} MB of counts) cycled step by step, "
                         "launches back to back",
                   "entry": "musr_chi2_grad_async: theta by value, results in device memory, evaluations queued",
                   "parallelism": f"replicas x{world}"},
        "roofline": rl,
        "clocks": clk,
        "e2e": _short(e2e),
        "gpu_launches": args.steps,  # one objective kernel launch per step
        "flushed_step_us": _r(flushed_us),
        "device_theta_step_us": _r(device_theta_us),
        "host_enqueue_us_per_step": _r(1e6 * enqueue / args.steps),
        "pipe_rates_per_s": _short(peaks["rates"]),
    }
    details = {"wall_s": wall}
    if others:
        details["other_configs"] = others
        c2 = others["cfg_16x65536"]
        line["cfg_16x65536"] = _short(
            {"chi2_grad_us_flushed": c2["chi2_grad_us"], "chi2_grad_us_b2b_l2": c2["chi2_grad_us_b2b_l2"],
             "gn_us_flushed": c2["gn_us"], "gn_us_b2b_l2": c2["gn_us_b2b_l2"], "value_us_flushed": c2["value_us"],
             "deviance_grad_us_flushed": c2["deviance_grad_us"], "chi2_grad_us_queued_l2": c2["chi2_grad_us_queued_l2"],
             "gn_us_queued_l2": c2["gn_us_queued_l2"]})
        line["cfg_32x131072_gn_us"] = _r(others["cfg_32x131072_gn_us"])
        line["cfg_32x131072_gn_us_queued_l2"] = _r(others["cfg_32x131072_gn_us_queued_l2"])
        f4 = others["cfg_32x131072_fits"]
        line["cfg_32x131072_fits_per_s"] = _short({k: v["fits_per_s"] for k, v in f4.items()})
    if batched:
        details["batched"] = batched
        line["batched_value"] = _short({"bin_evals_per_s": batched["value"], "frac": batched["roofline"]["frac"],
                                        "pipe": batched["roofline"]["pipe"]})
    if batched_grad:
        details["batched_grad"] = batched_grad
        line["batched_grad"] = _short({"bin_evals_per_s": batched_grad["value"],
                                       "frac": batched_grad["roofline"]["frac"],
                                       "pipe": batched_grad["roofline"]["pipe"]})
    if learned:
        details["learned_start"] = learned
        line["learned_start"] = _short(learned_summary(learned))
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = _short(cpu_baseline(lay, data, thetas))
    print(json.dumps(_short(details)), file=sys.stderr, flush=True)
    print(json.dumps(line), flush=True)
    run.close()


def run_sharded(args):
    """Strong scaling: the headline run split by histogram over the ranks
    (one GPU each); one step = chi2 + gradient of the whole run, every rank
    evaluating its shard through the library's host call and the shards'
    1 + P sums combined by an all-gather added in rank order."""
    import torch
    import torch.distributed as dist
    world, rank, local = dist_setup(args.gpus)
    if not dist.is_initialized():  # one rank: a process group of its own
        import tempfile
        pg_file = os.path.join(tempfile.mkdtemp(), "pg")
        dist.init_process_group("gloo", init_method=f"file://{pg_file}", rank=0, world_size=1)
    from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_VALUE_GRAD
    from paper_1604_02334_gb300.shard import ShardedRun
    lay, theta, seed = make_workload()
    from paper_1604_02334_gb300 import Run
    with Run(lay) as mrun:
        mean = mrun.model(theta).astype(np.float64)
    data = W.poisson_counts(mean, seed)  # the same run on every rank
    sr = ShardedRun(lay, data)
    g = W.rng(seed + 11)
    thetas = [W.perturb(theta, lay.free, 0.01, g) for _ in range(args.steps + args.warmup)]
    for i in range(args.warmup):
        sr.chi2_grad(thetas[i], MUSR_CHI2, MUSR_VALUE_GRAD)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(world)
    t0 = time.perf_counter()
    for j in range(args.steps):
        sr.chi2_grad(thetas[args.warmup + j], MUSR_CHI2, MUSR_VALUE_GRAD)
    barrier(world)
    el = max_over_ranks(time.perf_counter() - t0, world)
    clk = clocks.stop()
    sr.close()
    if rank != 0:
        return
    value = lay.total_bins * args.steps / el
    P = lay.n_params
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": "f32 eval, exact fixed-point sums per shard, f64 combine in rank order",
        "data": "synthetic (Poisson counts of the model, numpy PCG64)",
        "config": {"workload": WORKLOAD, "bins": lay.total_bins, "params": P,
                   "l2": "host calls, one whole-run evaluation per step (counts resident per shard)",
                   "parallelism": f"histogram shards x{world}, all-gather of 1 + P sums"},
        "clocks": clk,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": world * P * 8,
                "d2h_bytes_per_step": world * (1 + P) * 8},
        "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true")
    ap.add_argument("--learned-steps", type=int, default=32768,
                    help="proposer training steps for the learned-start A/B (0: skip it)")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: split the run by histogram over the ranks instead of replicas")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
