#!/usr/bin/env python
"""Benchmark: chi2 + gradient bin-evaluations per second on one GB300.

Workload: 16 detector histograms x 65536 bins of 0.1953125 ns (12.8 us),
theory = exponentially damped line + Gaussian-damped line (B1 + dB) + static
Gaussian Kubo-Toyabe, 56 parameters (40 free), Poisson counts.  One step is
one evaluation of chi2 and its gradient over every bin (objective kernel in
adjoint mode), for a fresh parameter vector; L2 is flushed (256 MB write)
between steps, outside the timed events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun): every rank runs an independent replica (the path has no
exchange step); value = all ranks' bin-evaluations / max-over-ranks time.
Prints one JSON line on rank 0.
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
WORKLOAD = "16 hist x 65536 bins, 2 lines + static GKT, 56 params (40 free), chi2 + gradient"

# FP32-pipe FLOPs per bin of the adjoint (value + gradient) code for this
# signature (1 exponential line, 1 Gaussian line, Kubo-Toyabe), counted by
# ncu on one launch of the batched adjoint kernel over 67,108,864 bins, where
# per-launch costs are negligible: 73.34 M FFMA and 28.45 M other FP32 warp
# instructions, i.e. (2 x 73.34 + 28.45) x 32 / 67.108864 = 83.5 FLOP / bin
# (FMA = 2).  The single-run kernel executes the same per-bin code.
FLOPS_PER_BIN_GRAD = 83.5
# DRAM bytes (read + write) of one eval_kernel<1,1,0,1,kGrad> launch of this
# workload, from the ncu capture summarised in
# profiles/eval_kernel_grad_16x65536.md (4,278,784 B read, 0 written); to be
# re-measured whenever that kernel changes.
TRAFFIC_BYTES_GRAD_LAUNCH = 4278784
# FP32-pipe FLOPs per bin-evaluation of the value-only batched kernel on the
# 64-run workload (batch_kernel<1,1,0,1>), counted by ncu on one launch of
# 2,720,958,581 bin-evaluations: 1978.5 M FFMA and 902.0 M other FP32 warp
# instructions, (2 x 1978.5 + 902.0) x 32 / 2720.96 = 57.1 FLOP per
# bin-evaluation (profiles/batch_kernel_value_64runs.md).
FLOPS_PER_BINEVAL_VALUE_BATCH = 57.1
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    return SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


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
SAMPLE_BINS = 8192  # leading bins of each of the 16 histograms


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
    lay, theta, seed = W.config_multi_detector()
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


def batched_throughput(dev, rank, reps=5):
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
    peak = fp32_peak_tflops()
    achieved = FLOPS_PER_BINEVAL_VALUE_BATCH * binevals / (med * 1e-3) / 1e12
    return {"workload": "64 runs, K~U{1..32} x M~U[2^14,2^17] bins, P+1 vectors each",
            "bins": int(sum(br.layout.total_bins for br in runs)), "bin_evals": int(binevals),
            "ms": med, "value": binevals / (med * 1e-3), "unit": "bin-evals/s (chi2, value only)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "batch_kernel<1,1,0,1>",
                         "note": "host-timed (includes the launch), L2 flushed before each"}}


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


def other_configs(rank):
    """The remaining workloads of the measurement plan, each a small extra:
    single histogram (fits/s, latency), -2lnL on the benchmark workload, the
    paper's Table 1 shapes, and the 32 x 131072 gradient workload (adjoint vs
    central-difference fits)."""
    from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD, MUSR_FIT_LM, MUSR_POISSON,
                                        MUSR_VALUE, MUSR_VALUE_GRAD, Run)
    res = {}
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
    # benchmark workload, Poisson deviance, value + gradient
    lay, theta, seed = make_workload()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        us, rate = _device_rate(run, theta, MUSR_POISSON, MUSR_VALUE_GRAD)
        us_v, rate_v = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
    res["multi_16x65536"] = {"poisson_grad_us": us, "poisson_grad_bin_evals_per_s": rate,
                             "chi2_value_us": us_v, "chi2_value_bin_evals_per_s": rate_v}
    # same shape with the second line a stretched exponential exp(-(lambda t)^beta), 41 free
    lay, theta, seed = W.config_stretched()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        us, rate = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE_GRAD)
        us_v, rate_v = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
    res["stretched_16x65536"] = {"chi2_grad_us": us, "chi2_grad_bin_evals_per_s": rate,
                                 "chi2_value_us": us_v, "chi2_value_bin_evals_per_s": rate_v}
    # the paper's Table 1 shapes: chi2 value per evaluation (its Table 1 times one chi2 per "Iter.")
    sweep = []
    for M in W.SWEEP_BINS:
        lay, theta, seed = W.config_sweep(M)
        with Run(lay) as m:
            mean = m.model(theta).astype(np.float64)
        with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
            us, rate = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE)
            us_g, rate_g = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE_GRAD)
        sweep.append({"bins": f"16x{M}", "chi2_us": us, "chi2_bin_evals_per_s": rate,
                      "chi2_grad_us": us_g, "chi2_grad_bin_evals_per_s": rate_g})
    res["table1_shapes"] = sweep
    # 32 x 131072, 72 free: value + gradient rate; fits from 1 % perturbed starts
    lay, theta, seed = W.config_gradient()
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        us, rate = _device_rate(run, theta, MUSR_CHI2, MUSR_VALUE_GRAD)
        g = W.rng(seed + 31 + rank)
        starts = [W.perturb(theta, lay.free, 0.01, g) for _ in range(5)]
        fits = {"lm_adjoint_gn": _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_LM),
                "bfgs_adjoint": _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_BFGS),
                "bfgs_central_differences": _fit_rate(run, starts, MUSR_CHI2, lay.free, MUSR_FIT_BFGS_FD)}
    res["gradient_32x131072"] = {"chi2_grad_us": us, "chi2_grad_bin_evals_per_s": rate, "fits": fits}
    # the benchmark theory as a user expression compiled at run time (FP64 kernel)
    from paper_1604_02334_gb300 import UserTheory
    lay, theta, seed = make_workload()
    t0 = time.perf_counter()
    th = UserTheory(W.MD_USER_EXPR)
    compile_s = time.perf_counter() - t0
    with Run(lay) as m:
        mean = m.model(theta).astype(np.float64)
    with Run(lay, W.poisson_counts(mean, seed + rank)) as run:
        th.eval(run, theta, MUSR_CHI2)
        reps = 20
        t0 = time.perf_counter()
        for _ in range(reps):
            th.eval(run, theta, MUSR_CHI2)
        us = 1e6 * (time.perf_counter() - t0) / reps
        nvec = 64
        thetas = np.repeat(theta[None, :], nvec, axis=0)
        th.eval(run, thetas, MUSR_CHI2)
        t0 = time.perf_counter()
        for _ in range(5):
            th.eval(run, thetas, MUSR_CHI2)
        us64 = 1e6 * (time.perf_counter() - t0) / 5
        t0 = time.perf_counter()
        th.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=1e-6)
        grad_ms = 1e3 * (time.perf_counter() - t0)
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
    res["user_theory_16x65536_fp32"] = {"chi2_64_vectors_us": us64_32,
                                        "chi2_bin_evals_per_s_64_vectors": 64 * lay.total_bins / (us64_32 * 1e-6),
                                        "forward_mode_gradient_40_directions_ms": fwd32_ms}
    res["user_theory_16x65536"] = {"compile_s": compile_s, "chi2_us_per_call": us,
                                   "chi2_bin_evals_per_s": lay.total_bins / (us * 1e-6),
                                   "chi2_64_vectors_us": us64,
                                   "chi2_bin_evals_per_s_64_vectors": 64 * lay.total_bins / (us64 * 1e-6),
                                   "fd_gradient_81_vectors_ms": grad_ms,
                                   "forward_mode_gradient_40_directions_ms": fwd_ms,
                                   "arithmetic": "fp64 (host call)"}
    return res


def batched_grad_throughput(dev, rank, n_runs=64, reps=5):
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
    peak = fp32_peak_tflops()
    achieved = FLOPS_PER_BIN_GRAD * bins / (med * 1e-3) / 1e12
    b.close()
    for r in runs:
        r.close()
    return {"workload": f"{n_runs} runs x 16 hist x 65536 bins, chi2 + gradient, one launch", "bin_evals": bins,
            "ms": med, "value": bins / (med * 1e-3), "unit": "bin-evals/s",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "kernel": "gbatch_kernel<1,1,0,1,kGrad>"}}


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


def run_ours(args):
    import torch

    world, rank, local = dist_setup(args.gpus)
    from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_VALUE_GRAD, Run

    dev = torch.device("cuda", torch.cuda.current_device())
    lay, theta, seed = make_workload()
    P = lay.n_params
    # synthetic Poisson counts: mean from the library's model kernel, noise from numpy PCG64
    with Run(lay) as mrun:
        mean = mrun.model(theta).astype(np.float64)
    data = W.poisson_counts(mean, seed + rank)
    data_t = torch.tensor(data, dtype=torch.float32, device=dev)
    run = Run(lay, data_t)
    g = W.rng(seed + 11 + rank)
    n_vec = args.steps + args.warmup
    thetas = np.stack([W.perturb(theta, lay.free, 0.01, g) for _ in range(n_vec)])
    thetas_t = torch.tensor(thetas, dtype=torch.float64, device=dev)
    outs = torch.empty((n_vec, 1 + P), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # one explicit (non-default) stream carries the flush, the events and the kernel
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream

    def step(i):
        run.chi2_grad_device(thetas_t[i], outs[i], MUSR_CHI2, MUSR_VALUE_GRAD, stream=sptr)

    for i in range(args.warmup):
        flush.fill_(i & 255)
        step(i)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for j in range(args.steps):
        flush.fill_((j + 1) & 255)
        starts[j].record(stream)
        step(args.warmup + j)
        ends[j].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_total = max_over_ranks(sum(step_ms) / 1e3, world)
    value = job_value(lay.total_bins * args.steps, sum(step_ms) / 1e3, world)
    mean_ms = 1e3 * t_total / args.steps

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
    batched = None if args.no_batched else batched_throughput(dev, rank)
    batched_grad = None if args.no_batched else batched_grad_throughput(dev, rank)
    learned = None if args.learned_steps <= 0 else learned_start_ab(dev, rank, args.learned_steps)
    others = None if args.no_other_configs else other_configs(rank)

    if rank != 0:
        run.close()
        return
    peak = fp32_peak_tflops()
    achieved = FLOPS_PER_BIN_GRAD * lay.total_bins / (mean_ms * 1e-3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 eval / f64 accumulate",
        "data": "synthetic (Poisson counts of the model, numpy PCG64)",
        "config": {"workload": WORKLOAD, "bins": lay.total_bins, "params": P,
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": TRAFFIC_BYTES_GRAD_LAUNCH,
                     "kernel": "eval_kernel<1,1,0,1,kGrad>",
                     "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 x 2070 MHz"},
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": args.steps,  # one objective kernel launch per step (the flush is a torch fill)
        "wall_s": wall,
    }
    if batched:
        line["batched"] = batched
    if batched_grad:
        line["batched_grad"] = batched_grad
    if learned:
        line["learned_start"] = learned
    if others:
        line["other_configs"] = others
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(lay, data, thetas)
    print(json.dumps(line), flush=True)
    run.close()


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
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
