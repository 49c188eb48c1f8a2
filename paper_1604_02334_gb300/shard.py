"""Histogram-sharded runs over several GPUs, one rank per GPU.

The objective of Sec. 4.1 (Eq. 3 chi2, Eq. 4 deviance), its gradient and its
Gauss-Newton matrix are sums over histograms, so a run split by histogram
over the ranks of a process group (the multi-GPU extension the paper's Sec. 6
names as future work) evaluates its shard with the library on each rank's
GPU and adds the shards' sums: one exchange of 1 + P (+ P^2) FP64 values per
evaluation.  The exchange is an all-gather whose parts every rank adds in
rank order, so every rank holds bitwise the same result and a fit driven by
it (musr_fit_eval) takes the same steps on every rank.

This module marshals arguments and moves the small partial vectors between
ranks (torch.distributed); every bin is evaluated by the library's kernels.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _lib
from ._lib import MUSR_CHI2, MUSR_FIT_LM, MUSR_OK, MUSR_VALUE, MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN


def partition_histograms(n_bins, world):
    """Histogram indices of each rank: the largest histograms first, each to
    the rank with the fewest bins so far (the lowest rank on ties), every
    rank's list in ascending order.  Deterministic: every rank computes the
    same partition."""
    nb = np.asarray(n_bins, dtype=np.int64)
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in sorted(range(nb.shape[0]), key=lambda i: (-int(nb[i]), i)):
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += int(nb[k])
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def shard_layout(layout, hists):
    """The run restricted to histograms `hists` (same parameters and components)."""
    hists = np.asarray(hists, dtype=np.int64)
    return dataclasses.replace(layout, n_bins=layout.n_bins[hists].copy(),
                               map=np.ascontiguousarray(layout.map[hists]))


def shard_data(layout, data, hists):
    """The counts of histograms `hists`, concatenated in that order."""
    offs = np.r_[0, np.cumsum(layout.n_bins)]
    d = np.asarray(data)
    if len(hists) == 0:
        return d[:0].copy()
    return np.concatenate([d[offs[k]:offs[k + 1]] for k in hists])


class ShardedRun:
    """One rank's share of a histogram-sharded run.

    layout, data: the whole run (every rank passes the same); the rank keeps
    the histograms partition_histograms gives it.  evaluate(theta, obj, mode)
    of the shard defaults to the library on this rank's current GPU (a Run of
    the shard); a callable with the same signature returning
    (value, grad or None, gn or None) can stand in for it.  group: the
    torch.distributed process group (default: the world).
    """

    def __init__(self, layout, data, group=None, evaluate=None):
        import torch.distributed as dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.layout = layout
        self.P = layout.n_params
        self.hists = partition_histograms(layout.n_bins, self.world)[self.rank]
        self.local_layout = shard_layout(layout, self.hists)
        self.run = None
        if evaluate is None and len(self.hists) > 0:
            from . import Run
            self.run = Run(self.local_layout, shard_data(layout, data, self.hists))
            evaluate = self._evaluate_run
        self._evaluate = evaluate

    def _evaluate_run(self, theta, obj, mode):
        if mode == MUSR_VALUE:
            return self.run.chi2(theta, obj), None, None
        v, g, H = self.run.chi2_grad(theta, obj, gn=mode == MUSR_VALUE_GRAD_GN)
        return v, g, H

    def _local(self, theta, obj, mode):
        n = 1 + (self.P if mode >= MUSR_VALUE_GRAD else 0) + (self.P * self.P if mode == MUSR_VALUE_GRAD_GN else 0)
        out = np.zeros(n)
        if self._evaluate is None:  # a rank without histograms adds zeros
            return out
        v, g, H = self._evaluate(np.asarray(theta, dtype=np.float64), obj, mode)
        out[0] = v
        if mode >= MUSR_VALUE_GRAD:
            out[1:1 + self.P] = g
        if mode == MUSR_VALUE_GRAD_GN:
            out[1 + self.P:] = np.asarray(H).ravel()
        return out

    def combine(self, part):
        """Sum of every rank's `part` (FP64), added in rank order on every rank."""
        import torch
        import torch.distributed as dist
        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.as_tensor(np.ascontiguousarray(part, dtype=np.float64), device=dev)
        parts = [torch.empty_like(t) for _ in range(self.world)]
        dist.all_gather(parts, t, group=self.group)
        total = parts[0].clone()
        for x in parts[1:]:
            total += x
        return total.cpu().numpy()

    def chi2_grad(self, theta, obj=MUSR_CHI2, mode=MUSR_VALUE_GRAD):
        """(value, grad, gn) of the whole run; grad / gn None below their mode."""
        tot = self.combine(self._local(theta, obj, mode))
        g = tot[1:1 + self.P] if mode >= MUSR_VALUE_GRAD else None
        H = tot[1 + self.P:].reshape(self.P, self.P) if mode == MUSR_VALUE_GRAD_GN else None
        return float(tot[0]), g, H

    def fit(self, theta0, obj=MUSR_CHI2, free=None, method=MUSR_FIT_LM, max_iter=500, edm_tol=1e-8, mu0=1e-3):
        """musr_fit_eval over the sharded evaluation: (theta, info, cov), the same on every rank."""
        return fit_eval(self.P, self.layout.total_bins, lambda th, mode: self.chi2_grad(th, obj, mode), theta0,
                        free=free, method=method, max_iter=max_iter, edm_tol=edm_tol, mu0=mu0)

    def close(self):
        if self.run is not None:
            self.run.close()
            self.run = None


def fit_eval(n_params, n_bins_total, evaluate, theta0, free=None, method=MUSR_FIT_LM, max_iter=500, edm_tol=1e-8,
             mu0=1e-3):
    """musr_fit_eval with evaluate(theta, mode) -> (value, grad, gn) supplying
    every evaluation (grad / gn may be None below their mode): (theta, info, cov)."""
    P = int(n_params)
    th = np.ascontiguousarray(theta0, dtype=np.float64).copy()
    fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
    nf = P if fm is None else int(fm.sum())
    cov = np.zeros((nf, nf))
    o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, 0.0)
    r = _lib.musr_fit_result()
    r.cov = cov.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    errors = []

    def cb(_user, mode, theta_p, value_p, grad_p, gn_p):
        try:
            theta = np.ctypeslib.as_array(theta_p, shape=(P,)).copy()
            v, g, H = evaluate(theta, mode)
            value_p[0] = v
            if mode >= MUSR_VALUE_GRAD:
                np.ctypeslib.as_array(grad_p, shape=(P,))[:] = g
            if mode == MUSR_VALUE_GRAD_GN:
                np.ctypeslib.as_array(gn_p, shape=(P * P,))[:] = np.asarray(H).ravel()
            return MUSR_OK if np.isfinite(v) else _lib.MUSR_ENONFINITE
        except Exception as e:  # noqa: BLE001 - re-raised after the fit
            errors.append(e)
            return _lib.MUSR_EINVAL

    fn = _lib.musr_eval_fn(cb)
    st = _lib.load().musr_fit_eval(P, int(n_bins_total), ctypes.cast(fn, ctypes.c_void_p), None,
                                   th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                   ctypes.byref(o), ctypes.byref(r))
    if errors:
        raise errors[0]
    info = {"value": r.value, "ndf": r.ndf, "edm": r.edm, "mu": r.mu, "iters": r.iters, "evals": r.n_evals,
            "status": st}
    return th, info, cov
