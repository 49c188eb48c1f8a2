"""GB300 (sm_103a) engine for the muSR fit objective of Locans et al. (Sec. 4).

The compute lives in libmusr.so (CUDA kernels behind the C ABI of
include/musr.h).  This package is a thin binding: :mod:`._lib` declares the
C entry points under their own names, :class:`Run` marshals numpy / torch
buffers into them, and :class:`Chi2` exposes the adjoint kernel as a
``torch.autograd.Function``.  PyTorch is used for device memory and streams
only.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (MUSR_CHI2, MUSR_F32, MUSR_F64, MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD, MUSR_FIT_LM,
                   MUSR_POISSON, MUSR_VALUE, MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN, MusrError, check)

__all__ = ["Run", "Chi2", "MusrError", "MUSR_CHI2", "MUSR_POISSON", "load"]


def load():
    """Load libmusr.so (raises ImportError if it has not been built)."""
    return _lib.load()


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _torch_stream_ptr():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Run:
    """A run: K histograms on the device plus their layout (Sec. 4.1 Eq. 1-2).

    ``layout`` is any object with the attributes n_bins, t0_us, dt_us,
    tau_us, gamma, n_params, map (K x W int32) and comp (C x 6 int32:
    kind, amp, rate, field, field2, phase map columns).  ``data`` is a numpy
    array (FP32 / FP64) or a CUDA torch tensor of sum(n_bins) counts, or None.
    ``stream``: 'torch' to work on torch's current stream, None for a stream
    of the run's own.
    """

    def __init__(self, layout, data=None, stream=None):
        lib = _lib.load()
        self.layout = layout
        self._nb = np.ascontiguousarray(layout.n_bins, dtype=np.int64)
        self._map = np.ascontiguousarray(layout.map, dtype=np.int32)
        comp = np.ascontiguousarray(layout.comp, dtype=np.int32).reshape(-1, 6)
        self._comp = (_lib.musr_component * max(1, comp.shape[0]))()
        for i, row in enumerate(comp):
            self._comp[i] = _lib.musr_component(*[int(x) for x in row])
        d = _lib.musr_run_desc()
        d.n_hist = int(self._nb.shape[0])
        d.n_bins = self._nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.t0_us, d.dt_us = float(layout.t0_us), float(layout.dt_us)
        d.tau_us, d.gamma_mhz_per_g = float(layout.tau_us), float(layout.gamma)
        d.n_params = int(layout.n_params)
        d.map_width = int(self._map.shape[1])
        d.map = self._map.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.n_comp = int(comp.shape[0])
        d.comp = ctypes.cast(self._comp, ctypes.POINTER(_lib.musr_component))
        keep = None
        if data is None:
            d.data = None
        elif _is_torch(data):
            assert data.is_cuda and data.is_contiguous()
            d.data_dtype = MUSR_F64 if str(data.dtype) == "torch.float64" else MUSR_F32
            d.data = ctypes.c_void_p(data.data_ptr())
            d.data_on_device = 1
        else:
            keep = np.ascontiguousarray(data)
            if keep.dtype not in (np.float32, np.float64):
                keep = keep.astype(np.float64)
            d.data_dtype = MUSR_F64 if keep.dtype == np.float64 else MUSR_F32
            d.data = keep.ctypes.data_as(ctypes.c_void_p)
        if stream == "torch":
            d.stream = _torch_stream_ptr()
        elif stream is not None:
            d.stream = ctypes.c_void_p(int(stream))
        self._desc = d
        h = ctypes.c_void_p()
        check(lib.musr_create_run(ctypes.byref(d), ctypes.byref(h)), "musr_create_run")
        self.handle = h
        self.P = int(layout.n_params)
        self.total_bins = int(self._nb.sum())
        del keep

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.load().musr_destroy_run(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- data ----------------------------------------------------------------
    def set_data(self, data):
        lib = _lib.load()
        if _is_torch(data):
            dt = MUSR_F64 if str(data.dtype) == "torch.float64" else MUSR_F32
            check(lib.musr_set_data(self.handle, dt, ctypes.c_void_p(data.data_ptr()), 1), "musr_set_data")
        else:
            a = np.ascontiguousarray(data)
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
            dt = MUSR_F64 if a.dtype == np.float64 else MUSR_F32
            check(lib.musr_set_data(self.handle, dt, a.ctypes.data_as(ctypes.c_void_p), 0), "musr_set_data")

    # -- evaluation (host pointers, synchronous) -----------------------------
    def chi2(self, theta, obj=MUSR_CHI2, raise_on_error=True):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        v = np.zeros(1)
        st = _lib.load().musr_chi2(self.handle, int(obj), _dptr(th), _dptr(v))
        if raise_on_error:
            check(st, "musr_chi2")
            return float(v[0])
        return float(v[0]), st

    def chi2_grad(self, theta, obj=MUSR_CHI2, gn=False):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        v = np.zeros(1)
        g = np.zeros(self.P)
        H = np.zeros((self.P, self.P)) if gn else None
        st = _lib.load().musr_chi2_grad(self.handle, int(obj), _dptr(th), _dptr(v), _dptr(g),
                                        _dptr(H) if gn else None)
        check(st, "musr_chi2_grad")
        return float(v[0]), g, H

    def model(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        out = np.zeros(self.total_bins, dtype=np.float32)
        check(_lib.load().musr_model(self.handle, _dptr(th), out.ctypes.data_as(ctypes.c_void_p), 0),
              "musr_model")
        return out

    # -- evaluation (device pointers, asynchronous on torch's stream) ---------
    def chi2_grad_device(self, theta_dev, out_dev, obj=MUSR_CHI2, mode=MUSR_VALUE_GRAD,
                         status_dev=None, stream=None):
        """theta_dev: CUDA FP64 tensor [P]; out_dev: CUDA FP64 tensor, 1 (+P (+P*P)) long."""
        st = ctypes.c_void_p(int(stream)) if stream is not None else _torch_stream_ptr()
        check(_lib.load().musr_chi2_grad_device(
            self.handle, int(obj), int(mode), ctypes.c_void_p(theta_dev.data_ptr()),
            ctypes.c_void_p(out_dev.data_ptr()),
            ctypes.c_void_p(status_dev.data_ptr()) if status_dev is not None else None, st),
            "musr_chi2_grad_device")

    # -- synthetic data ------------------------------------------------------
    def generate(self, thetas_dev, rebin, seed, out_dev, sample_offset=0, log1p_out=False,
                 mu_dev=None, stream=None):
        """Poisson histograms of the theory, summed over groups of `rebin` bins,
        for every row of thetas_dev (CUDA FP64 [n, P]) into out_dev (CUDA FP32)."""
        st = ctypes.c_void_p(int(stream)) if stream is not None else _torch_stream_ptr()
        n = int(thetas_dev.shape[0])
        check(_lib.load().musr_generate(self.handle, ctypes.c_void_p(thetas_dev.data_ptr()), n, int(rebin),
                                        int(seed) & 0xffffffffffffffff, int(sample_offset),
                                        1 if log1p_out else 0, ctypes.c_void_p(out_dev.data_ptr()),
                                        ctypes.c_void_p(mu_dev.data_ptr()) if mu_dev is not None else None,
                                        st), "musr_generate")

    # -- fit ----------------------------------------------------------------
    def fit(self, theta0, obj=MUSR_CHI2, free=None, method=MUSR_FIT_LM, max_iter=500,
            edm_tol=1e-8, mu0=1e-3, fd_rel_h=0.0):
        th = np.ascontiguousarray(theta0, dtype=np.float64).copy()
        fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        nf = self.P if fm is None else int(fm.sum())
        cov = np.zeros((nf, nf))
        o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, fd_rel_h)
        r = _lib.musr_fit_result()
        r.cov = _dptr(cov)
        st = _lib.load().musr_fit(self.handle, int(obj), _dptr(th),
                                  fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                  ctypes.byref(o), ctypes.byref(r))
        info = {"value": r.value, "ndf": r.ndf, "edm": r.edm, "mu": r.mu, "iters": r.iters,
                "evals": r.n_evals, "status": st}
        return th, info, cov


def _make_chi2_function():
    import torch

    class Chi2(torch.autograd.Function):
        """Objective value with the adjoint kernel's gradient as its backward.

        forward(theta [P] CUDA FP64, run, obj) -> scalar; one launch computes the
        value and d obj / d theta together; backward returns grad_out * grad.
        """

        @staticmethod
        def forward(ctx, theta, run, obj=MUSR_CHI2):
            theta = theta.detach().contiguous()
            out = torch.empty(1 + run.P, dtype=torch.float64, device=theta.device)
            run.chi2_grad_device(theta, out, obj, MUSR_VALUE_GRAD)
            ctx.save_for_backward(out[1:])
            return out[0].clone()

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g, None, None

    return Chi2


class _LazyChi2:
    _fn = None

    def __getattr__(self, name):
        if _LazyChi2._fn is None:
            _LazyChi2._fn = _make_chi2_function()
        return getattr(_LazyChi2._fn, name)


Chi2 = _LazyChi2()


class Batch:
    """A batched-evaluation plan over several runs (musr_batch_*).

    ``max_vec[r]`` parameter vectors of run r are evaluated per launch; the
    first evaluation autotunes the launch shape.
    """

    def __init__(self, runs, max_vec):
        lib = _lib.load()
        self.runs = list(runs)
        self.max_vec = np.ascontiguousarray(max_vec, dtype=np.int32)
        handles = (ctypes.c_void_p * len(self.runs))(*[r.handle.value for r in self.runs])
        h = ctypes.c_void_p()
        check(lib.musr_batch_create(handles, len(self.runs),
                                    self.max_vec.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    ctypes.byref(h)), "musr_batch_create")
        self.handle = h
        self.n_values = int(self.max_vec.sum())
        self.n_theta = int(sum(int(v) * r.P for v, r in zip(self.max_vec, self.runs)))

    def eval(self, thetas, obj=MUSR_CHI2, n_vec=None):
        th = np.ascontiguousarray(thetas, dtype=np.float64).ravel()
        nv = self.max_vec if n_vec is None else np.ascontiguousarray(n_vec, dtype=np.int32)
        out = np.zeros(int(nv.sum()))
        check(_lib.load().musr_batch_eval(self.handle, int(obj), _dptr(th),
                                          nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(out)),
              "musr_batch_eval")
        return out

    def eval_device(self, thetas_dev, values_dev, obj=MUSR_CHI2):
        """thetas_dev / values_dev: CUDA FP64 tensors (every run at max_vec vectors)."""
        check(_lib.load().musr_batch_eval_device(self.handle, int(obj),
                                                 ctypes.c_void_p(thetas_dev.data_ptr()),
                                                 ctypes.c_void_p(values_dev.data_ptr())),
              "musr_batch_eval_device")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.load().musr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def poisson_sample(mu_dev, seed, counts_dev, stream=None):
    """counts_dev[i] ~ Poisson(mu_dev[i]) (CUDA FP32 in, CUDA int32 out)."""
    st = ctypes.c_void_p(int(stream)) if stream is not None else _torch_stream_ptr()
    check(_lib.load().musr_poisson_sample(ctypes.c_void_p(mu_dev.data_ptr()), int(mu_dev.numel()),
                                          int(seed) & 0xffffffffffffffff,
                                          ctypes.c_void_p(counts_dev.data_ptr()), st),
          "musr_poisson_sample")


def chi2_batch(runs, thetas, n_vec, obj=MUSR_CHI2):
    """One-shot musr_chi2_batch: plan, evaluate, free."""
    lib = _lib.load()
    handles = (ctypes.c_void_p * len(runs))(*[r.handle.value for r in runs])
    nv = np.ascontiguousarray(n_vec, dtype=np.int32)
    th = np.ascontiguousarray(thetas, dtype=np.float64).ravel()
    out = np.zeros(int(nv.sum()))
    check(lib.musr_chi2_batch(handles, len(runs), int(obj), _dptr(th),
                              nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(out)),
          "musr_chi2_batch")
    return out
