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


def _comp_rows(comp) -> np.ndarray:
    """Component table as C x 7 int32 rows (a 6-column table gets beta = -1)."""
    c = np.asarray(comp, dtype=np.int32)
    c = c.reshape(-1, c.shape[-1] if c.ndim == 2 and c.shape[0] else 7)
    if c.shape[1] == 6:
        c = np.concatenate([c, np.full((c.shape[0], 1), -1, dtype=np.int32)], axis=1)
    if c.shape[1] != 7:
        raise ValueError("component rows need 6 or 7 columns")
    return np.ascontiguousarray(c)


class Run:
    """A run: K histograms on the device plus their layout (Sec. 4.1 Eq. 1-2).

    ``layout`` is any object with the attributes n_bins, t0_us, dt_us,
    tau_us, gamma, n_params, map (K x W int32) and comp (C x 7 int32:
    kind, amp, rate, field, field2, phase, beta map columns; C x 6 without
    beta is accepted), and optionally funcs (a list of function-array
    expressions over p[i]; map entries -2 - j read function j).  ``data`` is a numpy
    array (FP32 / FP64) or a CUDA torch tensor of sum(n_bins) counts, or None.
    ``stream``: 'torch' to work on torch's current stream, None for a stream
    of the run's own.
    """

    def __init__(self, layout, data=None, stream=None):
        lib = _lib.load()
        self.layout = layout
        self._nb = np.ascontiguousarray(layout.n_bins, dtype=np.int64)
        self._map = np.ascontiguousarray(layout.map, dtype=np.int32)
        comp = _comp_rows(layout.comp)
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
        funcs = [str(f).encode() for f in (getattr(layout, "funcs", None) or [])]
        self._funcs = (ctypes.c_char_p * max(1, len(funcs)))(*funcs)
        d.n_funcs = len(funcs)
        d.funcs = ctypes.cast(self._funcs, ctypes.POINTER(ctypes.c_char_p)) if funcs else None
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

    def chi2_grad_async(self, theta, out_dev, obj=MUSR_CHI2, mode=MUSR_VALUE_GRAD, status_dev=None,
                        stream=None):
        """theta: host FP64 vector [P], passed by value (reusable on return);
        out_dev: CUDA FP64 tensor, 1 (+P (+P*P)) long; queued on the stream."""
        # plain integers for the pointers: this call is made once per queued
        # evaluation and its host cost bounds the queue's rate
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if th.shape != (self.P,):
            raise ValueError(f"theta must hold {self.P} values")
        st = int(stream) if stream is not None else _torch_stream_ptr()
        rc = _lib.load().musr_chi2_grad_async(self.handle, int(obj), int(mode), th.ctypes.data, out_dev.data_ptr(),
                                             status_dev.data_ptr() if status_dev is not None else None, st)
        if rc:
            check(rc, "musr_chi2_grad_async")

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

    def fit_multistart(self, starts, obj=MUSR_CHI2, free=None, method=MUSR_FIT_LM, max_iter=500,
                       edm_tol=1e-8, mu0=1e-3, fd_rel_h=0.0):
        """musr_fit_multistart: the best of the fits from each row of starts."""
        st_ = np.ascontiguousarray(np.atleast_2d(starts), dtype=np.float64)
        assert st_.shape[1] == self.P
        fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        nf = self.P if fm is None else int(fm.sum())
        cov = np.zeros((nf, nf))
        th = np.zeros(self.P)
        o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, fd_rel_h)
        r = _lib.musr_fit_result()
        r.cov = _dptr(cov)
        st = _lib.load().musr_fit_multistart(self.handle, int(obj), _dptr(st_), st_.shape[0],
                                             fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                                             if fm is not None else None,
                                             ctypes.byref(o), _dptr(th), ctypes.byref(r))
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


def pipe_rates():
    """musr_pipe_rates: measured thread-level operations per second of the
    current device's FP32 FMA (scalar and packed pairs) and SFU ex2, sin, cos,
    rcp, lg2, as a dict keyed by those names."""
    out = np.zeros(_lib.MUSR_RATE_COUNT)
    check(_lib.load().musr_pipe_rates(_dptr(out), out.shape[0]), "musr_pipe_rates")
    return dict(zip(_lib.MUSR_RATE_NAMES, (float(x) for x in out)))


def function_eval(expr, theta):
    """musr_function_eval: (value, gradient) of one function-array expression at theta (host only)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    v = ctypes.c_double()
    g = np.zeros(th.shape[0])
    check(_lib.load().musr_function_eval(str(expr).encode(), th.shape[0], _dptr(th) if th.shape[0] else None,
                                         ctypes.byref(v), _dptr(g) if th.shape[0] else None),
          "musr_function_eval")
    return v.value, g


def gemm_bf16(a, b, bias=None, relu=False, out_f32=None, out_bf16=None, err=None, stream=None, ws=None):
    """out = act(a @ b.T + bias) on the tensor cores; a [m, k], b [n, k] CUDA bf16.
    ws: optional CUDA float32 scratch that enables split-K for products with few output tiles."""
    import torch
    m, k = a.shape
    n = b.shape[0]
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=a.device)
    ldc = (out_f32 if out_f32 is not None else out_bf16).shape[1]
    st = ctypes.c_void_p(int(stream)) if stream is not None else _torch_stream_ptr()
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    check(_lib.load().musr_gemm_bf16(p(a), p(b), m, n, k, p(bias), 1 if relu else 0, p(out_f32), p(out_bf16),
                                     ldc, p(ws), ws.numel() if ws is not None else 0, p(err), st),
          "musr_gemm_bf16")
    return err


def _fit_infos(res):
    return [{"value": x.value, "ndf": x.ndf, "edm": x.edm, "mu": x.mu, "iters": x.iters, "evals": x.n_evals,
             "status": x.status} for x in res]


def fit_multistart_batch(runs, starts, obj=MUSR_CHI2, free=None, max_iter=500, edm_tol=1e-8, mu0=1e-3,
                         method=MUSR_FIT_LM):
    """musr_fit_multistart_batch: starts[r] is an (n_starts, P_r) array per run.
    Returns (list of theta, list of info dicts)."""
    runs = list(runs)
    n_starts = int(np.asarray(starts[0]).shape[0])
    flat = np.ascontiguousarray(np.concatenate([np.asarray(st_, dtype=np.float64).reshape(n_starts, -1).ravel()
                                                for st_ in starts]))
    fm = None
    if free is not None:
        fm = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.uint8).ravel() for f in free]))
    out = np.zeros(sum(r.P for r in runs))
    o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, 0.0)
    res = (_lib.musr_fit_result * len(runs))()
    handles = (ctypes.c_void_p * len(runs))(*[r.handle.value for r in runs])
    st = _lib.load().musr_fit_multistart_batch(handles, len(runs), int(obj), _dptr(flat), n_starts,
                                               fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                                               if fm is not None else None, ctypes.byref(o), _dptr(out), res)
    if st not in (0, -7, -5, -4):
        check(st, "musr_fit_multistart_batch")
    offs = np.r_[0, np.cumsum([r.P for r in runs])]
    return [out[offs[i]:offs[i + 1]].copy() for i in range(len(runs))], _fit_infos(res)


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


class Mlp:
    """The learned start proposer's network (musr_mlp_*): BF16 tensor-core
    layers n_in -> n_hidden (x n_hidden_layers, ReLU) -> n_out, FP32 master
    weights, Adam.  Inputs, targets and outputs are CUDA FP32 tensors."""

    def __init__(self, n_in, n_hidden, n_hidden_layers, n_out, max_batch, in_scale=1.0, seed=0):
        self._lib = _lib.load()
        self.handle = ctypes.c_void_p()
        check(self._lib.musr_mlp_create(n_in, n_hidden, n_hidden_layers, n_out, max_batch, float(in_scale),
                                        int(seed), ctypes.byref(self.handle)), "musr_mlp_create")
        self.n_in, self.n_hidden, self.n_hidden_layers, self.n_out = n_in, n_hidden, n_hidden_layers, n_out
        n = ctypes.c_int64()
        check(self._lib.musr_mlp_n_params(self.handle, ctypes.byref(n)), "musr_mlp_n_params")
        self.n_params = int(n.value)

    def layer_shapes(self):
        """[(out, in)] per layer, in the order of the flat parameter vector."""
        dims = [self.n_in] + [self.n_hidden] * self.n_hidden_layers + [self.n_out]
        return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]

    def _flat(self, fn):
        out = np.zeros(self.n_params, dtype=np.float32)
        check(fn(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "musr_mlp params")
        return out

    def get_params(self):
        return self._flat(self._lib.musr_mlp_get_params)

    def get_grads(self):
        return self._flat(self._lib.musr_mlp_get_grads)

    def set_params(self, flat):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        assert f.shape == (self.n_params,)
        check(self._lib.musr_mlp_set_params(self.handle, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_mlp_set_params")

    def _check_x(self, x, width):
        import torch
        if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.dim() != 2 or x.shape[1] != width:
            raise ValueError(f"expected a contiguous CUDA float32 tensor [batch, {width}]")

    def activation(self, layer, batch):
        """Layer `layer`'s activations of the last forward pass, host FP32."""
        w = self.n_in if layer == 0 else (self.n_out if layer == self.n_hidden_layers + 1 else self.n_hidden)
        out = np.zeros((batch, w), dtype=np.float32)
        check(self._lib.musr_mlp_get_activation(self.handle, int(layer), int(batch),
                                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_mlp_get_activation")
        return out

    def forward(self, x, out=None):
        import torch
        self._check_x(x, self.n_in)
        b = x.shape[0]
        if out is None:
            out = torch.empty((b, self.n_out), dtype=torch.float32, device=x.device)
        check(self._lib.musr_mlp_forward(self.handle, ctypes.c_void_p(x.data_ptr()), b,
                                         ctypes.c_void_p(out.data_ptr()), _torch_stream_ptr()), "musr_mlp_forward")
        return out

    def backward(self, x, t):
        self._check_x(x, self.n_in)
        self._check_x(t, self.n_out)
        loss = ctypes.c_float()
        check(self._lib.musr_mlp_backward(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                          x.shape[0], ctypes.byref(loss), _torch_stream_ptr()), "musr_mlp_backward")
        return float(loss.value)

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        check(self._lib.musr_mlp_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps),
                                      _torch_stream_ptr()), "musr_mlp_adam")

    def train_step(self, x, t, lr):
        self._check_x(x, self.n_in)
        self._check_x(t, self.n_out)
        loss = ctypes.c_float()
        check(self._lib.musr_mlp_train_step(self.handle, ctypes.c_void_p(x.data_ptr()),
                                            ctypes.c_void_p(t.data_ptr()), x.shape[0], float(lr),
                                            ctypes.byref(loss), _torch_stream_ptr()), "musr_mlp_train_step")
        return float(loss.value)

    def close(self):
        if self.handle:
            self._lib.musr_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Proposer:
    """Learned start proposer (musr_proposer_*): an MLP trained on device-
    generated histograms of `layout`'s shape for parameters uniform in
    [lo, hi]; proposals for runs of that layout; learned-start fits."""

    def __init__(self, layout, lo, hi, rebin=64, n_hidden=512, n_hidden_layers=3, batch=512, in_scale=1.0,
                 seed=1, box_margin=0.25):
        self._lib = _lib.load()
        self.layout = layout  # keeps the layout run alive
        self.P = layout.P
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        assert self.lo.shape == (self.P,) and self.hi.shape == (self.P,)
        o = _lib.musr_proposer_opts(rebin, n_hidden, n_hidden_layers, batch, in_scale, seed, box_margin)
        self.handle = ctypes.c_void_p()
        check(self._lib.musr_proposer_create(layout.handle, _dptr(self.lo), _dptr(self.hi), ctypes.byref(o),
                                             ctypes.byref(self.handle)), "musr_proposer_create")
        self.batch = batch
        nf, nl, ni = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(self._lib.musr_proposer_info(self.handle, ctypes.byref(nf), ctypes.byref(nl), ctypes.byref(ni)),
              "musr_proposer_info")
        self.n_features, self.n_learned, self.n_inputs = int(nf.value), int(nl.value), int(ni.value)

    def norm(self):
        """(mu, inv_sigma) of the feature standardisation, FP32 host arrays."""
        mu = np.zeros(self.n_features, dtype=np.float32)
        isig = np.zeros(self.n_features, dtype=np.float32)
        check(self._lib.musr_proposer_get_norm(self.handle, mu.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               isig.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_proposer_get_norm")
        return mu, isig

    def set_norm(self, mu, inv_sigma):
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        isig = np.ascontiguousarray(inv_sigma, dtype=np.float32)
        check(self._lib.musr_proposer_set_norm(self.handle, mu.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                               isig.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_proposer_set_norm")

    def sample(self, n, offset=0, with_targets=True):
        """Training parameter vectors (and targets) for sample indices offset.., CUDA tensors."""
        import torch
        th = torch.empty((n, self.P), dtype=torch.float64, device="cuda")
        n_learned = int((self.hi > self.lo).sum())
        tg = torch.empty((n, n_learned), dtype=torch.float32, device="cuda") if with_targets else None
        check(self._lib.musr_proposer_sample(self.handle, int(n), int(offset), ctypes.c_void_p(th.data_ptr()),
                                             ctypes.c_void_p(tg.data_ptr()) if tg is not None else None,
                                             _torch_stream_ptr()), "musr_proposer_sample")
        return th, tg

    def features(self, runs):
        """The network's input rows (standardised log counts) for runs, CUDA FP32 [len(runs), n_features]."""
        import torch
        runs = list(runs)
        n_features = self.n_features
        handles = (ctypes.c_void_p * len(runs))(*[r.handle.value for r in runs])
        out = torch.empty((len(runs), n_features), dtype=torch.float32, device="cuda")
        check(self._lib.musr_proposer_features(self.handle, handles, len(runs), ctypes.c_void_p(out.data_ptr()),
                                               _torch_stream_ptr()), "musr_proposer_features")
        return out

    def train(self, n_steps, lr_start=1e-3, lr_end=1e-4):
        losses = np.zeros(max(int(n_steps), 1), dtype=np.float32)
        check(self._lib.musr_proposer_train(self.handle, int(n_steps), float(lr_start), float(lr_end),
                                            losses.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_proposer_train")
        return losses[:int(n_steps)]

    def mlp_params(self):
        """The network's flat FP32 parameter vector (host copy)."""
        m = ctypes.c_void_p()
        check(self._lib.musr_proposer_mlp(self.handle, ctypes.byref(m)), "musr_proposer_mlp")
        n = ctypes.c_int64()
        check(self._lib.musr_mlp_n_params(m, ctypes.byref(n)), "musr_mlp_n_params")
        out = np.zeros(int(n.value), dtype=np.float32)
        check(self._lib.musr_mlp_get_params(m, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
              "musr_mlp_get_params")
        return out

    def propose(self, runs):
        runs = list(runs)
        handles = (ctypes.c_void_p * len(runs))(*[r.handle.value for r in runs])
        out = np.zeros((len(runs), self.P))
        check(self._lib.musr_proposer_propose(self.handle, handles, len(runs), _dptr(out)), "musr_proposer_propose")
        return out

    def fit(self, run, obj=MUSR_CHI2, free=None, chi2ndf_max=1.2, fallback_starts=None, method=MUSR_FIT_LM,
            max_iter=500, edm_tol=1e-8, mu0=1e-3, fd_rel_h=0.0):
        """musr_fit_learned: (theta, info, cov); info["fallback"] tells whether the plain fit ran."""
        fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        nf = self.P if fm is None else int(fm.sum())
        cov = np.zeros((nf, nf))
        th = np.zeros(self.P)
        fb = None if fallback_starts is None else np.ascontiguousarray(np.atleast_2d(fallback_starts),
                                                                       dtype=np.float64)
        o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, fd_rel_h)
        r = _lib.musr_fit_result()
        r.cov = _dptr(cov)
        used = ctypes.c_int32()
        st = self._lib.musr_fit_learned(self.handle, run.handle, int(obj),
                                        fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                        ctypes.byref(o), float(chi2ndf_max), _dptr(fb) if fb is not None else None,
                                        0 if fb is None else fb.shape[0], _dptr(th), ctypes.byref(r),
                                        ctypes.byref(used))
        info = {"value": r.value, "ndf": r.ndf, "edm": r.edm, "mu": r.mu, "iters": r.iters,
                "evals": r.n_evals, "status": st, "fallback": bool(used.value), "fallback_stage": int(used.value)}
        return th, info, cov

    def fit_batch(self, gbatch, obj=MUSR_CHI2, free=None, chi2ndf_max=1.2, fallback_starts=None, max_iter=500,
                  edm_tol=1e-8, mu0=1e-3, method=MUSR_FIT_LM):
        """musr_fit_learned_batch over the runs of `gbatch` (a GBatch with GN):
        (list of theta, list of info dicts with "fallback")."""
        n = len(gbatch.runs)
        fm = None
        if free is not None:
            fm = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.uint8).ravel() for f in free]))
        fb, n_fb = None, 0
        if fallback_starts is not None:
            n_fb = int(np.asarray(fallback_starts[0]).shape[0])
            fb = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).reshape(n_fb, -1).ravel()
                                                      for x in fallback_starts]))
        out = np.zeros(int(gbatch.theta_off[-1]))
        o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, 0.0)
        res = (_lib.musr_fit_result * n)()
        used = np.zeros(n, dtype=np.int32)
        st = self._lib.musr_fit_learned_batch(self.handle, gbatch.handle, int(obj),
                                              fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
                                              if fm is not None else None, ctypes.byref(o), float(chi2ndf_max),
                                              _dptr(fb) if fb is not None else None, n_fb, _dptr(out), res,
                                              used.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if st not in (0, -7, -5, -4):
            check(st, "musr_fit_learned_batch")
        infos = _fit_infos(res)
        for i, u in zip(infos, used):
            i["fallback"] = bool(u)
            i["fallback_stage"] = int(u)
        offs = gbatch.theta_off
        return [out[offs[i]:offs[i + 1]].copy() for i in range(n)], infos

    def close(self):
        if self.handle:
            self._lib.musr_proposer_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GBatch:
    """Batched adjoint evaluation and lockstep LM fits of many runs
    (musr_gbatch_*, musr_fit_batch); one parameter vector per entry."""

    def __init__(self, runs, with_gn=True):
        self._lib = _lib.load()
        self.runs = list(runs)
        self.P = [r.P for r in self.runs]
        self.theta_off = np.r_[0, np.cumsum(self.P)].astype(np.int64)
        self.with_gn = bool(with_gn)
        handles = (ctypes.c_void_p * len(self.runs))(*[r.handle.value for r in self.runs])
        self.handle = ctypes.c_void_p()
        check(self._lib.musr_gbatch_create(handles, len(self.runs), 1 if with_gn else 0, ctypes.byref(self.handle)),
              "musr_gbatch_create")

    def out_sizes(self, mode):
        return [1 + p + (p * p if mode == MUSR_VALUE_GRAD_GN else 0) for p in self.P]

    def _flat(self, thetas):
        flat = np.concatenate([np.asarray(t, dtype=np.float64).ravel() for t in thetas])
        assert flat.shape[0] == self.theta_off[-1]
        return np.ascontiguousarray(flat)

    def eval(self, thetas, obj=MUSR_CHI2, mode=MUSR_VALUE_GRAD, active=None):
        """[(value, grad, gn or None) or None if inactive], flags."""
        flat = self._flat(thetas)
        sizes = self.out_sizes(mode)
        out = np.full(int(np.sum(sizes)), np.nan)
        flags = np.zeros(len(self.runs), dtype=np.int32)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        check(self._lib.musr_gbatch_eval(self.handle, int(obj), int(mode), _dptr(flat),
                                         act.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if act is not None else None,
                                         _dptr(out), flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
              "musr_gbatch_eval")
        res, o = [], 0
        for r, (p, n) in enumerate(zip(self.P, sizes)):
            if act is not None and not act[r]:
                res.append(None)
            else:
                v = out[o:o + n]
                res.append((float(v[0]), v[1:1 + p].copy(),
                            v[1 + p:].reshape(p, p).copy() if mode == MUSR_VALUE_GRAD_GN else None))
            o += n
        return res, flags

    def eval_device(self, thetas_dev, out_dev, obj=MUSR_CHI2, mode=MUSR_VALUE_GRAD, flags_dev=None, stream=None):
        st = ctypes.c_void_p(int(stream)) if stream is not None else _torch_stream_ptr()
        check(self._lib.musr_gbatch_eval_device(self.handle, int(obj), int(mode), ctypes.c_void_p(thetas_dev.data_ptr()),
                                                ctypes.c_void_p(out_dev.data_ptr()),
                                                ctypes.c_void_p(flags_dev.data_ptr()) if flags_dev is not None else None,
                                                st), "musr_gbatch_eval_device")

    def fit(self, thetas, obj=MUSR_CHI2, free=None, max_iter=500, edm_tol=1e-8, mu0=1e-3, method=MUSR_FIT_LM):
        """Lockstep fits (LM, or BFGS with method=MUSR_FIT_BFGS): (list of theta, list of info dicts)."""
        flat = self._flat(thetas)
        fm = None
        if free is not None:
            fm = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.uint8).ravel() for f in free]))
        o = _lib.musr_fit_opts(method, max_iter, edm_tol, mu0, 0.0)
        res = (_lib.musr_fit_result * len(self.runs))()
        st = self._lib.musr_fit_batch(self.handle, int(obj), _dptr(flat),
                                      fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                      ctypes.byref(o), res)
        if st not in (0, -7, -5, -4):
            check(st, "musr_fit_batch")
        ths = [flat[self.theta_off[r]:self.theta_off[r + 1]].copy() for r in range(len(self.runs))]
        infos = [{"value": x.value, "ndf": x.ndf, "edm": x.edm, "mu": x.mu, "iters": x.iters, "evals": x.n_evals,
                  "status": x.status} for x in res]
        return ths, infos

    def close(self):
        if self.handle:
            self._lib.musr_gbatch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UserTheory:
    """A user-defined asymmetry A_k(t) compiled at run time (musr_utheory_*):
    expr is a C expression over t, p, m and f (see include/musr.h)."""

    def __init__(self, expr, n_funcs=0, fp32=False):
        self._lib = _lib.load()
        self.n_funcs = int(n_funcs)
        self.fp32 = bool(fp32)
        self.handle = ctypes.c_void_p()
        st = self._lib.musr_utheory_create(expr.encode(), self.n_funcs, MUSR_F32 if fp32 else MUSR_F64,
                                           ctypes.byref(self.handle))
        if st != 0:
            log = self._lib.musr_utheory_log(None)
            raise MusrError(st, "musr_utheory_create" + (": " + log.decode(errors="replace") if log else ""))
        self.expr = expr

    @property
    def log(self):
        return self._lib.musr_utheory_log(self.handle).decode(errors="replace")

    def _funcs(self, funcs, n):
        if self.n_funcs == 0:
            return None
        f = np.ascontiguousarray(np.broadcast_to(np.asarray(funcs, dtype=np.float64), (n, self.n_funcs)))
        return f

    def eval(self, run, thetas, obj=MUSR_CHI2, funcs=None):
        th = np.ascontiguousarray(np.atleast_2d(thetas), dtype=np.float64)
        n = th.shape[0]
        f = self._funcs(funcs, n)
        out = np.zeros(n)
        check(self._lib.musr_utheory_eval(self.handle, run.handle, int(obj), _dptr(th),
                                          _dptr(f) if f is not None else None, n, _dptr(out)), "musr_utheory_eval")
        return out

    def grad(self, run, theta, obj=MUSR_CHI2, funcs=None, free=None, rel_h=1e-6):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        f = self._funcs(funcs, 1)
        fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        v = ctypes.c_double()
        g = np.zeros(th.shape[0])
        check(self._lib.musr_utheory_grad(self.handle, run.handle, int(obj), _dptr(th),
                                          _dptr(f) if f is not None else None,
                                          fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                          float(rel_h), ctypes.byref(v), _dptr(g)), "musr_utheory_grad")
        return float(v.value), g

    def fit(self, run, theta0, obj=MUSR_CHI2, funcs=None, free=None, max_iter=500, fd_rel_h=1e-4):
        th = np.ascontiguousarray(theta0, dtype=np.float64).copy()
        f = self._funcs(funcs, 1)
        fm = None if free is None else np.ascontiguousarray(free, dtype=np.uint8)
        nf = th.shape[0] if fm is None else int(fm.sum())
        cov = np.zeros((nf, nf))
        o = _lib.musr_fit_opts(MUSR_FIT_BFGS_FD, max_iter, 0.0, 0.0, fd_rel_h)
        r = _lib.musr_fit_result()
        r.cov = _dptr(cov)
        st = self._lib.musr_utheory_fit(self.handle, run.handle, int(obj), _dptr(th),
                                        _dptr(f) if f is not None else None,
                                        fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)) if fm is not None else None,
                                        ctypes.byref(o), ctypes.byref(r))
        info = {"value": r.value, "ndf": r.ndf, "edm": r.edm, "iters": r.iters, "evals": r.n_evals, "status": st}
        return th, info, cov

    def close(self):
        if self.handle:
            self._lib.musr_utheory_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
