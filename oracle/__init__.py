"""FP64 CPU oracle for the muSR fit objective (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may import this package.  The GPU library never does, and
this package never imports the GPU library: the two share no code.

The arithmetic lives in ``musr_oracle.c`` (plain C, FP64, Neumaier sums),
built on demand with gcc into ``liboracle.so`` beside it.  Each wrapper below
states the passage of the paper it follows; see the C file's header for the
readings taken where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "musr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ENONFINITE, EDOMAIN, ENOCONV = 0, -1, -2, -4, -5, -7
CHI2, POISSON = 0, 1


def build(force: bool = False) -> str:
    """Compile musr_oracle.c with gcc (OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            lp = ctypes.POINTER(ctypes.c_int64)
            layout = [ctypes.c_int, lp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, ctypes.c_int, ip]
            lib.orc_model.argtypes = layout + [dp, dp]
            lib.orc_objective.argtypes = layout + [dp, dp, ctypes.c_int, dp]
            lib.orc_gradient.argtypes = layout + [dp, dp, ctypes.c_int, dp, dp, dp]
            lib.orc_gradient_fd.argtypes = layout + [dp, dp, ctypes.c_int, ctypes.c_double, dp]
            lib.orc_fit.argtypes = layout + [dp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_uint8),
                                             ctypes.c_int, ctypes.c_double, dp, dp]
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.orc_philox4x32_10.restype = None
            lib.orc_poisson.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_int32)]
            lib.orc_poisson.restype = None
            lib.orc_rebinned_mean.argtypes = layout + [dp, ctypes.c_int, ctypes.c_int, dp]
            lib.orc_sample_thetas.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                              ctypes.c_uint64, dp, ctypes.POINTER(ctypes.c_float)]
            lib.orc_sample_thetas.restype = None
            for f in (lib.orc_model, lib.orc_objective, lib.orc_gradient, lib.orc_gradient_fd,
                      lib.orc_fit, lib.orc_rebinned_mean):
                f.restype = ctypes.c_int
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_num_threads.argtypes = [ctypes.c_int]
            lib.orc_set_num_threads.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _layout_args(lay):
    nb = np.ascontiguousarray(lay.n_bins, dtype=np.int64)
    mp = np.ascontiguousarray(lay.map, dtype=np.int32)
    cp = np.asarray(lay.comp, dtype=np.int32)
    cp = cp.reshape(-1, cp.shape[-1] if cp.ndim == 2 and cp.shape[0] else 7)
    if cp.shape[1] == 6:  # rows without the stretched line's beta column
        cp = np.concatenate([cp, np.full((cp.shape[0], 1), -1, dtype=np.int32)], axis=1)
    cp = np.ascontiguousarray(cp)
    keep = (nb, mp, cp)
    args = [lay.n_hist, nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), lay.t0_us, lay.dt_us,
            lay.tau_us, lay.gamma, lay.n_params, lay.map_width,
            mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), lay.n_comp,
            cp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))]
    return args, keep


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle status {code}")
        self.code = code


def num_threads() -> int:
    return int(_load().orc_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the oracle's following calls."""
    _load().orc_set_num_threads(int(n))


def model(lay, theta) -> np.ndarray:
    """Eq. 1 theory N^j(t_n) for every bin of every histogram (FP64)."""
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.zeros(lay.total_bins)
    st = lib.orc_model(*args, _dp(th), _dp(out))
    if st:
        raise OracleError(st)
    return out


def objective(lay, data, theta, obj=CHI2, raise_on_error=True):
    """Eq. 3 chi2 (sigma^2 = max(d, 1)) or Eq. 4 Poisson deviance, FP64 compensated."""
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    d = np.ascontiguousarray(data, dtype=np.float64)
    v = np.zeros(1)
    st = lib.orc_objective(*args, _dp(d), _dp(th), int(obj), _dp(v))
    if st and raise_on_error:
        raise OracleError(st)
    return (float(v[0]), st) if not raise_on_error else float(v[0])


def gradient(lay, data, theta, obj=CHI2, with_gn=True):
    """Value, analytic gradient and Gauss-Newton matrix (FP64)."""
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    d = np.ascontiguousarray(data, dtype=np.float64)
    P = lay.n_params
    v = np.zeros(1)
    g = np.zeros(P)
    H = np.zeros((P, P)) if with_gn else None
    st = lib.orc_gradient(*args, _dp(d), _dp(th), int(obj), _dp(v), _dp(g),
                          _dp(H) if with_gn else None)
    if st:
        raise OracleError(st)
    return float(v[0]), g, H


def gradient_fd(lay, data, theta, obj=CHI2, rel_h=1e-6):
    """Central finite differences of the objective, h = rel_h * max(|theta_j|, 1)."""
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    d = np.ascontiguousarray(data, dtype=np.float64)
    g = np.zeros(lay.n_params)
    st = lib.orc_gradient_fd(*args, _dp(d), _dp(th), int(obj), float(rel_h), _dp(g))
    if st:
        raise OracleError(st)
    return g


def fit(lay, data, theta0, obj=CHI2, free=None, max_iter=500, edm_tol=1e-8):
    """Levenberg-Marquardt fit over the free parameters (FP64).

    Returns (theta, stats dict, covariance of the free parameters).
    """
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(theta0, dtype=np.float64).copy()
    d = np.ascontiguousarray(data, dtype=np.float64)
    fm = np.ascontiguousarray(lay.free if free is None else free, dtype=np.uint8)
    nf = int(fm.sum())
    stats = np.zeros(8)
    cov = np.zeros((nf, nf))
    st = lib.orc_fit(*args, _dp(d), int(obj), _dp(th),
                     fm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), int(max_iter),
                     float(edm_tol), _dp(stats), _dp(cov))
    info = {"value": stats[0], "ndf": stats[1], "iters": int(stats[2]), "evals": int(stats[3]),
            "edm": stats[4], "mu": stats[5], "status": int(st)}
    return th, info, cov


def philox4x32_10(counter, key):
    """Philox4x32-10 block for a 4-word counter and 2-word key (Salmon et al. 2011)."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xffffffff for x in counter])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def poisson(mu, seed):
    """Poisson variates for FP32 means mu[i] (inversion below 12, PTRS above)."""
    lib = _load()
    m = np.ascontiguousarray(mu, dtype=np.float32)
    out = np.zeros(m.shape[0], dtype=np.int32)
    lib.orc_poisson(m.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), m.shape[0], int(seed),
                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


def rebinned_mean(lay, thetas, rebin):
    """Sums of the Eq. 1 theory over groups of `rebin` bins, per parameter vector (FP64)."""
    lib = _load()
    args, keep = _layout_args(lay)
    th = np.ascontiguousarray(np.atleast_2d(thetas), dtype=np.float64)
    per = int(sum((int(m) + rebin - 1) // rebin for m in lay.n_bins))
    out = np.zeros(th.shape[0] * per)
    st = lib.orc_rebinned_mean(*args, _dp(th), th.shape[0], int(rebin), _dp(out))
    if st:
        raise OracleError(st)
    return out.reshape(th.shape[0], per)


def sample_thetas(lo, hi, n, seed, offset=0):
    """Uniform training parameter vectors of the learned start proposer and
    their targets 2u - 1 (entries with hi > lo; others fixed at lo)."""
    lib = _load()
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    hi = np.ascontiguousarray(hi, dtype=np.float64)
    P = lo.shape[0]
    th = np.zeros((n, P))
    tg = np.zeros((n, int((hi > lo).sum())), dtype=np.float32)
    lib.orc_sample_thetas(_dp(lo), _dp(hi), P, int(n), int(seed), int(offset), _dp(th),
                          tg.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return th, tg


def rebin_sums(lay, data, rebin):
    """Counts summed over groups of `rebin` bins, per histogram in order, the
    last group of a histogram possibly short (FP64); list of arrays per histogram."""
    d = np.asarray(data, dtype=np.float64)
    out, o = [], 0
    for m in lay.n_bins:
        m = int(m)
        h = d[o:o + m]
        o += m
        out.append(np.array([h[g0:g0 + rebin].sum() for g0 in range(0, m, rebin)]))
    return out


def proposer_features(lay, data, rebin, mu=None, inv_sigma=None):
    """Input features of the learned start proposer (FP64): for every group g
    of histogram k, log(1 + c_kg) - log(1 + C_k), then log(1 + C_k) for every
    k, with C_k the histogram's total; standardised as (x - mu) * inv_sigma
    when those are given."""
    sums = rebin_sums(lay, data, rebin)
    tot = np.array([s.sum() for s in sums])
    u = np.concatenate([np.log1p(s) - np.log1p(t) for s, t in zip(sums, tot)])
    x = np.concatenate([u, np.log1p(tot)])
    if mu is not None:
        x = (x - np.asarray(mu, dtype=np.float64)) * np.asarray(inv_sigma, dtype=np.float64)
    return x
