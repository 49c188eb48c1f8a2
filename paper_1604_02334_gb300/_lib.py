"""ctypes binding of libmusr.so: the C ABI of include/musr.h, same names.

Argument marshalling only: every step of the evaluation runs in the
library's CUDA kernels.  Importing this module fails loudly if libmusr.so
has not been built (``python -m paper_1604_02334_gb300.build``); there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmusr.so")

MUSR_OK = 0
MUSR_EINVAL = -1
MUSR_ENOMEM = -2
MUSR_ECUDA = -3
MUSR_ENONFINITE = -4
MUSR_EDOMAIN = -5
MUSR_ETIMEOUT = -6
MUSR_ENOCONV = -7
MUSR_ENOTSUP = -8

MUSR_TF_EXP, MUSR_TF_GAUSS, MUSR_KT_STATIC_GAUSS, MUSR_TF_STRETCHED = 0, 1, 2, 3
MUSR_CHI2, MUSR_POISSON = 0, 1
MUSR_F32, MUSR_F64 = 0, 1
MUSR_VALUE, MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN = 0, 1, 2
MUSR_FIT_LM, MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD = 0, 1, 2
MUSR_NOALLOC_SCRATCH_BYTES = 32 << 20
MUSR_NOALLOC_MAX_HIST = 64
MUSR_NOALLOC_MAX_PARAMS = 256
MUSR_RATE_NAMES = ("ffma", "ffma2", "ex2", "sin", "cos", "rcp", "lg2")
MUSR_RATE_COUNT = len(MUSR_RATE_NAMES)
MUSR_GAMMA_MU_MHZ_PER_G = 0.013554
MUSR_TAU_MU_US = 2.197


class musr_component(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("kind", "amp", "rate", "field", "field2", "phase", "beta")]


class musr_run_desc(ctypes.Structure):
    _fields_ = [
        ("n_hist", ctypes.c_int32),
        ("n_bins", ctypes.POINTER(ctypes.c_int64)),
        ("t0_us", ctypes.c_double),
        ("dt_us", ctypes.c_double),
        ("tau_us", ctypes.c_double),
        ("gamma_mhz_per_g", ctypes.c_double),
        ("n_params", ctypes.c_int32),
        ("map_width", ctypes.c_int32),
        ("map", ctypes.POINTER(ctypes.c_int32)),
        ("n_comp", ctypes.c_int32),
        ("comp", ctypes.POINTER(musr_component)),
        ("data_dtype", ctypes.c_int32),
        ("data", ctypes.c_void_p),
        ("data_on_device", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("n_funcs", ctypes.c_int32),
        ("funcs", ctypes.POINTER(ctypes.c_char_p)),
    ]


class musr_fit_opts(ctypes.Structure):
    _fields_ = [
        ("method", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("edm_tol", ctypes.c_double),
        ("mu0", ctypes.c_double),
        ("fd_rel_h", ctypes.c_double),
    ]


class musr_fit_result(ctypes.Structure):
    _fields_ = [
        ("value", ctypes.c_double),
        ("ndf", ctypes.c_double),
        ("edm", ctypes.c_double),
        ("mu", ctypes.c_double),
        ("iters", ctypes.c_int32),
        ("n_evals", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("n_free", ctypes.c_int32),
        ("cov", ctypes.POINTER(ctypes.c_double)),
    ]


class musr_proposer_opts(ctypes.Structure):
    _fields_ = [
        ("rebin", ctypes.c_int32),
        ("n_hidden", ctypes.c_int32),
        ("n_hidden_layers", ctypes.c_int32),
        ("batch", ctypes.c_int32),
        ("in_scale", ctypes.c_float),
        ("seed", ctypes.c_uint64),
        ("box_margin", ctypes.c_float),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_vp = ctypes.c_void_p
_run = ctypes.c_void_p

# name -> (restype, argtypes); the complete list of symbols include/musr.h declares
SIGNATURES = {
    "musr_create_run": (ctypes.c_int, [ctypes.POINTER(musr_run_desc), ctypes.POINTER(_run)]),
    "musr_destroy_run": (ctypes.c_int, [_run]),
    "musr_run_info": (ctypes.c_int, [_run, _i32p, ctypes.POINTER(ctypes.c_int64), _i32p]),
    "musr_set_data": (ctypes.c_int, [_run, ctypes.c_int32, _vp, ctypes.c_int32]),
    "musr_chi2": (ctypes.c_int, [_run, ctypes.c_int, _dp, _dp]),
    "musr_chi2_grad": (ctypes.c_int, [_run, ctypes.c_int, _dp, _dp, _dp, _dp]),
    "musr_chi2_grad_device": (ctypes.c_int, [_run, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "musr_chi2_grad_async": (ctypes.c_int, [_run, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "musr_model": (ctypes.c_int, [_run, _dp, _vp, ctypes.c_int32]),
    "musr_chi2_batch": (ctypes.c_int, [ctypes.POINTER(_run), ctypes.c_int32, ctypes.c_int, _dp,
                                       _i32p, _dp]),
    "musr_batch_create": (ctypes.c_int, [ctypes.POINTER(_run), ctypes.c_int32, _i32p,
                                         ctypes.POINTER(_vp)]),
    "musr_batch_destroy": (ctypes.c_int, [_vp]),
    "musr_batch_eval": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _i32p, _dp]),
    "musr_batch_eval_device": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp]),
    "musr_fit": (ctypes.c_int, [_run, ctypes.c_int, _dp, _u8p, ctypes.POINTER(musr_fit_opts),
                                ctypes.POINTER(musr_fit_result)]),
    "musr_gbatch_create": (ctypes.c_int, [ctypes.POINTER(_run), ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(_vp)]),
    "musr_gbatch_destroy": (ctypes.c_int, [_vp]),
    "musr_gbatch_eval": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _dp, _u8p, _dp, _i32p]),
    "musr_gbatch_eval_device": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp]),
    "musr_fit_batch": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _u8p, ctypes.POINTER(musr_fit_opts),
                                      ctypes.POINTER(musr_fit_result)]),
    "musr_fit_multistart_batch": (ctypes.c_int, [ctypes.POINTER(_run), ctypes.c_int32, ctypes.c_int, _dp,
                                                 ctypes.c_int32, _u8p, ctypes.POINTER(musr_fit_opts), _dp,
                                                 ctypes.POINTER(musr_fit_result)]),
    "musr_fit_learned_batch": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _u8p, ctypes.POINTER(musr_fit_opts),
                                              ctypes.c_double, _dp, ctypes.c_int32, _dp,
                                              ctypes.POINTER(musr_fit_result), _i32p]),
    "musr_fit_multistart": (ctypes.c_int, [_run, ctypes.c_int, _dp, ctypes.c_int32, _u8p,
                                           ctypes.POINTER(musr_fit_opts), _dp, ctypes.POINTER(musr_fit_result)]),
    "musr_proposer_create": (ctypes.c_int, [_run, _dp, _dp, ctypes.POINTER(musr_proposer_opts),
                                            ctypes.POINTER(_vp)]),
    "musr_proposer_destroy": (ctypes.c_int, [_vp]),
    "musr_proposer_mlp": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "musr_proposer_sample": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_uint64, _vp, _vp, _vp]),
    "musr_proposer_features": (ctypes.c_int, [_vp, ctypes.POINTER(_run), ctypes.c_int32, _vp, _vp]),
    "musr_proposer_info": (ctypes.c_int, [_vp, _i32p, _i32p, _i32p]),
    "musr_proposer_get_norm": (ctypes.c_int, [_vp, _fp, _fp]),
    "musr_proposer_set_norm": (ctypes.c_int, [_vp, _fp, _fp]),
    "musr_proposer_train": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _fp]),
    "musr_proposer_propose": (ctypes.c_int, [_vp, ctypes.POINTER(_run), ctypes.c_int32, _dp]),
    "musr_fit_learned": (ctypes.c_int, [_vp, _run, ctypes.c_int, _u8p, ctypes.POINTER(musr_fit_opts),
                                        ctypes.c_double, _dp, ctypes.c_int32, _dp,
                                        ctypes.POINTER(musr_fit_result), _i32p]),
    "musr_poisson_sample": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_uint64, _vp, _vp]),
    "musr_generate": (ctypes.c_int, [_run, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_int32, _vp, _vp, _vp]),
    "musr_gemm_bf16": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _vp,
                                      ctypes.c_int32, _vp, _vp, ctypes.c_int32, _vp, ctypes.c_int64, _vp, _vp]),
    "musr_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "musr_mlp_destroy": (ctypes.c_int, [_vp]),
    "musr_mlp_n_params": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64)]),
    "musr_mlp_set_params": (ctypes.c_int, [_vp, _fp]),
    "musr_mlp_get_params": (ctypes.c_int, [_vp, _fp]),
    "musr_mlp_get_grads": (ctypes.c_int, [_vp, _fp]),
    "musr_mlp_get_activation": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, _fp]),
    "musr_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp]),
    "musr_mlp_backward": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _vp]),
    "musr_mlp_adam": (ctypes.c_int, [_vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp]),
    "musr_mlp_train_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_float,
                                           ctypes.POINTER(ctypes.c_float), _vp]),
    "musr_utheory_create": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_vp)]),
    "musr_utheory_destroy": (ctypes.c_int, [_vp]),
    "musr_utheory_log": (ctypes.c_char_p, [_vp]),
    "musr_utheory_eval": (ctypes.c_int, [_vp, _run, ctypes.c_int, _dp, _dp, ctypes.c_int32, _dp]),
    "musr_utheory_grad": (ctypes.c_int, [_vp, _run, ctypes.c_int, _dp, _dp, _u8p, ctypes.c_double, _dp, _dp]),
    "musr_utheory_fit": (ctypes.c_int, [_vp, _run, ctypes.c_int, _dp, _dp, _u8p, ctypes.POINTER(musr_fit_opts),
                                        ctypes.POINTER(musr_fit_result)]),
    "musr_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "musr_version": (ctypes.c_char_p, []),
    "musr_function_eval": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int32, _vp, _vp, _vp]),
    "musr_last_cuda_error": (ctypes.c_char_p, []),
    "musr_chi2_grad_noalloc": (ctypes.c_int, [ctypes.POINTER(musr_run_desc), ctypes.c_int, ctypes.c_int,
                                              _vp, _vp, _vp, _vp]),
    "musr_pipe_rates": (ctypes.c_int, [_dp, ctypes.c_int32]),
    "musr_fit_eval": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, _vp, _vp, _dp, _u8p,
                                     ctypes.POINTER(musr_fit_opts), ctypes.POINTER(musr_fit_result)]),
}

# int eval(void* user, int mode, const double* theta, double* value, double* grad, double* gn)
musr_eval_fn = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, _dp, _dp, _dp, _dp)

_lib = None


def load():
    """Load libmusr.so and declare every entry point (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -m paper_1604_02334_gb300.build` "
                "(the library has no CPU fallback)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class MusrError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        msg = load().musr_strerror(code).decode()
        if code in (MUSR_ECUDA, MUSR_ENOMEM):
            msg += " [" + load().musr_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {msg} ({code})" if where else f"{msg} ({code})")
        self.code = code


def check(code: int, where: str = "") -> int:
    if code != MUSR_OK:
        raise MusrError(code, where)
    return code


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(load(), name)
    raise AttributeError(name)
