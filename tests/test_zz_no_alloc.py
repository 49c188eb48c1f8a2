"""The allocation-free entry point, musr_chi2_grad_noalloc.

Some callers cannot allocate device memory -- for example a plug-in whose host
framework owns the whole device memory pool, or acquisition software that
forbids allocation once it is running -- so the library offers one entry point
that keeps all of its scratch in a fixed, static device array.  These checks
call it through the C ABI, with buffers the test allocates beforehand, and
compare its output with the regular device entry point (musr_chi2_grad_device
on a run) at the tolerances the other GPU tests use: objective relative error
<= 1e-6, gradient ||g - g_ref|| / ||g_ref|| <= 1e-4.  Two calls in a row check
that the shared scratch is reset between calls.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
torch = pytest.importorskip("torch")
from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_POISSON, Run, _lib  # noqa: E402


def noalloc_desc(lay, data_dev):
    """A musr_run_desc over device FP32 data (kept alive by the returned tuple)."""
    nb = np.ascontiguousarray(lay.n_bins, dtype=np.int64)
    mp = np.ascontiguousarray(lay.map, dtype=np.int32)
    comp = (_lib.musr_component * lay.n_comp)(*[_lib.musr_component(*map(int, r)) for r in lay.comp])
    d = _lib.musr_run_desc()
    d.n_hist = lay.n_hist
    d.n_bins = nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    d.t0_us, d.dt_us, d.tau_us, d.gamma_mhz_per_g = lay.t0_us, lay.dt_us, lay.tau_us, lay.gamma
    d.n_params, d.map_width = lay.n_params, lay.map_width
    d.map = mp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.n_comp = lay.n_comp
    d.comp = ctypes.cast(comp, ctypes.POINTER(_lib.musr_component))
    d.data_dtype = _lib.MUSR_F32
    d.data = ctypes.c_void_p(data_dev.data_ptr())
    d.data_on_device = 1
    return d, (nb, mp, comp, data_dev)


@pytest.mark.parametrize("stretched", [False, True])
@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_noalloc_matches_device_entry_point_twice(obj, stretched):
    lib = _lib.load()
    dev = torch.device("cuda:0")
    lay, theta, seed = W.config_stretched(16, 5000) if stretched else W.config_multi_detector(16, 5000)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    data_dev = torch.tensor(d, dtype=torch.float32, device=dev)
    P = lay.n_params
    thetas = [W.perturb(theta, lay.free, 0.01, W.rng(seed + i)) for i in (1, 2)]
    desc, keep = noalloc_desc(lay, data_dev)
    stream = torch.cuda.current_stream()
    with Run(lay, data_dev) as run:
        for th in thetas:  # two calls in a row through the shared scratch array
            th_dev = torch.tensor(th, dtype=torch.float64, device=dev)
            out = torch.full((1 + P,), float("nan"), dtype=torch.float64, device=dev)
            status = torch.full((1,), -1, dtype=torch.int32, device=dev)
            rc = lib.musr_chi2_grad_noalloc(ctypes.byref(desc), obj, _lib.MUSR_VALUE_GRAD,
                                            ctypes.c_void_p(th_dev.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(status.data_ptr()),
                                            ctypes.c_void_p(stream.cuda_stream))
            assert rc == _lib.MUSR_OK, lib.musr_strerror(rc)
            ref = torch.empty(1 + P, dtype=torch.float64, device=dev)
            run.chi2_grad_device(th_dev, ref, obj, _lib.MUSR_VALUE_GRAD)
            torch.cuda.synchronize()
            o, r = out.cpu().numpy(), ref.cpu().numpy()
            assert int(status.item()) == 0
            assert rel_err(o[0], r[0]) <= 1e-6
            assert grad_rel_err(o[1:], r[1:]) <= 1e-4


def test_noalloc_rejects_what_does_not_fit():
    lib = _lib.load()
    dev = torch.device("cuda:0")
    lay, theta, _ = W.config_multi_detector(65, 8)  # more histograms than the stated limit
    data_dev = torch.ones(lay.total_bins, dtype=torch.float32, device=dev)
    desc, keep = noalloc_desc(lay, data_dev)
    th = torch.tensor(theta, dtype=torch.float64, device=dev)
    out = torch.empty(1 + lay.n_params, dtype=torch.float64, device=dev)
    rc = lib.musr_chi2_grad_noalloc(ctypes.byref(desc), MUSR_CHI2, _lib.MUSR_VALUE_GRAD,
                                    ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                    None, None)
    assert rc == _lib.MUSR_ENOTSUP
