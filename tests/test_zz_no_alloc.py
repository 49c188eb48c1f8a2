"""The allocation-free entry point, musr_chi2_grad_noalloc.

Some callers cannot allocate device memory -- for example a plug-in whose host
framework owns the whole device memory pool, or acquisition software that
forbids allocation once it is running -- so the library offers one entry point
that keeps all of its scratch in a fixed, static device array.  These checks
call it through the C ABI, with buffers the test allocates beforehand, and
compare its output with the regular device entry point (musr_chi2_grad_device
on a run) and with the FP64 oracle at the tolerances the other GPU tests use:
objective relative error <= 1e-6, gradient 1e-4 norm-wise and per component.
Two calls in a row check that the shared scratch is reset between calls.
Cases: plain and stretched runs, both objectives, value-only mode, uneven
histogram lengths, 64 histograms filling the scratch array almost to its
size, one just too large for it (refused), and a call under stream capture
(refused).  After a first call (which loads the entry point's code and with
it the array), further calls leave the device's free memory and torch's
allocator unchanged.

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


def call_noalloc(lib, desc, obj, mode, th_dev, out, status, stream):
    return lib.musr_chi2_grad_noalloc(ctypes.byref(desc), obj, mode, ctypes.c_void_p(th_dev.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(status.data_ptr()) if status is not None else None,
                                      ctypes.c_void_p(stream.cuda_stream))


def check_against_references(lay, d, data_dev, thetas, obj, mode):
    """Two calls in a row: each against the run's device entry point and the
    oracle; device free memory and torch's allocator unchanged over both."""
    lib = _lib.load()
    dev = torch.device("cuda:0")
    P = lay.n_params
    n_out = 1 + (P if mode == _lib.MUSR_VALUE_GRAD else 0)
    desc, keep = noalloc_desc(lay, data_dev)
    stream = torch.cuda.current_stream()
    oobj = oracle.CHI2 if obj == MUSR_CHI2 else oracle.POISSON
    th_devs = [torch.tensor(th, dtype=torch.float64, device=dev) for th in thetas]
    outs = [torch.full((n_out,), float("nan"), dtype=torch.float64, device=dev) for _ in thetas]
    stats = [torch.full((1,), -1, dtype=torch.int32, device=dev) for _ in thetas]
    refs = [torch.empty(n_out, dtype=torch.float64, device=dev) for _ in thetas]
    # a first call on this device loads the entry point's code and its array
    rc = call_noalloc(lib, desc, obj, mode, th_devs[0], outs[0], stats[0], stream)
    assert rc == _lib.MUSR_OK, lib.musr_strerror(rc)
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for th_dev, out, st in zip(th_devs, outs, stats):  # two calls through the shared scratch array
        out.fill_(float("nan"))
        st.fill_(-1)
        rc = call_noalloc(lib, desc, obj, mode, th_dev, out, st, stream)
        assert rc == _lib.MUSR_OK, lib.musr_strerror(rc)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    with Run(lay, data_dev) as run:
        for th, th_dev, out, st, ref in zip(thetas, th_devs, outs, stats, refs):
            run.chi2_grad_device(th_dev, ref, obj, mode)
            torch.cuda.synchronize()
            o, r = out.cpu().numpy(), ref.cpu().numpy()
            assert int(st.item()) == 0
            assert rel_err(o[0], r[0]) <= 1e-6
            if mode == _lib.MUSR_VALUE_GRAD:
                assert grad_rel_err(o[1:], r[1:]) <= 1e-4
                rv, rg, _ = oracle.gradient(lay, d, th, oobj, with_gn=False)
                assert grad_rel_err(o[1:], rg) <= 1e-4
            else:
                rv = oracle.objective(lay, d, th, oobj)
            assert rel_err(o[0], rv) <= 1e-6


@pytest.mark.parametrize("stretched", [False, True])
@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_noalloc_matches_device_entry_point_and_oracle_twice(obj, stretched):
    dev = torch.device("cuda:0")
    lay, theta, seed = W.config_stretched(16, 5000) if stretched else W.config_multi_detector(16, 5000)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    thetas = [W.perturb(theta, lay.free, 0.01, W.rng(seed + i)) for i in (1, 2)]
    check_against_references(lay, d, torch.tensor(d, dtype=torch.float32, device=dev), thetas, obj,
                             _lib.MUSR_VALUE_GRAD)


def test_noalloc_value_mode_uneven_histograms():
    """Value only, histograms of uneven, non-tile-aligned lengths (an empty one too)."""
    dev = torch.device("cuda:0")
    nb = [5000, 12345, 0, 777, 40001, 8, 65536, 3]
    lay = W.multi_detector_layout(len(nb), nb, window_us=12.8)
    g = W.rng(404)
    theta = W.multi_detector_theta(lay, g)
    d = W.poisson_counts(oracle.model(lay, theta), 405)
    thetas = [W.perturb(theta, lay.free, 0.01, g) for _ in range(2)]
    data_dev = torch.tensor(d, dtype=torch.float32, device=dev)
    for obj in (MUSR_CHI2, MUSR_POISSON):
        check_against_references(lay, d, data_dev, thetas, obj, _lib.MUSR_VALUE)
    check_against_references(lay, d, data_dev, thetas, MUSR_CHI2, _lib.MUSR_VALUE_GRAD)


def test_noalloc_near_the_scratch_limit():
    """64 histograms (the stated maximum) of 128000 bins: the padded counts
    alone fill 98 % of the scratch array."""
    dev = torch.device("cuda:0")
    lay = W.multi_detector_layout(64, 128000, window_us=12.8)
    assert lay.total_bins * 4 > 0.97 * _lib.MUSR_NOALLOC_SCRATCH_BYTES
    g = W.rng(406)
    theta = W.multi_detector_theta(lay, g)
    d = W.poisson_counts(oracle.model(lay, theta), 407)
    thetas = [W.perturb(theta, lay.free, 0.01, g) for _ in range(2)]
    check_against_references(lay, d, torch.tensor(d, dtype=torch.float32, device=dev), thetas, MUSR_CHI2,
                             _lib.MUSR_VALUE_GRAD)


def _refusal_inputs(lay):
    dev = torch.device("cuda:0")
    data_dev = torch.ones(lay.total_bins, dtype=torch.float32, device=dev)
    desc, keep = noalloc_desc(lay, data_dev)
    th = torch.tensor(W.multi_detector_theta(lay, W.rng(1)), dtype=torch.float64, device=dev)
    out = torch.empty(1 + lay.n_params, dtype=torch.float64, device=dev)
    return desc, keep, th, out


def _call(desc, th, out, stream_ptr=None):
    return _lib.load().musr_chi2_grad_noalloc(ctypes.byref(desc), MUSR_CHI2, _lib.MUSR_VALUE_GRAD,
                                              ctypes.c_void_p(th.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              None, ctypes.c_void_p(stream_ptr) if stream_ptr else None)


def test_noalloc_rejects_what_does_not_fit():
    # more histograms than the stated limit
    desc, keep, th, out = _refusal_inputs(W.config_multi_detector(65, 8)[0])
    assert _call(desc, th, out) == _lib.MUSR_ENOTSUP
    # 64 histograms whose counts alone are the array's size: no room for the tables
    lay = W.multi_detector_layout(64, 131072, window_us=12.8)
    assert lay.total_bins * 4 >= _lib.MUSR_NOALLOC_SCRATCH_BYTES
    desc, keep, th, out = _refusal_inputs(lay)
    assert _call(desc, th, out) == _lib.MUSR_ENOTSUP


def test_noalloc_refuses_a_capturing_stream():
    """Its host-side table uploads cannot be captured into a graph: refused."""
    desc, keep, th, out = _refusal_inputs(W.multi_detector_layout(4, 1000, window_us=12.8))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(g, stream=s):
        out.zero_()
        rc = _call(desc, th, out, s.cuda_stream)
    assert rc == _lib.MUSR_ENOTSUP
