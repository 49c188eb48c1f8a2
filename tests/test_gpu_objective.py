"""GPU parity: the CUDA objective / adjoint kernels against the FP64 oracle.

Tolerances (stated for the FP32-evaluation / FP64-accumulation design):
  * chi2 and the Poisson deviance: relative error <= 1e-6;
  * gradient: ||g_gpu - g_oracle|| / ||g_oracle|| <= 1e-4 at a perturbed theta
    (at the minimum g ~ 0 and a relative bound is meaningless);
  * Gauss-Newton matrix: Frobenius relative error <= 1e-4;
  * model N per bin: relative error <= 2e-6 (a few FP32 ulps);
  * noise-free data: chi2_gpu <= sum (eps N)^2 / max(d, 1) with eps = 4e-7.
All calls go through the C ABI (libmusr.so via ctypes).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err

pytestmark = pytest.mark.gpu

gpu = pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_POISSON, Run  # noqa: E402
from paper_1604_02334_gb300 import _lib  # noqa: E402

OBJS = [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)]


def poisson_data(lay, theta, seed):
    return W.poisson_counts(oracle.model(lay, theta), seed)


@pytest.fixture(scope="module")
def md_small():
    """16 detectors x 5000 bins: several tiles per histogram and a ragged tail."""
    lay, theta, seed = W.config_multi_detector(16, 5000)
    d = poisson_data(lay, theta, seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 7))
    return lay, theta, th, d


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_single_histogram_objective(obj, oobj):
    lay, theta, seed = W.config_single()
    d = poisson_data(lay, theta, seed)  # FP64 counts
    th = W.perturb(theta, lay.free, 0.05, W.rng(seed))
    with Run(lay, d) as run:
        for t in (theta, th):
            v = run.chi2(t, obj)
            ref = oracle.objective(lay, d, t, oobj)
            assert rel_err(v, ref) <= 1e-6, (v, ref)


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_multi_detector_value_grad_gn(md_small, obj, oobj):
    lay, theta, th, d = md_small
    with Run(lay, d.astype(np.float32)) as run:
        v, g, H = run.chi2_grad(th, obj, gn=True)
        v0 = run.chi2(th, obj)
    rv, rg, rH = oracle.gradient(lay, d, th, oobj)
    assert rel_err(v, rv) <= 1e-6
    assert rel_err(v0, v) <= 1e-7  # value-only and adjoint launches (tilings differ per mode)
    assert grad_rel_err(g, rg) <= 1e-4
    assert np.linalg.norm(H - rH) / np.linalg.norm(rH) <= 1e-4


def test_gradient_matches_oracle_central_differences(md_small):
    """The adjoint gradient against FP64 central differences (h = 1e-6 relative)."""
    lay, theta, th, d = md_small
    with Run(lay, d) as run:
        _, g, _ = run.chi2_grad(th, MUSR_CHI2)
    gfd = oracle.gradient_fd(lay, d, th, oracle.CHI2, rel_h=1e-6)
    assert grad_rel_err(g, gfd) <= 1e-4


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_full_size_multi_detector(obj, oobj):
    """16 x 65536 bins, the benchmark's workload, at the launch configuration it times."""
    lay, theta, seed = W.config_multi_detector()
    d = poisson_data(lay, theta, seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 1))
    with Run(lay, d.astype(np.float32)) as run:
        v, g, H = run.chi2_grad(th, obj, gn=True)
        vt = run.chi2(theta, obj)
    rv, rg, rH = oracle.gradient(lay, d, th, oobj, with_gn=True)
    assert rel_err(v, rv) <= 1e-6
    assert grad_rel_err(g, rg) <= 1e-4
    assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
    assert rel_err(vt, oracle.objective(lay, d, theta, oobj)) <= 1e-6


def test_model_matches_oracle(md_small):
    lay, theta, th, d = md_small
    with Run(lay) as run:
        n = run.model(th)
    ref = oracle.model(lay, th)
    np.testing.assert_allclose(n, ref, rtol=2e-6, atol=1e-6)


def test_noise_free_chi2_bound():
    lay, theta, _ = W.config_multi_detector(4, 3000)
    ref = oracle.model(lay, theta)
    d = ref.astype(np.float32).astype(np.float64)
    with Run(lay, d) as run:
        v = run.chi2(theta, MUSR_CHI2)
    bound = np.sum((4e-7 * ref) ** 2 / np.maximum(d, 1.0)) + np.sum((d - ref) ** 2 / np.maximum(d, 1.0))
    assert 0.0 <= v <= bound


def fp32_model_bound(lay, d, th, oobj, eps=4e-7):
    """First-order bound on |obj_gpu - obj| when every model value carries a
    relative error eps (a few FP32 ulps): sum |d obj/dN| eps N + (eps N)^2 c.
    Used where too few bins exist for rounding errors to average out."""
    n = oracle.model(lay, th)
    dn = eps * np.abs(n)
    if oobj == oracle.CHI2:
        w = 1.0 / np.maximum(d, 1.0)
        return float(np.sum(2 * np.abs(d - n) * w * dn + dn * dn * w))
    return float(np.sum(2 * np.abs(1 - d / n) * dn + dn * dn * np.maximum(d, 1) / n ** 2))


@pytest.mark.parametrize("nb", [[1], [7], [8], [9], [0, 5, 0, 2047, 2048, 2049, 13], [16385, 3]])
def test_ragged_and_empty_histograms(nb):
    """Empty, single-bin and ragged histograms.  Below 4096 bins the value is held
    to the FP32 error-propagation bound instead of 1e-6 relative."""
    lay = W.multi_detector_layout(len(nb), nb, window_us=12.8)
    theta = W.multi_detector_theta(lay, W.rng(len(nb)))
    d = poisson_data(lay, theta, 99)
    th = W.perturb(theta, lay.free, 0.02, W.rng(5))
    with Run(lay, d) as run:
        for obj, oobj in OBJS:
            v, g, H = run.chi2_grad(th, obj, gn=True)
            rv, rg, rH = oracle.gradient(lay, d, th, oobj)
            if lay.total_bins >= 4096:
                assert rel_err(v, rv) <= 1e-6
            else:
                assert abs(v - rv) <= max(1e-6 * abs(rv), fp32_model_bound(lay, d, th, oobj))
            assert grad_rel_err(g, rg) <= 1e-4
            assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)


def test_no_histograms():
    lay = W.multi_detector_layout(1, [1])
    lay.n_bins = np.zeros(0, dtype=np.int64)
    lay.map = np.zeros((0, lay.map_width), dtype=np.int32)
    with Run(lay, np.zeros(0)) as run:
        v, g, _ = run.chi2_grad(np.ones(lay.n_params), MUSR_CHI2)
    assert v == 0.0 and not g.any()


def test_bitwise_repeatable(md_small):
    lay, theta, th, d = md_small
    with Run(lay, d) as run:
        a = run.chi2_grad(th, MUSR_CHI2, gn=True)
        b = run.chi2_grad(th, MUSR_CHI2, gn=True)
    assert a[0] == b[0]
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_histogram_permutation(md_small):
    lay, theta, th, d = md_small
    perm = np.random.default_rng(3).permutation(lay.n_hist)
    offs = np.r_[0, np.cumsum(lay.n_bins)]
    dp = np.concatenate([d[offs[k]:offs[k + 1]] for k in perm])
    with Run(lay, d) as r1, Run(lay.permuted(perm), dp) as r2:
        for obj, _ in OBJS:
            a, ga, _ = r1.chi2_grad(th, obj)
            b, gb, _ = r2.chi2_grad(th, obj)
            assert rel_err(a, b) <= 1e-6
            assert grad_rel_err(ga, gb) <= 1e-4


def test_poisson_domain_and_nonfinite():
    lay, theta, seed = W.config_single()
    d = poisson_data(lay, theta, seed)
    with Run(lay, d) as run:
        bad = theta.copy()
        bad[0] = -100.0  # N < 0 with d > 0
        v, st = run.chi2(bad, MUSR_POISSON, raise_on_error=False)
        assert st == _lib.MUSR_EDOMAIN and v == math.inf
        # chi2 is defined for any N
        assert math.isfinite(run.chi2(bad, MUSR_CHI2))
        nan = theta.copy()
        nan[3] = float("nan")
        _, st = run.chi2(nan, MUSR_CHI2, raise_on_error=False)
        assert st == _lib.MUSR_ENONFINITE
        # the run stays usable after errors
        assert rel_err(run.chi2(theta, MUSR_POISSON), oracle.objective(lay, d, theta, oracle.POISSON)) <= 1e-6


def test_device_path_and_autograd(md_small):
    torch = pytest.importorskip("torch")
    from paper_1604_02334_gb300 import Chi2
    lay, theta, th, d = md_small
    dev = torch.device("cuda:0")
    data_t = torch.tensor(d, dtype=torch.float32, device=dev)
    with Run(lay, data_t, stream="torch") as run:
        v_host, g_host, _ = run.chi2_grad(th, MUSR_CHI2)
        t = torch.tensor(th, dtype=torch.float64, device=dev, requires_grad=True)
        v = Chi2.apply(t, run, MUSR_CHI2)
        (gt,) = torch.autograd.grad(v * 3.0, t)
        ref = torch.empty(1 + lay.n_params, dtype=torch.float64, device=dev)
        run.chi2_grad_device(t.detach(), ref, MUSR_CHI2, 1)
        torch.cuda.synchronize()
        # autograd plumbing is exact against the device entry point it wraps
        assert float(v.detach()) == float(ref[0])
        np.testing.assert_array_equal(gt.cpu().numpy(), 3.0 * ref[1:].cpu().numpy())
        # device calls stage constants with FP32 functions, host calls in FP64
        assert rel_err(float(v.detach()), v_host) <= 1e-7
        assert grad_rel_err(ref[1:].cpu().numpy(), g_host) <= 1e-6
        # a caller's buffer full of NaN: the Gauss-Newton entries without
        # sources must come back as 0, the others as the oracle's
        P = lay.n_params
        out = torch.full((1 + P + P ** 2,), float("nan"), dtype=torch.float64, device=dev)
        st = torch.zeros(1, dtype=torch.int32, device=dev)
        run.chi2_grad_device(t.detach(), out, MUSR_POISSON, 2, st)
        torch.cuda.synchronize()
        rv, rg, rH = oracle.gradient(lay, d, th, oracle.POISSON, with_gn=True)
        o = out.cpu().numpy()
        assert rel_err(o[0], rv) <= 1e-6 and int(st.item()) == 0
        assert grad_rel_err(o[1:1 + P], rg) <= 1e-4
        H = o[1 + P:].reshape(P, P)
        assert np.all(np.isfinite(H))
        assert np.array_equal(H, H.T)
        assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)


def test_async_entry_queued_back_to_back(md_small):
    """Host-theta evaluations queued back to back on one stream, each one's
    staging and bin loop free to run while the previous kernel finishes
    (modes and objectives mixed, device-entry calls interleaved): queued
    twice, the results are equal bit for bit; they match the device entry's
    at the same theta (the queued tiling may differ, so FP32 lane sums round
    differently: value 1e-6, gradient 1e-5, GN 1e-5), the interleaved device
    calls equal the device entry's bit for bit, the Gauss-Newton entries
    without sources come back 0 in a NaN buffer, and the results match the
    oracle."""
    torch = pytest.importorskip("torch")
    lay, theta, th, d = md_small
    P = lay.n_params
    n = 1 + P + P * P
    J = 24
    dev = torch.device("cuda:0")
    ths = [W.perturb(theta, lay.free, 0.01, W.rng(300 + j)) for j in range(J)]
    cases = [((MUSR_CHI2, MUSR_POISSON)[j % 2], j % 3) for j in range(J)]
    width = [1, 1 + P, n]
    with Run(lay, d) as run:
        s = torch.cuda.Stream(device=dev)
        ths_t = [torch.tensor(t, dtype=torch.float64, device=dev) for t in ths]
        ref = torch.full((J, n), float("nan"), dtype=torch.float64, device=dev)
        for j, (obj, mode) in enumerate(cases):
            run.chi2_grad_device(ths_t[j], ref[j], obj, mode, stream=s.cuda_stream)
        s.synchronize()
        outs = []
        for rep in range(2):
            out = torch.full((J, n), float("nan"), dtype=torch.float64, device=dev)
            st = torch.full((J,), -1, dtype=torch.int32, device=dev)
            mixed = torch.full((J, n), float("nan"), dtype=torch.float64, device=dev)
            for j, (obj, mode) in enumerate(cases):
                run.chi2_grad_async(ths[j], out[j], obj, mode, st[j:j + 1], stream=s.cuda_stream)
                if j % 5 == 0:  # a device-entry call between queued ones
                    run.chi2_grad_device(ths_t[j], mixed[j], obj, mode, stream=s.cuda_stream)
            s.synchronize()
            assert not st.any().item()
            outs.append(out.cpu().numpy())
        o, r, m = outs[0], ref.cpu().numpy(), mixed.cpu().numpy()
        assert np.array_equal(o, outs[1], equal_nan=True)
        for j, (obj, mode) in enumerate(cases):
            w = width[mode]
            assert rel_err(o[j, 0], r[j, 0]) <= 1e-6, j
            if mode >= 1:
                assert grad_rel_err(o[j, 1:1 + P], r[j, 1:1 + P]) <= 1e-5, j
            if mode == 2:
                Ho, Hr = o[j, 1 + P:].reshape(P, P), r[j, 1 + P:].reshape(P, P)
                assert np.linalg.norm(Ho - Hr) <= 1e-5 * np.linalg.norm(Hr), j
            assert np.all(np.isnan(o[j, w:]))
            if j % 5 == 0:
                assert np.array_equal(m[j, :w], r[j, :w]), j
        for j in (0, 1, 2, 5):
            obj, mode = cases[j]
            rv, rg, rH = oracle.gradient(lay, d, ths[j], (oracle.CHI2, oracle.POISSON)[j % 2], with_gn=True)
            assert rel_err(o[j, 0], rv) <= 1e-6
            if mode >= 1:
                assert grad_rel_err(o[j, 1:1 + P], rg) <= 1e-4
            if mode == 2:
                H = o[j, 1 + P:].reshape(P, P)
                assert np.array_equal(H, H.T)
                assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
        # host-side checks: nothing is launched
        bad = ths[0].copy()
        bad[0] = np.nan
        with pytest.raises(_lib.MusrError) as ei:
            run.chi2_grad_async(bad, out[0], MUSR_CHI2, 1)
        assert ei.value.code == _lib.MUSR_ENONFINITE
        with pytest.raises(ValueError):
            run.chi2_grad_async(ths[0][:-1], out[0], MUSR_CHI2, 1)


def test_set_data_from_device_fp64(md_small):
    torch = pytest.importorskip("torch")
    lay, theta, th, d = md_small
    with Run(lay, d) as run:
        a = run.chi2(th, MUSR_CHI2)
        run.set_data(torch.tensor(d, dtype=torch.float64, device="cuda:0"))
        b = run.chi2(th, MUSR_CHI2)
    assert a == b


def test_concurrent_runs_on_host_threads():
    """Runs are independent: four host threads, each with its own run, evaluate
    concurrently (ctypes releases the GIL) and get, bit for bit, what the same
    calls give one after the other."""
    import threading
    cases = []
    for i in range(4):
        lay, theta, seed = W.config_multi_detector(8, 3000 + 1000 * i)
        d = poisson_data(lay, theta, seed + i)
        cases.append((lay, d, [W.perturb(theta, lay.free, 0.01, W.rng(seed + 10 * i + j)) for j in range(20)]))
    runs = [Run(lay, d) for lay, d, _ in cases]
    expected = [[run.chi2_grad(th, MUSR_CHI2, gn=(j % 2 == 1)) for j, th in enumerate(ths)]
                for run, (_, _, ths) in zip(runs, cases)]
    got = [None] * 4
    errors = []

    def work(i):
        try:
            got[i] = [runs[i].chi2_grad(th, MUSR_CHI2, gn=(j % 2 == 1)) for j, th in enumerate(cases[i][2])]
        except Exception as e:  # noqa: BLE001 -- reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for e_run, g_run in zip(expected, got):
        for (v0, g0, h0), (v1, g1, h1) in zip(e_run, g_run):
            assert v0 == v1 and np.array_equal(g0, g1)
            assert (h0 is None and h1 is None) or np.array_equal(h0, h1)
    for r in runs:
        r.close()
