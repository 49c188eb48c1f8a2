"""GPU parity of the stretched precession line, a exp(-(lambda t)^beta)
cos(2 pi gamma (B + B2) t + phi) (the stretched exponential of Sec. 4.2.1),
built into the FP32 objective / adjoint kernels, against the FP64 oracle.

Tolerances are those of the other lines: objective relative 1e-6, gradient
1e-4 norm-wise at a perturbed theta, Gauss-Newton matrix 1e-4 (Frobenius),
model 2e-6 relative per bin, fits within 1e-3 of the oracle's parameter
errors.  Every path that evaluates the theory is covered: single run (value,
gradient, GN, model), many runs x many vectors (value batch), many runs with
gradient (adjoint batch), the generator's rebinned means and the fit.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_LM, MUSR_POISSON, MUSR_VALUE_GRAD,  # noqa: E402
                                    MUSR_VALUE_GRAD_GN, GBatch, Run, chi2_batch)

OBJS = [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)]


def poisson_data(lay, theta, seed):
    return W.poisson_counts(oracle.model(lay, theta), seed)


@pytest.fixture(scope="module")
def st_small():
    """16 detectors x 5000 bins (several tiles and a ragged tail): exponential line,
    stretched line, Kubo-Toyabe term."""
    lay, theta, seed = W.config_stretched(16, 5000)
    d = poisson_data(lay, theta, seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 7))
    return lay, theta, th, d


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_value_grad_gn(st_small, obj, oobj):
    lay, theta, th, d = st_small
    with Run(lay, d.astype(np.float32)) as run:
        v, g, H = run.chi2_grad(th, obj, gn=True)
        v0 = run.chi2(th, obj)
    rv, rg, rH = oracle.gradient(lay, d, th, oobj)
    assert rel_err(v, rv) <= 1e-6
    assert rel_err(v0, v) <= 1e-7
    assert grad_rel_err(g, rg) <= 1e-4
    assert np.linalg.norm(H - rH) / np.linalg.norm(rH) <= 1e-4
    # the stretched line's own derivatives are each resolved, not hidden in the norm
    for name in ("A2", "lambda2", "beta"):
        j = lay.names.index(name)
        assert abs(g[j] - rg[j]) <= 1e-4 * max(abs(rg[j]), 1e-3 * np.abs(rg).max()), name


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_full_size(obj, oobj):
    """16 x 65536 bins with the stretched line in place of the Gaussian one."""
    lay, theta, seed = W.config_stretched()
    d = poisson_data(lay, theta, seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 1))
    with Run(lay, d.astype(np.float32)) as run:
        v, g, _ = run.chi2_grad(th, obj)
        vt = run.chi2(theta, obj)
    rv, rg, _ = oracle.gradient(lay, d, th, oobj, with_gn=False)
    assert rel_err(v, rv) <= 1e-6
    assert grad_rel_err(g, rg) <= 1e-4
    assert rel_err(vt, oracle.objective(lay, d, theta, oobj)) <= 1e-6


def test_model(st_small):
    lay, theta, th, d = st_small
    with Run(lay) as run:
        n = run.model(th)
    np.testing.assert_allclose(n, oracle.model(lay, th), rtol=2e-6, atol=1e-6)


def single_stretched_layout(n_bins=20000, dt=0.0005, t0=0.0):
    """One histogram with the stretched line alone: theta = [N0, bkg, A, lambda, B, phi, beta]."""
    lay = W.single_hist_layout(n_bins, dt, t0)
    lay.map = np.array([[0, 1, 2, 3, 4, 5, 6]], dtype=np.int32)
    lay.n_params = 7
    lay.names = ["N0", "bkg", "A", "lambda", "B", "phi", "beta"]
    lay.free = np.ones(7, dtype=np.uint8)
    lay.comp = W.comp_table([[W.TF_STRETCHED, 2, 3, 4, -1, 5, 6]])
    return lay


@pytest.mark.parametrize("t0", [0.0, 0.37])
@pytest.mark.parametrize("beta,lam", [(0.5, 1.2), (1.0, 0.7), (1.8, 2.5), (0.9, 0.0), (1.4, -0.3)])
def test_single_line_edge_cases(t0, beta, lam):
    """The line alone (no other component), a start offset t0, beta below, at and
    above 1, lambda = 0 and lambda < 0 (envelope 1, no derivative into lambda or
    beta)."""
    lay = single_stretched_layout(t0=t0)
    theta = np.array([3000.0, 4.0, 0.22, lam, 150.0, 0.3, beta])
    d = poisson_data(lay, theta, 5)
    th = theta.copy()
    th[[0, 2, 4]] *= [1.002, 1.05, 1.001]
    with Run(lay, d) as run:
        for obj, oobj in OBJS:
            v, g, H = run.chi2_grad(th, obj, gn=True)
            rv, rg, rH = oracle.gradient(lay, d, th, oobj)
            assert rel_err(v, rv) <= 1e-6
            assert grad_rel_err(g, rg) <= 1e-4
            assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
            if lam <= 0.0:
                assert g[3] == 0.0 and g[6] == 0.0
        np.testing.assert_allclose(run.model(th), oracle.model(lay, th), rtol=2e-6, atol=1e-6)


def test_value_batch():
    """Many runs x many vectors in one launch (value only)."""
    runs, data, vecs = [], [], []
    for i, (K, nb) in enumerate([(16, 20000), (3, 4099), (1, 65536)]):
        lay = W.multi_detector_layout(K, nb, 12.8, stretched=True)
        theta = W.multi_detector_theta(lay, W.rng(60 + i))
        d = poisson_data(lay, theta, 70 + i)
        th = W.perturb(theta, lay.free, 0.01, W.rng(80 + i))
        runs.append(lay)
        data.append(d)
        vecs.append(W.jacobian_vectors(th, lay.free, rel_h=1e-3)[:7])
    gruns = [Run(lay, d) for lay, d in zip(runs, data)]
    values = chi2_batch(gruns, np.concatenate([v.ravel() for v in vecs]), [v.shape[0] for v in vecs], MUSR_CHI2)
    o = 0
    for lay, d, v in zip(runs, data, vecs):
        for j in range(v.shape[0]):
            assert rel_err(values[o], oracle.objective(lay, d, v[j], oracle.CHI2)) <= 1e-6
            o += 1
    for r in gruns:
        r.close()


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_adjoint_batch(obj, oobj):
    """Many runs, one vector each, value + gradient (+ GN) in one launch."""
    cases = []
    for i, (K, nb) in enumerate([(16, 16384), (4, 5000), (2, 777)]):
        lay = W.multi_detector_layout(K, nb, 12.8, stretched=True)
        theta = W.multi_detector_theta(lay, W.rng(90 + i))
        d = poisson_data(lay, theta, 95 + i)
        cases.append((lay, d, W.perturb(theta, lay.free, 0.01, W.rng(99 + i))))
    gruns = [Run(lay, d) for lay, d, _ in cases]
    with GBatch(gruns) as b:
        for mode in (MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN):
            res, flags = b.eval([c[2] for c in cases], obj, mode)
            assert not np.any(flags)
            for (lay, d, th), (val, grad, gn) in zip(cases, res):
                v, g, H = oracle.gradient(lay, d, th, oobj, with_gn=True)
                if lay.total_bins >= 4096:
                    assert rel_err(val, v) <= 1e-6
                assert grad_rel_err(grad, g) <= 1e-4
                if mode == MUSR_VALUE_GRAD_GN:
                    assert np.linalg.norm(gn - H) <= 1e-4 * np.linalg.norm(H)
    for r in gruns:
        r.close()


def test_generator_means():
    """The generator's rebinned theory (the proposer's training data) with the stretched line."""
    torch = pytest.importorskip("torch")
    lay = W.multi_detector_layout(16, 4096, 12.8, stretched=True)
    g = W.rng(101)
    thetas = np.stack([W.multi_detector_theta(lay, g) for _ in range(4)])
    rebin = 64
    dev = torch.device("cuda:0")
    per = int(sum((int(m) + rebin - 1) // rebin for m in lay.n_bins))
    out = torch.empty((thetas.shape[0], per), dtype=torch.float32, device=dev)
    mu = torch.empty_like(out)
    with Run(lay) as r:
        r.generate(torch.tensor(thetas, device=dev), rebin, 3, out, mu_dev=mu)
        torch.cuda.synchronize()
    np.testing.assert_allclose(mu.cpu().numpy(), oracle.rebinned_mean(lay, thetas, rebin), rtol=2e-6, atol=1e-5)


def test_fit_matches_oracle_fit():
    """LM fit of 4 detectors x 16384 bins (17 free) from a 1 % perturbed start."""
    lay, theta, seed = W.config_stretched(4, 16384)
    d = poisson_data(lay, theta, seed)
    start = W.perturb(theta, lay.free, 0.01, W.rng(seed + 3))
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oracle.CHI2)
    assert info_o["status"] == 0
    with Run(lay, d) as run:
        th_g, info_g, _ = run.fit(start, MUSR_CHI2, free=lay.free, method=MUSR_FIT_LM)
    assert info_g["status"] == 0
    free = lay.free.astype(bool)
    sig = np.sqrt(np.diag(cov_o))
    assert np.max(np.abs(th_g[free] - th_o[free]) / sig) <= 1e-3
    assert rel_err(info_g["value"] / info_g["ndf"], info_o["value"] / info_o["ndf"]) <= 1e-6


def test_layout_limits():
    """Two stretched lines, or a stretched line beside two others, are outside the
    compiled signatures (MUSR_ENOTSUP); a beta column outside the map row is
    MUSR_EINVAL."""
    from paper_1604_02334_gb300 import MusrError
    from paper_1604_02334_gb300 import _lib
    lay = W.multi_detector_layout(2, 64, 12.8, stretched=True)
    two = lay.comp.copy()
    two[0] = [W.TF_STRETCHED, 3, 4, 5, -1, 2, 11]
    three = np.concatenate([lay.comp[:2], lay.comp[:1]])
    bad = lay.comp.copy()
    bad[1, 6] = lay.map_width
    for comp, code in ((two, _lib.MUSR_ENOTSUP), (three, _lib.MUSR_ENOTSUP), (bad, _lib.MUSR_EINVAL)):
        lay.comp = comp
        with pytest.raises(MusrError) as e:
            Run(lay)
        assert e.value.code == code
