"""GPU fits (musr_fit through the C ABI) against the FP64 oracle's fit.

Parity bar: every free parameter within 1e-3 of the oracle's parameter error
(sigma from its 2 H^-1 covariance), and chi2 / ndf within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import rel_err

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD,  # noqa: E402
                                    MUSR_FIT_LM, MUSR_POISSON, Run)


def check_fit_parity(th_gpu, info_gpu, th_or, info_or, cov_or, free, tol_sigma=1e-3):
    sig = np.sqrt(np.diag(cov_or))
    dev = np.abs(th_gpu[free] - th_or[free]) / sig
    assert dev.max() <= tol_sigma, dev
    assert rel_err(info_gpu["value"] / info_gpu["ndf"], info_or["value"] / info_or["ndf"]) <= 1e-6


@pytest.mark.parametrize("obj,oobj", [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)])
def test_single_histogram_fit(obj, oobj):
    """1 x 8192 bins, 6 free parameters, from a 5 % perturbed start."""
    lay, theta, seed = W.config_single()
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    start = W.perturb(theta, lay.free, 0.05, W.rng(seed))
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oobj)
    assert info_o["status"] == 0
    with Run(lay, d) as run:
        th_g, info_g, cov_g = run.fit(start, obj, method=MUSR_FIT_LM)
    assert info_g["status"] == 0
    free = lay.free.astype(bool)
    check_fit_parity(th_g, info_g, th_o, info_o, cov_o, free)
    np.testing.assert_allclose(np.sqrt(np.diag(cov_g)), np.sqrt(np.diag(cov_o)), rtol=1e-3)


def test_multi_detector_fit_lm():
    """4 detectors x 16384 bins, 16 free parameters, from a 1 % perturbed start."""
    lay, theta, seed = W.config_multi_detector(4, 16384)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    start = W.perturb(theta, lay.free, 0.01, W.rng(seed + 3))
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oracle.CHI2)
    assert info_o["status"] == 0
    with Run(lay, d) as run:
        th_g, info_g, _ = run.fit(start, MUSR_CHI2, free=lay.free)
    assert info_g["status"] == 0
    check_fit_parity(th_g, info_g, th_o, info_o, cov_o, lay.free.astype(bool))


@pytest.mark.parametrize("method", [MUSR_FIT_BFGS, MUSR_FIT_BFGS_FD])
def test_quasi_newton_fits_reach_the_same_minimum(method):
    """BFGS on the adjoint gradient and on central differences: the oracle's
    minimum, every parameter within 1e-3 sigma."""
    lay, theta, seed = W.config_single()
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    start = W.perturb(theta, lay.free, 0.02, W.rng(seed))
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oracle.CHI2)
    assert info_o["status"] == 0
    with Run(lay, d) as run:
        th_g, info_g, _ = run.fit(start, MUSR_CHI2, method=method, max_iter=2000)
    assert info_g["status"] == 0, info_g
    check_fit_parity(th_g, info_g, th_o, info_o, cov_o, lay.free.astype(bool))


def test_fit_pulls_are_unit_normal():
    """GPU deviance fits of 200 Poisson realisations of the single-histogram run
    (2048 bins), started at the truth: the pulls (theta_hat - theta_true) /
    sigma_hat have mean ~0 and spread ~1 (bounds ~4.5 standard errors) and pass
    a KS test against N(0, 1) for every parameter."""
    from scipy import stats
    lay, theta, _ = W.config_single()
    lay.n_bins = np.array([2048])
    lay.dt_us = 0.005
    mean = oracle.model(lay, theta)
    pulls = []
    with Run(lay, np.zeros(2048)) as run:
        for s in range(200):
            run.set_data(W.poisson_counts(mean, 5000 + s))
            th, info, cov = run.fit(theta, MUSR_POISSON)
            assert info["status"] == 0
            pulls.append((th - theta) / np.sqrt(np.diag(cov)))
    pulls = np.array(pulls)
    assert np.all(np.abs(pulls.mean(0)) < 0.32)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.22)
    for j in range(pulls.shape[1]):
        assert stats.kstest(pulls[:, j], "norm").pvalue > 1e-3
