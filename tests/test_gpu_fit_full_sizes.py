"""GPU fits at the sizes the benchmark fits, against the FP64 oracle's fit.

Workloads: 16 x 65536 bins (40 free parameters) and 32 x 131072 bins (72
free), Poisson counts, each fitted from the same 1 % perturbed start as the
benchmark's fits.  The oracle's Levenberg-Marquardt fit (FP64, EDM < 1e-8) is
the reference; the GPU fits are musr_fit through the C ABI with the adjoint
Levenberg-Marquardt and the adjoint BFGS.

Parity bar (the minimiser reaches the oracle's minimum): status MUSR_OK on
both sides, every free parameter within 1e-3 of the oracle's parameter error
sigma (from its covariance 2 H^-1), and chi2 / ndf within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import rel_err

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_LM, MUSR_POISSON, Run  # noqa: E402

CASES = {"16x65536": W.config_multi_detector, "32x131072": W.config_gradient}
_cache = {}


def oracle_case(name, obj):
    """(layout, counts, start, oracle theta, oracle info, oracle covariance), cached per case."""
    key = (name, obj)
    if key not in _cache:
        lay, theta, seed = CASES[name]()
        d = W.poisson_counts(oracle.model(lay, theta), seed)
        start = W.perturb(theta, lay.free, 0.01, W.rng(seed + 31))
        th_o, info_o, cov_o = oracle.fit(lay, d, start, obj)
        assert info_o["status"] == 0, info_o
        _cache[key] = (lay, d, start, th_o, info_o, cov_o)
    return _cache[key]


def check_fit_parity(th_gpu, info_gpu, th_or, info_or, cov_or, free, tol_sigma=1e-3):
    sig = np.sqrt(np.diag(cov_or))
    dev = np.abs(th_gpu[free] - th_or[free]) / sig
    assert dev.max() <= tol_sigma, (float(dev.max()), int(np.argmax(dev)))
    assert rel_err(info_gpu["value"] / info_gpu["ndf"], info_or["value"] / info_or["ndf"]) <= 1e-6


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("method", [MUSR_FIT_LM, MUSR_FIT_BFGS], ids=["lm", "bfgs"])
def test_chi2_fit_matches_oracle_fit(name, method):
    lay, d, start, th_o, info_o, cov_o = oracle_case(name, oracle.CHI2)
    with Run(lay, d.astype(np.float32)) as run:
        th_g, info_g, _ = run.fit(start, MUSR_CHI2, free=lay.free, method=method)
    assert info_g["status"] == 0, info_g
    check_fit_parity(th_g, info_g, th_o, info_o, cov_o, lay.free.astype(bool))


def test_deviance_fit_matches_oracle_fit():
    lay, d, start, th_o, info_o, cov_o = oracle_case("16x65536", oracle.POISSON)
    with Run(lay, d.astype(np.float32)) as run:
        th_g, info_g, _ = run.fit(start, MUSR_POISSON, free=lay.free, method=MUSR_FIT_LM)
    assert info_g["status"] == 0, info_g
    check_fit_parity(th_g, info_g, th_o, info_o, cov_o, lay.free.astype(bool))
