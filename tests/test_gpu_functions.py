"""GPU parity of runs with a function array (Sec. 4.2.1): map entries that
read expressions of the parameters, evaluated on the host per call, with the
kernels' gradient and Gauss-Newton matrix folded back onto the parameters by
the chain rule.  Tolerances as for plain runs (objective 1e-6 relative,
gradient and GN 1e-4, model 2e-6, fits within 1e-3 of the oracle's errors).
"""
import dataclasses

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err
from oracle import functions as of

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_LM, MUSR_POISSON, MusrError, Run,  # noqa: E402
                                    _lib, chi2_batch)

OBJS = [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)]


def function_layout(K=16, n_bins=5000):
    """Multi-detector run where A2 = A1 * r and sigma2 = sqrt(lambda1^2 + s^2)
    (r, s two new parameters): nonlinear functions of the parameters."""
    lay, theta, seed = W.config_multi_detector(K, n_bins)
    P = lay.n_params
    a1, l1 = lay.names.index("A1"), lay.names.index("lambda1")
    mp = lay.map.copy()
    mp[:, 6] = -2
    mp[:, 7] = -3
    lf = dataclasses.replace(lay, map=mp, n_params=P + 2, names=lay.names + ["r", "s"],
                             free=np.concatenate([lay.free, [1, 1]]).astype(np.uint8),
                             funcs=[f"p[{a1}] * p[{P}]", f"sqrt(p[{l1}] ^ 2 + p[{P + 1}] ^ 2)"])
    th = np.concatenate([theta, [1.2, 0.5]])
    return lf, th, seed


@pytest.fixture(scope="module")
def fcase():
    lf, th, seed = function_layout()
    d = W.poisson_counts(of.model(lf, th), seed)
    tp = W.perturb(th, lf.free, 0.01, W.rng(seed + 9))
    return lf, th, tp, d


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_value_grad_gn(fcase, obj, oobj):
    lf, th, tp, d = fcase
    with Run(lf, d.astype(np.float32)) as run:
        v, g, H = run.chi2_grad(tp, obj, gn=True)
        v0 = run.chi2(tp, obj)
    rv, rg, rH = of.gradient(lf, d, tp, oobj)
    assert rel_err(v, rv) <= 1e-6
    assert rel_err(v0, v) <= 1e-7
    assert grad_rel_err(g, rg) <= 1e-4
    assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
    for name in ("A1", "lambda1", "r", "s"):  # the parameters the functions read
        j = lf.names.index(name)
        assert abs(g[j] - rg[j]) <= 1e-4 * max(abs(rg[j]), 1e-3 * np.abs(rg).max()), name


def test_model(fcase):
    lf, th, tp, d = fcase
    with Run(lf) as run:
        n = run.model(tp)
    np.testing.assert_allclose(n, of.model(lf, tp), rtol=2e-6, atol=1e-6)


def test_linear_function_equals_the_plain_run():
    """B1 + dB as a function instead of the map's field / field2 pair: the same numbers."""
    lay, theta, seed = W.config_multi_detector(16, 5000)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    b1, db = lay.names.index("B1"), lay.names.index("dB")
    mp = np.concatenate([lay.map, np.full((lay.n_hist, 1), -2, dtype=np.int32)], axis=1)
    comp = lay.comp.copy()
    comp[1, 3], comp[1, 4] = mp.shape[1] - 1, -1
    lf = dataclasses.replace(lay, map=mp, comp=comp, funcs=[f"p[{b1}] + p[{db}]"])
    th = W.perturb(theta, lay.free, 0.01, W.rng(4))
    with Run(lay, d) as r0, Run(lf, d) as r1:
        v0, g0, H0 = r0.chi2_grad(th, MUSR_CHI2, gn=True)
        v1, g1, H1 = r1.chi2_grad(th, MUSR_CHI2, gn=True)
    assert rel_err(v1, v0) <= 1e-12
    assert grad_rel_err(g1, g0) <= 1e-10
    assert np.linalg.norm(H1 - H0) <= 1e-10 * np.linalg.norm(H0)


def test_fit_through_functions():
    """The field pair reparametrised as (B1, B2) with dB = B2 - B1 a function:
    the fit reaches the plain run's oracle minimum (mapped back)."""
    lay, theta, seed = W.config_multi_detector(4, 16384)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    start = W.perturb(theta, lay.free, 0.01, W.rng(seed + 3))
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oracle.CHI2)
    assert info_o["status"] == 0
    b1, db = lay.names.index("B1"), lay.names.index("dB")
    P = lay.n_params
    mp = lay.map.copy()
    mp[:, 8] = -2  # dB column -> function 0 = B2 - B1
    free = lay.free.copy()
    free[db] = 0   # dB itself no longer read
    lf = dataclasses.replace(lay, map=mp, n_params=P + 1, names=lay.names + ["B2"],
                             free=np.concatenate([free, [1]]).astype(np.uint8), funcs=[f"p[{P}] - p[{b1}]"])
    s = np.concatenate([start, [start[b1] + start[db]]])
    with Run(lf, d) as run:
        th_g, info_g, _ = run.fit(s, MUSR_CHI2, free=lf.free, method=MUSR_FIT_LM)
    assert info_g["status"] == 0
    mapped = th_g[:P].copy()
    mapped[db] = th_g[P] - th_g[b1]
    fr = lay.free.astype(bool)
    sig = np.sqrt(np.diag(cov_o))
    assert np.max(np.abs(mapped[fr] - th_o[fr]) / sig) <= 1e-3
    assert rel_err(info_g["value"], info_o["value"]) <= 1e-6


def test_errors():
    lf, th, _ = function_layout(2, 64)
    for bad in (["p[0] +"], ["p[999]"], ["q[1]"]):
        with pytest.raises(MusrError) as e:
            Run(dataclasses.replace(lf, funcs=bad + lf.funcs[1:]))
        assert e.value.code == _lib.MUSR_EINVAL
    mp = lf.map.copy()
    mp[0, 3] = -4  # a third function that does not exist
    with pytest.raises(MusrError) as e:
        Run(dataclasses.replace(lf, map=mp))
    assert e.value.code == _lib.MUSR_EINVAL
    d = np.ones(lf.total_bins)
    with Run(lf, d) as run:
        bad_th = th.copy()
        bad_th[-1] = float("nan")
        with pytest.raises(MusrError) as e:
            run.chi2(bad_th, MUSR_CHI2)
        assert e.value.code == _lib.MUSR_ENONFINITE
        with pytest.raises(MusrError) as e:  # the batched paths form no function values
            chi2_batch([run], th, [1], MUSR_POISSON)
        assert e.value.code == _lib.MUSR_ENOTSUP
    neg = dataclasses.replace(lf, funcs=[lf.funcs[0], f"log(p[{lf.n_params - 1}] - 10)"])
    with Run(neg, d) as run:
        with pytest.raises(MusrError) as e:
            run.chi2(th, MUSR_CHI2)
        assert e.value.code == _lib.MUSR_ENONFINITE
