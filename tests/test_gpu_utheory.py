"""User-defined theory functions compiled at run time (NVRTC): objective
parity with the FP64 expression oracle (FP64 variant: relative 1e-10, both
FP64 with different summation order; FP32 variant: relative 1e-5 — a model
error of ~5e-7 per bin from FP32 exp / cos and N0 rounding, summed with
partly coherent signs over ~1e6 bins of ~1e3 counts), agreement with the
built-in kernels for the same theory, forward-mode and central-difference
gradients against the oracle's analytic gradient of the equivalent built-in
model, a stretched exponential and the function array, out-of-range indices,
compile errors, and a fit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_POISSON, MusrError, Run, UserTheory  # noqa: E402
import oracle  # noqa: E402
from oracle import utheory as U  # noqa: E402
import workloads as W  # noqa: E402
from _gpu_util import grad_rel_err, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def md():
    lay = W.multi_detector_layout(4, [3000, 5000, 777, 4096], window_us=12.8)
    g = W.rng(21)
    theta = W.multi_detector_theta(lay, g)
    d = W.poisson_counts(oracle.model(lay, theta), 22)
    return lay, theta, d, g


@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_user_objective_matches_oracle_and_builtin(md, obj):
    lay, theta, d, g = md
    th = UserTheory(W.MD_USER_EXPR)
    thetas = np.stack([W.perturb(theta, lay.free, 0.01, g) for _ in range(5)])
    with Run(lay, d) as run:
        vals = th.eval(run, thetas, obj)
        for i in range(5):
            ref = U.objective(lay, d, thetas[i], W.MD_USER_EXPR, obj)
            assert rel_err(vals[i], ref) <= 1e-10
            builtin = run.chi2(thetas[i], obj)
            assert rel_err(vals[i], builtin) <= 1e-6
        # bitwise repeatable
        np.testing.assert_array_equal(th.eval(run, thetas, obj), vals)
    th.close()


@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_user_gradient_matches_oracle_analytic(md, obj):
    # forward-mode (exact) and central-difference gradients of the user theory
    # against the C oracle's analytic gradient of the same (built-in) model
    lay, theta, d, g = md
    th = UserTheory(W.MD_USER_EXPR)
    t1 = W.perturb(theta, lay.free, 0.01, g)
    with Run(lay, d) as run:
        v, gr = th.grad(run, t1, obj, free=lay.free, rel_h=0.0)
        vf, gf = th.grad(run, t1, obj, free=lay.free, rel_h=1e-6)
    vref, gref, _ = oracle.gradient(lay, d, t1, oracle.CHI2 if obj == MUSR_CHI2 else oracle.POISSON, with_gn=False)
    fr = lay.free.astype(bool)
    assert rel_err(v, vref) <= 1e-10 and rel_err(vf, vref) <= 1e-10
    assert grad_rel_err(gr[fr], gref[fr]) <= 1e-9
    assert not gr[~fr].any()
    assert grad_rel_err(gf[fr], gref[fr]) <= 1e-4
    th.close()


def test_stretched_exponential_and_function_array():
    lay = W.single_hist_layout()
    theta = W.single_hist_truth()
    # single-histogram map row: [N0, bkg, A0, lambda, B, phi]; beta through f[0]
    expr = "p[m[2]] * ge(t, p[m[3]], f[0]) * tf(t, p[m[5]], p[m[4]])"
    d = W.poisson_counts(U.model(lay, theta, expr, funcs=[0.7]), 31)
    th = UserTheory(expr, n_funcs=1)
    with Run(lay, d) as run:
        for beta in (0.5, 0.7, 1.0, 1.8):
            v = th.eval(run, theta, MUSR_POISSON, funcs=[beta])[0]
            ref = U.objective(lay, d, theta, expr, 1, funcs=[beta])
            assert rel_err(v, ref) <= 1e-10
        # forward-mode gradient of the stretched exponential against central
        # differences of the FP64 oracle (h = 1e-6 relative)
        _, gr = th.grad(run, theta, MUSR_POISSON, funcs=[0.7], rel_h=0.0)
    gfd = np.zeros_like(theta)
    for j in range(theta.shape[0]):
        h = 1e-6 * max(abs(theta[j]), 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        gfd[j] = (U.objective(lay, d, tp, expr, 1, funcs=[0.7]) - U.objective(lay, d, tm, expr, 1, funcs=[0.7])) / (2 * h)
    assert grad_rel_err(gr, gfd) <= 1e-6
    th.close()


def test_compile_errors_and_rejected_expressions():
    with pytest.raises(MusrError) as e:
        UserTheory("p[m[0]] * nosuchfunction(t)")
    assert "nosuchfunction" in str(e.value)
    for bad in ("t; x", "t == 1", "t{}", "\"s\""):
        with pytest.raises(MusrError):
            UserTheory(bad)


def test_user_fit_reaches_the_builtin_minimum():
    lay, truth, seed = W.config_single()
    d = W.poisson_counts(oracle.model(lay, truth), seed)
    expr = "p[m[2]] * se(t, p[m[3]]) * tf(t, p[m[5]], p[m[4]])"
    # the single-histogram map row is [N0, bkg, A0, lambda, B, phi]
    np.testing.assert_allclose(U.model(lay, truth, expr), oracle.model(lay, truth), rtol=1e-12)
    th = UserTheory(expr)
    start = W.perturb(truth, lay.free, 0.02, W.rng(5))
    with Run(lay, d) as run:
        tu, iu, _ = th.fit(run, start, MUSR_CHI2, free=lay.free)
        tb, ib, _ = run.fit(start, MUSR_CHI2, free=lay.free)
    assert iu["status"] == 0
    assert rel_err(iu["value"], ib["value"]) <= 1e-6
    th.close()


def test_calls_of_different_vector_counts(md):
    # alternating batch sizes reuse the scratch with different layouts
    lay, theta, d, g = md
    th = UserTheory(W.MD_USER_EXPR)
    with Run(lay, d) as run:
        v1 = th.eval(run, theta, MUSR_CHI2)[0]
        for n in (81, 1, 40, 3, 81, 1):
            v = th.eval(run, np.repeat(theta[None, :], n, axis=0), MUSR_CHI2)
            assert np.all(v == v1)
        _, g0 = th.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=1e-6)
        v2, g1 = th.grad(run, theta, MUSR_CHI2, free=lay.free, rel_h=0.0)
        assert v2 == v1
    th.close()


@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_fp32_variant_matches_oracle(md, obj):
    lay, theta, d, g = md
    th = UserTheory(W.MD_USER_EXPR, fp32=True)
    t1 = W.perturb(theta, lay.free, 0.01, g)
    with Run(lay, d) as run:
        v = th.eval(run, t1, obj)[0]
        vg, gr = th.grad(run, t1, obj, free=lay.free, rel_h=0.0)
    ref = U.objective(lay, d, t1, W.MD_USER_EXPR, obj)
    assert rel_err(v, ref) <= 1e-5 and vg == v
    vref, gref, _ = oracle.gradient(lay, d, t1, oracle.CHI2 if obj == MUSR_CHI2 else oracle.POISSON, with_gn=False)
    fr = lay.free.astype(bool)
    assert grad_rel_err(gr[fr], gref[fr]) <= 1e-3
    th.close()


def test_out_of_range_indices_are_flagged(md):
    lay, theta, d, g = md
    for expr in ("p[100000] * t", "p[m[40]] * t", "f[3] * t"):
        th = UserTheory(expr, n_funcs=1)
        with Run(lay, d) as run:
            v = th.eval(run, theta, MUSR_CHI2, funcs=[1.0])[0]
            assert v == np.inf
            with pytest.raises(MusrError):
                th.grad(run, theta, MUSR_CHI2, funcs=[1.0], rel_h=0.0)
        th.close()
