"""Pins of the FP64 oracle's stretched precession line, a ge(t, lambda, beta)
cos(2 pi gamma (B + B2) t + phi) component (the stretched exponential among
the predefined relaxation functions of Sec. 4.2.1), against facts fixed by
mathematics:

  * beta = 1 is the exponential line, beta = 2 with
    lambda = sigma / sqrt(2) the Gaussian line, bit for bit up to
    rounding, values and derivatives;
  * ge(1/lambda) = 1/e for every beta, ge(2/lambda) = exp(-2^beta);
  * lambda t <= 0 gives ge = 1 (the reading for a negative base, which has
    no real power);
  * the closed-form beta derivative at beta = 1, the analytic gradient against
    central differences of the objective, the Gauss-Newton matrix against the
    exact Hessian at zero residual;
  * 8-bin brute force at 50 digits (mpmath), and the user-theory evaluator
    (an independent implementation of "ge") on the same run.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import utheory as ou


def unit_layout(kind, n_bins=3001, dt=0.002):
    """N0 = 1, bkg = 0, no lifetime: N - 1 is the bare component.
    theta = [N0, bkg, a, rate, B, phi, beta]."""
    lay = W.single_hist_layout(n_bins, dt)
    lay.tau_us = 1e300
    lay.map = np.array([[0, 1, 2, 3, 4, 5, 6]], dtype=np.int32)
    lay.n_params = 7
    lay.names = ["N0", "bkg", "a", "rate", "B", "phi", "beta"]
    lay.free = np.ones(7, dtype=np.uint8)
    lay.comp = W.comp_table([[kind, 2, 3, 4, -1, 5, 6 if kind == W.TF_STRETCHED else -1]])
    return lay


def test_beta_one_is_the_exponential_line():
    """beta = 1: exp(-(lambda t)^1) = exp(-lambda t); model and the derivatives
    shared with the exponential line agree to rounding."""
    th = np.array([1.0, 0.0, 0.7, 0.9, 240.0, 0.35, 1.0])
    st, ex = unit_layout(W.TF_STRETCHED), unit_layout(W.TF_EXP)
    np.testing.assert_allclose(oracle.model(st, th), oracle.model(ex, th), rtol=1e-14, atol=1e-15)
    d = W.poisson_counts(oracle.model(ex, th) * 50.0, 3) / 50.0
    _, g_st, _ = oracle.gradient(st, d, th, oracle.CHI2, with_gn=False)
    _, g_ex, _ = oracle.gradient(ex, d, th, oracle.CHI2, with_gn=False)
    np.testing.assert_allclose(g_st[:6], g_ex[:6], rtol=1e-12, atol=1e-12 * np.abs(g_ex).max())
    assert g_ex[6] == 0.0


def test_beta_two_is_the_gaussian_line():
    """beta = 2, lambda = sigma / sqrt(2): exp(-(lambda t)^2) = exp(-(sigma t)^2 / 2);
    d/d lambda = sqrt(2) d/d sigma."""
    sigma = 1.3
    th_g = np.array([1.0, 0.0, 0.6, sigma, 180.0, -0.4, 0.0])
    th_s = th_g.copy()
    th_s[3] = sigma / math.sqrt(2.0)
    th_s[6] = 2.0
    st, ga = unit_layout(W.TF_STRETCHED), unit_layout(W.TF_GAUSS)
    np.testing.assert_allclose(oracle.model(st, th_s), oracle.model(ga, th_g), rtol=1e-13, atol=1e-14)
    d = np.full(st.total_bins, 1.2)
    _, g_s, _ = oracle.gradient(st, d, th_s, oracle.CHI2, with_gn=False)
    _, g_g, _ = oracle.gradient(ga, d, th_g, oracle.CHI2, with_gn=False)
    scale = np.abs(g_g[:6]).max()
    np.testing.assert_allclose(g_s[[0, 1, 2, 4, 5]], g_g[[0, 1, 2, 4, 5]], rtol=1e-10, atol=1e-11 * scale)
    assert g_s[3] == pytest.approx(math.sqrt(2.0) * g_g[3], rel=1e-10)


@pytest.mark.parametrize("beta", [0.45, 1.0, 1.7, 3.0])
def test_envelope_special_points(beta):
    """phi = 0, B = 0 leaves the envelope alone: ge(0) = 1, ge(1/lambda) = 1/e for
    every beta, ge(2/lambda) = exp(-2^beta)."""
    lam = 0.8
    dt = 1.0 / lam / 1000
    lay = unit_layout(W.TF_STRETCHED, n_bins=2001, dt=dt)
    th = np.array([1.0, 0.0, 1.0, lam, 0.0, 0.0, beta])
    s = oracle.model(lay, th) - 1.0
    assert s[0] == 1.0
    assert s[1000] == pytest.approx(math.exp(-1.0), rel=1e-13)
    assert s[2000] == pytest.approx(math.exp(-(2.0 ** beta)), rel=1e-12)


def test_nonpositive_rate_is_flat():
    """lambda <= 0: ge = 1, the line is the bare cosine (the exponential line at
    rate 0), and no derivative flows into lambda or beta."""
    st, ex = unit_layout(W.TF_STRETCHED), unit_layout(W.TF_EXP)
    for lam in (0.0, -0.4):
        th = np.array([1.0, 0.0, 0.5, lam, 300.0, 0.2, 0.7])
        th0 = th.copy()
        th0[3] = 0.0
        np.testing.assert_allclose(oracle.model(st, th), oracle.model(ex, th0), rtol=1e-15, atol=1e-15)
        d = np.full(st.total_bins, 1.5)
        _, g, _ = oracle.gradient(st, d, th, oracle.CHI2, with_gn=False)
        assert g[3] == 0.0 and g[6] == 0.0


def test_beta_derivative_closed_form_at_beta_one():
    """d/d beta of exp(-(lambda t)^beta) at beta = 1 is -(lambda t) ln(lambda t) e^{-lambda t};
    the chi2 gradient at d = 0 (sigma^2 = 1) is then 2 sum N dN/d beta."""
    lam = 1.1
    lay = unit_layout(W.TF_STRETCHED, n_bins=1500, dt=0.003)
    th = np.array([1.0, 0.0, 0.4, lam, 0.0, 0.0, 1.0])
    t = np.arange(lay.total_bins) * lay.dt_us
    x = lam * t
    with np.errstate(divide="ignore", invalid="ignore"):
        dn = np.where(x > 0, -0.4 * x * np.log(x) * np.exp(-x), 0.0)
    n = 1.0 + 0.4 * np.exp(-x)
    _, g, _ = oracle.gradient(lay, np.zeros(lay.total_bins), th, oracle.CHI2, with_gn=False)
    assert g[6] == pytest.approx(float(np.sum(2.0 * n * dn)), rel=1e-12)


@pytest.mark.parametrize("obj", [oracle.CHI2, oracle.POISSON])
def test_gradient_matches_central_differences(obj):
    """Hand-derived chain rule (including d/d lambda2 and d/d beta) vs FP64
    central differences of the objective on the stretched multi-detector run."""
    lay, theta, seed = W.config_stretched(3, 1200)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.03, W.rng(23))
    _, g, _ = oracle.gradient(lay, d, th, obj, with_gn=False)
    gfd = oracle.gradient_fd(lay, d, th, obj, rel_h=1e-6)
    np.testing.assert_allclose(g, gfd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


@pytest.mark.parametrize("obj", [oracle.CHI2, oracle.POISSON])
def test_gauss_newton_is_exact_hessian_at_zero_residual(obj):
    """Noise-free data: the Gauss-Newton matrix equals the exact Hessian, here
    from central differences of the analytic gradient."""
    lay, theta, _ = W.config_stretched(2, 600)
    d = oracle.model(lay, theta)
    _, _, H = oracle.gradient(lay, d, theta, obj)
    P = lay.n_params
    Hfd = np.zeros((P, P))
    for j in range(P):
        h = 1e-5 * max(abs(theta[j]), 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        Hfd[:, j] = (oracle.gradient(lay, d, tp, obj, False)[1] - oracle.gradient(lay, d, tm, obj, False)[1]) / (2 * h)
    np.testing.assert_allclose(H, Hfd, rtol=2e-5, atol=1e-6 * np.abs(H).max())


def test_brute_force_8_bins_mpmath():
    """8-bin inputs of the stretched run evaluated at 50 digits (mpmath)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    lay = W.multi_detector_layout(2, 8, window_us=3.0, stretched=True)
    theta = W.multi_detector_theta(lay, W.rng(9))
    d = np.array([3, 0, 7, 1, 2, 0, 5, 4, 9, 2, 0, 1, 6, 3, 8, 2], dtype=float)
    n = oracle.model(lay, theta)
    idx = {nm: i for i, nm in enumerate(lay.names)}
    mp = mpmath.mpf
    gam = mp(W.GAMMA_MU_MHZ_PER_G)
    chi = mp(0)
    dev = mp(0)
    for k in range(2):
        for i in range(8):
            t = mp(i) * mp(lay.dt_us)
            p = lambda s: mp(theta[idx[s]])  # noqa: E731
            phi = mp(theta[idx[f"phi_{k}"]])
            a1 = p("A1") * mpmath.exp(-p("lambda1") * t) * mpmath.cos(2 * mpmath.pi * gam * p("B1") * t + phi)
            u = p("lambda2") * t
            ge = mpmath.exp(-(u ** p("beta"))) if u > 0 else mp(1)
            a2 = p("A2") * ge * mpmath.cos(2 * mpmath.pi * gam * (p("B1") + p("dB")) * t + phi)
            x = (p("Delta_KT") * t) ** 2
            kt = p("A_KT") * (mp(1) / 3 + mp(2) / 3 * (1 - x) * mpmath.exp(-x / 2))
            nn = mp(theta[idx[f"N0_{k}"]]) * mpmath.exp(-t / mp(W.TAU_MU_US)) * (1 + a1 + a2 + kt) + \
                mp(theta[idx[f"bkg_{k}"]])
            assert float(nn) == pytest.approx(n[8 * k + i], rel=1e-14)
            dd = mp(d[8 * k + i])
            chi += (dd - nn) ** 2 / max(dd, mp(1))
            dev += 2 * nn if dd == 0 else 2 * ((nn - dd) + dd * mpmath.log(dd / nn))
    assert oracle.objective(lay, d, theta, oracle.CHI2) == pytest.approx(float(chi), rel=1e-14)
    assert oracle.objective(lay, d, theta, oracle.POISSON) == pytest.approx(float(dev), rel=1e-14)


ST_USER_EXPR = ("p[m[3]]*se(t,p[m[4]])*tf(t,p[m[2]],p[m[5]])"
                " + p[m[6]]*ge(t,p[m[7]],p[m[11]])*tf(t,p[m[2]],p[m[5]]+p[m[8]])"
                " + p[m[9]]*stg(t,p[m[10]])")


def test_matches_the_user_theory_evaluator():
    """The built-in stretched run and the same theory written as a user expression
    (the expression evaluator's own se / ge / tf / stg) give the same objectives."""
    lay, theta, seed = W.config_stretched(3, 2000)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    np.testing.assert_allclose(oracle.model(lay, theta), ou.model(lay, theta, ST_USER_EXPR), rtol=1e-13)
    for obj in (oracle.CHI2, oracle.POISSON):
        assert oracle.objective(lay, d, theta, obj) == pytest.approx(
            ou.objective(lay, d, theta, ST_USER_EXPR, obj), rel=1e-12)
