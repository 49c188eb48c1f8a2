"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test names what it pins.  Together they are chosen so that a plausible
slip anywhere in the oracle (a dropped term, a wrong sign, a wrong factor of
2 pi or gamma, a swapped index, a wrong weight) fails at least one of them.
None of them re-derives the oracle's value by retyping its formula.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W


def lifetime_only_layout(n_bins, dt, t0=0.0):
    """One histogram, no asymmetry components: N = N0 e^{-t/tau} + bkg."""
    lay = W.single_hist_layout(n_bins, dt, t0)
    lay.comp = np.zeros((0, 6), dtype=np.int32)
    return lay


def unit_signal_layout(kind, n_bins=4096, dt=0.001):
    """N0 = 1, bkg = 0, tau huge, one component: N - 1 is the bare component."""
    lay = W.single_hist_layout(n_bins, dt)
    lay.tau_us = 1e300
    if kind == W.KT_STATIC_GAUSS:
        lay.comp = np.array([[kind, 2, 3, -1, -1, -1]], dtype=np.int32)
    else:
        lay.comp = np.array([[kind, 2, 3, 4, -1, 5]], dtype=np.int32)
    return lay


def t_grid(lay):
    return lay.t0_us + np.arange(lay.total_bins) * lay.dt_us


# ---------------------------------------------------------------------------
# Eq. 1: theory function
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("t0", [0.0, 0.37])
def test_geometric_series_closed_form(t0):
    """A = 0, bkg = 0, N0 = 1, d = 0: sum_n e^{-(t0 + n dt)/tau} is a geometric series.

    deviance = 2 sum N = 2 e^{-t0/tau} (1 - r^M)/(1 - r),  r = e^{-dt/tau}
    chi2 (sigma^2 = 1 at d = 0) = sum N^2 = e^{-2 t0/tau} (1 - r^{2M})/(1 - r^2)
    """
    M, dt = 5000, 0.01
    lay = lifetime_only_layout(M, dt, t0)
    theta = np.array([1.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    d = np.zeros(M)
    r = math.exp(-dt / W.TAU_MU_US)
    c = math.exp(-t0 / W.TAU_MU_US)
    dev = oracle.objective(lay, d, theta, oracle.POISSON)
    chi = oracle.objective(lay, d, theta, oracle.CHI2)
    assert dev == pytest.approx(2 * c * (1 - r**M) / (1 - r), rel=1e-13)
    assert chi == pytest.approx(c * c * (1 - r ** (2 * M)) / (1 - r * r), rel=1e-13)


def test_lifetime_and_background():
    """N(t_n) = N0 e^{-t_n/tau} + bkg: N(0) = N0 + bkg, and N - bkg halves every tau ln 2."""
    dt = W.TAU_MU_US * math.log(2) / 100  # 100 bins per half-life
    lay = lifetime_only_layout(1001, dt)
    theta = np.array([800.0, 7.0, 0, 0, 0, 0])
    n = oracle.model(lay, theta)
    assert n[0] == pytest.approx(807.0, rel=1e-15)
    ratios = (n[100::100] - 7.0) / (n[:-100:100] - 7.0)
    np.testing.assert_allclose(ratios, 0.5, rtol=1e-12)


def test_kubo_toyabe_special_values():
    """Static Gaussian KT: G(0) = 1, G(t -> inf) = 1/3, minimum at Delta t = sqrt(3)
    with value 1/3 - (4/3) e^{-3/2} (the Kubo-Toyabe function with real-valued 1/3, 2/3)."""
    lay = unit_signal_layout(W.KT_STATIC_GAUSS, n_bins=200001, dt=1e-4)
    delta = 0.9
    theta = np.array([1.0, 0.0, 1.0, delta, 0.0, 0.0])
    g = oracle.model(lay, theta) - 1.0
    t = t_grid(lay)
    assert g[0] == pytest.approx(1.0, abs=1e-15)
    assert g[-1] == pytest.approx(1.0 / 3.0, abs=1e-12)  # Delta t = 18: e^{-162} negligible
    i = int(np.argmin(g))
    assert abs(t[i] - math.sqrt(3) / delta) <= lay.dt_us
    assert g[i] == pytest.approx(1 / 3 - 4 / 3 * math.exp(-1.5), abs=1e-8)
    assert 1 / 3 - 4 / 3 * math.exp(-1.5) == pytest.approx(0.035826, abs=1e-6)


@pytest.mark.parametrize("kind", [W.TF_EXP, W.TF_GAUSS])
def test_precession_special_points(kind):
    """cos(2 pi gamma B t + phi): value cos(phi) at t = 0, -sin(phi) after a quarter
    period T/4 = 1/(4 gamma B), period T exactly, and no relaxation when rate = 0."""
    B, phi = 200.0, 0.4
    period = 1.0 / (W.GAMMA_MU_MHZ_PER_G * B)
    n_per = 1000
    lay = unit_signal_layout(kind, n_bins=4 * n_per + 1, dt=period / n_per)
    theta = np.array([1.0, 0.0, 1.0, 0.0, B, phi])
    s = oracle.model(lay, theta) - 1.0
    assert s[0] == pytest.approx(math.cos(phi), abs=1e-14)
    assert s[n_per // 4] == pytest.approx(-math.sin(phi), abs=1e-12)
    assert s[n_per // 2] == pytest.approx(-math.cos(phi), abs=1e-12)
    np.testing.assert_allclose(s[n_per:], s[:-n_per], atol=1e-11)


def test_relaxation_envelopes():
    """At cos = 1 points (phi = 0, t = m T): exponential envelope e^{-lambda t},
    Gaussian envelope e^{-(sigma t)^2 / 2} (Sec. 4.2.1 relaxation functions, Eq. 5)."""
    B = 100.0
    period = 1.0 / (W.GAMMA_MU_MHZ_PER_G * B)
    n_per = 500
    for kind, rate, env in [(W.TF_EXP, 0.7, lambda t: np.exp(-0.7 * t)),
                            (W.TF_GAUSS, 0.45, lambda t: np.exp(-0.5 * (0.45 * t) ** 2))]:
        lay = unit_signal_layout(kind, n_bins=10 * n_per + 1, dt=period / n_per)
        theta = np.array([1.0, 0.0, 1.0, rate, B, 0.0])
        s = oracle.model(lay, theta) - 1.0
        peaks = s[::n_per]
        tp = np.arange(peaks.size) * period
        np.testing.assert_allclose(peaks, env(tp), rtol=1e-11)


def test_field_offset_adds_to_field():
    """field2 adds to the field: (B, dB) gives the same signal as B + dB alone."""
    lay1 = unit_signal_layout(W.TF_GAUSS, 3000, 0.003)
    lay2 = unit_signal_layout(W.TF_GAUSS, 3000, 0.003)
    lay2.map = np.array([[0, 1, 2, 3, 4, 5, 6]], dtype=np.int32)
    lay2.comp = np.array([[W.TF_GAUSS, 2, 3, 4, 6, 5]], dtype=np.int32)
    lay2.n_params = 7
    t1 = np.array([1.0, 0.0, 0.8, 0.3, 330.0, 1.1])
    t2 = np.array([1.0, 0.0, 0.8, 0.3, 300.0, 1.1, 30.0])
    np.testing.assert_allclose(oracle.model(lay1, t1), oracle.model(lay2, t2), rtol=0, atol=1e-12)


def test_precession_frequency_by_fft():
    """The spectrum of the precession signal peaks at gamma_mu B (numpy FFT)."""
    B = 250.0
    lay = unit_signal_layout(W.TF_EXP, n_bins=1 << 16, dt=0.0005)
    theta = np.array([1.0, 0.0, 1.0, 0.0, B, 0.2])
    s = oracle.model(lay, theta) - 1.0
    spec = np.abs(np.fft.rfft(s))
    freqs = np.fft.rfftfreq(s.size, lay.dt_us)
    assert abs(freqs[np.argmax(spec)] - W.GAMMA_MU_MHZ_PER_G * B) <= freqs[1]


def test_mapped_multi_detector_matches_single_histograms():
    """Map indirection (Eq. 2, the map array of Sec. 4.2.1): each histogram of a 3-detector run equals
    a standalone single-histogram run with its own N0, bkg, phase and the shared rest."""
    lay = W.multi_detector_layout(3, [700, 500, 900], window_us=5.0)
    lay.comp = lay.comp[:1].copy()  # TF_EXP line only, so the single layout can express it
    theta = W.multi_detector_theta(lay, W.rng(5))
    full = oracle.model(lay, theta)
    off = 0
    idx = {n: i for i, n in enumerate(lay.names)}
    for k in range(3):
        single = W.single_hist_layout(int(lay.n_bins[k]), lay.dt_us)
        th = np.array([theta[idx[f"N0_{k}"]], theta[idx[f"bkg_{k}"]], theta[idx["A1"]],
                       theta[idx["lambda1"]], theta[idx["B1"]], theta[idx[f"phi_{k}"]]])
        part = oracle.model(single, th)
        np.testing.assert_array_equal(full[off:off + part.size], part)
        off += part.size


# ---------------------------------------------------------------------------
# Eq. 3 / Eq. 4 objectives
# ---------------------------------------------------------------------------
def test_noise_free_data_gives_zero():
    """chi2 = 0 and deviance = 0 when d equals the noise-free FP64 model."""
    lay, theta, _ = W.config_multi_detector(4, 3000)
    d = oracle.model(lay, theta)
    assert oracle.objective(lay, d, theta, oracle.CHI2) == 0.0
    assert oracle.objective(lay, d, theta, oracle.POISSON) == 0.0


def test_deviance_equals_scipy_log_likelihood_ratio():
    """Eq. 4 read as -2 ln(L(N)/L_saturated): equals -2 sum [logpmf(d; N) - logpmf(d; d)]
    with scipy's Poisson log-pmf (which includes d = 0 bins, where logpmf(0; 0) = 0)."""
    lay, theta, seed = W.config_multi_detector(3, 2000)
    mean = oracle.model(lay, theta)
    d = W.poisson_counts(mean * 0.01, seed)  # low counts, many zeros
    mean_fit = oracle.model(lay, theta * np.where(lay.free.astype(bool), 0.0101, 1.0))
    # evaluate at a theta whose model is mean_fit
    th = theta * np.where(lay.free.astype(bool), 0.0101, 1.0)
    dev = oracle.objective(lay, d, th, oracle.POISSON)
    ref = -2.0 * np.sum(stats.poisson.logpmf(d, mean_fit) - stats.poisson.logpmf(d, d))
    assert (d == 0).sum() > 100
    assert dev == pytest.approx(ref, rel=1e-10)


def test_deviance_domain():
    """N <= 0 where d > 0 has no Poisson likelihood: the oracle reports EDOMAIN."""
    lay = lifetime_only_layout(10, 0.1)
    d = np.ones(10)
    theta = np.array([-5.0, 0.0, 0, 0, 0, 0])
    v, st = oracle.objective(lay, d, theta, oracle.POISSON, raise_on_error=False)
    assert st == oracle.EDOMAIN and v == math.inf


def test_chi2_weighted_mean_minimum():
    """Constant theory N = bkg: the chi2 minimum over bkg is the weighted mean with
    weights 1/max(d, 1) (closed form), which pins the sigma^2 = max(d, 1) reading."""
    lay = lifetime_only_layout(3000, 0.01)
    d = W.poisson_counts(np.full(3000, 3.0), 11)
    theta0 = np.array([0.0, 2.0, 0, 0, 0, 0])
    free = np.array([0, 1, 0, 0, 0, 0], dtype=np.uint8)
    th, info, cov = oracle.fit(lay, d, theta0, oracle.CHI2, free, edm_tol=1e-16)
    w = 1.0 / np.maximum(d, 1.0)
    assert info["status"] == 0
    # a value-driven minimiser locates the minimum to ~sqrt(2 eps f / H) ~ 1e-8 relative
    assert th[1] == pytest.approx(np.sum(w * d) / np.sum(w), rel=1e-8)
    # parameter error of a weighted mean: 1 / sqrt(sum w)
    assert math.sqrt(cov[0, 0]) == pytest.approx(1 / math.sqrt(np.sum(w)), rel=1e-8)


def test_poisson_mle_of_constant_is_sample_mean():
    """Deviance fit of a constant mean: the MLE is the sample mean (closed form)."""
    lay = lifetime_only_layout(2500, 0.01)
    d = W.poisson_counts(np.full(2500, 2.2), 12)
    th, info, _ = oracle.fit(lay, d, np.array([0.0, 1.0, 0, 0, 0, 0]), oracle.POISSON,
                             np.array([0, 1, 0, 0, 0, 0], dtype=np.uint8), edm_tol=1e-16)
    assert info["status"] == 0
    assert th[1] == pytest.approx(d.mean(), rel=1e-8)


def test_linear_parameters_match_weighted_least_squares():
    """With only N0 and bkg free the theory is linear in them: the chi2 fit equals
    numpy's weighted linear least squares on the design [shape, 1]."""
    lay, theta, seed = W.config_single()
    lay.n_bins = np.array([3000])
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    free = np.array([1, 1, 0, 0, 0, 0], dtype=np.uint8)
    start = theta.copy()
    start[:2] = [500.0, 1.0]
    th, info, _ = oracle.fit(lay, d, start, oracle.CHI2, free, edm_tol=1e-16)
    shape = oracle.model(lay, np.r_[1.0, 0.0, theta[2:]])
    w = 1.0 / np.sqrt(np.maximum(d, 1.0))
    X = np.stack([shape, np.ones_like(shape)], 1) * w[:, None]
    sol, *_ = np.linalg.lstsq(X, d * w, rcond=None)
    np.testing.assert_allclose(th[:2], sol, rtol=1e-8)


def test_histogram_permutation_invariance():
    """The objective is a sum over histograms: reordering them with their map rows
    changes nothing (exactly, up to compensated-summation rounding)."""
    lay, theta, seed = W.config_multi_detector(5, 1500)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.02, W.rng(3))
    perm = [3, 0, 4, 2, 1]
    offs = np.r_[0, np.cumsum(lay.n_bins)]
    dp = np.concatenate([d[offs[k]:offs[k + 1]] for k in perm])
    lp = lay.permuted(perm)
    for obj in (oracle.CHI2, oracle.POISSON):
        a = oracle.objective(lay, d, th, obj)
        b = oracle.objective(lp, dp, th, obj)
        assert a == pytest.approx(b, rel=1e-15)


def test_chi2_per_dof_at_truth():
    """With Poisson data at the generating parameters, chi2/ndf = 1 within a few
    sqrt(2/ndf).  A 2 us window keeps every mean above ~80 counts, where the
    sigma^2 = d weighting is unbiased to O(1/N)."""
    lay, theta, seed = W.config_multi_detector(4, 20000, window_us=2.0)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    n = d.size
    chi = oracle.objective(lay, d, theta, oracle.CHI2)
    assert abs(chi / n - 1.0) < 5 * math.sqrt(2.0 / n) + 0.01


def test_brute_force_8_bins_mpmath():
    """8-bin inputs evaluated independently at 50 digits (mpmath): the FP64 oracle
    agrees to ~1e-15 relative on the theory and both objectives."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    lay = W.multi_detector_layout(2, 8, window_us=3.0)
    theta = W.multi_detector_theta(lay, W.rng(8))
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
            p = lambda s: mp(theta[idx[s]])
            phi = mp(theta[idx[f"phi_{k}"]])
            a1 = p("A1") * mpmath.exp(-p("lambda1") * t) * mpmath.cos(2 * mpmath.pi * gam * p("B1") * t + phi)
            a2 = p("A2") * mpmath.exp(-(p("sigma2") * t) ** 2 / 2) * mpmath.cos(
                2 * mpmath.pi * gam * (p("B1") + p("dB")) * t + phi)
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


# ---------------------------------------------------------------------------
# Gradient and Gauss-Newton matrix
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("obj", [oracle.CHI2, oracle.POISSON])
def test_analytic_gradient_matches_central_differences(obj):
    """Hand-derived chain rule vs FP64 central differences of the objective itself,
    for every parameter (including fixed phases and the field offset dB)."""
    lay, theta, seed = W.config_multi_detector(3, 1200)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.03, W.rng(21))
    _, g, _ = oracle.gradient(lay, d, th, obj, with_gn=False)
    gfd = oracle.gradient_fd(lay, d, th, obj, rel_h=1e-6)
    scale = np.abs(g).max()
    np.testing.assert_allclose(g, gfd, rtol=1e-5, atol=1e-6 * scale)


@pytest.mark.parametrize("obj", [oracle.CHI2, oracle.POISSON])
def test_gauss_newton_is_exact_hessian_at_zero_residual(obj):
    """With noise-free data the residual vanishes, so the Gauss-Newton matrix equals
    the exact Hessian; compare with central differences of the analytic gradient."""
    lay, theta, _ = W.config_multi_detector(2, 800)
    d = oracle.model(lay, theta)
    _, _, H = oracle.gradient(lay, d, theta, obj)
    P = lay.n_params
    Hfd = np.zeros((P, P))
    for j in range(P):
        h = 1e-5 * max(abs(theta[j]), 1.0)
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        Hfd[:, j] = (oracle.gradient(lay, d, tp, obj, False)[1] -
                     oracle.gradient(lay, d, tm, obj, False)[1]) / (2 * h)
    np.testing.assert_allclose(H, Hfd, rtol=2e-5, atol=1e-6 * np.abs(H).max())


# ---------------------------------------------------------------------------
# Fit
# ---------------------------------------------------------------------------
def test_fit_recovers_noise_free_truth():
    """LM on noise-free data from a 5 % perturbed start returns the generating
    parameters (to ~1e-8 relative) with chi2 ~ 0."""
    lay, theta, seed = W.config_single()
    d = oracle.model(lay, theta)
    start = W.perturb(theta, lay.free, 0.05, W.rng(seed))
    th, info, _ = oracle.fit(lay, d, start, oracle.CHI2)
    assert info["status"] == 0
    np.testing.assert_allclose(th, theta, rtol=1e-7)
    assert info["value"] < 1e-10


def test_fit_pulls_are_unit_normal():
    """Poisson data at known truth, fitted by the Poisson deviance (maximum
    likelihood) from the truth: the pulls (theta_hat - theta_true)/sigma_hat over
    240 seeds have mean ~0 and std ~1 (bounds ~4.5 standard errors: 1/sqrt(240) on
    the mean, 1/sqrt(480) on the std) and pass a KS test against N(0, 1).  (The
    chi2 with sigma^2 = d is biased low on the background by the low-count tail,
    as expected of Neyman's chi2.)"""
    lay, theta, _ = W.config_single()
    lay.n_bins = np.array([2048])
    lay.dt_us = 0.005
    mean = oracle.model(lay, theta)
    pulls = []
    for s in range(240):
        d = W.poisson_counts(mean, 1000 + s)
        th, info, cov = oracle.fit(lay, d, theta, oracle.POISSON)
        assert info["status"] == 0
        pulls.append((th - theta) / np.sqrt(np.diag(cov)))
    pulls = np.array(pulls)
    assert np.all(np.abs(pulls.mean(0)) < 0.3)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.2)
    for j in range(pulls.shape[1]):
        assert stats.kstest(pulls[:, j], "norm").pvalue > 1e-3
