"""Pins of the user-theory oracle: C typing of literals, the predefined muSR
functions against closed forms and against each other, and the
multi-detector theory written as an expression against the C oracle's
built-in components (two independent implementations)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import utheory as U

T = np.linspace(0.0, 12.8, 2001)


def ev(expr, p=(), m=(), f=None):
    return U.Expression(expr).evaluate(T, np.asarray(p, dtype=float), np.asarray(m, dtype=int), f)


def test_c_integer_division_and_literals():
    np.testing.assert_array_equal(ev("1/3 + 0*t"), 0.0)
    np.testing.assert_array_equal(ev("-7/2 + 0*t"), -3.0)
    np.testing.assert_allclose(ev("1.0/3 + 0*t"), 1.0 / 3.0, rtol=1e-15)
    np.testing.assert_allclose(ev("2*t"), 2.0 * T, rtol=0)


def test_predefined_functions_closed_forms():
    lam, beta, sig = 0.7, 1.0, 1.3
    np.testing.assert_allclose(ev("ge(t, p[0], p[1])", [lam, 1.0]), ev("se(t, p[0])", [lam]), rtol=1e-14)
    # ge with beta = 2 is the Gaussian with sigma = sqrt(2) lambda
    np.testing.assert_allclose(ev("ge(t, p[0], p[1])", [lam, 2.0]), ev("sg(t, p[0])", [math.sqrt(2) * lam]),
                               rtol=1e-13, atol=1e-300)
    # ge at lambda t = 1 is 1/e for any beta
    np.testing.assert_allclose(U.ge(np.array([1.0 / lam]), lam, 0.37), math.exp(-1), rtol=1e-15)
    np.testing.assert_allclose(ev("se(t, p[0])", [lam]), np.exp(-lam * T), rtol=1e-15)
    # static Gaussian Kubo-Toyabe: 1 at t = 0, minimum 1/3 - 4/3 e^{-3/2} at sigma t = sqrt(3), 1/3 at infinity
    assert U.stg(np.array([0.0]), sig)[0] == 1.0
    tm = math.sqrt(3) / sig
    np.testing.assert_allclose(U.stg(np.array([tm]), sig), 1 / 3 - 4 / 3 * math.exp(-1.5), rtol=1e-14)
    assert abs(U.stg(np.array([1e3]), sig)[0] - 1 / 3) < 1e-15
    # precession: cos(phi) at t = 0 and one period at 1 / (gamma B)
    np.testing.assert_allclose(U.tf(np.array([0.0]), 0.3, 250.0), math.cos(0.3), rtol=1e-15)
    per = 1.0 / (U.GAMMA_MHZ_PER_G * 250.0)
    np.testing.assert_allclose(U.tf(np.array([per]), 0.3, 250.0), math.cos(0.3), rtol=1e-12)
    assert beta == 1.0


@pytest.mark.parametrize("obj", [oracle.CHI2, oracle.POISSON])
def test_multi_detector_expression_matches_builtin_oracle(obj):
    lay = W.multi_detector_layout(4, [3000, 5000, 777, 4096], window_us=12.8)
    theta = W.multi_detector_theta(lay, W.rng(3))
    m_user = U.model(lay, theta, W.MD_USER_EXPR)
    m_c = oracle.model(lay, theta)
    np.testing.assert_allclose(m_user, m_c, rtol=1e-12, atol=0)
    d = W.poisson_counts(m_c, 11)
    v_user = U.objective(lay, d, theta, W.MD_USER_EXPR, obj)
    v_c = oracle.objective(lay, d, theta, obj)
    assert v_user == pytest.approx(v_c, rel=1e-11)


def test_function_array_and_rejections():
    np.testing.assert_allclose(ev("f[0] * t + f[1]", f=[2.0, 0.5]), 2.0 * T + 0.5, rtol=1e-15)
    for bad in ("t; x", "t == 1", "__import__('os')", "t{0}", "q[0]"):
        with pytest.raises(ValueError):
            ev(bad)
