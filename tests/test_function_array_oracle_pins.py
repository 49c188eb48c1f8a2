"""Pins of the oracle's function array (oracle/functions.py, Sec. 4.2.1):

  * an identity function reproduces the plain run exactly;
  * a linear function B1 + dB in place of the map's two-entry field sum gives
    the same objective, gradient and Gauss-Newton matrix as the C oracle's own
    sum (two independent routes to one number);
  * the chain-rule gradient of a nonlinear function equals central
    differences of the objective taken through the functions themselves;
  * the expression evaluator's precedence and associativity.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from oracle import functions as of


def with_field_function(lay):
    """The multi-detector run with the Gaussian line's field read from function 0 =
    B1 + dB (a new map column holding -2) instead of the field / field2 pair."""
    names = lay.names
    b1, db = names.index("B1"), names.index("dB")
    mp = np.concatenate([lay.map, np.full((lay.n_hist, 1), -2, dtype=np.int32)], axis=1)
    comp = lay.comp.copy()
    comp[1, 3], comp[1, 4] = mp.shape[1] - 1, -1
    import dataclasses
    return dataclasses.replace(lay, map=mp, comp=comp, funcs=[f"p[{b1}] + p[{db}]"])


@pytest.mark.parametrize("expr,val", [("1 + 2 * 3", 7.0), ("(1 + 2) * 3", 9.0), ("2 ^ 3 ^ 2", 512.0),
                                      ("-2 ^ 2", -4.0), ("2 ^ -1", 0.5), ("pow(4, 0.5) + abs(-3)", 5.0),
                                      ("p[1] / p[0] - 1", 1.0)])
def test_expression_values(expr, val):
    assert of.value(expr, [2.0, 4.0]) == pytest.approx(val, rel=1e-15)


def test_identity_function_is_the_plain_run():
    lay, theta, seed = W.config_multi_detector(3, 1500)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    j = lay.names.index("A2")
    import dataclasses
    mp = lay.map.copy()
    mp[:, 6] = -2
    lf = dataclasses.replace(lay, map=mp, funcs=[f"p[{j}]"])
    for obj in (oracle.CHI2, oracle.POISSON):
        v0, g0, H0 = oracle.gradient(lay, d, theta, obj)
        v1, g1, H1 = of.gradient(lf, d, theta, obj)
        assert v1 == pytest.approx(v0, rel=1e-14)
        np.testing.assert_allclose(g1, g0, rtol=1e-9, atol=1e-9 * np.abs(g0).max())
        np.testing.assert_allclose(H1, H0, rtol=1e-9, atol=1e-9 * np.abs(H0).max())


def test_linear_function_matches_the_two_entry_field_sum():
    lay, theta, seed = W.config_multi_detector(3, 1500)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    lf = with_field_function(lay)
    np.testing.assert_allclose(of.model(lf, theta), oracle.model(lay, theta), rtol=1e-14)
    for obj in (oracle.CHI2, oracle.POISSON):
        v0, g0, H0 = oracle.gradient(lay, d, theta, obj)
        v1, g1, H1 = of.gradient(lf, d, theta, obj)
        assert v1 == pytest.approx(v0, rel=1e-13)
        np.testing.assert_allclose(g1, g0, rtol=1e-8, atol=1e-9 * np.abs(g0).max())
        np.testing.assert_allclose(H1, H0, rtol=1e-8, atol=1e-9 * np.abs(H0).max())


def test_nonlinear_chain_rule_matches_central_differences():
    """A2 = A1 * r (r a new parameter) and sigma2 = sqrt(lambda1^2 + s^2): the
    chain-rule gradient against central differences of the objective itself."""
    import dataclasses
    lay, theta, seed = W.config_multi_detector(2, 1200)
    names = lay.names + ["r", "s"]
    P = lay.n_params
    th = np.concatenate([theta, [1.3, 0.4]])
    a1, l1 = lay.names.index("A1"), lay.names.index("lambda1")
    mp = lay.map.copy()
    mp[:, 6] = -2   # A2 column -> function 0
    mp[:, 7] = -3   # sigma2 column -> function 1
    lf = dataclasses.replace(lay, map=mp, n_params=P + 2, names=names,
                             free=np.concatenate([lay.free, [1, 1]]).astype(np.uint8),
                             funcs=[f"p[{a1}] * p[{P}]", f"sqrt(p[{l1}] ^ 2 + p[{P + 1}] ^ 2)"])
    d = W.poisson_counts(of.model(lf, th), seed)
    for obj in (oracle.CHI2, oracle.POISSON):
        _, g, _ = of.gradient(lf, d, th, obj, with_gn=False)
        fd = np.zeros_like(g)
        for j in range(th.shape[0]):
            h = 1e-6 * max(abs(th[j]), 1.0)
            tp, tm = th.copy(), th.copy()
            tp[j] += h
            tm[j] -= h
            fd[j] = (of.objective(lf, d, tp, obj) - of.objective(lf, d, tm, obj)) / (2 * h)
        np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_jacobian_row_against_closed_form():
    th = [0.7, 2.0, 3.0]
    row = of.jacobian_row("p[0] * exp(p[1]) / p[2]", th)
    e = math.exp(2.0)
    np.testing.assert_allclose(row, [e / 3.0, 0.7 * e / 3.0, -0.7 * e / 9.0], rtol=1e-10)
