"""The library's function-array expressions (musr_function_eval, host code,
no GPU): values and exact derivatives against closed forms, operator
precedence and associativity, and rejection of malformed input."""
import math

import numpy as np
import pytest

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MusrError, function_eval  # noqa: E402

TH = np.array([0.7, -1.3, 2.5, 4.0])


@pytest.mark.parametrize("expr,value,grad", [
    ("p[0] + p[1]", 0.7 - 1.3, [1, 1, 0, 0]),
    ("1 + 2 * 3", 7.0, [0, 0, 0, 0]),
    ("(1 + 2) * 3", 9.0, [0, 0, 0, 0]),
    ("2 ^ 3 ^ 2", 512.0, [0, 0, 0, 0]),            # right-associative
    ("-p[3] ^ 2", -16.0, [0, 0, 0, -8.0]),          # power before unary minus
    ("p[3] ^ -0.5", 0.5, [0, 0, 0, -0.5 * 4.0 ** -1.5]),
    ("p[0] * p[2] / p[3]", 0.7 * 2.5 / 4, [2.5 / 4, 0, 0.7 / 4, -0.7 * 2.5 / 16]),
    ("pow(p[2], p[0])", 2.5 ** 0.7, [2.5 ** 0.7 * math.log(2.5), 0, 0.7 * 2.5 ** -0.3, 0]),
    ("exp(p[1]) + log(p[3]) + sqrt(p[3])", math.exp(-1.3) + math.log(4) + 2.0, [0, math.exp(-1.3), 0, 0.25 + 0.25]),
    ("sin(p[0]) * cos(p[2])", math.sin(0.7) * math.cos(2.5),
     [math.cos(0.7) * math.cos(2.5), 0, -math.sin(0.7) * math.sin(2.5), 0]),
    ("tan(p[0]) + atan(p[1]) + abs(p[1])", math.tan(0.7) + math.atan(-1.3) + 1.3,
     [1 / math.cos(0.7) ** 2, 1 / (1 + 1.69) - 1.0, 0, 0]),
    ("2.5e-1 * p[3] - .5", 0.5, [0, 0, 0, 0.25]),
])
def test_values_and_derivatives(expr, value, grad):
    v, g = function_eval(expr, TH)
    assert v == pytest.approx(value, rel=1e-14, abs=1e-15)
    np.testing.assert_allclose(g, grad, rtol=1e-13, atol=1e-15)


def test_derivatives_match_central_differences():
    expr = "p[0] * exp(-p[3] / p[2]) + pow(p[2] * p[2] + 1, 0.25) * sin(p[1] - p[0])"
    _, g = function_eval(expr, TH)
    for j in range(TH.shape[0]):
        h = 1e-6 * max(abs(TH[j]), 1.0)
        tp, tm = TH.copy(), TH.copy()
        tp[j] += h
        tm[j] -= h
        fd = (function_eval(expr, tp)[0] - function_eval(expr, tm)[0]) / (2 * h)
        assert g[j] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("expr", ["", "p[4]", "p[-1]", "p[0", "q[0]", "1 +", "(1", "foo(1)", "pow(1)",
                                  "p[0]; p[1]", "1 2", "exp 1"])
def test_rejects_malformed(expr):
    with pytest.raises(MusrError):
        function_eval(expr, TH)


def test_non_finite_value():
    with pytest.raises(MusrError):
        function_eval("log(p[1])", TH)
