"""FP64 oracle for user-defined theory functions (test infrastructure only:
the test-suite and the benchmark's CPU leg may import it; the GPU library
never does and this module imports nothing of it).

Sec. 4.2.1 of the paper: the asymmetry A_k(t) of a histogram is a C
expression over t (us), the parameter array p, the histogram's map row m and
a function array f, using the predefined muSR functions of the
user-function language (se, ge, sg, stg, tf: exponential, stretched
exponential, Gaussian and static Gaussian Kubo-Toyabe relaxation, precession),
written from their definitions, plus the C math functions.  This module
evaluates such an expression directly from its syntax tree with numpy, in
FP64, vectorised over t, keeping C's typing of literals (an int / int
division truncates toward zero, as in the compiled kernel), and forms
N_k(t) = p[m[0]] exp(-t/tau) (1 + A_k(t)) + p[m[1]] and the objectives of
Eq. 3 (chi2, sigma^2 = max(d, 1)) and Eq. 4 (Poisson deviance) from their
definitions.
"""
from __future__ import annotations

import ast
import math

import numpy as np

GAMMA_MHZ_PER_G = 0.013554  # muon gyromagnetic ratio / (2 pi)


def se(t, lam):
    return np.exp(-lam * t)


def ge(t, lam, beta):
    x = lam * t
    return np.where(x > 0.0, np.exp(-np.power(np.maximum(x, 0.0), beta)), 1.0)


def sg(t, sigma):
    x = sigma * t
    return np.exp(-0.5 * x * x)


def stg(t, sigma):
    x2 = (sigma * t) ** 2
    return 1.0 / 3.0 + 2.0 / 3.0 * (1.0 - x2) * np.exp(-0.5 * x2)


def tf(t, phi, field):
    return np.cos(2.0 * math.pi * GAMMA_MHZ_PER_G * field * t + phi)


_FUNCS = {
    "se": se, "ge": ge, "sg": sg, "stg": stg, "tf": tf,
    "exp": np.exp, "log": np.log, "sqrt": np.sqrt, "cos": np.cos, "sin": np.sin, "tan": np.tan,
    "pow": np.power, "fabs": np.abs, "tanh": np.tanh, "cosh": np.cosh, "sinh": np.sinh,
    "atan": np.arctan, "atan2": np.arctan2, "fmin": np.minimum, "fmax": np.maximum,
}


class _Value:
    """An evaluated sub-expression: array or scalar, and whether C types it int."""

    def __init__(self, v, is_int):
        self.v = v
        self.is_int = is_int


def _c_div(a: _Value, b: _Value) -> _Value:
    if a.is_int and b.is_int:
        q = abs(int(a.v)) // abs(int(b.v))
        return _Value(q if (int(a.v) >= 0) == (int(b.v) >= 0) else -q, True)
    return _Value(np.asarray(a.v, dtype=np.float64) / b.v, False)


class Expression:
    """A parsed user expression; evaluate(t, p, m, f) returns A(t) (FP64)."""

    def __init__(self, text: str):
        allowed = set("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789_.+-*/()[], \t\n")
        if not text or any(c not in allowed for c in text):
            raise ValueError("characters outside the expression alphabet")
        self.text = text
        self.tree = ast.parse(text, mode="eval")

    def evaluate(self, t, p, m, f=None):
        t = np.asarray(t, dtype=np.float64)
        r = self._eval(self.tree.body, t, np.asarray(p, dtype=np.float64), np.asarray(m), f)
        return np.broadcast_to(np.asarray(r.v, dtype=np.float64), t.shape).astype(np.float64)

    def _eval(self, node, t, p, m, f) -> _Value:
        if isinstance(node, ast.Constant) and isinstance(node.value, (int, float)) and not isinstance(node.value, bool):
            return _Value(node.value, isinstance(node.value, int))
        if isinstance(node, ast.Name):
            if node.id == "t":
                return _Value(t, False)
            raise ValueError(f"unknown name {node.id}")
        if isinstance(node, ast.Subscript) and isinstance(node.value, ast.Name):
            idx = self._eval(node.slice, t, p, m, f)
            if not idx.is_int:
                raise ValueError("array index must be an integer")
            i = int(idx.v)
            if node.value.id == "p":
                return _Value(float(p[i]), False)
            if node.value.id == "m":
                return _Value(int(m[i]), True)
            if node.value.id == "f":
                return _Value(float(f[i]), False)
            raise ValueError(f"unknown array {node.value.id}")
        if isinstance(node, ast.UnaryOp) and isinstance(node.op, (ast.USub, ast.UAdd)):
            a = self._eval(node.operand, t, p, m, f)
            return _Value(-a.v if isinstance(node.op, ast.USub) else a.v, a.is_int)
        if isinstance(node, ast.BinOp) and isinstance(node.op, (ast.Add, ast.Sub, ast.Mult, ast.Div)):
            a = self._eval(node.left, t, p, m, f)
            b = self._eval(node.right, t, p, m, f)
            if isinstance(node.op, ast.Div):
                return _c_div(a, b)
            both = a.is_int and b.is_int
            if isinstance(node.op, ast.Add):
                return _Value(a.v + b.v, both)
            if isinstance(node.op, ast.Sub):
                return _Value(a.v - b.v, both)
            return _Value(a.v * b.v, both)
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in _FUNCS:
            args = [np.asarray(self._eval(a, t, p, m, f).v, dtype=np.float64) for a in node.args]
            return _Value(_FUNCS[node.func.id](*args), False)
        raise ValueError(f"unsupported syntax: {ast.dump(node)[:60]}")


def model(lay, theta, expr: str, funcs=None) -> np.ndarray:
    """Eq. 1 with the user asymmetry for every bin of every histogram (FP64)."""
    e = Expression(expr)
    theta = np.asarray(theta, dtype=np.float64)
    out = []
    for k, nb in enumerate(lay.n_bins):
        t = lay.t0_us + np.arange(int(nb), dtype=np.float64) * lay.dt_us
        mrow = np.asarray(lay.map[k])
        a = e.evaluate(t, theta, mrow, funcs)
        out.append(theta[mrow[0]] * np.exp(-t / lay.tau_us) * (1.0 + a) + theta[mrow[1]])
    return np.concatenate(out) if out else np.zeros(0)


def objective(lay, data, theta, expr: str, obj: int = 0, funcs=None) -> float:
    """Eq. 3 chi2 (obj 0) or Eq. 4 Poisson deviance (obj 1) with the user theory;
    +inf where the deviance has no likelihood."""
    n = model(lay, theta, expr, funcs)
    d = np.asarray(data, dtype=np.float64)
    if obj == 0:
        return float(np.sum((d - n) ** 2 / np.maximum(d, 1.0)))
    if np.any((d > 0) & ~(n > 0)) or np.any(n < 0):
        return math.inf
    pos = d > 0
    term = np.where(pos, (n - d) + d * np.log(np.where(pos, d, 1.0) / np.where(pos, n, 1.0)), n)
    return float(2.0 * np.sum(term))
