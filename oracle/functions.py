"""FP64 oracle of the function array (Sec. 4.2.1): values that the theory reads
through the map but that are functions of the parameters.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
baseline).  Shares no code with the CUDA library.

The paper's framework computes the function array from the parameters before
each evaluation and passes it to the kernel beside the parameter array.  Here:
  * a function is an arithmetic expression over p[i] with + - * / ^ (power,
    right-associative, above unary minus), parentheses and the functions exp
    log sqrt sin cos tan atan abs pow, evaluated by Python's own expression
    evaluator over a whitelisted syntax tree ('^' is rewritten to '**');
  * a map entry -2 - j stands for function j; the run is evaluated as an
    extended run whose parameter vector is [theta, f(theta)] and whose map
    points those entries at the appended slots;
  * derivatives follow the chain rule, d/dtheta = A^T d/d[theta, f] with
    A = [I; J], J = df/dtheta from a fourth-order central difference of each
    function (error ~1e-11 relative, far inside the gradient tolerance); the
    Gauss-Newton matrix of the composition is A^T H A.
"""
from __future__ import annotations

import ast
import dataclasses
import math

import numpy as np

import oracle

_FUNCS = {"exp": math.exp, "log": math.log, "sqrt": math.sqrt, "sin": math.sin, "cos": math.cos,
          "tan": math.tan, "atan": math.atan, "abs": abs, "fabs": abs, "pow": math.pow}
_NODES = (ast.Expression, ast.BinOp, ast.UnaryOp, ast.Call, ast.Name, ast.Load, ast.Constant, ast.Subscript,
          ast.Add, ast.Sub, ast.Mult, ast.Div, ast.Pow, ast.USub, ast.UAdd)


def _tree(expr: str) -> ast.Expression:
    tree = ast.parse(expr.replace("^", "**"), mode="eval")
    for node in ast.walk(tree):
        if not isinstance(node, _NODES):
            raise ValueError(f"unsupported syntax in {expr!r}")
        if isinstance(node, ast.Name) and node.id != "p" and node.id not in _FUNCS:
            raise ValueError(f"unknown name {node.id!r}")
    return tree


def value(expr: str, theta) -> float:
    """f(theta) for one function-array expression."""
    code = compile(_tree(expr), "<function>", "eval")
    return float(eval(code, {"__builtins__": {}}, dict(_FUNCS, p=list(map(float, theta)))))


def jacobian_row(expr: str, theta) -> np.ndarray:
    """df/dtheta by the fourth-order central difference (f(-2h) - 8f(-h) + 8f(h) - f(2h)) / 12h."""
    theta = np.asarray(theta, dtype=np.float64)
    row = np.zeros(theta.shape[0])
    for j in range(theta.shape[0]):
        if f"p[{j}]" not in expr.replace(" ", ""):
            continue
        h = 1e-3 * max(abs(theta[j]), 1.0)
        v = []
        for s in (-2, -1, 1, 2):
            t = theta.copy()
            t[j] += s * h
            v.append(value(expr, t))
        row[j] = (v[0] - 8.0 * v[1] + 8.0 * v[2] - v[3]) / (12.0 * h)
    return row


def extended(lay, theta):
    """(layout, theta) of the extended run: theta followed by the function values,
    map entries -2 - j pointing at slot P + j."""
    funcs = list(getattr(lay, "funcs", None) or [])
    P = int(lay.n_params)
    ext = np.concatenate([np.asarray(theta, dtype=np.float64), [value(f, theta) for f in funcs]])
    mp = np.array(lay.map, dtype=np.int32, copy=True)
    fmask = mp <= -2
    mp[fmask] = P + (-2 - mp[fmask])
    lay_x = dataclasses.replace(lay, map=mp, n_params=P + len(funcs),
                                names=list(lay.names) + [f"f{j}" for j in range(len(funcs))],
                                free=np.concatenate([lay.free, np.zeros(len(funcs), dtype=np.uint8)]),
                                funcs=[])
    return lay_x, ext


def chain(lay, theta) -> np.ndarray:
    """A = [I; J], the derivative of [theta, f(theta)] with respect to theta."""
    funcs = list(getattr(lay, "funcs", None) or [])
    P = int(lay.n_params)
    A = np.zeros((P + len(funcs), P))
    A[:P] = np.eye(P)
    for j, f in enumerate(funcs):
        A[P + j] = jacobian_row(f, theta)
    return A


def model(lay, theta) -> np.ndarray:
    lx, tx = extended(lay, theta)
    return oracle.model(lx, tx)


def objective(lay, data, theta, obj=oracle.CHI2) -> float:
    lx, tx = extended(lay, theta)
    return oracle.objective(lx, data, tx, obj)


def gradient(lay, data, theta, obj=oracle.CHI2, with_gn=True):
    """(value, gradient, GN matrix or None) with respect to theta, by the chain rule."""
    lx, tx = extended(lay, theta)
    v, g, H = oracle.gradient(lx, data, tx, obj, with_gn=with_gn)
    A = chain(lay, theta)
    return v, A.T @ g, (A.T @ H @ A if with_gn else None)
