"""NumPy FP64 oracle for the learned start proposer's MLP (test infrastructure
only: the test-suite and the benchmark's CPU leg may import it; the GPU
library never does and this module imports nothing of it).

The network is a plain multilayer perceptron, layer l computing
z = a W_l^T + b_l, hidden layers a = max(z, 0), the last layer linear, trained
on the mean squared error with Adam (Kingma and Ba, 2015).  The precision the
proposer fixes is BF16 weights and BF16 tensor-core operands with wider
accumulation, so with ``bf16=True`` this oracle rounds to BF16 (round to
nearest even, through FP32) exactly where a tensor-core operand is formed:
the scaled input, the weights, the hidden activations, and the back-propagated
errors dZ that enter the weight- and input-gradient products.  Bias gradients
and the loss use the unrounded errors.  Everything else is FP64.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even) via FP32; returns FP64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def split_params(flat, shapes):
    """Flat vector (per layer W [out x in] row-major, then b [out]) -> [(W, b)]."""
    out, o = [], 0
    flat = np.asarray(flat, dtype=np.float64)
    for (n_out, n_in) in shapes:
        w = flat[o:o + n_out * n_in].reshape(n_out, n_in)
        o += n_out * n_in
        b = flat[o:o + n_out]
        o += n_out
        out.append((w, b))
    assert o == flat.shape[0]
    return out


def join_params(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for (w, b) in layers])


def forward(layers, x, in_scale=1.0, bf16=True):
    """Activations [a_0 = scaled input, a_1, ..., a_{L-1}] and the output y."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    a = r(np.asarray(x, dtype=np.float64) * in_scale) if bf16 else np.asarray(x, np.float64) * in_scale
    acts = [a]
    for li, (w, b) in enumerate(layers):
        z = acts[-1] @ r(w).T + b
        if li == len(layers) - 1:
            return acts, z
        acts.append(r(np.maximum(z, 0.0)))
    raise AssertionError("no layers")


def loss_and_grads(layers, x, t, in_scale=1.0, bf16=True):
    """MSE loss mean((y - t)^2) and its gradient with respect to every W and b."""
    acts, y = forward(layers, x, in_scale, bf16)
    return backward(layers, acts, y, t, bf16)


def backward(layers, acts, y, t, bf16=True):
    """Back-propagation of the MSE loss from given activations and output."""
    r = bf16_round if bf16 else (lambda v: np.asarray(v, dtype=np.float64))
    acts = [np.asarray(a, dtype=np.float64) for a in acts]
    y = np.asarray(y, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    e = y - t
    loss = float(np.mean(e * e))
    dz = 2.0 * e / e.size
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        w, _ = layers[li]
        dzr = r(dz)
        grads[li] = (dzr.T @ acts[li], dz.sum(axis=0))
        if li > 0:
            dh = dzr @ r(w)
            dz = dh * (acts[li] > 0)
    return loss, grads


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (bias-corrected moments); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
