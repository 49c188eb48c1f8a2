"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import workloads as W


def rel_err(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grad_rel_err(g, ref):
    """Gradient error against the oracle's, as the larger of the norm-wise
    relative error ||g - ref|| / ||ref|| and the per-component error
    max_j |g_j - ref_j| / ||ref||_inf, so that `<= 1e-4` states both
    tolerances: 1e-4 norm-wise, and no component off by more than 1e-4 of the
    largest one (a wrong small component cannot hide under the norm)."""
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    norm = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300)
    comp = np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300) if ref.size else 0.0
    return float(max(norm, comp))


def split_by_hist(lay, x):
    offs = np.r_[0, np.cumsum(lay.n_bins)]
    return [x[offs[k]:offs[k + 1]] for k in range(lay.n_hist)]


def ragged_layout(n_bins, n_hist=None):
    """Multi-detector layout with explicitly uneven histogram sizes."""
    nb = list(n_bins)
    return W.multi_detector_layout(len(nb), nb, window_us=12.8)
