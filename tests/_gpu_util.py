"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np

import workloads as W


def rel_err(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def grad_rel_err(g, ref):
    """||g - ref|| / ||ref|| (the gradient tolerance is stated norm-wise)."""
    return float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300))


def split_by_hist(lay, x):
    offs = np.r_[0, np.cumsum(lay.n_bins)]
    return [x[offs[k]:offs[k + 1]] for k in range(lay.n_hist)]


def ragged_layout(n_bins, n_hist=None):
    """Multi-detector layout with explicitly uneven histogram sizes."""
    nb = list(n_bins)
    return W.multi_detector_layout(len(nb), nb, window_us=12.8)
