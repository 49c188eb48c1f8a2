"""Seeded synthetic workloads for the muSR fit objective.

This module describes the inputs only: histogram layouts (bin counts, time
grid, parameter map, component list), parameter vectors drawn from stated
ranges, and Poisson / normal random draws from numpy's PCG64 generator.  It
holds none of the method's arithmetic (no theory function, no objective): the
means handed to :func:`poisson_counts` are computed by whoever calls it.

Both the FP64 oracle (tests) and the GPU library (tests, benchmark) take their
inputs from here, so neither ever produces the other's inputs.

Layout conventions (Sec. 4.1 Eq. 2 and the map array of Sec. 4.2.1):
  * theta is the global FP64 parameter vector;
  * every histogram k has a map row of ``map_width`` entries, each an index
    into theta (or -1 for the constant 0); column 0 is N0, column 1 is Nbkg;
  * every theory component names the map columns it reads:
    (kind, amp, rate, field, field2, phase, beta), -1 when unused.  The field
    is theta[field] + theta[field2]; beta is the exponent of a stretched line.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

TF_EXP = 0
TF_GAUSS = 1
KT_STATIC_GAUSS = 2
TF_STRETCHED = 3

CHI2 = 0
POISSON = 1

# gamma_mu / 2 pi in MHz per gauss, and the muon lifetime in microseconds
GAMMA_MU_MHZ_PER_G = 0.013554
TAU_MU_US = 2.197

BASE_SEED = 16040233


@dataclasses.dataclass
class RunLayout:
    n_bins: np.ndarray  # int64 [n_hist]
    t0_us: float
    dt_us: float
    tau_us: float
    gamma: float
    n_params: int
    map: np.ndarray  # int32 [n_hist, map_width]
    comp: np.ndarray  # int32 [n_comp, 7]
    names: List[str]
    free: np.ndarray  # uint8 [n_params]
    # function array (Sec. 4.2.1): expressions over p[i]; a map entry -2 - j reads function j
    funcs: List[str] = dataclasses.field(default_factory=list)

    @property
    def n_hist(self) -> int:
        return int(self.n_bins.shape[0])

    @property
    def map_width(self) -> int:
        return int(self.map.shape[1])

    @property
    def n_comp(self) -> int:
        return int(self.comp.shape[0])

    @property
    def total_bins(self) -> int:
        return int(self.n_bins.sum())

    @property
    def n_free(self) -> int:
        return int(self.free.sum())

    def permuted(self, perm: Sequence[int]) -> "RunLayout":
        """Same run with histograms reordered (map rows move with them)."""
        perm = np.asarray(perm, dtype=np.int64)
        return dataclasses.replace(
            self, n_bins=self.n_bins[perm].copy(), map=self.map[perm].copy()
        )


def comp_table(comp) -> np.ndarray:
    """Component rows as int32 [n_comp, 7]; 6-column rows (no beta) get beta = -1."""
    rows = [[int(x) for x in r] + [-1] * (7 - len(r)) for r in comp]
    return np.ascontiguousarray(np.asarray(rows, dtype=np.int32).reshape(-1, 7))


def _layout(n_bins, dt_us, map_rows, comp, names, free, t0_us=0.0):
    return RunLayout(
        n_bins=np.asarray(n_bins, dtype=np.int64),
        t0_us=float(t0_us),
        dt_us=float(dt_us),
        tau_us=TAU_MU_US,
        gamma=GAMMA_MU_MHZ_PER_G,
        n_params=len(names),
        map=np.ascontiguousarray(np.asarray(map_rows, dtype=np.int32)),
        comp=comp_table(comp),
        names=list(names),
        free=np.asarray(free, dtype=np.uint8),
    )


# ---------------------------------------------------------------------------
# Single-histogram workload: one damped precession signal
# ---------------------------------------------------------------------------
def single_hist_layout(n_bins: int = 8192, dt_us: float = 0.00125, t0_us: float = 0.0) -> RunLayout:
    """1 histogram: N0 e^{-t/tau}[1 + A0 e^{-lambda t} cos(2 pi gamma B t + phi)] + bkg.

    theta = [N0, bkg, A0, lambda, B, phi]; 6 free parameters.
    """
    names = ["N0", "bkg", "A0", "lambda", "B", "phi"]
    map_rows = [[0, 1, 2, 3, 4, 5]]
    comp = [[TF_EXP, 2, 3, 4, -1, 5]]
    return _layout([n_bins], dt_us, map_rows, comp, names, [1] * 6, t0_us)


def single_hist_truth() -> np.ndarray:
    return np.array([1000.0, 5.0, 0.25, 0.5, 100.0, 0.3])


# ---------------------------------------------------------------------------
# Multi-detector workload: two precession lines + static Gaussian Kubo-Toyabe
# ---------------------------------------------------------------------------
# column order of every map row
MD_COLS = ["N0", "bkg", "phi", "A1", "lambda1", "B1", "A2", "sigma2", "dB", "A_KT", "Delta_KT"]
SHARED_NAMES = ["A1", "lambda1", "B1", "A2", "sigma2", "dB", "A_KT", "Delta_KT"]
SHARED_RANGES = {
    "A1": (0.05, 0.15),
    "lambda1": (0.1, 2.0),
    "B1": (50.0, 500.0),
    "A2": (0.05, 0.15),
    "sigma2": (0.1, 2.0),
    "dB": (5.0, 50.0),
    "A_KT": (0.02, 0.08),
    "Delta_KT": (0.1, 1.0),
    # the stretched-line variant: second line exp(-(lambda2 t)^beta) instead of the Gaussian
    "lambda2": (0.1, 2.0),
    "beta": (0.5, 2.0),
}
# shared parameters of the stretched-line variant, in map-column order after phi
ST_SHARED_NAMES = ["A1", "lambda1", "B1", "A2", "lambda2", "dB", "A_KT", "Delta_KT", "beta"]
N0_RANGE = (200.0, 5000.0)
BKG_RANGE = (1.0, 20.0)
MD_COMPONENTS = [
    [TF_EXP, 3, 4, 5, -1, 2],
    [TF_GAUSS, 6, 7, 5, 8, 2],
    [KT_STATIC_GAUSS, 9, 10, -1, -1, -1],
]
# map row [N0, bkg, phi, A1, lambda1, B1, A2, lambda2, dB, A_KT, Delta_KT, beta]
MD_ST_COMPONENTS = [
    [TF_EXP, 3, 4, 5, -1, 2, -1],
    [TF_STRETCHED, 6, 7, 5, 8, 2, 11],
    [KT_STATIC_GAUSS, 9, 10, -1, -1, -1, -1],
]


# The multi-detector theory written as a user expression over the map row
# [N0, bkg, phi, A1, lambda1, B1, A2, sigma2, dB, A_KT, Delta_KT] (MD_COLS).
MD_USER_EXPR = ("p[m[3]]*se(t,p[m[4]])*tf(t,p[m[2]],p[m[5]])"
                " + p[m[6]]*sg(t,p[m[7]])*tf(t,p[m[2]],p[m[5]]+p[m[8]])"
                " + p[m[9]]*stg(t,p[m[10]])")


def multi_detector_layout(
    n_hist: int = 16,
    n_bins=65536,
    window_us: float = 12.8,
    shared_bkg: bool = False,
    t0_us: float = 0.0,
    stretched: bool = False,
) -> RunLayout:
    """K detector histograms sharing the physics parameters.

    theta = [N0_0..N0_{K-1}, bkg_0..bkg_{K-1} (or one shared bkg),
             phi_0..phi_{K-1} (fixed, 2 pi k / K), A1, lambda1, B1, A2, sigma2,
             dB, A_KT, Delta_KT].
    The second line's field is B1 + dB.  Free: N0, bkg and the 8 shared ones.
    ``stretched``: the second line relaxes as exp(-(lambda2 t)^beta) and the
    shared block is A1, lambda1, B1, A2, lambda2, dB, A_KT, Delta_KT, beta
    (9 free).
    ``n_bins`` is an int or a per-histogram sequence; dt = window / max(n_bins).
    """
    if np.isscalar(n_bins):
        nb = [int(n_bins)] * n_hist
    else:
        nb = [int(x) for x in n_bins]
        assert len(nb) == n_hist
    dt = window_us / max(nb)
    names = [f"N0_{k}" for k in range(n_hist)]
    n_bkg = 1 if shared_bkg else n_hist
    names += ["bkg"] if shared_bkg else [f"bkg_{k}" for k in range(n_hist)]
    names += [f"phi_{k}" for k in range(n_hist)]
    base = len(names)
    shared = ST_SHARED_NAMES if stretched else SHARED_NAMES
    names += shared
    rows = []
    for k in range(n_hist):
        bkg_idx = n_hist if shared_bkg else n_hist + k
        phi_idx = n_hist + n_bkg + k
        rows.append([k, bkg_idx, phi_idx] + [base + j for j in range(len(shared))])
    free = [1] * (n_hist + n_bkg) + [0] * n_hist + [1] * len(shared)
    comp = MD_ST_COMPONENTS if stretched else MD_COMPONENTS
    return _layout(nb, dt, rows, comp, names, free, t0_us)


def multi_detector_theta(layout: RunLayout, rng: np.random.Generator) -> np.ndarray:
    """Draw a parameter vector uniformly from the stated ranges; phases 2 pi k/K."""
    K = layout.n_hist
    theta = np.zeros(layout.n_params)
    for j, name in enumerate(layout.names):
        if name.startswith("N0_"):
            theta[j] = rng.uniform(*N0_RANGE)
        elif name.startswith("bkg"):
            theta[j] = rng.uniform(*BKG_RANGE)
        elif name.startswith("phi_"):
            k = int(name.split("_")[1])
            theta[j] = 2.0 * math.pi * k / K
        else:
            theta[j] = rng.uniform(*SHARED_RANGES[name])
    return theta


def range_centre_theta(layout: RunLayout) -> np.ndarray:
    """Default start: centre of every range (phases at their fixed values)."""
    K = layout.n_hist
    theta = np.zeros(layout.n_params)
    for j, name in enumerate(layout.names):
        if name.startswith("N0_"):
            theta[j] = 0.5 * sum(N0_RANGE)
        elif name.startswith("bkg"):
            theta[j] = 0.5 * sum(BKG_RANGE)
        elif name.startswith("phi_"):
            theta[j] = 2.0 * math.pi * int(name.split("_")[1]) / K
        else:
            theta[j] = 0.5 * sum(SHARED_RANGES[name])
    return theta


def multi_detector_box(layout: RunLayout):
    """(lo, hi) of the uniform prior of multi_detector_theta; phases fixed (lo == hi)."""
    lo = np.zeros(layout.n_params)
    hi = np.zeros(layout.n_params)
    K = layout.n_hist
    for j, name in enumerate(layout.names):
        if name.startswith("N0_"):
            lo[j], hi[j] = N0_RANGE
        elif name.startswith("bkg"):
            lo[j], hi[j] = BKG_RANGE
        elif name.startswith("phi_"):
            lo[j] = hi[j] = 2.0 * math.pi * int(name.split("_")[1]) / K
        else:
            lo[j], hi[j] = SHARED_RANGES[name]
    return lo, hi


def default_starts(layout: RunLayout, n_grid: int = 10) -> np.ndarray:
    """Plain fit starts: the range centre with B1 at the centres of n_grid
    equal slices of its range (a multi-start grid over the precession field)."""
    base = range_centre_theta(layout)
    j = layout.names.index("B1")
    b_lo, b_hi = SHARED_RANGES["B1"]
    starts = np.repeat(base[None, :], n_grid, axis=0)
    starts[:, j] = b_lo + (np.arange(n_grid) + 0.5) * (b_hi - b_lo) / n_grid
    return starts


def perturb(theta: np.ndarray, free: np.ndarray, rel: float, rng: np.random.Generator) -> np.ndarray:
    """theta * (1 + rel * z), z ~ N(0, 1), free entries only."""
    z = rng.standard_normal(theta.shape[0])
    out = theta.copy()
    m = free.astype(bool)
    out[m] = theta[m] * (1.0 + rel * z[m])
    return out


def poisson_counts(mean: np.ndarray, seed: int) -> np.ndarray:
    """Poisson draws (as FP64 counts) for the given per-bin means."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.poisson(np.maximum(mean, 0.0)).astype(np.float64)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------
def config_single():
    """1 x 8192 bins of 1.25 ns, 6 free parameters (seed BASE_SEED + 0)."""
    return single_hist_layout(), single_hist_truth(), BASE_SEED + 0


def config_multi_detector(n_hist=16, n_bins=65536, window_us=12.8, seed_offset=1):
    """16 x 65536 bins of 0.1953125 ns, 40 free parameters (seed BASE_SEED + 1)."""
    lay = multi_detector_layout(n_hist, n_bins, window_us)
    theta = multi_detector_theta(lay, rng(BASE_SEED + seed_offset))
    return lay, theta, BASE_SEED + seed_offset


# histogram lengths of the paper's Table 1 data sets (16 detectors each)
SWEEP_BINS = (85320, 106650, 142200, 213300, 426601)


def config_stretched(n_hist=16, n_bins=65536, window_us=12.8):
    """16 x 65536 bins, the second line a stretched exponential, 41 free parameters
    (seed BASE_SEED + 6)."""
    lay = multi_detector_layout(n_hist, n_bins, window_us, stretched=True)
    theta = multi_detector_theta(lay, rng(BASE_SEED + 6))
    return lay, theta, BASE_SEED + 6


def config_sweep(n_bins: int, window_us: float = 10.0):
    """16 x n_bins bins over a 10 us window (seed BASE_SEED + 4); the paper's data-set shapes."""
    return config_multi_detector(16, n_bins, window_us, seed_offset=4)


def config_gradient(n_hist=32, n_bins=131072, window_us=12.8):
    """32 x 131072 bins, 72 free parameters (seed BASE_SEED + 3)."""
    return config_multi_detector(n_hist, n_bins, window_us, seed_offset=3)


@dataclasses.dataclass
class BatchRun:
    layout: RunLayout
    theta: np.ndarray
    seed: int


def config_batched(n_runs: int = 64, seed_offset: int = 2, min_bins: int = 16384,
                   max_bins: int = 131072, max_hist: int = 32) -> List[BatchRun]:
    """64 independent runs of uneven size: K ~ U{1..32}, bins ~ U[2^14, 2^17].

    K <= 20: per-detector N0 and bkg (2K + 8 free); K > 20: per-detector N0 and
    one shared bkg (K + 9 free), so no run has more than 48 free parameters.
    """
    g = rng(BASE_SEED + seed_offset)
    runs = []
    for r in range(n_runs):
        K = int(g.integers(1, max_hist + 1))
        nb = int(g.integers(min_bins, max_bins + 1))
        lay = multi_detector_layout(K, nb, 12.8, shared_bkg=K > 20)
        theta = multi_detector_theta(lay, g)
        runs.append(BatchRun(lay, theta, BASE_SEED + 1000 * (seed_offset + 1) + r))
    return runs


def jacobian_vectors(theta: np.ndarray, free: np.ndarray, rel_h: float = 1e-6) -> np.ndarray:
    """theta and theta + h_j e_j for every free j: the (P_free + 1) vector set."""
    idx = np.nonzero(free)[0]
    vecs = [theta.copy()]
    for j in idx:
        v = theta.copy()
        v[j] += rel_h * max(abs(theta[j]), 1.0)
        vecs.append(v)
    return np.stack(vecs)
