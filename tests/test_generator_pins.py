"""Pins of the oracle's synthetic-data generator (CPU).

Philox4x32-10 is pinned by the statistical properties a counter-based
generator must have (uniform words, full avalanche of counter and key bits,
no collisions); the Poisson sampler against scipy's Poisson pmf (goodness of
fit, mean and variance) on both of its branches; the rebinned means against
the geometric-series closed form.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
import workloads as W


def test_philox_known_answer_vectors():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert oracle.philox4x32_10(w[0:4], w[4:6]) == w[6:10]
        n += 1
    assert n == 3


def test_philox_words_are_uniform():
    words = np.array([oracle.philox4x32_10([i, 7, 0, 3], [11, 13]) for i in range(1 << 14)],
                     dtype=np.uint64).ravel()
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4
    bits = np.unpackbits(words.astype(">u4").view(np.uint8))
    assert abs(bits.mean() - 0.5) < 0.005


def test_philox_avalanche_and_no_collisions():
    rng = np.random.default_rng(1)
    base_c = [int(x) for x in rng.integers(0, 2**32, 4)]
    key = [int(x) for x in rng.integers(0, 2**32, 2)]
    ref = np.array(oracle.philox4x32_10(base_c, key), dtype=np.uint32)
    flips = []
    for w in range(4):
        for b in range(32):
            c = list(base_c)
            c[w] ^= 1 << b
            out = np.array(oracle.philox4x32_10(c, key), dtype=np.uint32)
            flips.append(int(np.unpackbits((out ^ ref).view(np.uint8)).sum()))
    for w in range(2):
        for b in range(32):
            k = list(key)
            k[w] ^= 1 << b
            out = np.array(oracle.philox4x32_10(base_c, k), dtype=np.uint32)
            flips.append(int(np.unpackbits((out ^ ref).view(np.uint8)).sum()))
    flips = np.array(flips)
    assert abs(flips.mean() - 64) < 2.5 and flips.min() > 30
    seen = {tuple(oracle.philox4x32_10([i, 0, 0, 0], key)) for i in range(20000)}
    assert len(seen) == 20000


@pytest.mark.parametrize("mu", [0.3, 2.5, 11.99, 12.0, 37.5, 600.0, 2.0e4])
def test_poisson_goodness_of_fit(mu):
    n = 60000
    k = oracle.poisson(np.full(n, mu, dtype=np.float32), seed=int(mu * 1000) + 5)
    # mean and variance (z-tests)
    assert abs(k.mean() - mu) < 5 * math.sqrt(mu / n)
    assert abs(k.var() / mu - 1.0) < 5 * math.sqrt(2.0 / n) + 0.01
    # chi-square against the pmf over the central range, tails pooled
    lo = int(max(0, math.floor(mu - 5 * math.sqrt(mu) - 2)))
    hi = int(math.ceil(mu + 5 * math.sqrt(mu) + 2))
    edges = np.arange(lo, hi + 1)
    obs = np.array([(k < lo).sum()] + [(k == e).sum() for e in edges] + [(k > hi).sum()], dtype=float)
    pmf = stats.poisson.pmf(edges, mu)
    exp = np.r_[stats.poisson.cdf(lo - 1, mu), pmf, stats.poisson.sf(hi, mu)] * n
    keep = exp >= 5
    o = np.r_[obs[keep], obs[~keep].sum()]
    e = np.r_[exp[keep], exp[~keep].sum()]
    if e[-1] < 5:
        o, e = o[:-1], e[:-1]
    chi2 = ((o - e) ** 2 / e).sum()
    p = stats.chi2.sf(chi2, len(o) - 1)
    assert p > 1e-5, (mu, chi2, len(o))


def test_poisson_edge_means():
    k = oracle.poisson(np.array([0.0, -1.0, 1e-30, 1e-6], dtype=np.float32), 3)
    assert k[0] == 0 and k[1] == 0 and k[2] == 0 and k[3] in (0, 1)
    big = oracle.poisson(np.full(20000, 3.0e6, dtype=np.float32), 4)
    assert abs(big.mean() - 3.0e6) < 5 * math.sqrt(3.0e6 / 20000)


def test_rebinned_mean_geometric_closed_form():
    """Lifetime-only theory, N0 = 1, bkg = 0: a group of r bins starting at bin j r
    sums to q^{j r} (1 - q^r) / (1 - q), q = e^{-dt/tau} (the last group is short)."""
    M, r, dt = 1000, 64, 0.002
    lay = W.single_hist_layout(M, dt)
    lay.comp = np.zeros((0, 6), dtype=np.int32)
    mu = oracle.rebinned_mean(lay, np.array([1.0, 0.0, 0, 0, 0, 0]), r)[0]
    q = math.exp(-dt / W.TAU_MU_US)
    ref = [q ** j0 * (1 - q ** min(r, M - j0)) / (1 - q) for j0 in range(0, M, r)]
    np.testing.assert_allclose(mu, ref, rtol=1e-13)


# ---------------------------------------------------------------------------
# Training parameter vectors of the learned start proposer, and its features
# ---------------------------------------------------------------------------
def test_sample_thetas_box_uniform_and_fixed_entries():
    from scipy import stats
    lo = np.array([200.0, 1.0, 0.7, 50.0, 0.1])
    hi = np.array([5000.0, 20.0, 0.7, 500.0, 2.0])
    th, tg = oracle.sample_thetas(lo, hi, 20000, seed=11)
    assert np.all(th[:, 2] == 0.7)
    learned = [0, 1, 3, 4]
    assert tg.shape == (20000, 4)
    for q, j in enumerate(learned):
        u = (th[:, j] - lo[j]) / (hi[j] - lo[j])
        assert np.all((u > 0) & (u < 1))
        assert stats.kstest(u, "uniform").pvalue > 1e-3
        np.testing.assert_allclose(tg[:, q], 2 * u - 1, rtol=0, atol=1e-6)
    # entries sharing a Philox block (q = 0, 1) and across blocks are uncorrelated
    c = np.corrcoef(tg.T)
    assert np.all(np.abs(c - np.eye(4)) < 0.05)


def test_sample_thetas_offset_is_a_shift():
    lo = np.zeros(3)
    hi = np.array([1.0, 2.0, 3.0])
    a, ta = oracle.sample_thetas(lo, hi, 10, seed=5, offset=0)
    b, tb = oracle.sample_thetas(lo, hi, 4, seed=5, offset=6)
    np.testing.assert_array_equal(a[6:], b)
    np.testing.assert_array_equal(ta[6:], tb)
    c, _ = oracle.sample_thetas(lo, hi, 10, seed=6, offset=0)
    assert not np.any(a == c)


def test_sample_thetas_known_word_mapping():
    # u is built from the documented Philox words, checked against the pinned block function
    lo = np.array([0.0, 0.0, 0.0])
    hi = np.array([1.0, 1.0, 1.0])
    th, _ = oracle.sample_thetas(lo, hi, 1, seed=(3 << 32) | 9, offset=(1 << 32) + 5)
    w = oracle.philox4x32_10([5, 1, 0, 0xfffffffe], [9 ^ 0x0A5F00D1, 3])
    w2 = oracle.philox4x32_10([5, 1, 1, 0xfffffffe], [9 ^ 0x0A5F00D1, 3])
    u = [((w[0] >> 5) * 2.0 ** 26 + (w[1] >> 6) + 0.5) / 2.0 ** 53,
         ((w[2] >> 5) * 2.0 ** 26 + (w[3] >> 6) + 0.5) / 2.0 ** 53,
         ((w2[0] >> 5) * 2.0 ** 26 + (w2[1] >> 6) + 0.5) / 2.0 ** 53]
    np.testing.assert_array_equal(th[0], u)


def test_proposer_features_brute_force():
    from workloads import multi_detector_layout
    lay = multi_detector_layout(n_hist=2, n_bins=[10, 7], window_us=1.0)
    data = np.arange(17, dtype=np.float64)
    sums = [[0 + 1 + 2 + 3, 4 + 5 + 6 + 7, 8 + 9], [10 + 11 + 12 + 13, 14 + 15 + 16]]
    tot = [sum(sums[0]), sum(sums[1])]
    assert tot == [45, 91]
    want = np.array([np.log1p(c) - np.log1p(tot[k]) for k in range(2) for c in sums[k]] + list(np.log1p(tot)))
    np.testing.assert_array_equal(oracle.proposer_features(lay, data, 4), want)
    mu = np.arange(7.0)
    isig = np.full(7, 2.0)
    np.testing.assert_array_equal(oracle.proposer_features(lay, data, 4, mu, isig), (want - mu) * 2.0)
