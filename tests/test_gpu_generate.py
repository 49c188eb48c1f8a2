"""GPU parity of the synthetic-data generator.

* Poisson sampler: bit-exact against the oracle's sampler on the same FP32
  means (integer output; both sides take every decision in FP32 in the same
  operation order), over both branches (inversion below 12, PTRS above).
* Fused generator (theory summed over groups of bins, then a count per group):
  group means within 2e-6 relative of the oracle's FP64 sums; counts
  statistically Poisson around those means; log1p output consistent; draws a
  pure function of (seed, sample, histogram, group).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
torch = pytest.importorskip("torch")
from paper_1604_02334_gb300 import Run, poisson_sample  # noqa: E402


def test_poisson_sampler_bit_exact():
    g = np.random.default_rng(5)
    mu = np.concatenate([
        np.zeros(10), g.uniform(0, 1, 20000), g.uniform(1, 12, 20000),
        np.full(5000, 11.999999), np.full(5000, 12.0), g.uniform(12, 100, 20000),
        g.uniform(100, 1e4, 20000), g.uniform(1e4, 5e5, 20000)]).astype(np.float32)
    ref = oracle.poisson(mu, seed=0x1234_5678_9abc)
    mu_d = torch.tensor(mu, device="cuda:0")
    out = torch.empty(mu.size, dtype=torch.int32, device="cuda:0")
    poisson_sample(mu_d, 0x1234_5678_9abc, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got, ref), np.flatnonzero(got != ref)[:10]


@pytest.fixture(scope="module")
def gen_case():
    lay = W.multi_detector_layout(16, 4096, window_us=12.8)
    g = W.rng(77)
    thetas = np.stack([W.multi_detector_theta(lay, g) for _ in range(8)])
    return lay, thetas


def generate(lay, thetas, rebin, seed, offset=0, log1p=False):
    dev = torch.device("cuda:0")
    per = int(sum((int(m) + rebin - 1) // rebin for m in lay.n_bins))
    th = torch.tensor(thetas, device=dev)
    out = torch.empty((thetas.shape[0], per), dtype=torch.float32, device=dev)
    mu = torch.empty_like(out)
    with Run(lay) as r:
        r.generate(th, rebin, seed, out, sample_offset=offset, log1p_out=log1p, mu_dev=mu)
        torch.cuda.synchronize()
    return out.cpu().numpy(), mu.cpu().numpy()


@pytest.mark.parametrize("rebin", [64, 1, 13])
def test_generator_means_match_oracle(gen_case, rebin):
    lay, thetas = gen_case
    _, mu = generate(lay, thetas, rebin, seed=9)
    ref = oracle.rebinned_mean(lay, thetas, rebin)
    np.testing.assert_allclose(mu, ref, rtol=2e-6, atol=1e-5)


def test_generator_counts_are_poisson_and_reproducible(gen_case):
    lay, thetas = gen_case
    cnt, mu = generate(lay, thetas, 64, seed=21)
    assert np.all(cnt == np.floor(cnt)) and cnt.min() >= 0
    z = (cnt - mu) / np.sqrt(mu)
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / z.size) + 0.02
    again, _ = generate(lay, thetas, 64, seed=21)
    assert np.array_equal(cnt, again)
    other, _ = generate(lay, thetas, 64, seed=21, offset=8)
    assert not np.array_equal(cnt, other)
    logc, _ = generate(lay, thetas, 64, seed=21, log1p=True)
    np.testing.assert_allclose(logc, np.log1p(cnt), rtol=2e-7, atol=0)
