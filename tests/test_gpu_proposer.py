"""Learned start proposer on the GPU: its training inputs and features
against the oracle (bit-exact parameter draws, features to FP32 rounding),
training on device-generated data, and the learned-start fit with its
fallback against fits from the truth."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, Proposer, Run  # noqa: E402
import oracle  # noqa: E402
import workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def small():
    # 8 detectors x 8192 bins over 12.8 us; 512 features at rebin 128
    lay = W.multi_detector_layout(8, 8192, window_us=12.8)
    lo, hi = W.multi_detector_box(lay)
    run = Run(lay)
    prop = Proposer(run, lo, hi, rebin=128, n_hidden=256, n_hidden_layers=2, batch=256, seed=123)
    yield lay, lo, hi, run, prop
    prop.close()
    run.close()


def test_training_draws_match_oracle_bitwise(small):
    lay, lo, hi, run, prop = small
    th, tg = prop.sample(300, offset=1000)
    torch.cuda.synchronize()
    ref_th, ref_tg = oracle.sample_thetas(lo, hi, 300, seed=123, offset=1000)
    np.testing.assert_array_equal(th.cpu().numpy(), ref_th)
    np.testing.assert_array_equal(tg.cpu().numpy(), ref_tg)


def test_features_match_oracle(small):
    # device: FP32 log1p (<= 1 ulp) of exact group sums, an FP32 log of the
    # exact total, two FP32 subtractions and a product with inv_sigma; the
    # bound adds those roundings, scaled by inv_sigma, with a 1.5x margin
    lay, lo, hi, run, prop = small
    mu, isig = prop.norm()
    g = W.rng(5)
    runs, refs, raw = [], [], []
    for i in range(3):
        theta = W.multi_detector_theta(lay, g)
        d = W.poisson_counts(oracle.model(lay, theta), 50 + i)
        runs.append(Run(lay, d))
        refs.append(oracle.proposer_features(lay, d, 128, mu, isig))
        raw.append(oracle.proposer_features(lay, d, 128))
    got = prop.features(runs).cpu().double().numpy()
    assert got.shape == (3, prop.n_features)
    ref = np.stack(refs)
    a = np.abs(np.stack(raw))
    eps = 2.0 ** -23
    G = prop.n_features - lay.n_hist
    L = np.concatenate([np.repeat(a[:, G:], [int(-(-m // 128)) for m in lay.n_bins], axis=1), a[:, G:]], axis=1)
    logc = np.where(np.arange(prop.n_features) < G, a + L, 0.0)
    tol = 1.5 * eps * (isig * (1.5 * logc + 0.5 * L + 0.5 * a + 0.5 * np.abs(a - mu)) + 0.5 * np.abs(ref))
    assert np.all(np.abs(got - ref) <= tol), float(np.max(np.abs(got - ref) / tol))
    for r in runs:
        r.close()


def test_standardisation_of_training_features(small):
    # fresh training samples, standardised: per-feature mean ~ 0 and sd ~ 1
    lay, lo, hi, run, prop = small
    g = W.rng(15)
    feats = []
    for i in range(64):
        theta = W.multi_detector_theta(lay, g)
        with Run(lay, W.poisson_counts(oracle.model(lay, theta), 100 + i)) as r:
            feats.append(prop.features([r]).cpu().double().numpy()[0])
    f = np.stack(feats)
    assert np.median(np.abs(f.mean(axis=0))) < 0.3
    sd = f.std(axis=0)
    assert 0.7 < np.median(sd) < 1.3


def test_training_lowers_the_loss(small):
    lay, lo, hi, run, prop = small
    losses = prop.train(400, 2e-3, 2e-4)
    assert np.all(np.isfinite(losses))
    first, last = float(np.mean(losses[:20])), float(np.mean(losses[-20:]))
    # targets are uniform on [-1, 1] (MSE 1/3 for a constant 0): within 400
    # steps the network must explain a clear part of the variance
    assert last < 0.85 * first and last < 0.3


def test_proposals_inside_box_and_fixed_entries(small):
    lay, lo, hi, run, prop = small
    g = W.rng(6)
    theta = W.multi_detector_theta(lay, g)
    with Run(lay, W.poisson_counts(oracle.model(lay, theta), 7)) as r:
        p = prop.propose([r, r])
    assert p.shape == (2, lay.n_params)
    np.testing.assert_array_equal(p[0], p[1])
    assert np.all(p[0] >= lo) and np.all(p[0] <= hi)
    fixed = hi == lo
    np.testing.assert_array_equal(p[0][fixed], lo[fixed])
    # after training, N0 proposals carry information: error below the prior's spread
    j = [i for i, n in enumerate(lay.names) if n.startswith("N0_")]
    assert np.sqrt(np.mean((p[0][j] - theta[j]) ** 2)) < 0.5 * (hi[j[0]] - lo[j[0]]) / np.sqrt(12)


def test_fit_learned_fallback_and_agreement(small):
    lay, lo, hi, run, prop = small
    g = W.rng(8)
    theta = W.multi_detector_theta(lay, g)
    d = W.poisson_counts(oracle.model(lay, theta), 9)
    free = lay.free
    with Run(lay, d) as r:
        ref, ri, _ = r.fit(theta, MUSR_CHI2, free=free, edm_tol=1e-10)
        starts = np.stack([theta, W.range_centre_theta(lay)])
        # threshold 0: the fallback must run, and its best start is the truth
        th0, i0, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=0.0, fallback_starts=starts, edm_tol=1e-10)
        assert i0["fallback"]
        assert abs(i0["value"] - ri["value"]) <= 1e-6 * ri["value"]
        # no fallback allowed: a learned fit alone
        th1, i1, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=1e300, fallback_starts=starts, edm_tol=1e-10)
        assert not i1["fallback"]
        assert np.isfinite(i1["value"]) and i1["value"] >= ri["value"] * (1 - 1e-6)
        # multistart picks the best of its starts
        thm, im, _ = r.fit_multistart(starts, MUSR_CHI2, free=free, edm_tol=1e-10)
        assert abs(im["value"] - ri["value"]) <= 1e-6 * ri["value"]
