"""What the learned start proposer gains (16 detectors x 65536 bins, 40 free
parameters, uniform prior box): trained on device-generated histograms, its
proposals lead the LM fit to the same minimum as a fit started at the truth
(chi2 within 1e-6 relative) at least as often as the plain fit from the range
centre with a 10-point B1 grid, and in a small fraction of its time.  On two
runs the minimum is also checked against the FP64 oracle's fit."""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, GBatch, Proposer, Run, fit_multistart_batch  # noqa: E402
import oracle  # noqa: E402
import workloads as W  # noqa: E402

TRAIN_STEPS = 16384   # 8.4M generated histograms, ~30 s on one GB300
N_RUNS = 16


@pytest.fixture(scope="module")
def trained():
    lay = W.multi_detector_layout(16, 65536, 12.8)
    lo, hi = W.multi_detector_box(lay)
    layout = Run(lay)
    prop = Proposer(layout, lo, hi, seed=W.BASE_SEED + 5)
    losses = prop.train(TRAIN_STEPS, 1e-3, 3e-5)
    yield lay, lo, hi, layout, prop, losses
    prop.close()
    layout.close()


def _held_out(lay, layout, n, seed):
    g = W.rng(seed)
    thetas = np.stack([W.multi_detector_theta(lay, g) for _ in range(n)])
    data = torch.empty((n, lay.total_bins), dtype=torch.float32, device="cuda")
    layout.generate(torch.tensor(thetas, device="cuda"), 1, seed, data, sample_offset=0, log1p_out=False)
    torch.cuda.synchronize()
    return thetas, data


def test_learned_start_beats_plain_fit(trained):
    lay, lo, hi, layout, prop, losses = trained
    assert np.mean(losses[-100:]) < 0.2 * np.mean(losses[:100])
    thetas, data = _held_out(lay, layout, N_RUNS, W.BASE_SEED + 1005)
    starts = W.default_starts(lay)
    free = lay.free
    ok_l, ok_p, t_l, t_p, it_l, it_p = [], [], 0.0, 0.0, [], []
    for i in range(N_RUNS):
        with Run(lay, data[i].contiguous()) as r:
            _, ref, _ = r.fit(thetas[i], MUSR_CHI2, free=free)
            t0 = time.perf_counter()
            _, il, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=1.2, fallback_starts=starts)
            t1 = time.perf_counter()
            _, ip, _ = r.fit_multistart(starts, MUSR_CHI2, free=free)
            t2 = time.perf_counter()
        t_l += t1 - t0
        t_p += t2 - t1
        it_l.append(il["iters"])
        it_p.append(ip["iters"])
        ok_l.append(abs(il["value"] - ref["value"]) <= 1e-6 * ref["value"])
        ok_p.append(abs(ip["value"] - ref["value"]) <= 1e-6 * ref["value"])
    print(f"learned: success {np.mean(ok_l):.2f}, {t_l / N_RUNS * 1e3:.1f} ms/fit, {np.mean(it_l):.1f} iters; "
          f"plain: success {np.mean(ok_p):.2f}, {t_p / N_RUNS * 1e3:.1f} ms/fit, {np.mean(it_p):.1f} iters")
    assert np.mean(ok_l) >= 0.85
    assert np.mean(ok_l) >= np.mean(ok_p) - 0.07
    assert t_l < 0.2 * t_p
    assert np.mean(it_l) < 0.1 * np.mean(it_p)


def test_batched_learned_start_beats_batched_plain_fit(trained):
    # both arms batched: all runs' learned starts fitted in lockstep, against all
    # (run, start) pairs of the plain multi-start grid fitted in lockstep
    lay, lo, hi, layout, prop, losses = trained
    thetas, data = _held_out(lay, layout, N_RUNS, W.BASE_SEED + 1008)
    starts = W.default_starts(lay)
    free = lay.free
    runs = [Run(lay, data[i].contiguous()) for i in range(N_RUNS)]
    with GBatch(runs) as b:
        _, ref = b.fit(list(thetas), MUSR_CHI2, free=[free] * N_RUNS)
        t0 = time.perf_counter()
        _, il = prop.fit_batch(b, MUSR_CHI2, free=[free] * N_RUNS, chi2ndf_max=1.2, fallback_starts=[starts] * N_RUNS)
        t1 = time.perf_counter()
    _, ip = fit_multistart_batch(runs, [starts] * N_RUNS, MUSR_CHI2, free=[free] * N_RUNS)
    t2 = time.perf_counter()
    ok_l = [abs(a["value"] - r["value"]) <= 1e-6 * r["value"] for a, r in zip(il, ref)]
    ok_p = [abs(a["value"] - r["value"]) <= 1e-6 * r["value"] for a, r in zip(ip, ref)]
    print(f"batched learned: success {np.mean(ok_l):.2f}, {(t1 - t0) / N_RUNS * 1e3:.2f} ms/fit; "
          f"batched plain: success {np.mean(ok_p):.2f}, {(t2 - t1) / N_RUNS * 1e3:.2f} ms/fit")
    assert np.mean(ok_l) >= 0.85
    assert np.mean(ok_l) >= np.mean(ok_p) - 0.07
    assert (t1 - t0) < 0.2 * (t2 - t1)
    for r in runs:
        r.close()


def test_learned_fit_reaches_the_oracle_minimum(trained):
    # inputs from the oracle's model and numpy's Poisson draws (host side)
    lay, lo, hi, layout, prop, losses = trained
    g = W.rng(W.BASE_SEED + 1006)
    free = lay.free
    for i in range(2):
        theta = W.multi_detector_theta(lay, g)
        d = W.poisson_counts(oracle.model(lay, theta), W.BASE_SEED + 1007 + i)
        _, oi, _ = oracle.fit(lay, d, theta, oracle.CHI2, free=free)
        with Run(lay, d) as r:
            _, il, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=1.2, fallback_starts=W.default_starts(lay))
        assert abs(il["value"] / il["ndf"] - oi["value"] / oi["ndf"]) <= 1e-6 * oi["value"] / oi["ndf"]


def test_fallback_stages_keep_the_best(trained):
    """A run whose field lies outside the prior box widened by a quarter of its
    width: every fit ends outside it, so both fallback stages run (the grid
    with the proposal's values for what it does not scan, then the plain
    grid) and the result is the best of the three fits."""
    lay, lo, hi, layout, prop, losses = trained
    theta = W.multi_detector_theta(lay, W.rng(W.BASE_SEED + 1010))
    theta[lay.names.index("B1")] = 700.0
    d = W.poisson_counts(oracle.model(lay, theta), W.BASE_SEED + 1011)
    starts = W.default_starts(lay)
    free = lay.free
    with Run(lay, d) as r:
        _, il, _ = prop.fit(r, MUSR_CHI2, free=free, chi2ndf_max=1.2, fallback_starts=starts)
        p0 = prop.propose([r])[0]
        _, only_learned, _ = r.fit(p0, MUSR_CHI2, free=free)
        _, only_plain, _ = r.fit_multistart(starts, MUSR_CHI2, free=free)
        with GBatch([r]) as b:
            _, ib = prop.fit_batch(b, MUSR_CHI2, free=[free], chi2ndf_max=1.2, fallback_starts=[starts])
    assert il["fallback_stage"] == 2 and ib[0]["fallback_stage"] == 2
    best = min(only_learned["value"], only_plain["value"])
    assert il["value"] <= best * (1 + 1e-9)
    assert ib[0]["value"] <= best * (1 + 1e-6)
