"""Batched adjoint evaluation (many runs, one launch) against the FP64 oracle
with the single-run tolerances (relative 1e-6 on the objective, 1e-4
norm-wise on the gradient and the GN matrix), inactive entries left alone,
bitwise repeatability, and lockstep LM fits against single fits and the
oracle's fit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_POISSON, MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN,  # noqa: E402
                                    GBatch, Run)
import oracle  # noqa: E402
import workloads as W  # noqa: E402
from _gpu_util import grad_rel_err, rel_err  # noqa: E402


@pytest.fixture(scope="module")
def runs():
    # uneven runs of one signature: 2..16 histograms, ragged bin counts
    g = W.rng(321)
    specs = [(16, [65536] * 16), (3, [5000, 12345, 777]), (8, list(g.integers(1000, 40000, 8))), (2, [8, 4099])]
    out = []
    for i, (K, nb) in enumerate(specs):
        lay = W.multi_detector_layout(K, [int(x) for x in nb], window_us=12.8)
        theta = W.multi_detector_theta(lay, g)
        d = W.poisson_counts(oracle.model(lay, theta), 900 + i)
        th = W.perturb(theta, lay.free, 0.01, g)
        out.append((lay, d, th))
    return out


@pytest.mark.parametrize("obj", [MUSR_CHI2, MUSR_POISSON])
def test_gbatch_matches_oracle(runs, obj):
    gruns = [Run(lay, d) for lay, d, _ in runs]
    # the first run twice (as for two start points), then the others
    order = [0, 1, 0, 2, 3]
    with GBatch([gruns[i] for i in order]) as b:
        for mode in (MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN):
            res, flags = b.eval([runs[i][2] for i in order], obj, mode)
            assert not np.any(flags)
            for e, i in enumerate(order):
                lay, d, th = runs[i]
                v, g, H = oracle.gradient(lay, d, th, obj, with_gn=True)
                val, grad, gn = res[e]
                if lay.total_bins >= 4096:
                    assert rel_err(val, v) <= 1e-6
                assert grad_rel_err(grad, g) <= 1e-4
                if mode == MUSR_VALUE_GRAD_GN:
                    assert np.linalg.norm(gn - H) <= 1e-4 * np.linalg.norm(H)
            # bitwise repeatable
            res2, _ = b.eval([runs[i][2] for i in order], obj, mode)
            for a, c in zip(res, res2):
                assert a[0] == c[0] and np.array_equal(a[1], c[1])
    for r in gruns:
        r.close()


def test_gbatch_inactive_entries_and_device_entry(runs):
    gruns = [Run(lay, d) for lay, d, _ in runs]
    with GBatch(gruns, with_gn=False) as b:
        thetas = [th for _, _, th in runs]
        full, _ = b.eval(thetas, MUSR_CHI2, MUSR_VALUE_GRAD)
        part, _ = b.eval(thetas, MUSR_CHI2, MUSR_VALUE_GRAD, active=[0, 1, 0, 1])
        assert part[0] is None and part[2] is None
        assert part[1][0] == full[1][0] and part[3][0] == full[3][0]
        flat = torch.tensor(np.concatenate(thetas), device="cuda")
        out = torch.empty(int(np.sum(b.out_sizes(MUSR_VALUE_GRAD))), dtype=torch.float64, device="cuda")
        b.eval_device(flat, out, MUSR_CHI2, MUSR_VALUE_GRAD)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        off = 0
        for e, n in enumerate(b.out_sizes(MUSR_VALUE_GRAD)):
            assert o[off] == full[e][0]
            np.testing.assert_array_equal(o[off + 1:off + n], full[e][1])
            off += n
        with pytest.raises(Exception):
            b.eval(thetas, MUSR_CHI2, MUSR_VALUE_GRAD_GN)  # not prepared without GN
    for r in gruns:
        r.close()


def test_gbatch_gn_device_entry_into_a_nan_buffer(runs):
    """The batched Gauss-Newton evaluation into a caller's buffer full of NaN:
    every entry comes back, the entries without sources as 0, equal to the
    host entry point's results."""
    gruns = [Run(lay, d) for lay, d, _ in runs]
    with GBatch(gruns, with_gn=True) as b:
        thetas = [th for _, _, th in runs]
        full, _ = b.eval(thetas, MUSR_CHI2, MUSR_VALUE_GRAD_GN)
        flat = torch.tensor(np.concatenate(thetas), device="cuda")
        sizes = b.out_sizes(MUSR_VALUE_GRAD_GN)
        out = torch.full((int(np.sum(sizes)),), float("nan"), dtype=torch.float64, device="cuda")
        b.eval_device(flat, out, MUSR_CHI2, MUSR_VALUE_GRAD_GN)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        off = 0
        for e, n in enumerate(sizes):
            P = len(full[e][1])
            assert o[off] == full[e][0]
            np.testing.assert_array_equal(o[off + 1:off + 1 + P], full[e][1])
            H = o[off + 1 + P:off + n].reshape(P, P)
            assert np.all(np.isfinite(H)) and np.array_equal(H, H.T)
            np.testing.assert_array_equal(H, full[e][2])
            off += n
    for r in gruns:
        r.close()


def test_fit_batch_matches_single_fits_and_oracle(runs):
    """Lockstep LM fits of every run (the 16 x 65536 one included) converge
    (status MUSR_OK), equal the single fits, and lie within 1e-3 sigma of the
    oracle's fit."""
    sel = [0, 1, 2, 3]
    gruns = [Run(runs[i][0], runs[i][1]) for i in sel]
    with GBatch(gruns) as b:
        ths, infos = b.fit([runs[i][2] for i in sel], MUSR_CHI2, free=[runs[i][0].free for i in sel])
    for e, i in enumerate(sel):
        lay, d, th = runs[i]
        single, si, cov = gruns[e].fit(th, MUSR_CHI2, free=lay.free)
        assert infos[e]["status"] == 0, (i, infos[e])
        assert si["status"] == 0, (i, si)
        assert rel_err(infos[e]["value"], si["value"]) <= 1e-6
        ref, oi, ocov = oracle.fit(lay, d, th, oracle.CHI2, free=lay.free)
        sig = np.sqrt(np.diag(ocov))
        fr = lay.free.astype(bool)
        assert np.all(np.abs(ths[e][fr] - ref[fr]) <= 1e-3 * sig + 1e-12 * np.abs(ref[fr]))
    for r in gruns:
        r.close()


def test_multistart_batch_matches_sequential_multistart(runs):
    from paper_1604_02334_gb300 import fit_multistart_batch
    sel = [1, 2]
    gruns = [Run(runs[i][0], runs[i][1]) for i in sel]
    starts = [np.stack([runs[i][2], W.range_centre_theta(runs[i][0])]) for i in sel]
    ths, infos = fit_multistart_batch(gruns, starts, MUSR_CHI2, free=[runs[i][0].free for i in sel])
    for e, i in enumerate(sel):
        _, si, _ = gruns[e].fit_multistart(starts[e], MUSR_CHI2, free=runs[i][0].free)
        assert rel_err(infos[e]["value"], si["value"]) <= 1e-6
    for r in gruns:
        r.close()


def test_gbatch_edge_cases():
    g = W.rng(77)
    # a run whose histograms include empty ones and one of 8 bins
    lay = W.multi_detector_layout(4, [0, 8, 0, 3000], window_us=12.8)
    theta = W.multi_detector_theta(lay, g)
    d = W.poisson_counts(oracle.model(lay, theta), 5)
    # a run where the deviance has no likelihood: N = 0 under counts
    lay2 = W.multi_detector_layout(2, [500, 700], window_us=12.8)
    th2 = W.multi_detector_theta(lay2, g)
    d2 = W.poisson_counts(oracle.model(lay2, th2), 6)
    bad = th2.copy()
    bad[0] = 0.0
    bad[2] = 0.0  # N0 and bkg of histogram 0 -> N = 0 where d > 0
    r1, r2 = Run(lay, d), Run(lay2, d2)
    with GBatch([r1, r2, r2]) as b:
        res, flags = b.eval([theta, bad, th2], MUSR_POISSON, MUSR_VALUE_GRAD_GN)
        v, gr, H = oracle.gradient(lay, d, theta, oracle.POISSON, with_gn=True)
        assert grad_rel_err(res[0][1], gr) <= 1e-4
        assert flags[0] == 0 and flags[2] == 0
        assert flags[1] & 1
        v2, g2, _ = oracle.gradient(lay2, d2, th2, oracle.POISSON, with_gn=False)
        assert grad_rel_err(res[2][1], g2) <= 1e-4
    r1.close()
    r2.close()


def test_gbatch_rejects_a_run_without_histograms():
    from paper_1604_02334_gb300 import MusrError
    from workloads import RunLayout  # noqa: F401
    import dataclasses
    lay = W.multi_detector_layout(1, [100], window_us=12.8)
    empty = dataclasses.replace(lay, n_bins=np.zeros(0, dtype=np.int64), map=np.zeros((0, lay.map_width), np.int32))
    r = Run(empty)
    with pytest.raises(MusrError):
        GBatch([r])
    r.close()


def test_fit_batch_bfgs_reaches_the_lm_minimum(runs):
    from paper_1604_02334_gb300 import MUSR_FIT_BFGS
    sel = [1, 2]
    gruns = [Run(runs[i][0], runs[i][1]) for i in sel]
    starts = [runs[i][2] for i in sel]
    free = [runs[i][0].free for i in sel]
    with GBatch(gruns) as b:
        _, lm = b.fit(starts, MUSR_CHI2, free=free)
        _, bf = b.fit(starts, MUSR_CHI2, free=free, method=MUSR_FIT_BFGS)
    with GBatch(gruns, with_gn=False) as b2:
        _, bf2 = b2.fit(starts, MUSR_CHI2, free=free, method=MUSR_FIT_BFGS)
    for e in range(len(sel)):
        _, single, _ = gruns[e].fit(starts[e], MUSR_CHI2, free=free[e], method=MUSR_FIT_BFGS)
        assert bf[e]["status"] == 0 and bf2[e]["status"] in (0, -7)
        assert rel_err(bf[e]["value"], lm[e]["value"]) <= 1e-6
        assert rel_err(bf2[e]["value"], lm[e]["value"]) <= 1e-6
        assert rel_err(bf[e]["value"], single["value"]) <= 1e-6
    for r in gruns:
        r.close()
