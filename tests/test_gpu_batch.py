"""GPU parity of the batched persistent kernel (many runs x many vectors).

Each batched value is held to the same bar as a single evaluation: relative
error <= 1e-6 against the FP64 oracle (runs of >= 4096 bins), and <= 1e-7
against the single-run kernel, whose per-bin arithmetic it shares.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import rel_err

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_POISSON, Batch, Run, chi2_batch  # noqa: E402


def small_batched_runs(n_runs=6, seed_offset=40):
    """Uneven runs in the shape of the batched workload, scaled down so the
    oracle finishes in seconds: K in 1..8, bins in [4096, 12000]."""
    return W.config_batched(n_runs, seed_offset, min_bins=4096, max_bins=12000, max_hist=8)


@pytest.fixture(scope="module")
def batch_case():
    runs = small_batched_runs()
    data, vecs = [], []
    for br in runs:
        d = W.poisson_counts(oracle.model(br.layout, br.theta), br.seed)
        data.append(d)
        th = W.perturb(br.theta, br.layout.free, 0.01, W.rng(br.seed + 1))
        vecs.append(W.jacobian_vectors(th, br.layout.free, rel_h=1e-3)[:9])  # up to 9 vectors
    return runs, data, vecs


@pytest.mark.parametrize("obj,oobj", [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)])
def test_batch_matches_oracle_and_single(batch_case, obj, oobj):
    runs, data, vecs = batch_case
    gruns = [Run(br.layout, d) for br, d in zip(runs, data)]
    n_vec = [v.shape[0] for v in vecs]
    values = chi2_batch(gruns, np.concatenate([v.ravel() for v in vecs]), n_vec, obj)
    o = 0
    for br, d, v, gr in zip(runs, data, vecs, gruns):
        for j in range(v.shape[0]):
            ref = oracle.objective(br.layout, d, v[j], oobj)
            assert rel_err(values[o], ref) <= 1e-6, (o, values[o], ref)
            assert rel_err(values[o], gr.chi2(v[j], obj)) <= 1e-7
            o += 1
    for gr in gruns:
        gr.close()


def test_batch_plan_reuse_autotune_device_and_repeatability(batch_case):
    torch = pytest.importorskip("torch")
    runs, data, vecs = batch_case
    gruns = [Run(br.layout, d) for br, d in zip(runs, data)]
    max_vec = [v.shape[0] for v in vecs]
    flat = np.concatenate([v.ravel() for v in vecs])
    with Batch(gruns, max_vec) as b:
        a1 = b.eval(flat, MUSR_CHI2)        # autotunes, then evaluates
        a2 = b.eval(flat, MUSR_CHI2)
        assert np.array_equal(a1, a2)       # fixed-order reduction: bitwise repeatable
        th_d = torch.tensor(flat, dtype=torch.float64, device="cuda:0")
        out_d = torch.empty(b.n_values, dtype=torch.float64, device="cuda:0")
        b.eval_device(th_d, out_d, MUSR_CHI2)
        torch.cuda.synchronize()
        assert np.array_equal(out_d.cpu().numpy(), a1)
        # fewer vectors than planned
        nv = [max(1, m // 2) for m in max_vec]
        sub = np.concatenate([v[:n].ravel() for v, n in zip(vecs, nv)])
        a3 = b.eval(sub, MUSR_CHI2, nv)
        o, o1 = 0, 0
        for m, n in zip(max_vec, nv):
            np.testing.assert_array_equal(a3[o:o + n], a1[o1:o1 + n])
            o += n
            o1 += m
    for gr in gruns:
        gr.close()


def test_batch_domain_error_is_per_vector():
    lay, theta, seed = W.config_single()
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    bad = theta.copy()
    bad[0] = -50.0
    with Run(lay, d) as r:
        v = chi2_batch([r], np.stack([theta, bad, theta]).ravel(), [3], MUSR_POISSON)
        assert math.isinf(v[1]) and v[0] == v[2] and math.isfinite(v[0])
        ref = oracle.objective(lay, d, theta, oracle.POISSON)
        assert rel_err(v[0], ref) <= 1e-6
