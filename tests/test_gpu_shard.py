"""Histogram-sharded evaluation on the GPU: the run split into shards, each a
run of its own on cuda:0 (one process, no collective: the shards' sums are
added in shard order as ranks would), against the unsharded run and the FP64
oracle; and a fit driven through musr_fit_eval by the shards' sums against
musr_fit on the whole run and the oracle's fit."""
import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err

pytestmark = pytest.mark.gpu
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_LM, MUSR_POISSON,  # noqa: E402
                                    MUSR_VALUE_GRAD, MUSR_VALUE_GRAD_GN, Run)
from paper_1604_02334_gb300.shard import fit_eval, partition_histograms, shard_data, shard_layout  # noqa: E402


def shard_runs(lay, data, n):
    parts = partition_histograms(lay.n_bins, n)
    return [Run(shard_layout(lay, h), shard_data(lay, data, h).astype(np.float32)) for h in parts if len(h)]


def sharded_eval(runs, P):
    def ev(theta, mode):
        v, g, H = 0.0, np.zeros(P), np.zeros((P, P))
        for r in runs:  # shard order, as the ranks' all-gather adds them
            rv, rg, rH = r.chi2_grad(theta, ev.obj, gn=mode == MUSR_VALUE_GRAD_GN)
            v += rv
            g += rg
            if rH is not None:
                H += rH
        return v, g, H
    return ev


@pytest.mark.parametrize("obj,oobj", [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)])
def test_shards_add_up_to_the_run(obj, oobj):
    lay, theta, seed = W.config_multi_detector(16, 65536)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 5))
    runs = shard_runs(lay, d, 2)
    ev = sharded_eval(runs, lay.n_params)
    ev.obj = obj
    v, g, H = ev(th, MUSR_VALUE_GRAD_GN)
    with Run(lay, d.astype(np.float32)) as whole:
        wv, wg, wH = whole.chi2_grad(th, obj, gn=True)
    rv, rg, rH = oracle.gradient(lay, d, th, oobj, with_gn=True)
    assert rel_err(v, wv) <= 1e-6 and rel_err(v, rv) <= 1e-6
    assert grad_rel_err(g, wg) <= 1e-4 and grad_rel_err(g, rg) <= 1e-4
    assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
    for r in runs:
        r.close()


@pytest.mark.parametrize("method", [MUSR_FIT_LM, MUSR_FIT_BFGS], ids=["lm", "bfgs"])
def test_sharded_fit_matches_the_run_and_the_oracle(method):
    lay, theta, seed = W.config_multi_detector(16, 65536)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    start = W.perturb(theta, lay.free, 0.01, W.rng(seed + 31))
    runs = shard_runs(lay, d, 3)
    ev = sharded_eval(runs, lay.n_params)
    ev.obj = MUSR_CHI2
    th_s, info_s, _ = fit_eval(lay.n_params, lay.total_bins, ev, start, free=lay.free, method=method)
    th_o, info_o, cov_o = oracle.fit(lay, d, start, oracle.CHI2)
    assert info_s["status"] == 0 and info_o["status"] == 0
    sig = np.sqrt(np.diag(cov_o))
    fr = lay.free.astype(bool)
    assert np.max(np.abs(th_s[fr] - th_o[fr]) / sig) <= 1e-3
    assert rel_err(info_s["value"] / info_s["ndf"], info_o["value"] / info_o["ndf"]) <= 1e-6
    for r in runs:
        r.close()
