"""Histogram-sharded evaluation and fits (the multi-GPU extension) on CPU:
world size 2 and 3 on the gloo backend, each rank's shard evaluated by the
FP64 oracle in place of its GPU.  Checks the partition, that the combined
value / gradient / Gauss-Newton matrix equal the oracle's on the whole run,
that the combination is bitwise the same on every rank, and that LM and BFGS
fits driven through musr_fit_eval (host-only) reach the oracle's fit of the
whole run and return the same parameters on every rank."""
import json
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case(n_hist):
    lay = W.multi_detector_layout(n_hist, [1500 + 377 * k for k in range(n_hist)], window_us=12.8)
    theta = W.multi_detector_theta(lay, W.rng(606))
    return lay, theta


def test_partition_covers_every_histogram_once_and_balances():
    from paper_1604_02334_gb300.shard import partition_histograms
    nb = [5000, 100, 7000, 3000, 3000, 250, 9000]
    for world in (1, 2, 3, 8):
        parts = partition_histograms(nb, world)
        assert len(parts) == world
        flat = np.sort(np.concatenate(parts))
        assert np.array_equal(flat, np.arange(len(nb)))
        loads = [int(np.sum(np.asarray(nb)[p])) if len(p) else 0 for p in parts]
        assert max(loads) - min(loads) <= max(nb)
        assert partition_histograms(nb, world)[0].tolist() == parts[0].tolist()  # deterministic


def _worker(rank, world, port, n_hist, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import oracle
    from paper_1604_02334_gb300 import MUSR_CHI2, MUSR_FIT_BFGS, MUSR_FIT_LM, MUSR_VALUE, MUSR_VALUE_GRAD_GN
    from paper_1604_02334_gb300.shard import ShardedRun, shard_data, shard_layout
    lay, theta = _case(n_hist)
    data = W.poisson_counts(oracle.model(lay, theta), 607)

    def make_eval(sl, sd):
        def ev(th, obj, mode):
            if mode == MUSR_VALUE:
                return oracle.objective(sl, sd, th, obj), None, None
            v, g, H = oracle.gradient(sl, sd, th, obj, with_gn=mode == MUSR_VALUE_GRAD_GN)
            return v, g, H
        return ev

    from paper_1604_02334_gb300.shard import partition_histograms
    hists = partition_histograms(lay.n_bins, world)[rank]
    ev = make_eval(shard_layout(lay, hists), shard_data(lay, data, hists)) if len(hists) else None
    sr = ShardedRun(lay, data, evaluate=ev)
    th = W.perturb(theta, lay.free, 0.01, W.rng(608))
    res = {"hists": sr.hists.tolist()}
    for obj in (oracle.CHI2, oracle.POISSON):
        v, g, H = sr.chi2_grad(th, obj, MUSR_VALUE_GRAD_GN)
        res[f"v{obj}"], res[f"g{obj}"], res[f"H{obj}"] = v, g.tolist(), H.ravel().tolist()
    start = W.perturb(theta, lay.free, 0.02, W.rng(609))
    for name, method in (("lm", MUSR_FIT_LM), ("bfgs", MUSR_FIT_BFGS)):
        t_fit, info, _ = sr.fit(start, MUSR_CHI2, free=lay.free, method=method)
        res[name] = {"theta": t_fit.tolist(), "status": info["status"], "value": info["value"], "ndf": info["ndf"]}
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_hist", [(2, 5), (3, 2)])
def test_sharded_evaluation_and_fit_match_the_whole_run(tmp_path, world, n_hist):
    import oracle
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, n_hist, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    lay, theta = _case(n_hist)
    data = W.poisson_counts(oracle.model(lay, theta), 607)
    th = W.perturb(theta, lay.free, 0.01, W.rng(608))
    assert sorted(sum((r["hists"] for r in res), [])) == list(range(n_hist))
    for obj in (oracle.CHI2, oracle.POISSON):
        v, g, H = oracle.gradient(lay, data, th, obj, with_gn=True)
        for r in res:  # bitwise the same on every rank
            assert r[f"v{obj}"] == res[0][f"v{obj}"] and r[f"g{obj}"] == res[0][f"g{obj}"]
            assert r[f"H{obj}"] == res[0][f"H{obj}"]
        assert abs(res[0][f"v{obj}"] - v) <= 1e-12 * abs(v)
        assert np.linalg.norm(np.array(res[0][f"g{obj}"]) - g) <= 1e-10 * np.linalg.norm(g)
        assert np.linalg.norm(np.array(res[0][f"H{obj}"]).reshape(H.shape) - H) <= 1e-12 * np.linalg.norm(H)
    start = W.perturb(theta, lay.free, 0.02, W.rng(609))
    th_o, info_o, cov_o = oracle.fit(lay, data, start, oracle.CHI2)
    assert info_o["status"] == 0
    sig = np.sqrt(np.diag(cov_o))
    fr = lay.free.astype(bool)
    for name in ("lm", "bfgs"):
        for r in res:
            assert r[name]["status"] == 0 and r[name]["theta"] == res[0][name]["theta"]
        t = np.array(res[0][name]["theta"])
        assert np.max(np.abs(t[fr] - th_o[fr]) / sig) <= 1e-3, name
        assert res[0][name]["ndf"] == lay.total_bins - int(fr.sum())
