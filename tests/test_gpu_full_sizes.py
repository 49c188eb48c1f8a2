"""GPU parity at the full sizes of the measured configurations, in the launch
configurations the benchmark times:

  * 32 x 131072 bins, 72 free parameters (the gradient workload): value,
    gradient and Gauss-Newton matrix against the FP64 oracle for both
    objectives;
  * the paper's Table 1 histogram lengths (16 x 85320 ... 16 x 426601): chi2
    against the oracle;
  * the batched workload (64 uneven runs x (P+1) vectors, 2.7e9
    bin-evaluations in one launch, the autotuned shape): sampled outputs --
    every vector of the three smallest runs and the base vector of the three
    largest -- against the oracle, which computes them one by one;
  * the batched adjoint over 64 runs of 16 x 65536: sampled runs' values and
    gradients against the oracle;
  * the limits: one histogram of 2^24 bins, and 1024 histograms with 3080
    parameters (beyond the Gauss-Newton limit of 1024).
Tolerances as elsewhere: objective relative 1e-6, gradient 1e-4 norm-wise and
per component (of the largest), GN matrix 1e-4 Frobenius.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from _gpu_util import grad_rel_err, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import (MUSR_CHI2, MUSR_POISSON, MUSR_VALUE_GRAD, Batch, GBatch,  # noqa: E402
                                    Run)

OBJS = [(MUSR_CHI2, oracle.CHI2), (MUSR_POISSON, oracle.POISSON)]


@pytest.mark.parametrize("obj,oobj", OBJS)
def test_gradient_workload_32x131072(obj, oobj):
    """Value, gradient (norm-wise and per component) and Gauss-Newton matrix
    (Frobenius relative 1e-4) of the 32 x 131072 workload against the oracle."""
    lay, theta, seed = W.config_gradient()
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 1))
    with Run(lay, d.astype(np.float32)) as run:
        v, g, _ = run.chi2_grad(th, obj)
        vh, gh, H = run.chi2_grad(th, obj, gn=True)
        # queued host-theta evaluations back to back (as the benchmark times
        # them: each one's bin loop may overlap the previous one's reduction,
        # in the queued tiling), the measured theta between perturbed ones,
        # against the device entry (FP32 lane sums round differently between
        # tilings: value 1e-6, gradient 1e-5) and the oracle
        P = lay.n_params
        ths = [W.perturb(theta, lay.free, 0.01, W.rng(seed + 40 + j)) for j in range(5)]
        ths[2] = th
        out = torch.full((5, 1 + P), float("nan"), dtype=torch.float64, device="cuda:0")
        ref = torch.full((5, 1 + P), float("nan"), dtype=torch.float64, device="cuda:0")
        st = torch.full((5,), -1, dtype=torch.int32, device="cuda:0")
        for j in range(5):
            run.chi2_grad_async(ths[j], out[j], obj, MUSR_VALUE_GRAD, st[j:j + 1])
        torch.cuda.synchronize()
        for j in range(5):
            run.chi2_grad_device(torch.tensor(ths[j], device="cuda:0"), ref[j], obj, MUSR_VALUE_GRAD)
        torch.cuda.synchronize()
        qa, qr = out.cpu().numpy(), ref.cpu().numpy()
        assert not st.any().item()
        for j in range(5):
            assert rel_err(qa[j, 0], qr[j, 0]) <= 1e-6
            assert grad_rel_err(qa[j, 1:], qr[j, 1:]) <= 1e-5
    rv, rg, rH = oracle.gradient(lay, d, th, oobj, with_gn=True)
    assert rel_err(v, rv) <= 1e-6
    assert grad_rel_err(g, rg) <= 1e-4
    assert rel_err(vh, rv) <= 1e-6
    assert grad_rel_err(gh, rg) <= 1e-4
    assert np.linalg.norm(H - rH) <= 1e-4 * np.linalg.norm(rH)
    assert rel_err(qa[2, 0], rv) <= 1e-6
    assert grad_rel_err(qa[2, 1:], rg) <= 1e-4


@pytest.mark.parametrize("M", [W.SWEEP_BINS[0], W.SWEEP_BINS[-1]])
def test_table1_shapes(M):
    lay, theta, seed = W.config_sweep(M)
    d = W.poisson_counts(oracle.model(lay, theta), seed)
    th = W.perturb(theta, lay.free, 0.01, W.rng(seed + 2))
    with Run(lay, d.astype(np.float32)) as run:
        for obj, oobj in OBJS:
            assert rel_err(run.chi2(th, obj), oracle.objective(lay, d, th, oobj)) <= 1e-6


def test_batched_workload_sampled():
    runs = W.config_batched()
    dev = torch.device("cuda:0")
    data, vecs, gruns = [], [], []
    for br in runs:
        d = W.poisson_counts(oracle.model(br.layout, br.theta), br.seed)
        data.append(d)
        gruns.append(Run(br.layout, torch.tensor(d, dtype=torch.float32, device=dev)))
        vecs.append(W.jacobian_vectors(br.theta, br.layout.free, 1e-6))
    mv = [v.shape[0] for v in vecs]
    with Batch(gruns, mv) as b:
        th = torch.tensor(np.concatenate([v.ravel() for v in vecs]), device=dev)
        out = torch.empty(b.n_values, dtype=torch.float64, device=dev)
        b.eval_device(th, out)  # tunes the launch shape, as in the benchmark
        b.eval_device(th, out)
        torch.cuda.synchronize()
        values = out.cpu().numpy()
    offs = np.r_[0, np.cumsum(mv)]
    size = [br.layout.total_bins for br in runs]
    order = np.argsort(size)
    for r in order[:3]:
        for j in range(mv[r]):
            ref = oracle.objective(runs[r].layout, data[r], vecs[r][j], oracle.CHI2)
            assert rel_err(values[offs[r] + j], ref) <= 1e-6, (r, j)
    for r in order[-3:]:
        ref = oracle.objective(runs[r].layout, data[r], vecs[r][0], oracle.CHI2)
        assert rel_err(values[offs[r]], ref) <= 1e-6, r
    for g in gruns:
        g.close()


def test_batched_adjoint_64x16x65536_sampled():
    lay = W.multi_detector_layout(16, 65536, 12.8)
    g = W.rng(W.BASE_SEED + 77)
    n_runs = 64
    thetas = [W.multi_detector_theta(lay, g) for _ in range(n_runs)]
    sample = [0, 31, 63]
    data = [W.poisson_counts(oracle.model(lay, t), 7000 + i) for i, t in enumerate(thetas)]
    runs = [Run(lay, d.astype(np.float32)) for d in data]
    th = [W.perturb(t, lay.free, 0.01, g) for t in thetas]
    with GBatch(runs, with_gn=False) as b:
        res, flags = b.eval(th, MUSR_CHI2, MUSR_VALUE_GRAD)
    assert not np.any(flags)
    for i in sample:
        v, gr, _ = oracle.gradient(lay, data[i], th[i], oracle.CHI2, with_gn=False)
        assert rel_err(res[i][0], v) <= 1e-6
        assert grad_rel_err(res[i][1], gr) <= 1e-4
    for r in runs:
        r.close()


def test_maximum_histogram_length():
    """One histogram at the per-histogram limit of 2^24 bins (t up to 21 us with
    1.25 ns bins): value and gradient against the oracle."""
    lay = W.single_hist_layout(1 << 24, 0.00125)
    theta = W.single_hist_truth()
    d = W.poisson_counts(oracle.model(lay, theta), 31)
    th = W.perturb(theta, lay.free, 0.01, W.rng(32))
    with Run(lay, d.astype(np.float32)) as run:
        for obj, oobj in OBJS:
            v, g, _ = run.chi2_grad(th, obj)
            rv, rg, _ = oracle.gradient(lay, d, th, oobj, with_gn=False)
            assert rel_err(v, rv) <= 1e-6
            assert grad_rel_err(g, rg) <= 1e-4


def test_many_histograms_many_parameters():
    """1024 histograms of 777 bins with per-histogram N0, background and phase:
    3080 parameters (theta through device memory, role rows from the device
    table), beyond the Gauss-Newton limit (1024): value and gradient only."""
    lay = W.multi_detector_layout(1024, 777, 12.8)
    theta = W.multi_detector_theta(lay, W.rng(33))
    d = W.poisson_counts(oracle.model(lay, theta), 34)
    th = W.perturb(theta, lay.free, 0.01, W.rng(35))
    assert lay.n_params > 1024
    with Run(lay, d.astype(np.float32)) as run:
        for obj, oobj in OBJS:
            v, g, _ = run.chi2_grad(th, obj)
            rv, rg, _ = oracle.gradient(lay, d, th, oobj, with_gn=False)
            assert rel_err(v, rv) <= 1e-6
            assert grad_rel_err(g, rg) <= 1e-4
