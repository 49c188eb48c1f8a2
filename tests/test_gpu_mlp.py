"""GPU parity of the proposer MLP (BF16 tensor-core forward, backward and
Adam) against the NumPy oracle with the same BF16 rounding points.

Forward, layer by layer: the oracle takes the device's own BF16 input
activation of each layer, so the only difference is FP32 against FP64
accumulation before one rounding.  A BF16 result therefore equals the
oracle's or lies one BF16 ulp away (a rounding flip, expected in well under 1%
of the elements); the FP32 output agrees to 1e-5 of its scale.

Backward: the oracle back-propagates from the device's activations.  Flips
of the BF16-rounded errors dZ (as above) move the gradients downstream of
them by up to one BF16 ulp times the weights met, a few 1e-3 of a tensor's
scale; without a flip an element agrees to ~1e-5.  So: at least 90% of the
elements within 2e-4 of the scale, all within 1e-2."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import Mlp, MusrError  # noqa: E402
from oracle import mlp as omlp  # noqa: E402

DEV = torch.device("cuda:0")


def _bf16_ulp(x):
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -126)))
    return 2.0 ** (e - 7)


def _close(got, ref):
    scale = float(np.abs(ref).max()) + 1e-30
    d = np.abs(np.asarray(got, dtype=np.float64) - ref) / scale
    assert d.max() <= 1e-2, f"max deviation {d.max():.3g} of scale"
    assert np.mean(d > 2e-4) <= 0.1, f"{np.mean(d > 2e-4):.3%} of elements beyond 2e-4 of scale"


CASES = [(128, 128, 1, 10, 128, 1.0), (1024, 256, 3, 40, 256, 0.25), (16384, 512, 3, 40, 128, 0.125)]


@pytest.mark.parametrize("n_in,n_hid,n_hl,n_out,batch,scale", CASES)
def test_forward_backward_match_oracle(n_in, n_hid, n_hl, n_out, batch, scale):
    net = Mlp(n_in, n_hid, n_hl, n_out, max_batch=batch, in_scale=scale, seed=n_in + n_hid)
    rng = np.random.default_rng(n_in)
    x = (rng.standard_normal((batch, n_in)) * 2.0 + 1.0).astype(np.float32)
    t = rng.standard_normal((batch, n_out)).astype(np.float32)
    layers = omlp.split_params(net.get_params(), net.layer_shapes())
    y = net.forward(torch.from_numpy(x).to(DEV)).cpu().double().numpy()
    acts = [net.activation(l, batch).astype(np.float64) for l in range(n_hl + 1)]
    np.testing.assert_array_equal(acts[0], omlp.bf16_round(x.astype(np.float64) * scale))
    for li, (w, b) in enumerate(layers):
        z = acts[li] @ omlp.bf16_round(w).T + b
        if li == len(layers) - 1:
            np.testing.assert_allclose(y, z, rtol=0, atol=1e-5 * np.abs(z).max())
            break
        ref = omlp.bf16_round(np.maximum(z, 0.0))
        got = acts[li + 1]
        diff = np.abs(got - ref)
        # one BF16 ulp, or a pre-activation within accumulation error of 0 on either side of the ReLU
        tol = np.maximum(_bf16_ulp(np.maximum(np.abs(ref), np.abs(got))) * 1.0001, 1e-5 * np.abs(ref).max())
        assert np.all(diff <= tol), f"layer {li}"
        assert np.mean(diff > 0) < 0.01, f"layer {li}: {np.mean(diff > 0):.3%} flipped"
    loss = net.backward(torch.from_numpy(x).to(DEV), torch.from_numpy(t).to(DEV))
    acts = [net.activation(l, batch).astype(np.float64) for l in range(n_hl + 1)]
    y = net.activation(n_hl + 1, batch).astype(np.float64)
    loss_ref, grads_ref = omlp.backward(layers, acts, y, t, bf16=True)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    got = omlp.split_params(net.get_grads(), net.layer_shapes())
    for (gw, gb), (rw, rb) in zip(got, grads_ref):
        _close(gw, rw)
        _close(gb, rb)
    net.close()


def test_adam_step_matches_oracle():
    net = Mlp(256, 128, 2, 12, max_batch=128, in_scale=0.5, seed=7)
    rng = np.random.default_rng(8)
    x = torch.from_numpy(rng.standard_normal((128, 256)).astype(np.float32)).to(DEV)
    t = torch.from_numpy(rng.standard_normal((128, 12)).astype(np.float32)).to(DEV)
    p = net.get_params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for step in range(1, 4):
        net.backward(x, t)
        g = net.get_grads().astype(np.float64)
        net.adam(1e-3)
        p, m, v = omlp.adam_step(p, g, m, v, step, 1e-3)
        got = net.get_params().astype(np.float64)
        np.testing.assert_allclose(got, p, rtol=0, atol=1e-6 * np.abs(p).max())


def test_training_fits_a_linear_teacher():
    # targets are a fixed random linear map of the inputs: the loss must fall
    # by 10x within 300 Adam steps
    rng = np.random.default_rng(9)
    net = Mlp(128, 256, 2, 8, max_batch=256, in_scale=1.0, seed=10)
    teacher = rng.standard_normal((8, 128)) / np.sqrt(128)
    losses = []
    for s in range(300):
        xb = rng.standard_normal((256, 128)).astype(np.float32)
        tb = (xb @ teacher.T).astype(np.float32)
        losses.append(net.train_step(torch.from_numpy(xb).to(DEV), torch.from_numpy(tb).to(DEV), 1e-3))
    assert np.mean(losses[-20:]) < 0.1 * np.mean(losses[:5])


def test_bad_shapes_rejected():
    with pytest.raises(MusrError):
        Mlp(100, 128, 1, 8, 128)      # n_in not a multiple of 64
    with pytest.raises(MusrError):
        Mlp(128, 100, 1, 8, 128)      # hidden width not a multiple of 128
    with pytest.raises(MusrError):
        Mlp(128, 128, 1, 200, 128)    # too many outputs
    net = Mlp(128, 128, 1, 8, 128)
    with pytest.raises(MusrError):
        net.forward(torch.zeros((64, 128), device=DEV))   # batch not a multiple of 128
    net.close()
