"""Pins of the NumPy MLP oracle against things other than itself: torch's
float32 -> bfloat16 conversion (round to nearest even), closed-form outputs
of hand-set networks, central finite differences of the FP64 loss, and
torch.optim.Adam."""
import numpy as np
import pytest

from oracle import mlp

torch = pytest.importorskip("torch")


def test_bf16_round_matches_torch_including_ties():
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-20, 20, 20000), [0.0, -0.0, 1.0, -1.0]])
    # exact ties: low 16 bits of the FP32 pattern == 0x8000, both parities of bit 16
    u = (rng.integers(0x3f000000, 0x41000000, 4000, dtype=np.int64) & ~0xFFFF) | 0x8000
    x = np.concatenate([x, u.astype(np.uint32).view(np.float32).astype(np.float64)])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).double().numpy()
    np.testing.assert_array_equal(mlp.bf16_round(x), ref)


def test_forward_closed_form():
    # 2 -> 2 (ReLU) -> 1: h = relu([x0 - x1, x1 - x0] + [0.5, 0]); y = h0 + 2 h1 - 1
    layers = [(np.array([[1.0, -1.0], [-1.0, 1.0]]), np.array([0.5, 0.0])),
              (np.array([[1.0, 2.0]]), np.array([-1.0]))]
    x = np.array([[3.0, 1.0], [1.0, 3.0], [0.0, 0.0]])
    _, y = mlp.forward(layers, x, bf16=False)
    np.testing.assert_array_equal(y[:, 0], [1.5, 3.0, -0.5])
    # input scale multiplies before the first layer
    _, y2 = mlp.forward(layers, x / 4.0, in_scale=4.0, bf16=False)
    np.testing.assert_array_equal(y2, y)
    # BF16 rounding of operands: 1 + 2^-9 rounds to 1 (tie to even), 1 + 3 * 2^-9 to 1 + 2^-7
    lin = [(np.array([[1.0]]), np.array([0.0]))]
    _, y3 = mlp.forward(lin, np.array([[1 + 2.0 ** -9], [1 + 3 * 2.0 ** -9]]), bf16=True)
    np.testing.assert_array_equal(y3[:, 0], [1.0, 1 + 2.0 ** -7])


def _net(rng, dims):
    return [(rng.standard_normal((dims[i + 1], dims[i])) / np.sqrt(dims[i]), rng.standard_normal(dims[i + 1]) * 0.1)
            for i in range(len(dims) - 1)]


@pytest.mark.parametrize("dims", [[5, 7, 3], [6, 8, 8, 4], [4, 9, 9, 9, 2]])
def test_gradients_match_central_differences(dims):
    rng = np.random.default_rng(len(dims))
    layers = _net(rng, dims)
    x = rng.standard_normal((11, dims[0]))
    t = rng.standard_normal((11, dims[-1]))
    _, grads = mlp.loss_and_grads(layers, x, t, in_scale=0.7, bf16=False)
    flat = mlp.join_params(layers)
    shapes = [w.shape for (w, _) in layers]
    g_an = mlp.join_params(grads)
    h = 1e-6
    g_fd = np.zeros_like(flat)
    for j in range(flat.shape[0]):
        p = flat.copy()
        p[j] += h
        lp, _ = mlp.loss_and_grads(mlp.split_params(p, shapes), x, t, 0.7, bf16=False)
        p[j] -= 2 * h
        lm, _ = mlp.loss_and_grads(mlp.split_params(p, shapes), x, t, 0.7, bf16=False)
        g_fd[j] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(g_an, g_fd, rtol=1e-6, atol=1e-8 * np.abs(g_fd).max())


def test_loss_is_mean_squared_error():
    layers = [(np.eye(3), np.zeros(3))]
    x = np.array([[1.0, 2.0, 3.0], [0.0, 0.0, 0.0]])
    t = np.array([[1.0, 2.0, 5.0], [1.0, 0.0, 0.0]])
    loss, _ = mlp.loss_and_grads(layers, x, t, bf16=False)
    assert loss == pytest.approx((4.0 + 1.0) / 6.0, rel=1e-15)


def test_adam_matches_torch():
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal(50)
    gs = [rng.standard_normal(50) * s for s in (1.0, 1e-3, 10.0, 0.0)]
    p = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    q, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step, g in enumerate(gs, start=1):
        opt.zero_grad()
        p.grad = torch.tensor(g)
        opt.step()
        q, m, v = mlp.adam_step(q, g, m, v, step, 1e-2)
        np.testing.assert_allclose(q, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_split_join_roundtrip():
    rng = np.random.default_rng(4)
    layers = _net(rng, [4, 6, 3])
    flat = mlp.join_params(layers)
    back = mlp.split_params(flat, [(6, 4), (3, 6)])
    for (w, b), (w2, b2) in zip(layers, back):
        np.testing.assert_array_equal(w, w2)
        np.testing.assert_array_equal(b, b2)
