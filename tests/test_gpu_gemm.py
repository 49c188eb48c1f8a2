"""GPU parity of the tcgen05 BF16 GEMM against a float64 CPU matmul of the
same BF16 inputs.  FP32 accumulation of K products: relative error
<= 2e-5 * sqrt(K / 64) of the output scale; BF16 outputs to 1 BF16 ulp."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
pytest.importorskip("paper_1604_02334_gb300")
from paper_1604_02334_gb300 import gemm_bf16  # noqa: E402


@pytest.mark.parametrize("m,n,k,relu,bias", [(128, 128, 64, False, False), (256, 384, 1024, True, True),
                                              (512, 128, 16384, False, True), (128, 256, 192, True, False)])
def test_gemm_matches_cpu(m, n, k, relu, bias):
    g = torch.Generator().manual_seed(m + n + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    bv = torch.randn(n, generator=g) if bias else None
    ref = a.double() @ b.double().T
    if bias:
        ref = ref + bv.double()
    if relu:
        ref = ref.clamp_min(0)
    dev = torch.device("cuda:0")
    out = torch.full((m, n), float("nan"), dtype=torch.float32, device=dev)
    outb = torch.empty((m, n), dtype=torch.bfloat16, device=dev)
    err = gemm_bf16(a.to(dev), b.to(dev), bv.to(dev) if bias else None, relu, out, outb)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    scale = float(np.sqrt(k))
    np.testing.assert_allclose(out.cpu().double().numpy(), ref.numpy(), rtol=0,
                               atol=2e-5 * scale * np.sqrt(k / 64) + 1e-6)
    np.testing.assert_allclose(outb.cpu().double().numpy(), out.cpu().to(torch.bfloat16).double().numpy(),
                               rtol=0, atol=0)


def test_gemm_rejects_bad_shapes():
    from paper_1604_02334_gb300 import MusrError
    dev = torch.device("cuda:0")
    a = torch.zeros(100, 64, dtype=torch.bfloat16, device=dev)
    b = torch.zeros(128, 64, dtype=torch.bfloat16, device=dev)
    out = torch.empty(100, 128, device=dev)
    with pytest.raises(MusrError):
        gemm_bf16(a, b, out_f32=out)


@pytest.mark.parametrize("m,n,k,ws_floats,ldc", [(128, 512, 16384, 152 * 128 * 128, 512),   # 29 slices of 9 K tiles
                                                 (128, 128, 320, 152 * 128 * 128, 136),    # 5 slices of 1 K tile
                                                 (256, 256, 4096, 3 * 256 * 256, 264),     # workspace caps at 3
                                                 (128, 256, 1024, 100, 256)])              # too small: unsplit
def test_gemm_split_k_matches_cpu(m, n, k, ws_floats, ldc):
    """Split-K (partial tiles in the workspace, slice-order reduction, then bias
    and ReLU) against the same float64 reference; the row stride ldc > n checks
    that the reduction writes with the output's stride and leaves the padding."""
    g = torch.Generator().manual_seed(7 * m + n + k)
    a = torch.randn(m, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    bv = torch.randn(n, generator=g)
    ref = (a.double() @ b.double().T + bv.double()).clamp_min(0)
    dev = torch.device("cuda:0")
    out = torch.full((m, ldc), float("nan"), dtype=torch.float32, device=dev)
    outb = torch.zeros((m, ldc), dtype=torch.bfloat16, device=dev)
    ws = torch.full((ws_floats,), float("nan"), dtype=torch.float32, device=dev)
    err = gemm_bf16(a.to(dev), b.to(dev), bv.to(dev), True, out, outb, ws=ws)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    o = out.cpu().double().numpy()
    np.testing.assert_allclose(o[:, :n], ref.numpy(), rtol=0, atol=2e-5 * np.sqrt(k) * np.sqrt(k / 64) + 1e-6)
    assert np.isnan(o[:, n:]).all()
    np.testing.assert_allclose(outb[:, :n].cpu().double().numpy(), out[:, :n].cpu().to(torch.bfloat16).double().numpy(),
                               rtol=0, atol=0)
    assert (outb[:, n:].cpu() == 0).all()
    # deterministic: a second call gives the same bits
    out2 = torch.empty_like(out)
    gemm_bf16(a.to(dev), b.to(dev), bv.to(dev), True, out2, None, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(out[:, :n], out2[:, :n])
