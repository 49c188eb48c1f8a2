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
