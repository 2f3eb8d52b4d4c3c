"""GPU checks of the batched (tensor-core) path against plain references."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2511_22460_gb300 import ebr  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("n,B,d", [(1000, 64, 64), (333, 256, 128), (4096, 32, 64),
                                   (129, 96, 128)])
def test_tcgen05_gemm_matches_fp64(n, B, d):
    g = torch.Generator().manual_seed(n + B + d)
    A = (torch.randn(n, d, generator=g) / d ** 0.5).to(torch.bfloat16)
    U = (torch.randn(B, d, generator=g) / d ** 0.5).to(torch.bfloat16)
    out = torch.full((n, B), float("nan"), dtype=torch.float32, device=DEV)
    ebr.debug_gemm_bf16(A.to(DEV).view(torch.int16), U.to(DEV).view(torch.int16), out)
    ref = A.double() @ U.double().T  # products of BF16 values are exact in FP64
    mag = A.double().abs() @ U.double().abs().T
    err = (out.cpu().double() - ref).abs()
    assert torch.all(err <= 1e-6 * mag + 1e-30), float((err / (mag + 1e-30)).max())


@pytest.mark.parametrize("n,B,d", [(1000, 64, 64), (333, 256, 128), (4096, 32, 64),
                                   (129, 96, 128), (300, 256, 64)])
def test_tcgen05_fp8_gemm_matches_fp64(n, B, d):
    """kind::f8f6f4 with E4M3 operands (64-byte rows use the 64-byte swizzle,
    128-byte rows the 128-byte one) against FP64 sums of the decoded codes'
    products, which are exact in FP64."""
    import oracle
    rng = np.random.default_rng(n + B + d)
    A, _ = oracle.quantize_fp8_rows((rng.standard_normal((n, d)) / d ** 0.5).astype(np.float32))
    U, _ = oracle.quantize_fp8_rows((rng.standard_normal((B, d)) / d ** 0.5).astype(np.float32))
    out = torch.full((n, B), float("nan"), dtype=torch.float32, device=DEV)
    ebr.debug_gemm_e4m3(torch.from_numpy(A).to(DEV), torch.from_numpy(U).to(DEV), out)
    tab = oracle.fp8_e4m3_value(np.arange(256, dtype=np.uint8))  # every code's value
    Av, Uv = tab[A], tab[U]
    ref = Av @ Uv.T
    mag = np.abs(Av) @ np.abs(Uv).T
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    worst = float((err / (mag + 1e-30)).max())
    assert np.all(err <= 1e-6 * mag + 1e-30), worst


def test_bounded_wait_gives_up_and_reports_timeout():
    """A device wait that nothing ends returns EBR_ETIMEDOUT after its limit;
    the context stays usable (the tensor-core check runs right after)."""
    import time
    t0 = time.perf_counter()
    rc = ebr.debug_wait_timeout(20_000)  # 20 ms
    assert rc == ebr.EBR_ETIMEDOUT
    assert time.perf_counter() - t0 < 5.0
    assert ebr.debug_wait_timeout(0) == ebr.EBR_EINVAL
    test_tcgen05_gemm_matches_fp64(1000, 64, 64)
