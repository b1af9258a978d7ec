"""The tcgen05 FP32 product used for the dense blocks of the coarse-level block
elimination: three-term TF32 split accumulated in FP32, checked against an FP64
product (FP32-class accuracy, far below the ~1e-3 of a single TF32 product), with
beta accumulation, several tiles in both dimensions and several k chunks."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


def _tf32(x):
    """x rounded to TF32 (10 explicit mantissa bits, nearest, ties away)."""
    b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return b.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,k", [(128, 128, 32), (256, 384, 96), (1024, 1024, 1024)])
def test_gemm_matches_fp64(ras, m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k)).astype(np.float32)
    B = rng.standard_normal((k, n)).astype(np.float32)
    C0 = rng.standard_normal((m, n)).astype(np.float32)
    ref = 0.75 * (A.astype(np.float64) @ B.astype(np.float64)) - 0.5 * C0.astype(np.float64)
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    Cd = torch.tensor(C0, device="cuda")
    ras.gemm_f32(Ad, Bd, Cd, alpha=0.75, beta=-0.5)
    out = Cd.cpu().numpy().astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    err = np.abs(out - ref).max() / scale.max()
    one_pass = np.abs(_tf32(A) @ _tf32(B) - A.astype(np.float64) @ B.astype(np.float64)).max() / scale.max()
    assert err < 1e-5 and err < 0.2 * one_pass, (err, one_pass)


def test_gemm_rejects_unsupported_shapes(ras):
    A = torch.zeros((100, 32), device="cuda")
    B = torch.zeros((32, 128), device="cuda")
    C = torch.zeros((100, 128), device="cuda")
    with pytest.raises(ras.RasError) as e:
        ras.gemm_f32(A, B, C)
    assert e.value.status == ras.RAS_EINVAL
