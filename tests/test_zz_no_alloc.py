"""ras_norm2_noalloc: the entry point for callers that cannot allocate device
memory at call time (a framework owning all device memory through its own
pool, a latency-critical loop that cannot afford an allocation). Its partial
sums live in a static device array in the library; it must give the same norm
as residual_eval's (which uses library-allocated scratch), bit for bit (the
same grid, accumulation and fixed-order finalisation), on two calls in a row.

This file is collected last on purpose, and passes both alone in a fresh
process and after the other GPU tests (the per-device address lookup happens
on the first call)."""
import numpy as np
import pytest
import torch

from paper_2007_13966_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ras():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_13966_gb300 import ras as R
    R.lib()
    return R


@pytest.mark.parametrize("dims", [(24, 20, 12), (128, 128, 64)])
def test_noalloc_norm_matches_residual_eval(ras, dims):
    res = syn.small_3d(*dims, seed=11)
    gp = ras.Problem(res)
    N = res.grid.n
    p = torch.tensor(syn.random_pressure(res, 5), device="cuda")
    p_l = 0.98 * p
    F = torch.zeros(N, dtype=torch.float64, device="cuda")
    ref = gp.residual_eval(p, p_l, p_l, res.dt, 1, F, want_norm=True)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):   # the static scratch keeps the previous call's contents
        out.fill_(float("nan"))
        ras.norm2_noalloc(F, out)
        torch.cuda.synchronize()
        assert out.item() == ref


def test_noalloc_rejects_sizes_beyond_the_maximum(ras):
    import ctypes as C
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = ras.lib().ras_norm2_noalloc(C.c_void_p(x.data_ptr()), C.c_longlong(2 ** 31),
                                     C.c_void_p(out.data_ptr()), None)
    assert st == ras.RAS_EINVAL
    ras.norm2_noalloc(x[:0], out)
    torch.cuda.synchronize()
    assert out.item() == 0.0
