"""The allocation-free block GEMM (hs_gemm_static) against the context-based one (hs_gemm).

hs_gemm_static serves callers that may not allocate device memory (their own
memory manager owns it all, or cudaMalloc's synchronisation is not acceptable
in their loop): it keeps its scratch in a static device array. This file runs
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from paper_2410_11596_gb300 import _lib as L  # noqa: E402

pytestmark = pytest.mark.gpu

# same bounds as tests/test_gpu_tc.py: |C - C_ref| <= tol * sum_k |A_ik| |B_jk|
TOL = {L.HS_PREC_TF32X3: 2 ** -18, L.HS_PREC_TF32: 2 ** -9, L.HS_PREC_BF16X3: 2 ** -14}


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("prec", [L.HS_PREC_TF32X3, L.HS_PREC_TF32, L.HS_PREC_BF16X3])
def test_static_scratch_gemm_matches_context_gemm_twice(ctx, prec):
    shapes = [(300, 200, 100), (129, 257, 70)]
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):            # two calls in a row reuse the same static scratch
        for (M, N, K) in shapes:
            rng = np.random.default_rng(100 * call + M + N + K)
            A = torch.from_numpy(rng.standard_normal((M, K))).cuda()
            B = torch.from_numpy(rng.standard_normal((N, K))).cuda()
            C_ctx = torch.empty((M, N), dtype=torch.float64, device="cuda")
            C_sta = torch.full((M, N), np.nan, dtype=torch.float64, device="cuda")
            L.hs_gemm(ctx.handle, prec, A, B, C_ctx)
            L.hs_gemm_static(prec, A, B, C_sta, status, ctx.stream.cuda_stream)
            ctx.sync()
            torch.cuda.synchronize()
            assert int(status.item()) == 0
            a, b = A.cpu().numpy(), B.cpu().numpy()
            bound = TOL[prec] * (np.abs(a) @ np.abs(b).T)
            c1, c2 = C_ctx.cpu().numpy(), C_sta.cpu().numpy()
            assert np.isfinite(c2).all()
            assert (np.abs(c2 - c1) <= bound).all()
            assert (np.abs(c2 - a @ b.T) <= bound).all()


def test_static_scratch_limit_is_enforced(ctx):
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    M, N, K = 4096, 4096, 512    # 2 * 8192 * 512 * 4 bytes = 32 MiB > 16 MiB
    A = torch.zeros((M, K), dtype=torch.float64, device="cuda")
    B = torch.zeros((N, K), dtype=torch.float64, device="cuda")
    C = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    with pytest.raises(L.HsError) as e:
        L.hs_gemm_static(L.HS_PREC_TF32X3, A, B, C, status, ctx.stream.cuda_stream)
    assert e.value.status == -2
    assert "static scratch" in str(e.value)
