"""Batched CTMRG (hs_ctmrg_move_batched): many independent instances moved concurrently."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from paper_2410_11596_gb300 import _lib as L, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    ensure_library()


@pytest.mark.parametrize("precision,eig", [("f64", "f64"), ("tf32x3", "subspace")])
def test_batched_equals_one_by_one(precision, eig):
    """Each instance of a batch (mixed D and chi, real and complex) ends in the same
    state as when it is moved alone: the batch shares nothing between instances."""
    from paper_2410_11596_gb300.api import CTMRG, BatchedCTMRG, Context
    specs = [(2, 8, False), (3, 18, False), (2, 12, True), (3, 27, False), (2, 16, False)]
    tensors = [inputs.random_ipeps(2, D, 500 + i, complex_valued=c) for i, (D, _, c) in enumerate(specs)]
    chis = [chi for _, chi, _ in specs]
    batch = BatchedCTMRG(tensors, chis, precision=precision, eig=eig, nthreads=3)
    batch.run(12)
    h = inputs.heisenberg_bond()
    ctx = Context(0)
    for A, chi, m in zip(tensors, chis, batch.members):
        c = CTMRG(ctx, A, chi, precision=precision, eig=eig)
        c.run(12)
        assert (m.env.chi_even, m.env.chi_odd) == (c.env.chi_even, c.env.chi_odd)
        assert abs(m.energy(h) - c.energy(h)) <= 1e-13
    assert len(batch.latencies_ms) == 12 and all(len(x) == len(specs) for x in batch.latencies_ms)
    batch.close()
    ctx.close()


def test_batched_rejects_shared_context():
    from paper_2410_11596_gb300.api import CTMRG, Context
    ctx = Context(0)
    A = inputs.random_ipeps(2, 2, 7)
    c1, c2 = CTMRG(ctx, A, 8), CTMRG(ctx, A, 8)
    with pytest.raises(L.HsError):
        L.hs_ctmrg_move_batched([ctx.handle, ctx.handle], [c1.a, c2.a], [c1.env, c2.env], [8, 8], 2)
    ctx.close()
