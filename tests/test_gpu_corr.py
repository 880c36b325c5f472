"""Correlation length on the GPU (hs_correlation_length) against the oracle's definition."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from oracle import doublelayer as dl, observables as ob  # noqa: E402
from paper_2410_11596_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


# cases with a gapped transfer spectrum (|lambda_2| < |lambda_1|); the random D=4
# workload has lambda_2 = -lambda_1, so its xi is not defined
@pytest.mark.parametrize("name,A,chi,moves,precision,tol", [
    ("ising_b0.3", inputs.ising_ipeps(0.3), 16, 60, "f64", 1e-9),
    ("workload1", inputs.workload_tensor(1), 16, 30, "f64", 1e-9),
    ("random_D3", inputs.random_ipeps(2, 3, 7), 18, 30, "f64", 1e-9),
    ("workload1_tf32x3", inputs.workload_tensor(1), 16, 30, "tf32x3", 1e-5),
])
def test_correlation_length_matches_oracle(ctx, name, A, chi, moves, precision, tol):
    """xi from the library's Lanczos on the GPU equals the oracle's ARPACK value of the
    same transfer matrix (the environment the GPU built, copied to the host)."""
    from paper_2410_11596_gb300.api import CTMRG
    c = CTMRG(ctx, A, chi, precision=precision, eig="f64")
    c.run(moves)
    xi = c.correlation_length()
    _, T = c.dense_env()
    xi_ref = ob.correlation_length(T.cpu().numpy(), dl.double_layer(A))
    print(f"{name}: xi = {xi:.12f} oracle {xi_ref:.12f}")
    assert np.isfinite(xi) and xi > 0
    assert abs(xi - xi_ref) <= tol * xi_ref
