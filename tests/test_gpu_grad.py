"""Gradient of the bond energy through the CTMRG iterations (hs_ctmrg_energy_grad behind
torch.autograd): the energy against the oracle, and directional derivatives along C4v-symmetric
directions against central finite differences of the oracle's whole CTMRG run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from oracle import ctmrg as oc, doublelayer as dl, observables as ob  # noqa: E402
from paper_2410_11596_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


def _oracle_energy(A, chi, moves):
    r = oc.run(dl.double_layer(A), chi, moves)
    return ob.bond_energy(ob.two_site_rdm(r.C, r.T, A), inputs.heisenberg_bond()), r.min_gap


@pytest.mark.parametrize("basis", ["hermitian", "dense"])
@pytest.mark.parametrize("k,chi,moves", [(1, 12, 8), (1, 16, 12)])
def test_gradient_through_iterations_matches_finite_differences(ctx, basis, k, chi, moves):
    """D=2 (workload 1). The central differences use the oracle (step 1e-5 along a unit direction:
    truncation error ~1e-10 of the derivative, checked by halving the step), so the bound is
    1e-6 relative."""
    from paper_2410_11596_gb300.api import ctmrg_energy
    A = inputs.workload_tensor(k)
    h = inputs.heisenberg_bond()
    At = torch.from_numpy(A.copy()).cuda().requires_grad_(True)
    E = ctmrg_energy(ctx, At, chi, moves, h, basis)
    E.backward()
    g = At.grad.cpu().numpy()
    e_ref, gap = _oracle_energy(A, chi, moves)
    assert gap > 1e-6
    assert E.item() == pytest.approx(e_ref, abs=1e-10)
    rng = np.random.default_rng(70 + chi)
    eps = 1e-5
    for _ in range(4):
        v = inputs.d4_symmetrize(rng.standard_normal(A.shape))
        v /= np.linalg.norm(v)
        fd = (_oracle_energy(A + eps * v, chi, moves)[0] - _oracle_energy(A - eps * v, chi, moves)[0]) / (2 * eps)
        print(f"{basis} chi={chi}: <g, v> = {float(np.sum(g * v)):.10e}, central difference = {fd:.10e}")
        assert float(np.sum(g * v)) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_gradient_bases_agree(ctx):
    """The Hermitian and the dense basis run the same CTMRG (same kept states); their gradients,
    projected on C4v-symmetric directions, agree to rounding."""
    from paper_2410_11596_gb300 import _lib as L
    A = inputs.workload_tensor(1)
    Ad = torch.from_numpy(A.copy()).cuda()
    hd = torch.from_numpy(inputs.heisenberg_bond()).cuda()
    out = []
    for basis in (L.HS_BASIS_HERMITIAN, L.HS_BASIS_DENSE):
        dA = torch.empty_like(Ad)
        e = L.hs_ctmrg_energy_grad(ctx.handle, Ad, 2, 2, basis, 12, 8, hd, dA)
        out.append((e, inputs.d4_symmetrize(dA.cpu().numpy())))
    assert out[0][0] == pytest.approx(out[1][0], abs=1e-12)
    np.testing.assert_allclose(out[0][1], out[1][1], atol=1e-9 * np.abs(out[1][1]).max())
