"""Hand-written adjoint of the RDM/energy contraction (hs_rdm_vjp) behind torch.autograd."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import ensure_library  # noqa: E402
from oracle import adjoint, ctmrg as oc, doublelayer as dl  # noqa: E402
from paper_2410_11596_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    ensure_library()
    from paper_2410_11596_gb300.api import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("k,chi,moves,basis", [(1, 16, 12, "hermitian"), (2, 32, 15, "hermitian"),
                                               (1, 16, 12, "dense")])
def test_energy_gradient(ctx, k, chi, moves, basis):
    from paper_2410_11596_gb300.api import CTMRG, bond_energy
    A = inputs.workload_tensor(k)
    h = inputs.heisenberg_bond()
    ctm = CTMRG(ctx, A, chi, basis=basis)
    ctm.run(moves)
    At = torch.from_numpy(A.copy()).cuda().requires_grad_(True)
    e = bond_energy(ctm, At, h)
    e.backward()
    g = At.grad.cpu().numpy()
    # (1) dense gradient: torch autograd on the oracle's own environment
    r = oc.run(dl.double_layer(A), chi, moves)
    g_ref = adjoint.energy_gradient(r.C, r.T, A, h)
    assert np.abs(g - g_ref).max() <= 1e-8 * np.abs(g_ref).max()
    # (2) central differences, h = 1e-6, on 64 seeded coordinates, environment fixed
    rng = np.random.default_rng(100 + k)
    eps = 1e-6
    hd = torch.from_numpy(h).cuda()
    Ad = torch.from_numpy(A).cuda()
    for flat in rng.choice(A.size, size=min(64, A.size), replace=False):
        dv = torch.zeros(A.size, dtype=torch.float64, device="cuda")
        dv[flat] = eps
        dv = dv.reshape(A.shape)
        _, tp = ctm.rdm2_of(Ad + dv, hd)
        _, tm = ctm.rdm2_of(Ad - dv, hd)
        fd = float(tp[1] / tp[0] - tm[1] / tm[0]) / (2 * eps)
        assert g.reshape(-1)[flat] == pytest.approx(fd, rel=1e-5, abs=1e-8)
    # (3) four random directional derivatives
    for _ in range(4):
        v = rng.standard_normal(A.shape)
        vd = torch.from_numpy(v).cuda()
        _, tp = ctm.rdm2_of(Ad + eps * vd, hd)
        _, tm = ctm.rdm2_of(Ad - eps * vd, hd)
        fd = float(tp[1] / tp[0] - tm[1] / tm[0]) / (2 * eps)
        assert float(np.sum(g * v)) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def _complex_gradient_checks(ctx, k, chi, moves, n_fd, dense_ref):
    from paper_2410_11596_gb300.api import CTMRG, bond_energy
    A = inputs.workload_tensor(k)
    h = inputs.heisenberg_bond()
    ctm = CTMRG(ctx, A, chi)
    ctm.run(moves)
    At = torch.from_numpy(A.copy()).cuda().requires_grad_(True)
    e = bond_energy(ctm, At, h)
    e.backward()
    g = At.grad.cpu().numpy()
    if dense_ref:
        # dense gradient: torch autograd of the oracle's network on this environment
        C, T = ctm.dense_env()
        g_ref = adjoint.energy_gradient(C.cpu().numpy(), T.cpu().numpy(), A, h)
        assert np.abs(g - g_ref).max() <= 1e-9 * np.abs(g_ref).max()
    rng = np.random.default_rng(200 + k)
    eps = 1e-6
    hd = torch.from_numpy(h).cuda()
    Ad = torch.from_numpy(A).cuda()

    def energy(X):
        _, tr = ctm.rdm2_of(X, hd)
        return float(torch.real(tr[1] / tr[0]))

    for flat in rng.choice(A.size, size=min(n_fd, A.size), replace=False):
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            dv = torch.zeros(A.size, dtype=torch.complex128, device="cuda")
            dv[flat] = unit * eps
            dv = dv.reshape(A.shape)
            fd = (energy(Ad + dv) - energy(Ad - dv)) / (2 * eps)
            assert part(g.reshape(-1)[flat]) == pytest.approx(fd, rel=1e-5, abs=1e-8)
    for _ in range(4):
        v = rng.standard_normal(A.shape) + 1j * rng.standard_normal(A.shape)
        vd = torch.from_numpy(v).cuda()
        fd = (energy(Ad + eps * vd) - energy(Ad - eps * vd)) / (2 * eps)
        # directional derivative along v: Re <g, v> with g = dE/dRe + i dE/dIm
        assert float(np.sum(g.real * v.real + g.imag * v.imag)) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_complex_energy_gradient_small(ctx):
    """Complex A (Sec. II.C): adjoint of the graded environment's rho vs the dense autograd
    gradient and central differences (h = 1e-6) in the real and imaginary directions."""
    _complex_gradient_checks(ctx, 6, 27, 20, 64, True)


def test_complex_energy_gradient_full_size(ctx):
    """Complex workload at full size (D=5, chi=100, 40 moves): finite differences on 16
    coordinates (both parts) and four directional derivatives."""
    _complex_gradient_checks(ctx, 5, 100, 40, 16, False)


@pytest.mark.parametrize("cplx", [False, True])
def test_rdm_vjp_with_the_energy_cotangent_equals_energy_vjp(ctx, cplx):
    """hs_rdm_vjp fed the cotangent of E = Re Tr(rho h)/Tr rho gives hs_energy_vjp's gradient."""
    from paper_2410_11596_gb300.api import CTMRG
    A = inputs.workload_tensor(6 if cplx else 1)
    ctm = CTMRG(ctx, A, 27 if cplx else 16)
    ctm.run(8)
    h = torch.from_numpy(inputs.heisenberg_bond()).cuda()
    if cplx:
        At = torch.from_numpy(A).cuda()
    else:
        At = torch.from_numpy(A.copy()).cuda()
    _, tr = ctm.rdm2_of(At, h)
    eye = torch.eye(4, dtype=tr.dtype, device="cuda")
    drho = 0.7 * (torch.conj(1.0 / tr[0]) * h.t().to(tr.dtype) - torch.conj(tr[1] / tr[0] ** 2) * eye)
    g1 = ctm.rdm2_vjp(At, drho).cpu().numpy()
    g2 = ctm.energy_vjp(At, h, 0.7).cpu().numpy()
    assert np.abs(g1 - g2).max() <= 1e-12 * np.abs(g1).max()
