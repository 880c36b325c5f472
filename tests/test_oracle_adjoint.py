"""Pin of the oracle's energy gradient: torch autograd vs central differences of the numpy oracle."""
import numpy as np
import pytest

from oracle import adjoint, ctmrg, doublelayer as dl, observables as ob
from paper_2410_11596_gb300 import inputs


def _energy_np(C, T, A, h):
    return ob.bond_energy(ob.two_site_rdm(C, T, A), h)


def test_autograd_matches_finite_differences():
    A = inputs.workload_tensor(1)
    h = inputs.heisenberg_bond()
    r = ctmrg.run(dl.double_layer(A), 16, 10)
    g = adjoint.energy_gradient(r.C, r.T, A, h)
    rng = np.random.default_rng(3)
    eps = 1e-6
    for flat in rng.choice(A.size, size=12, replace=False):
        e = np.zeros(A.size)
        e[flat] = eps
        e = e.reshape(A.shape)
        fd = (_energy_np(r.C, r.T, A + e, h) - _energy_np(r.C, r.T, A - e, h)) / (2 * eps)
        assert g.reshape(-1)[flat] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    assert _energy_np(r.C, r.T, A, h) == pytest.approx(
        float(adjoint.energy_torch(*(__import__("torch").tensor(x) for x in (r.C, r.T, A, h)))), rel=1e-13)


def test_product_state_gradient_closed_form():
    """Product state, D = 1: E = <S>^2 per component, dE/dphi known in closed form."""
    phi = np.array([0.6, 0.3])
    A = inputs.product_state_ipeps(phi, 1)
    h = inputs.heisenberg_bond()
    r = ctmrg.run(dl.double_layer(A), 4, 3)
    g = adjoint.energy_gradient(r.C, r.T, A, h)[:, 0, 0, 0, 0]
    n2 = phi @ phi
    S = [np.array([[0, 0.5], [0.5, 0]]), np.diag([0.5, -0.5])]    # S^y vanishes for real phi
    grad = np.zeros(2)
    for s in S:
        m = phi @ s @ phi / n2
        dm = (2 * s @ phi) / n2 - (phi @ s @ phi) * 2 * phi / n2 ** 2
        grad += 2 * m * dm
    np.testing.assert_allclose(g, grad, rtol=1e-10, atol=1e-13)


def test_complex_gradient_matches_finite_differences():
    """Complex A: the gradient dE/dRe A + i dE/dIm A against central differences of the
    numpy oracle in the real and in the imaginary direction (h = 1e-6)."""
    A = inputs.workload_tensor(6)
    h = inputs.heisenberg_bond()
    r = ctmrg.run(dl.double_layer(A), 12, 8)
    g = adjoint.energy_gradient(r.C, r.T, A, h)
    rng = np.random.default_rng(4)
    eps = 1e-6
    for flat in rng.choice(A.size, size=8, replace=False):
        e = np.zeros(A.size, dtype=complex)
        e[flat] = eps
        e = e.reshape(A.shape)
        fr = (_energy_np(r.C, r.T, A + e, h) - _energy_np(r.C, r.T, A - e, h)) / (2 * eps)
        fi = (_energy_np(r.C, r.T, A + 1j * e, h) - _energy_np(r.C, r.T, A - 1j * e, h)) / (2 * eps)
        assert g.reshape(-1)[flat].real == pytest.approx(fr, rel=1e-6, abs=1e-9)
        assert g.reshape(-1)[flat].imag == pytest.approx(fi, rel=1e-6, abs=1e-9)
