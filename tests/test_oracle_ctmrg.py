"""Pins of the dense C4v CTMRG oracle (Sec. II.A, III.A): closed forms, Onsager, brute force."""
import numpy as np
import pytest

from oracle import ctmrg, doublelayer as dl, observables as ob
from paper_2410_11596_gb300 import inputs
from pins import contract_patch, onsager_log_z, onsager_nn

SPIN = [np.array([[0, 0.5], [0.5, 0]]), np.array([[0, -0.5j], [0.5j, 0]]), np.diag([0.5, -0.5])]


@pytest.mark.parametrize("D", [1, 4])
def test_product_state_energy_closed_form(D):
    """Product state: E = sum_a <phi|S^a|phi>^2 / <phi|phi>^2, also when embedded at D = 4."""
    phi = np.array([0.6, 0.1 + 0.8j])
    A = inputs.product_state_ipeps(phi, D)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 8, 4)
    rho = ob.two_site_rdm(r.C, r.T, A)
    n2 = np.vdot(phi, phi).real
    closed = sum((np.vdot(phi, s @ phi).real / n2) ** 2 for s in SPIN)
    assert ob.bond_energy(rho, inputs.heisenberg_bond()) == pytest.approx(closed, abs=1e-14)
    sz = np.vdot(phi, np.diag([1.0, -1.0]) @ phi).real / n2
    assert ob.bond_energy(rho, inputs.sz_sz_bond()) == pytest.approx(sz * sz, abs=1e-14)


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_free_energy_and_bond_correlation(beta):
    """Norm network of the Ising iPEPS = 2D Ising partition function (Onsager)."""
    A = inputs.ising_ipeps(beta)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 32, 120)
    assert ob.log_kappa(r.C, r.T, a).real == pytest.approx(onsager_log_z(beta), abs=1e-9)
    rho = ob.two_site_rdm(r.C, r.T, A)
    assert ob.bond_energy(rho, inputs.sz_sz_bond()) == pytest.approx(onsager_nn(beta), abs=1e-9)


def _hole(extra_dims):
    n = int(np.prod(extra_dims))
    return np.eye(n).reshape(tuple(extra_dims) * 2)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [0, 1, 2])
def test_environment_equals_finite_patch_without_truncation(n, cplx):
    """chi >= chi0 q^n: eps after n moves equals the (2n+3)^2 traced-boundary patch."""
    A = inputs.random_ipeps(2, 2, 7, complex_valued=cplx)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 64, n)
    eps = ob.one_site_environment(r.C, r.T)
    L = 2 * n + 3
    hole = _hole((4, 4, 4, 4))
    ex = contract_patch(lambda i, j: ("open", hole) if (i == n + 1 and j == n + 1) else a, L, L, 2)
    e1, e2 = eps / np.linalg.norm(eps), ex / np.linalg.norm(ex)
    np.testing.assert_allclose(e1, e2, atol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [0, 1])
def test_two_site_rdm_equals_finite_patch_without_truncation(n, cplx):
    A = inputs.random_ipeps(2, 2, 8, complex_valued=cplx)
    a = dl.double_layer(A)
    a_open = dl.open_double_layer(A)
    r = ctmrg.run(a, 64, n)
    rho = ob.two_site_rdm(r.C, r.T, A)
    rows, cols = 2 * n + 3, 2 * n + 4
    sites = {(n + 1, n + 1), (n + 1, n + 2)}
    ex = contract_patch(lambda i, j: ("open", a_open) if (i, j) in sites else a, rows, cols, 2)
    ex = ex.transpose(0, 2, 1, 3).reshape(4, 4)          # [s1, s1', s2, s2'] -> [(s1 s2), (s1' s2')]
    np.testing.assert_allclose(rho / np.trace(rho), ex / np.trace(ex), atol=1e-13)


def test_symmetry_error_definition():
    """Eq. (4) for eps = H + t K (H Hermitian, K anti-Hermitian parts): S_err = t ||K|| / ||H||."""
    rng = np.random.default_rng(1)
    D = 2
    e = rng.standard_normal((4,) * 4) + 1j * rng.standard_normal((4,) * 4)
    H = 0.5 * (e + ob.dagger_env(e, D))
    K = 0.5 * (e - ob.dagger_env(e, D))
    assert ob.symmetry_error(H, D) < 1e-15
    for t in (1e-6, 0.3, 2.0):
        expect = t * np.linalg.norm(K) / np.linalg.norm(H)
        assert ob.symmetry_error(H + t * K, D) == pytest.approx(expect, rel=1e-12)


def test_gapped_workload1_dense_ctmrg_is_hermitian():
    """Without multiplets at the cut the dense truncation keeps S-symmetry up to rounding."""
    A = inputs.workload_tensor(1)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 16, 30)
    assert r.min_gap > 1e-9
    assert ob.symmetry_error(ob.one_site_environment(r.C, r.T), 2) < 1e-12
    assert ob.hermiticity_error(ob.two_site_rdm(r.C, r.T, A)) < 1e-12


def test_keep_all_when_boundary_small():
    A = inputs.random_ipeps(2, 2, 3)
    r = ctmrg.run(dl.double_layer(A), 16, 1)
    assert r.C.shape == (16, 16) and r.T.shape == (16, 4, 16)
    assert np.isinf(r.infos[0].gap)


def test_corner_spectrum_gauge_invariant():
    """Normalised corner spectrum is unchanged by an orthogonal change of the boundary basis."""
    A = inputs.random_ipeps(2, 2, 4)
    r = ctmrg.run(dl.double_layer(A), 8, 6)
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((8, 8)))
    np.testing.assert_allclose(ob.corner_spectrum(Q.T @ r.C @ Q), ob.corner_spectrum(r.C), atol=1e-14)


def test_correlation_length_decoupled_chains_closed_form():
    """a[u,l,d,r] = M[u,d] M[l,r]: every row is an independent 1D chain with
    transfer matrix M and the boundary is an exact product state (chi = 1), so the
    column transfer matrix T-a-T is (v1^T M v1) M and xi = -1/ln|mu2/mu1|."""
    rng = np.random.default_rng(5)
    for q in (4, 9):  # q = D^2: the traced-boundary init pairs bra and ket
        X = rng.standard_normal((q, q))
        M = X @ X.T + 0.5 * np.eye(q)
        a = np.einsum("ud,lr->uldr", M, M)
        r = ctmrg.run(a, 1, 30)
        mu = np.sort(np.abs(np.linalg.eigvalsh(M)))[::-1]
        assert ob.correlation_length(r.T, a) == pytest.approx(-1.0 / np.log(mu[1] / mu[0]), rel=1e-12)


def test_correlation_length_ising_approaches_onsager():
    """High-temperature 2D Ising (K = beta = 0.2 < K_c): the axis correlation length is
    1/(ln coth K - 2K). At finite chi CTMRG underestimates it and the error shrinks with chi."""
    beta = 0.2
    exact = 1.0 / (np.log(1.0 / np.tanh(beta)) - 2.0 * beta)
    a = dl.double_layer(inputs.ising_ipeps(beta))
    errs = []
    for chi in (8, 16):
        r = ctmrg.run(a, chi, 120)
        errs.append(exact - ob.correlation_length(r.T, a))
    assert 0.0 < errs[1] < errs[0] < 0.02 * exact


def test_complex_rule_reduces_to_real_rule():
    """The SVD truncation used for complex tensors, fed a real tensor as complex,
    keeps the same states as the eigenvalue rule (singular values = |lambda|,
    U = V up to signs): same energy and corner spectrum after truncating moves."""
    A = inputs.random_ipeps(2, 3, seed=7)
    a = dl.double_layer(A)
    rr = ctmrg.run(a, 12, 20)
    rc = ctmrg.run(a.astype(complex), 12, 20)
    assert rr.min_gap > 1e-6
    h = inputs.heisenberg_bond()
    er = ob.bond_energy(ob.two_site_rdm(rr.C, rr.T, A), h)
    ec = ob.bond_energy(ob.two_site_rdm(rc.C, rc.T, A.astype(complex)), h)
    assert ec == pytest.approx(er, abs=1e-13)
    np.testing.assert_allclose(ob.corner_spectrum(rc.C), ob.corner_spectrum(rr.C), atol=1e-12)


@pytest.mark.parametrize("D,chi", [(2, 8), (3, 12)])
def test_complex_truncation_preserves_hermiticity(D, chi):
    """Complex A (Sec. II.C): the truncated environment keeps the bra-ket
    symmetry, so rho is Hermitian and S_err (Eq. (4)) vanishes to rounding."""
    A = inputs.random_ipeps(2, D, seed=11, complex_valued=True)
    a = dl.double_layer(A)
    r = ctmrg.run(a, chi, 30)
    assert r.min_gap > 1e-6
    assert ob.hermiticity_error(ob.two_site_rdm(r.C, r.T, A)) < 1e-11
    assert ob.symmetry_error(ob.one_site_environment(r.C, r.T), D) < 1e-11


def test_corner_spectrum_known_signed_values():
    """A symmetric corner with eigenvalues of both signs: the spectrum is |lambda| in
    descending order over the largest (a sign, an ordering or a missing division fails)."""
    lam = np.array([-3.0, 2.0, -0.5, 1.0, 0.25, -1.5])
    Q, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((6, 6)))
    C = Q @ np.diag(lam) @ Q.T
    expect = np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.25]) / 3.0
    np.testing.assert_allclose(ob.corner_spectrum(C), expect, atol=1e-14)


@pytest.mark.parametrize("cplx", [False, True])
def test_corner_spectrum_known_singular_values_non_normal(cplx):
    """An oriented (complex or non-symmetric) corner C = U diag(s) V^dagger: the spectrum is
    s / s_max; the moduli of its eigenvalues are different numbers here."""
    rng = np.random.default_rng(4)
    n = 7
    X = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Y = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    U, _ = np.linalg.qr(X)
    V, _ = np.linalg.qr(Y)
    s = np.array([5.0, 4.0, 2.5, 1.0, 0.7, 0.2, 0.01])
    C = U @ np.diag(s) @ V.conj().T
    np.testing.assert_allclose(ob.corner_spectrum(C), s / 5.0, atol=1e-13)
    mags = np.sort(np.abs(np.linalg.eigvals(C)))[::-1]
    assert np.abs(mags / mags[0] - s / 5.0).max() > 1e-3


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [1, 2])
def test_corner_spectrum_equals_quadrant_without_truncation(n, cplx):
    """chi >= q^(n+1): after n moves the corner is the (n+1) x (n+1) upper-left quadrant,
    traced on its outer legs, up to unitary changes of the boundary basis, so its spectrum is
    that of the brute-force quadrant matrix between the two cuts."""
    from pins import contract_quadrant
    A = inputs.random_ipeps(2, 2, 9, complex_valued=cplx)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 64, n)
    Q = contract_quadrant(a, n + 1, 2)
    s = np.linalg.svd(Q, compute_uv=False)
    assert r.C.shape == Q.shape
    np.testing.assert_allclose(ob.corner_spectrum(r.C), s / s[0], atol=1e-12)


@pytest.mark.parametrize("D", [1, 4])
def test_one_site_rdm_product_state_closed_form(D):
    """Product state: rho1 / Tr rho1 = |phi><phi| / <phi|phi>, also embedded at D = 4."""
    phi = np.array([0.6, 0.1 + 0.8j])
    A = inputs.product_state_ipeps(phi, D)
    r = ctmrg.run(dl.double_layer(A), 8, 4)
    rho = ob.one_site_rdm(r.C, r.T, A)
    np.testing.assert_allclose(rho / np.trace(rho), np.outer(phi, phi.conj()) / np.vdot(phi, phi).real, atol=1e-14)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n", [0, 1])
def test_one_site_rdm_equals_finite_patch_without_truncation(n, cplx):
    """chi >= chi0 q^n: rho1 after n moves equals the (2n+3)^2 traced-boundary patch whose
    centre site keeps its physical legs open."""
    A = inputs.random_ipeps(2, 2, 10, complex_valued=cplx)
    a = dl.double_layer(A)
    r = ctmrg.run(a, 64, n)
    rho = ob.one_site_rdm(r.C, r.T, A)
    L = 2 * n + 3
    ao = dl.open_double_layer(A)
    ex = contract_patch(lambda i, j: ("open", ao) if (i == n + 1 and j == n + 1) else a, L, L, 2)
    np.testing.assert_allclose(rho / np.trace(rho), ex / np.trace(ex), atol=1e-13)


def test_two_site_rdm_chunked_sum_is_the_same_sum():
    """Summing the bottom bond in slices gives the same rho (memory bound for large chi D^2)."""
    A = inputs.random_ipeps(2, 2, 12)
    r = ctmrg.run(dl.double_layer(A), 12, 6)
    full = ob.two_site_rdm(r.C, r.T, A)
    for c in (1, 5, 12):
        np.testing.assert_allclose(ob.two_site_rdm(r.C, r.T, A, chunk=c), full, rtol=1e-13, atol=1e-15)
