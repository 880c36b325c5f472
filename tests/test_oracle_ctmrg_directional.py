"""Pins of the directional (non-C4v) CTMRG oracle (Sec. II.A without the C4v assumption):
brute-force patches, the anisotropic Onsager solution, the Eckart-Young property of the
projectors and the reduction to the pinned C4v oracle."""
import numpy as np
import pytest

from oracle import ctmrg, ctmrg_directional as cd, doublelayer as dl, observables as ob
from paper_2410_11596_gb300 import inputs
from pins import contract_patch, onsager_log_z, onsager_log_z_aniso, onsager_nn, onsager_nn_aniso


def _asym(D=2, seed=11):
    return inputs.asymmetric_ipeps(2, D, inputs.SEED_BASE + 5000 + seed)


def test_onsager_aniso_helpers():
    """The anisotropic integrals reduce to the isotropic ones and the correlation is the
    derivative of the free energy (central difference)."""
    assert onsager_log_z_aniso(0.4, 0.4) == pytest.approx(onsager_log_z(0.4), abs=1e-14)
    assert onsager_nn_aniso(0.4, 0.4) == pytest.approx(onsager_nn(0.4), abs=1e-13)
    h = 1e-5
    fd = (onsager_log_z_aniso(0.3 + h, 0.5) - onsager_log_z_aniso(0.3 - h, 0.5)) / (2 * h)
    assert onsager_nn_aniso(0.3, 0.5) == pytest.approx(fd, abs=1e-9)


def test_init_is_rotation_covariant():
    """The eight traced-boundary formulas agree with each other through the frame rotation."""
    a = dl.double_layer(_asym())
    E = cd.init_environment(a)
    E1, a1 = cd.rotate(E, a)
    for x, y in zip(cd.init_environment(a1), E1):
        np.testing.assert_allclose(x, y, atol=1e-15)


def test_c4v_input_gives_the_c4v_init_and_equal_quarters():
    """With a C4v-symmetric double layer every corner is the C4v corner, every edge the C4v
    edge, and the four quarters are the C4v enlarged corner C'."""
    a = dl.double_layer(inputs.random_ipeps(2, 2, 7))
    E = cd.init_environment(a)
    C, T = ctmrg.init_environment(a)
    C, T = C / np.abs(C).max(), T / np.abs(T).max()
    for k in range(8):
        np.testing.assert_allclose(E[k], C if k % 2 == 0 else T, atol=1e-15)
    Cp = ctmrg.enlarged_corner(C, T, a)
    for e, b in cd.frames(E, a):
        np.testing.assert_allclose(cd.quarter(e, b), Cp, atol=1e-13)


def test_c4v_projector_is_the_eigenprojector():
    """C4v input: both quarters are the symmetric C', X = C'^2, so the oblique projector
    P_a P_b^T is the orthogonal projector on the chi eigenvectors of C' of largest |lambda|
    (the pinned C4v truncation) and the kept singular values are (|lambda| / |lambda_max|)^2.
    The oblique form carries S^-1: its rounding bound is 64 u s_max / s_chi."""
    a = dl.double_layer(inputs.random_ipeps(2, 2, 7))
    E = cd.init_environment(a)
    C, T = E[0], E[1]
    for chi in (4, 6):
        P, lam, info = ctmrg.truncate(ctmrg.enlarged_corner(C, T, a), chi)
        assert info.gap > 1e-5
        Pa, Pb, dinfo = cd.projectors(E, a, chi)
        tol = 64 * 2.0 ** -53 / dinfo.kept[-1]
        np.testing.assert_allclose(Pa @ Pb.T, P @ P.T, atol=tol)
        np.testing.assert_allclose(dinfo.kept, (np.abs(lam) / np.abs(lam[0])) ** 2, rtol=tol)


@pytest.mark.parametrize("chi", [5, 9])
def test_projectors_give_the_best_rank_chi_approximation(chi):
    """P_b^T P_a = 1 (so P_a P_b^T is a projector) and Q1^T P_a P_b^T Q4^T is the truncated
    SVD of X = Q1^T Q4^T: its error is the discarded singular weight (Eckart-Young). The
    same construction with P_a and P_b exchanged misses it. The oblique form carries S^-1,
    so its rounding bound is 64 u s_max / s_chi (u the FP64 unit roundoff)."""
    a = dl.double_layer(_asym())
    E = cd.init_environment(a)
    E, _ = cd.left_move(E, a, 16)             # a frame whose four sides differ
    E, a = cd.rotate(E, a)
    Q1, Q4 = cd.left_quarters(E, a)
    assert Q1.shape != Q4.T.shape              # top and bottom bonds differ: X is not square
    X = Q1.T @ Q4.T
    s = np.linalg.svd(X, compute_uv=False)
    Pa, Pb, info = cd.projectors(E, a, chi)
    np.testing.assert_allclose(Pb.T @ Pa, np.eye(chi), atol=64 * 2.0 ** -53 * s[0] / s[chi - 1])
    err = np.linalg.norm(X - Q1.T @ Pa @ Pb.T @ Q4.T)
    assert err == pytest.approx(np.sqrt(np.sum(s[chi:] ** 2)), rel=1e-8)
    np.testing.assert_allclose(info.kept, s[:chi] / s[0], rtol=1e-12)
    swapped = np.linalg.norm(X - Q1.T @ Pb @ Pa.T @ Q4.T)
    assert swapped > 1.5 * err


def _hole(extra_dims):
    n = int(np.prod(extra_dims))
    return np.eye(n).reshape(tuple(extra_dims) * 2)


@pytest.mark.parametrize("n", [0, 1, 2])
def test_environment_equals_finite_patch_without_truncation(n):
    """No truncation (chi never binds): after n sweeps eps is the (2n+3)^2 traced patch
    around one open site, for a tensor with no lattice symmetry. Exact to rounding for
    n <= 1; in the second sweep the 1e-12 s_max floor drops 7-9 of 64 states (s below the
    floor, not zero), which costs 7e-9, hence 1e-7 there."""
    A = _asym()
    a = dl.double_layer(A)
    r = cd.run(a, 4 ** (n + 2), n)
    assert all(len(i.kept) < 4 ** (n + 2) for i in r.infos)   # chi never binds
    eps = cd.one_site_environment(r.E)
    L = 2 * n + 3
    hole = _hole((4, 4, 4, 4))
    ex = contract_patch(lambda i, j: ("open", hole) if (i == n + 1 and j == n + 1) else a, L, L, 2)
    np.testing.assert_allclose(eps / np.linalg.norm(eps), ex / np.linalg.norm(ex),
                               atol=1e-12 if n <= 1 else 1e-7)


@pytest.mark.parametrize("n", [0, 1])
def test_rdms_equal_finite_patch_without_truncation(n):
    """One-site and both two-site RDMs against the brute-force patch with the sites open."""
    A = _asym()
    a = dl.double_layer(A)
    ao = dl.open_double_layer(A)                        # [s, s', u, l, d, r]
    r = cd.run(a, 4 ** (n + 2), n)
    assert all(len(i.kept) < 4 ** (n + 2) for i in r.infos)
    c = n + 1

    def patch(open_sites, rows, cols):
        return contract_patch(lambda i, j: ("open", ao) if (i, j) in open_sites else a, rows, cols, 2)

    rho1 = cd.one_site_rdm(r.E, A)
    ex1 = patch({(c, c)}, 2 * n + 3, 2 * n + 3)
    np.testing.assert_allclose(rho1 / np.trace(rho1), ex1 / np.trace(ex1), atol=1e-12)
    # horizontal pair: the patch is one column wider, the environment sees the same ring
    rh = cd.two_site_rdm_horizontal(r.E, A)
    exh = patch({(c, c), (c, c + 1)}, 2 * n + 3, 2 * n + 4).transpose(0, 2, 1, 3).reshape(4, 4)
    np.testing.assert_allclose(rh / np.trace(rh), exh / np.trace(exh), atol=1e-12)
    rv = cd.two_site_rdm_vertical(r.E, A)
    exv = patch({(c, c), (c + 1, c)}, 2 * n + 4, 2 * n + 3).transpose(0, 2, 1, 3).reshape(4, 4)
    np.testing.assert_allclose(rv / np.trace(rv), exv / np.trace(exv), atol=1e-12)


@pytest.mark.parametrize("bx,by", [(0.3, 0.5), (0.5, 0.7)])
def test_anisotropic_ising_matches_onsager(bx, by):
    """Couplings beta_x on horizontal and beta_y on vertical bonds (disordered and ordered
    phase): the free energy per site and the nearest-neighbour correlation along each
    direction from the anisotropic Onsager solution."""
    A = inputs.anisotropic_ising_ipeps(bx, by)
    a = dl.double_layer(A)
    r = cd.run(a, 24, 60)
    zz = inputs.sz_sz_bond()
    assert cd.log_kappa(r.E, a) == pytest.approx(onsager_log_z_aniso(bx, by), abs=1e-10)
    rh = cd.two_site_rdm_horizontal(r.E, A)
    rv = cd.two_site_rdm_vertical(r.E, A)
    assert ob.bond_energy(rh, zz) == pytest.approx(onsager_nn_aniso(bx, by), abs=1e-9)
    assert ob.bond_energy(rv, zz) == pytest.approx(onsager_nn_aniso(by, bx), abs=1e-9)


def test_c4v_input_converges_to_the_c4v_fixed_point():
    """A C4v tensor: the directional and the C4v schemes truncate differently move by move but
    approximate the same infinite network; at chi = 16 their bond energies agree to the
    truncation level and the directional environment stays C4v-symmetric."""
    A = inputs.random_ipeps(2, 2, inputs.SEED_BASE + 1)
    a = dl.double_layer(A)
    h = inputs.heisenberg_bond()
    r4 = ctmrg.run(a, 16, 60)
    e4 = ob.bond_energy(ob.two_site_rdm(r4.C, r4.T, A), h)
    rd = cd.run(a, 16, 30)
    eh = ob.bond_energy(cd.two_site_rdm_horizontal(rd.E, A), h)
    ev = ob.bond_energy(cd.two_site_rdm_vertical(rd.E, A), h)
    assert eh == pytest.approx(ev, abs=1e-10)
    assert eh == pytest.approx(e4, abs=1e-7)
