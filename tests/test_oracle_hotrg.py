"""Pins of the dense HOTRG oracle and its b-probe (Sec. II.A, III.A)."""
import numpy as np
import pytest

from oracle import doublelayer as dl, hotrg
from paper_2410_11596_gb300 import inputs
from pins import onsager_log_z


@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_free_energy(beta):
    a = dl.double_layer(inputs.ising_ipeps(beta))
    res = hotrg.run(a, 16, 30)
    assert hotrg.log_z_per_site(res) == pytest.approx(onsager_log_z(beta), abs=2e-9)


def test_b_probe_is_antisymmetric_under_swap():
    """b is odd under the bra-ket exchange of all legs, |b| even (Sec. III.A)."""
    D = 2
    b = hotrg.b_tensor(D)
    babs = hotrg.b_tensor(D, absolute=True)
    np.testing.assert_array_equal(dl.swap_all_legs(b, D), -b)
    np.testing.assert_array_equal(dl.swap_all_legs(babs, D), babs)
    assert np.count_nonzero(b) == D ** 8 - D ** 4


def test_b_error_zero_without_truncation():
    """One step at chi >= q^2 keeps every state, so the network stays Hermitian."""
    A = inputs.random_ipeps(2, 2, 12)
    a = dl.double_layer(A)
    assert hotrg.symmetry_error(a, 2, 16, 1) < 1e-13


@pytest.mark.parametrize("chi", [6, 8])
def test_b_error_vanishes_for_gapped_real_network(chi):
    """Real A: Gram eigenvectors are S-eigenvectors unless degenerate, so the b-probe stays ~0."""
    A = inputs.random_ipeps(2, 2, 12)
    a = dl.double_layer(A)
    assert hotrg.symmetry_error(a, 2, chi, 4) < 1e-13


def test_b_probe_detects_a_non_hermitian_network():
    """Replacing a by a + small S-odd part makes the b-probe non-zero, linearly in its size."""
    A = inputs.random_ipeps(2, 2, 12)
    a = dl.double_layer(A)
    odd = hotrg.b_tensor(2) * 1e-3
    e1 = hotrg.symmetry_error(a + odd, 2, 16, 1)
    e2 = hotrg.symmetry_error(a + 2 * odd, 2, 16, 1)
    assert e1 > 1e-8
    assert e2 / e1 == pytest.approx(2.0, rel=1e-2)


@pytest.mark.parametrize("mirror", [False, True])
def test_isometry_takes_the_side_that_discards_less(mirror):
    """The side rule on a network that is not mirror symmetric: the chosen isometry's
    truncation error ||M - V V^T M||^2 equals the smaller of the two best rank-chi errors
    (discarded squared singular values of the fused left and right matricisations, from an
    SVD), and the side is the right one unless the tensor is mirrored (l <-> r)."""
    chi = 4
    A = inputs.lopsided_ipeps()
    if mirror:
        A = A.transpose(0, 1, 4, 3, 2)
    a = dl.double_layer(A)
    a = a / np.abs(a).max()
    M = hotrg.stack_vertical(a, a)
    u, l1, l2, d, r1, r2 = M.shape
    mats = (M.transpose(1, 2, 0, 3, 4, 5).reshape(l1 * l2, -1), M.transpose(4, 5, 0, 1, 2, 3).reshape(r1 * r2, -1))
    best = [float(np.sum(np.linalg.svd(Mx, compute_uv=False)[chi:] ** 2)) for Mx in mats]
    assert best[0] > 10 * best[1] if not mirror else best[1] > 10 * best[0]
    V, _, side = hotrg.isometry(M, chi)
    assert side == (0 if mirror else 1)
    Mx = mats[side]
    resid = float(np.linalg.norm(Mx - V @ (V.T @ Mx)) ** 2)
    assert resid == pytest.approx(min(best), rel=1e-9)
    assert hotrg.run(dl.double_layer(A), chi, 2).sides[0] == side
