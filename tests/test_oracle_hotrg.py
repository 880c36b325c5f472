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
