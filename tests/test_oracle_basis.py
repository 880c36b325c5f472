"""Pins of the Hermitian basis, the swap S and the complex grading (Sec. II.B, II.C)."""
import os

import numpy as np
import pytest

from oracle import basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_d2_fixture():
    s = 1 / np.sqrt(2)
    rows = []
    for line in open(os.path.join(GOLDEN, "hermitian_basis_D2.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        tok = line.split()
        coeffs = [{"s": s, "-s": -s}.get(t, None) if t in ("s", "-s") else float(t) for t in tok[1:5]]
        rows.append((tok[0], np.array(coeffs)))
    return rows


def test_d2_basis_is_the_printed_one():
    """Sec. II.B prints the D=2 eigenbasis; the combined order (1 1'), (2 1'), (1 2'), (2 2')."""
    U = basis.hermitian_basis(2)
    par = basis.sector_parities(2)
    rows = _read_d2_fixture()
    assert len(rows) == 4
    for k, (p, vec) in enumerate(rows):
        assert (p == "odd") == bool(par[k])
        np.testing.assert_allclose(U[:, k], vec, atol=1e-15)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7])
def test_swap_is_an_involution_permutation(D):
    S = basis.swap_matrix(D)
    q = D * D
    np.testing.assert_array_equal(S @ S, np.eye(q))
    np.testing.assert_array_equal(S.sum(0), np.ones(q))
    np.testing.assert_array_equal(S, S.T)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7])
def test_sector_dims_from_spectrum_of_S(D):
    """Counting S's +1 and -1 eigenvalues gives D(D+1)/2 and D(D-1)/2 (Sec. II.B)."""
    w = np.linalg.eigvalsh(basis.swap_matrix(D))
    n_even = int(np.sum(np.isclose(w, 1.0)))
    n_odd = int(np.sum(np.isclose(w, -1.0)))
    assert (n_even, n_odd) == basis.sector_dims(D)
    assert n_even == D * (D + 1) // 2 and n_odd == D * (D - 1) // 2


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7])
def test_basis_orthonormal_and_diagonalises_S(D):
    U = basis.hermitian_basis(D)
    S = basis.swap_matrix(D)
    q = D * D
    np.testing.assert_allclose(U.T @ U, np.eye(q), atol=1e-14)
    sign = 1.0 - 2.0 * basis.sector_parities(D)
    np.testing.assert_allclose(U.T @ S @ U, np.diag(sign), atol=1e-14)


def test_graded_product_is_complex_multiplication():
    """Eq. (3) with f of Eq. (2) reproduces complex matrix products; [1, i] converts back."""
    rng = np.random.default_rng(11)
    b1 = rng.standard_normal((7, 5)) + 1j * rng.standard_normal((7, 5))
    b2 = rng.standard_normal((5, 4)) + 1j * rng.standard_normal((5, 4))
    c = basis.from_graded(basis.graded_matmul(basis.to_graded(b1), basis.to_graded(b2)))
    np.testing.assert_allclose(c, b1 @ b2, rtol=1e-14, atol=1e-14)
    np.testing.assert_array_equal(basis.from_graded(basis.to_graded(b1)), b1)


def test_f_tensor_entries():
    """Eq. (2): exactly four non-zero entries, one of them -1 (Im * Im -> Re)."""
    f = basis.F_TENSOR
    assert np.count_nonzero(f) == 4
    assert f[1, 1, 0] == -1.0 and f[0, 0, 0] == 1.0 and f[0, 1, 1] == 1.0 and f[1, 0, 1] == 1.0
