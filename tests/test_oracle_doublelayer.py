"""Pins of the double layer and its Hermitian-basis form (Sec. II.A-II.C)."""
import numpy as np
import pytest

from oracle import basis, doublelayer as dl
from paper_2410_11596_gb300 import inputs


def _parity_total(D):
    p = basis.sector_parities(D)
    return (p[:, None, None, None] + p[None, :, None, None] + p[None, None, :, None] + p[None, None, None, :]) % 2


@pytest.mark.parametrize("D", [1, 2, 3])
@pytest.mark.parametrize("cplx", [False, True])
def test_full_trace_is_norm_of_A(D, cplx):
    """Closing all four legs of a with delta(i, ibar) gives sum |A|^2."""
    A = inputs.random_ipeps(2, D, 3, complex_valued=cplx)
    a = dl.double_layer(A)
    v = np.zeros(D * D)
    for k in range(D):
        v[basis.combined_index(k, k, D)] = 1.0
    tr = np.einsum("uldr,u,l,d,r->", a, v, v, v, v)
    np.testing.assert_allclose(tr, np.sum(np.abs(A) ** 2), rtol=1e-14)


@pytest.mark.parametrize("cplx", [False, True])
def test_a_is_positive_as_ket_bra_matrix(cplx):
    """a = sum_s A_s A_s^dagger: Hermitian and positive semidefinite from ket to bra indices."""
    D = 2
    A = inputs.random_ipeps(2, D, 4, complex_valued=cplx)
    a = dl.double_layer(A).reshape((D, D) * 4)           # [ub, uk, lb, lk, db, dk, rb, rk]
    m = a.transpose(1, 3, 5, 7, 0, 2, 4, 6).reshape(D ** 4, D ** 4)
    np.testing.assert_allclose(m, m.conj().T, atol=1e-15)
    w = np.linalg.eigvalsh(m)
    assert w.min() > -1e-13
    assert np.linalg.matrix_rank(m, tol=1e-12) <= A.shape[0]


@pytest.mark.parametrize("D", [2, 3, 4])
def test_real_a_swap_invariant_and_block_sparse(D):
    """Real A: a is invariant under S on all legs (Fig. 1(e)); odd-total blocks of a~ vanish."""
    A = inputs.random_ipeps(2, D, 5)
    a = dl.double_layer(A)
    np.testing.assert_allclose(dl.swap_all_legs(a, D), a, atol=1e-15)
    at = dl.to_hermitian_basis(a, D)
    odd = _parity_total(D) == 1
    assert np.abs(at[odd]).max() <= 1e-15 * np.abs(at).max()
    assert np.abs(at[~odd]).max() > 0.1 * np.abs(at).max()
    np.testing.assert_allclose(dl.from_hermitian_basis(at, D), a, atol=1e-14)


@pytest.mark.parametrize("D", [2, 3])
def test_complex_a_graded(D):
    """Complex A: S maps a to conj(a); even-total blocks are real, odd-total imaginary (Sec. II.C)."""
    A = inputs.random_ipeps(2, D, 6, complex_valued=True)
    a = dl.double_layer(A)
    np.testing.assert_allclose(dl.swap_all_legs(a, D), np.conj(a), atol=1e-15)
    at = dl.to_hermitian_basis(a, D)
    odd = _parity_total(D) == 1
    scale = np.abs(at).max()
    assert np.abs(at[~odd].imag).max() <= 1e-15 * scale
    assert np.abs(at[odd].real).max() <= 1e-15 * scale
    assert np.abs(at[odd].imag).max() > 0.01 * scale


def test_d4_symmetrized_input_is_c4v():
    A = inputs.random_ipeps(2, 3, 9)
    for g in inputs.D4_LEG_PERMUTATIONS:
        np.testing.assert_allclose(np.transpose(A, (0, 1 + g[0], 1 + g[1], 1 + g[2], 1 + g[3])), A, atol=1e-15)
    assert np.abs(A).max() == 1.0
