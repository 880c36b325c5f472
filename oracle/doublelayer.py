"""Double-layer tensor a and its rotation into the Hermitian basis (Sec. II.A, II.B).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from .basis import hermitian_basis, swap_matrix


def double_layer(A: np.ndarray) -> np.ndarray:
    """a = sum_s A_s (x) conj(A_s), Sec. II.A and Fig. 1(b).

    A has shape (d, D, D, D, D) with legs (p, u, l, d, r). Each leg of a joins
    the ket index i (from A) and the bra index ibar (from conj A) into one
    index i + D*ibar of dimension D^2 (ket fastest, as in the listing of
    Sec. II.B). Returns a[U, L, D, R] of shape (D^2,)*4.
    """
    d, D = A.shape[0], A.shape[1]
    q = D * D
    # bra indices are the capitals; axis order (bra, ket) per leg gives bra*D + ket.
    a = np.einsum("puldr,pUVWX->UuVlWdXr", A, np.conj(A))
    if not np.iscomplexobj(A):
        a = a.real
    return np.ascontiguousarray(a.reshape(q, q, q, q))


def open_double_layer(A: np.ndarray) -> np.ndarray:
    """a_open[s, s', U, L, D, R] = A[s, ...] (x) conj(A[s', ...]): physical legs left open.

    Same combined-leg convention as double_layer. Used for reduced density
    matrices, which need the individual bra and ket tensors (Sec. II.B: such
    contractions are dense because A alone carries no Z2 symmetry).
    """
    d, D = A.shape[0], A.shape[1]
    q = D * D
    a = np.einsum("suldr,tUVWX->stUuVlWdXr", A, np.conj(A))
    return np.ascontiguousarray(a.reshape(d, d, q, q, q, q))


def rotate_legs(t: np.ndarray, U: np.ndarray, legs) -> np.ndarray:
    """Apply U^T to each listed leg of t: t'[.., X, ..] = sum_x U[x, X] t[.., x, ..]."""
    for ax in legs:
        t = np.moveaxis(np.tensordot(U, t, axes=([0], [ax])), 0, ax)
    return t


def to_hermitian_basis(a: np.ndarray, D: int) -> np.ndarray:
    """a~ = (U^T)^{(x)4} a: the double layer in the eigenbasis of S (Sec. II.B).

    Rows and columns of every leg are ordered as hermitian_basis(D): the
    D(D+1)/2 even states first, then the D(D-1)/2 odd states.
    """
    U = hermitian_basis(D)
    return rotate_legs(a, U, range(a.ndim))


def from_hermitian_basis(at: np.ndarray, D: int) -> np.ndarray:
    """Inverse of to_hermitian_basis: a = U^{(x)4} a~."""
    U = hermitian_basis(D)
    return rotate_legs(at, U.T, range(at.ndim))


def swap_all_legs(t: np.ndarray, D: int) -> np.ndarray:
    """Act with S on every leg of t (exchange bra and ket on all legs), Fig. 1(e,f)."""
    S = swap_matrix(D)
    for ax in range(t.ndim):
        t = np.moveaxis(np.tensordot(S, t, axes=([1], [ax])), 0, ax)
    return t
