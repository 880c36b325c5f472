"""Hermitian basis of one combined bra-ket leg (Sec. II.B) and the complex grading (Sec. II.C).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def combined_index(i: int, ibar: int, D: int) -> int:
    """Position of the pair (ket i, bra ibar) in a combined leg of dimension D^2.

    Sec. II.B lists the D = 2 combined basis as (1 1'), (2 1'), (1 2'), (2 2')
    (primes marking bra indices): the ket index runs fastest.
    """
    return i + D * ibar


def swap_matrix(D: int) -> np.ndarray:
    """The swap S of Sec. II.B, S_{i ibar j jbar} = delta(i, jbar) delta(ibar, j), as a D^2 x D^2 matrix.

    Row (i, ibar), column (j, jbar): it exchanges the ket and bra index of one
    combined leg.
    """
    q = D * D
    S = np.zeros((q, q))
    for i in range(D):
        for ib in range(D):
            for j in range(D):
                for jb in range(D):
                    if i == jb and ib == j:
                        S[combined_index(i, ib, D), combined_index(j, jb, D)] = 1.0
    return S


def sector_dims(D: int) -> tuple[int, int]:
    """(dim even, dim odd) = (D + (D^2 - D)/2, (D^2 - D)/2), Sec. II.B."""
    return D + (D * D - D) // 2, (D * D - D) // 2


def hermitian_basis(D: int) -> np.ndarray:
    """Eigenbasis U of S (columns), even sector first, then odd (Sec. II.B).

    Even: (k k') for k = 0..D-1, then (k l' + l k')/sqrt(2) for k < l in
    lexicographic order. Odd: (k l' - l k')/sqrt(2) for k < l, in the same order.
    Here (k l') is the state with ket k and bra l. Sec. II.B gives exactly this
    for D = 2: {(1 1'), (2 2'), (1 2' + 2 1')/sqrt2 | (1 2' - 2 1')/sqrt2}.
    """
    q = D * D
    cols = []
    for k in range(D):
        v = np.zeros(q)
        v[combined_index(k, k, D)] = 1.0
        cols.append(v)
    pairs = [(k, l) for k in range(D) for l in range(k + 1, D)]
    for sign in (+1.0, -1.0):
        for k, l in pairs:
            v = np.zeros(q)
            v[combined_index(k, l, D)] = 1.0 / np.sqrt(2.0)
            v[combined_index(l, k, D)] = sign / np.sqrt(2.0)
            cols.append(v)
    return np.stack(cols, axis=1)


def sector_parities(D: int) -> np.ndarray:
    """Parity (0 even, 1 odd) of each column of hermitian_basis(D)."""
    ne, no = sector_dims(D)
    return np.concatenate([np.zeros(ne, dtype=np.int64), np.ones(no, dtype=np.int64)])


#: The tensor f of Eq. (2), 0-based: f[p, q, r] with 0 = real slice, 1 = imaginary slice.
F_TENSOR = np.zeros((2, 2, 2))
F_TENSOR[0, 0, 0] = 1.0
F_TENSOR[1, 1, 0] = -1.0
F_TENSOR[0, 1, 1] = 1.0
F_TENSOR[1, 0, 1] = 1.0


def to_graded(b: np.ndarray) -> np.ndarray:
    """Eq. (1): append a leg q of dimension 2 holding Re b (q = 0) and Im b (q = 1)."""
    return np.stack([np.real(b), np.imag(b)], axis=-1).astype(np.float64)


def from_graded(bt: np.ndarray) -> np.ndarray:
    """Inverse of Eq. (1): contract the extra leg with the vector [1, i] (Sec. II.C)."""
    return bt @ np.array([1.0, 1.0j])


def graded_matmul(b1: np.ndarray, b2: np.ndarray) -> np.ndarray:
    """Eq. (3): c[i, k, r] = sum_{j, p, q} b1[i, j, p] b2[j, k, q] f[p, q, r] with f of Eq. (2)."""
    return np.einsum("ijp,jkq,pqr->ikr", b1, b2, F_TENSOR)
