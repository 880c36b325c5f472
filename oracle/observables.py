"""Observables from a converged C4v environment (Sec. III.A and Sec. III).

Test infrastructure only (see the package docstring).

Network pictures (C corner, T edge, a double layer, * the open site):

    one-site environment eps      two-site RDM rho
        C  T  C                     C  T  T  C
        T  *  T                     T  *  *  T
        C  T  C                     C  T  T  C
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import LinearOperator, eigs

from .basis import swap_matrix
from .doublelayer import open_double_layer


def half_ring(C: np.ndarray, T: np.ndarray) -> np.ndarray:
    """H[a, x, b] = sum C[a, c] T[c, x, e] C[e, b]: a row C-T-C with its two ends open."""
    return np.tensordot(np.tensordot(C, T, axes=([1], [0])), C, axes=([2], [0]))


def one_site_environment(C: np.ndarray, T: np.ndarray) -> np.ndarray:
    """eps[u, l, d, r]: Fig. 1(d) with the centre tensor removed (Sec. III.A).

    Upper half-ring H[a, u, b], left edge T[a, l, a'], right edge T[b, r, b'],
    lower half-ring H[a', d, b'].
    """
    H = half_ring(C, T)
    Y1 = np.tensordot(H, T, axes=([0], [0]))             # [u, b, l, a']
    Y2 = np.tensordot(Y1, T, axes=([1], [0]))            # [u, l, a', r, b']
    eps = np.tensordot(Y2, H, axes=([2, 4], [0, 2]))     # [u, l, r, d]
    return np.ascontiguousarray(eps.transpose(0, 1, 3, 2))


def dagger_env(eps: np.ndarray, D: int) -> np.ndarray:
    """eps^dagger: exchange bra and ket on every open leg and conjugate."""
    S = swap_matrix(D)
    t = eps
    for ax in range(t.ndim):
        t = np.moveaxis(np.tensordot(S, t, axes=([1], [ax])), 0, ax)
    return np.conj(t)


def symmetry_error(eps: np.ndarray, D: int) -> float:
    """S_err = ||eps - eps^dagger|| / ||eps + eps^dagger|| (Eq. (4)), Frobenius norms."""
    ed = dagger_env(eps, D)
    return float(np.linalg.norm(eps - ed) / np.linalg.norm(eps + ed))


def two_site_rdm(C: np.ndarray, T: np.ndarray, A: np.ndarray) -> np.ndarray:
    """rho[(s1 s2), (s1' s2')] of a horizontal bond, not normalised.

    Left block: the left column C-T-C, the two edges above and below site 1 and
    site 1 itself with its physical legs open; the right block likewise.
    They meet on the upper boundary bond, the shared bond m and the lower
    boundary bond.
    """
    d = A.shape[0]
    a_open = open_double_layer(A)                        # [s, s', u, l, d, r]
    E = half_ring(C, T)                                  # [t, x, b] column with open ends
    # left block
    Z1 = np.tensordot(E, T, axes=([0], [0]))             # [l, b, u, t']
    Z2 = np.tensordot(Z1, T, axes=([1], [0]))            # [l, u, t', d, b']
    LB = np.tensordot(Z2, a_open, axes=([0, 1, 3], [3, 2, 4]))   # [t', b', s1, s1', m]
    # right block (mirror image)
    Z1r = np.tensordot(E, T, axes=([0], [2]))            # [r, b, t', u2]
    Z2r = np.tensordot(Z1r, T, axes=([1], [2]))          # [r, t', u2, b', d2]
    RB = np.tensordot(Z2r, a_open, axes=([0, 2, 4], [5, 2, 4]))  # [t', b', s2, s2', m]
    rho = np.tensordot(LB, RB, axes=([0, 1, 4], [0, 1, 4]))      # [s1, s1', s2, s2']
    return rho.transpose(0, 2, 1, 3).reshape(d * d, d * d)


def bond_energy(rho: np.ndarray, h: np.ndarray) -> float:
    """E = Tr(rho h) / Tr(rho), real part."""
    return float(np.real(np.trace(rho @ h) / np.trace(rho)))


def hermiticity_error(rho: np.ndarray) -> float:
    """||rho - rho^dagger|| / ||rho||."""
    return float(np.linalg.norm(rho - rho.conj().T) / np.linalg.norm(rho))


def corner_spectrum(C: np.ndarray) -> np.ndarray:
    """Singular values of C divided by the largest, descending (gauge invariant)."""
    s = np.linalg.svd(C, compute_uv=False)
    return s / s[0]


def log_kappa(C: np.ndarray, T: np.ndarray, a: np.ndarray) -> complex:
    """ln kappa = ln(Z1 Z4 / Z2^2): the free energy per site, -beta f, of the norm network.

    Z1 = C T C / T a T / C T C, Z4 = Tr C^4 (corners only), Z2 = C T C / C T C
    (one column of edges). Invariant under rescaling C and T.
    """
    eps = one_site_environment(C, T)
    Z1 = np.sum(eps * a)
    Z4 = np.trace(C @ C @ C @ C)
    H = half_ring(C, T)
    Z2 = np.sum(H * H)
    return np.log(complex(Z1 * Z4 / Z2 ** 2))


def correlation_length(T: np.ndarray, a: np.ndarray, k: int = 2) -> float:
    """xi = -1 / ln|l2 / l1| of the column transfer matrix T-a-T.

    E[(alpha, l, beta), (alpha', r, beta')] = sum_{u, d} T[alpha, u, alpha'] a[u, l, d, r] T[beta, d, beta'].
    parity unpinned (no closed form is checked for it).
    """
    chi, q = T.shape[0], T.shape[1]
    n = chi * q * chi
    dt = np.result_type(T, a)

    def mv(v):
        v = v.reshape(chi, q, chi)
        W1 = np.tensordot(T, v, axes=([2], [0]))          # [alpha, u, r, beta']
        W2 = np.tensordot(W1, a, axes=([1, 2], [0, 3]))   # [alpha, beta', l, d]
        W3 = np.tensordot(W2, T, axes=([1, 3], [2, 1]))   # [alpha, l, beta]
        return W3.reshape(n)

    op = LinearOperator((n, n), matvec=mv, dtype=dt)
    vals = eigs(op, k=k, which="LM", return_eigenvectors=False, tol=1e-12)
    mags = np.sort(np.abs(vals))[::-1]
    if mags[1] == 0:
        return 0.0
    r = mags[1] / mags[0]
    return float(np.inf) if r >= 1.0 else float(-1.0 / np.log(r))
