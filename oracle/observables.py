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
    """H[a, x, b] = sum C[a, c] T[c, x, e] C[e, b]: corner, edge, corner along the
    boundary orientation, entering at a and leaving at b, bulk leg x open."""
    return np.tensordot(np.tensordot(C, T, axes=([1], [0])), C, axes=([2], [0]))


def one_site_environment(C: np.ndarray, T: np.ndarray) -> np.ndarray:
    """eps[u, l, d, r]: Fig. 1(d) with the centre tensor removed (Sec. III.A).

    The boundary ring, clockwise: upper half-ring H[a, u, b] (corner, top edge,
    corner), right edge T[b, r, b'], lower half-ring H[b', d, a'], left edge
    T[a', l, a].
    """
    H = half_ring(C, T)
    Y1 = np.tensordot(H, T, axes=([2], [0]))             # [a, u, r, b']
    Y2 = np.tensordot(Y1, H, axes=([3], [0]))            # [a, u, r, d, a']
    eps = np.tensordot(Y2, T, axes=([4, 0], [0, 2]))     # [u, r, d, l]
    return np.ascontiguousarray(eps.transpose(0, 3, 2, 1))


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


def one_site_rdm(C: np.ndarray, T: np.ndarray, A: np.ndarray) -> np.ndarray:
    """rho1[s, s'] of one site, not normalised: the one-site environment eps
    closed with the open double layer A_s (x) conj(A_s') (Sec. III.A)."""
    eps = one_site_environment(C, T)
    return np.einsum("stuldr,uldr->st", open_double_layer(A), eps)


def two_site_rdm(C: np.ndarray, T: np.ndarray, A: np.ndarray, chunk: int | None = None) -> np.ndarray:
    """rho[(s1 s2), (s1' s2')] of a horizontal bond, not normalised.

    The boundary ring, clockwise: corner, top edges above site 1 and site 2,
    corner, right edge, corner, bottom edges below site 2 and site 1, corner,
    left edge. Cut at the top bond t (between the two top edges) and the
    bottom bond b (between the two bottom edges): the left chain runs from b
    to t through the bottom edge below site 1, the left half-ring and the top
    edge above site 1; the right chain runs from t to b. Each chain is closed
    with its site's open double layer; the two halves share t, b and the bond
    m between the sites.

    chunk: the sum over the bottom bond b taken in slices of that many values
    (the same sum; it only bounds the memory of the chi^2 D^6 intermediates).
    """
    d = A.shape[0]
    chi = T.shape[0]
    a_open = open_double_layer(A)                        # [s, s', u, l, d, r]
    H = half_ring(C, T)                                  # [a, x, b]
    R1 = np.tensordot(T, H, axes=([2], [0]))             # [t, u2, r2, e]
    rho = 0
    step = chi if chunk is None else chunk
    for b0 in range(0, chi, step):
        bs = slice(b0, min(chi, b0 + step))
        # left chain L[b, d1, l1, u1, t] = T[b, d1, c] H[c, l1, e] T[e, u1, t]
        L1 = np.tensordot(T[bs], H, axes=([2], [0]))     # [b, d1, l1, e]
        L2 = np.tensordot(L1, T, axes=([3], [0]))        # [b, d1, l1, u1, t]
        LB = np.tensordot(L2, a_open, axes=([1, 2, 3], [4, 3, 2]))   # [b, t, s1, s1', m]
        # right chain R[t, u2, r2, d2, b] = T[t, u2, c] H[c, r2, e] T[e, d2, b]
        R2 = np.tensordot(R1, T[:, :, bs], axes=([3], [0]))          # [t, u2, r2, d2, b]
        RB = np.tensordot(R2, a_open, axes=([1, 2, 3], [2, 5, 4]))   # [t, b, s2, s2', m]
        rho = rho + np.tensordot(LB, RB, axes=([0, 1, 4], [1, 0, 4]))  # [s1, s1', s2, s2']
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
    (the upper and lower half-rings joined, their bulk legs contracted).
    Invariant under rescaling C and T.
    """
    eps = one_site_environment(C, T)
    Z1 = np.sum(eps * a)
    Z4 = np.trace(C @ C @ C @ C)
    H = half_ring(C, T)
    Z2 = np.einsum("axb,bxa->", H, H)
    return np.log(complex(Z1 * Z4 / Z2 ** 2))


def correlation_length(T: np.ndarray, a: np.ndarray, k: int = 2) -> float:
    """xi = -1 / ln|l2 / l1| of the column transfer matrix T-a-T.

    E[(alpha, l, beta), (alpha', r, beta')] = sum_{u, d} T[alpha, u, alpha'] a[u, l, d, r] T[beta', d, beta]:
    the top edge runs left to right, the bottom edge right to left (clockwise).
    Pinned by the closed form of decoupled chains (a = M (x) M, xi = -1/ln|mu2/mu1|)
    and by the high-temperature Ising correlation length approached from below.
    """
    chi, q = T.shape[0], T.shape[1]
    n = chi * q * chi
    dt = np.result_type(T, a)

    def mv(v):
        v = v.reshape(chi, q, chi)
        W1 = np.tensordot(T, v, axes=([2], [0]))          # [alpha, u, r, beta']
        W2 = np.tensordot(W1, a, axes=([1, 2], [0, 3]))   # [alpha, beta', l, d]
        W3 = np.tensordot(W2, T, axes=([1, 3], [0, 1]))   # [alpha, l, beta]
        return W3.reshape(n)

    op = LinearOperator((n, n), matvec=mv, dtype=dt)
    vals = eigs(op, k=k, which="LM", return_eigenvectors=False, tol=1e-12)
    mags = np.sort(np.abs(vals))[::-1]
    if mags[1] == 0:
        return 0.0
    r = mags[1] / mags[0]
    return float(np.inf) if r >= 1.0 else float(-1.0 / np.log(r))
