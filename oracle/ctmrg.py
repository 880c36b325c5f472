"""Dense C4v CTMRG in FP64 (Sec. II.A, Fig. 1(d)).

Test infrastructure only (see the package docstring).

One move grows the corner by one row and one column of double-layer tensors
(boundary dimension chi -> chi*D^2) and truncates back to chi with an
eigenvalue decomposition of the enlarged corner (Sec. II.A). With C4v symmetry
all four corners C[chi, chi] and all four edges T[chi, D^2, chi] are equal.

Index conventions (all tensors here are plain dense arrays):
  a[u, l, d, r]          double layer, legs up/left/down/right (double_layer()).
  T[alpha, x, beta]      edge: alpha and beta are the two boundary bonds, x the
                         bond into the bulk. Boundary tensors are oriented
                         clockwise around the lattice: alpha is the incoming
                         end, beta the outgoing one. As the left edge, alpha
                         points down, beta up and x right; as the top edge,
                         alpha is the left end and x points down.
  C[beta, gamma]         corner, incoming leg beta, outgoing leg gamma.
  C'[(alpha,d),(eps,r)]  enlarged upper-left corner: left edge T, corner C, top
                         edge T and the bulk a; rows are the incoming pair
                         (boundary bond alpha, bulk leg d), columns the
                         outgoing pair (eps, r).
For real tensors C4v makes T[alpha, x, beta] = T[beta, x, alpha] and C
symmetric, and the orientation plays no role.

Readings of points the paper leaves open (each is a convention; the
gauge-invariant results do not depend on it):
  * initial environment: traced boundary. The open outer legs of the first
    corner and edge are closed with the bra-ket identity delta(i, ibar), which
    is an even state of S;
  * truncation, real tensors: keep the chi eigenvalues of largest modulus of
    the symmetric C' (ties: lower index in the eigensolver's ascending order);
    P = V_kept, C_new = diag(lambda_kept), T_new = P^T (T a) P. If
    chi*D^2 <= chi all states are kept;
  * truncation, complex tensors: C' is complex symmetric but its eigenvalues
    come in complex-conjugate pairs of equal modulus, so "keep the chi largest"
    is not well defined for them. The move uses the singular value
    decomposition C' = U S V^dagger instead: keep the chi largest singular
    values, insert U_k U_k^dagger on every boundary bond, i.e. renormalise each
    boundary tensor as U_k^dagger (incoming leg) ... U_k (outgoing leg):
    C_new = U_k^dagger C' U_k, T_new = U_k^dagger (T a) U_k. This keeps the
    orientation and reduces to the real rule for real tensors (singular values
    |lambda|, U = V up to signs);
  * normalisation: C and T are divided by their largest modulus after every
    move.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .basis import combined_index


def traced_boundary_vector(D: int) -> np.ndarray:
    """delta(i, ibar) on one combined leg: sum_k |k k'> (an even state of S)."""
    v = np.zeros(D * D)
    for k in range(D):
        v[combined_index(k, k, D)] = 1.0
    return v


def init_environment(a: np.ndarray):
    """C0[d, r] = a[u, l, d, r] v[u] v[l] and T0[alpha=d, x=r, beta=u] = a[u, l, d, r] v[l]."""
    q = a.shape[0]
    D = int(round(np.sqrt(q)))
    v = traced_boundary_vector(D)
    C = np.einsum("uldr,u,l->dr", a, v, v)
    T = np.einsum("uldr,l->dru", a, v)
    return C, T


def enlarged_corner(C: np.ndarray, T: np.ndarray, a: np.ndarray) -> np.ndarray:
    """C'[(alpha,d),(eps,r)] = sum T[alpha,x,beta] C[beta,gamma] T[gamma,y,eps] a[y,x,d,r]."""
    chi, q = T.shape[0], T.shape[1]
    X1 = np.tensordot(T, C, axes=([2], [0]))            # [alpha, x, gamma]
    X2 = np.tensordot(X1, T, axes=([2], [0]))           # [alpha, x, y, eps]
    X3 = np.tensordot(X2, a, axes=([1, 2], [1, 0]))     # [alpha, eps, d, r]
    return X3.transpose(0, 2, 1, 3).reshape(chi * q, chi * q)


@dataclass
class MoveInfo:
    """Per-move record: eigenvalues kept and the relative gap at the cut."""
    kept: np.ndarray
    gap: float
    lam_cut: float
    lam_next: float
    n: int
    log_norm_C: float = 0.0
    log_norm_T: float = 0.0


def truncate(Cp: np.ndarray, chi: int):
    """Projector and kept spectrum of the enlarged corner (Sec. II.A).

    Real: eigh of the symmetric C' (symmetric by C4v; its symmetric part is
    taken explicitly), keep the chi eigenvalues of largest modulus,
    P = V[:, kept]; returns those eigenvalues in descending modulus.
    Complex: SVD C' = U S V^dagger, keep the chi largest singular values,
    P = U[:, :chi]; returns those singular values.
    Returns (P, kept, info).
    """
    n = Cp.shape[0]
    keep = min(chi, n)
    if np.iscomplexobj(Cp):
        U, sv, _ = np.linalg.svd(Cp)
        P = U[:, :keep]
        kept = sv[:keep]
        mags = sv
    else:
        w, V = np.linalg.eigh(0.5 * (Cp + Cp.T))
        order = np.argsort(-np.abs(w), kind="stable")
        lam = w[order]
        P = V[:, order[:keep]]
        kept = lam[:keep]
        mags = np.abs(lam)
    lam_cut = float(mags[keep - 1])
    lam_next = float(mags[keep]) if keep < n else 0.0
    gap = (lam_cut - lam_next) / float(mags[0]) if keep < n else np.inf
    return P, kept, MoveInfo(kept=np.array(kept), gap=gap, lam_cut=lam_cut, lam_next=lam_next, n=n)


def renormalize_edge(T: np.ndarray, a: np.ndarray, P: np.ndarray) -> np.ndarray:
    """T_new[a', r, b'] = sum conj(P[(alpha,d),a']) T[alpha,x,beta] a[u,x,d,r] P[(beta,u),b'].

    In the left-edge frame (alpha, d) is the incoming pair and (beta, u) the
    outgoing one. Contracted as Y = P^dagger T (over alpha), Z = Y a (over d
    and x), T_new = Z P (over beta and u). For real P this is P^T (T a) P.
    """
    chi, q = T.shape[0], T.shape[1]
    P3 = P.reshape(chi, q, P.shape[1])                   # [alpha, d, a']
    Y = np.tensordot(P3.conj(), T, axes=([0], [0]))      # [d, a', x, beta]
    Z = np.tensordot(Y, a, axes=([0, 2], [2, 1]))        # [a', beta, u, r]
    Tn = np.tensordot(Z, P3, axes=([1, 2], [0, 1]))      # [a', r, b']
    return Tn


def move(C: np.ndarray, T: np.ndarray, a: np.ndarray, chi: int):
    """One C4v CTMRG move: enlarge, truncate, renormalise, normalise."""
    Cp = enlarged_corner(C, T, a)
    P, lam, info = truncate(Cp, chi)
    if np.iscomplexobj(Cp):
        Cn = P.conj().T @ Cp @ P
    else:
        Cn = np.diag(lam)
    Tn = renormalize_edge(T, a, P)
    nC = np.abs(Cn).max()
    nT = np.abs(Tn).max()
    info.log_norm_C = float(np.log(nC))
    info.log_norm_T = float(np.log(nT))
    if not np.iscomplexobj(a):
        Cn, Tn = Cn.real, Tn.real
    return Cn / nC, Tn / nT, info


@dataclass
class CTMRGResult:
    C: np.ndarray
    T: np.ndarray
    infos: list = field(default_factory=list)

    @property
    def min_gap(self) -> float:
        g = [i.gap for i in self.infos if np.isfinite(i.gap)]
        return min(g) if g else np.inf


def run(a: np.ndarray, chi: int, moves: int) -> CTMRGResult:
    """Traced-boundary initialisation followed by `moves` CTMRG moves."""
    C, T = init_environment(a)
    nC, nT = np.abs(C).max(), np.abs(T).max()
    C, T = C / nC, T / nT
    res = CTMRGResult(C, T)
    for _ in range(moves):
        C, T, info = move(C, T, a, chi)
        res.infos.append(info)
    res.C, res.T = C, T
    return res
