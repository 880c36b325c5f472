"""Directional CTMRG without lattice symmetry, in FP64 (Sec. II.A).

Test infrastructure only (see the package docstring).

The paper runs CTMRG with C4v symmetry "for simplicity" (Sec. II.A): one
corner and one edge. Without that symmetry the environment of a one-site unit
cell has four distinct corners and four distinct edges, and every directional
move grows one side of the boundary by a column of double-layer tensors and
truncates it back with a pair of oblique projectors. The projectors come from
the singular value decomposition of the product of the two enlarged corners
(quarters) on the side being moved, cut along the bonds being truncated.

The environment is a list, clockwise from the upper-left corner:

    E = [C1, T1, C2, T2, C3, T3, C4, T4]        C1 T1 C2
                                                T4 a  T2
                                                C4 T3 C3

Every tensor is oriented clockwise as in ctmrg.py: a corner is C[in, out], an
edge T[in, x, out] with x its bulk leg. Written out:
  C1[left bond, top bond]      T1[top, x = up leg of a, top]
  C2[top, right]               T2[right, x = right leg of a, right]
  C3[right, bottom]            T3[bottom, x = down leg of a, bottom]
  C4[bottom, left]             T4[left, x = left leg of a, left]
so T1[alpha, x, beta] runs left to right, T2 top to bottom, T3 right to left
and T4 bottom to top.

Turning the lattice by 90 degrees counter-clockwise moves the top side to the
left: the environment becomes E[2:] + E[:2] and the double layer
a_rot[u, l, d, r] = a[l, d, r, u] (rotate()). Every directional move is
therefore written once, as a move of the left side (left_move()); a sweep is a
left move in each of the four frames reached by successive rotations, i.e. the
left, top, right and bottom sides in that order.

Readings of points the paper leaves open (the C4v scheme of ctmrg.py is the
special case; the gauge-invariant results do not depend on these):
  * initial environment: traced boundary, as in ctmrg.py, on every side;
  * projectors: the upper-left quarter Q1[i, j] and the lower-left quarter
    Q4[j', i] of the frame (quarter()) meet at the left-side cut i.
    X = Q1^T Q4^T = U S V^T; keep the chi largest singular values (and only
    those above 1e-12 s_max); P_a = Q4^T V S^-1/2 goes on the upper side of
    every left-side bond and P_b = Q1 U S^-1/2 on the lower side, so
    P_a P_b^T is the oblique projector that turns Q1^T (.) Q4^T into the best
    rank-chi approximation of X. (The product of the upper and lower halves,
    Q1 Q2 and Q4^T Q3^T, would use the whole ring, but its singular values
    are those of the quarters squared: at chi = 13 of D = 2 they already span
    twelve decades, and S^-1/2 then amplifies rounding beyond use in FP64);
  * normalisation: each updated tensor is divided by its largest modulus.
Real tensors only.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .ctmrg import traced_boundary_vector
from .doublelayer import open_double_layer

SV_CUTOFF = 1e-12  # singular values below this fraction of the largest are never kept


def rotate(E: list, a: np.ndarray):
    """The frame turned by 90 degrees counter-clockwise: the top side becomes the left side."""
    return E[2:] + E[:2], np.ascontiguousarray(a.transpose(3, 0, 1, 2))


def frames(E: list, a: np.ndarray) -> list:
    """The four frames [(E, a), rotate(E, a), rotate^2, rotate^3]."""
    out = [(list(E), a)]
    for _ in range(3):
        out.append(rotate(*out[-1]))
    return out


def init_environment(a: np.ndarray) -> list:
    """Traced boundary on every side: each corner is one double layer with its two outer legs
    closed by delta(i, ibar), each edge one double layer with its outer leg closed."""
    q = a.shape[0]
    v = traced_boundary_vector(int(round(np.sqrt(q))))
    C1 = np.einsum("uldr,u,l->dr", a, v, v)      # [in = down leg, out = right leg]
    T1 = np.einsum("uldr,u->ldr", a, v)          # [left, x = down, right]
    C2 = np.einsum("uldr,u,r->ld", a, v, v)      # [in = left leg, out = down leg]
    T2 = np.einsum("uldr,r->uld", a, v)          # [top, x = left, bottom]
    C3 = np.einsum("uldr,d,r->ul", a, v, v)      # [in = up leg, out = left leg]
    T3 = np.einsum("uldr,d->rul", a, v)          # [right, x = up, left]
    C4 = np.einsum("uldr,d,l->ru", a, v, v)      # [in = right leg, out = up leg]
    T4 = np.einsum("uldr,l->dru", a, v)          # [bottom, x = right, top]
    return [t / np.abs(t).max() for t in (C1, T1, C2, T2, C3, T3, C4, T4)]


def quarter(E: list, a: np.ndarray) -> np.ndarray:
    """Upper-left quarter of the frame as a matrix:
    Q[(alpha, d), (beta, r)] = sum T4[alpha, x, b] C1[b, g] T1[g, y, beta] a[y, x, d, r].

    Rows: the left-side bond below the quarter (alpha) and the down leg of a;
    columns: the top-side bond right of it (beta) and the right leg of a.
    """
    C1, T1, T4 = E[0], E[1], E[7]
    chiL, q, chiT = T4.shape[0], a.shape[0], T1.shape[2]
    X1 = np.tensordot(T4, C1, axes=([2], [0]))           # [alpha, x, g]
    X2 = np.tensordot(X1, T1, axes=([2], [0]))           # [alpha, x, y, beta]
    X3 = np.tensordot(X2, a, axes=([1, 2], [1, 0]))      # [alpha, beta, d, r]
    return X3.transpose(0, 2, 1, 3).reshape(chiL * q, chiT * q)


@dataclass
class MoveInfo:
    """Per directional move: kept singular values / s_max and the relative gap at the cut."""
    kept: np.ndarray
    gap: float
    s_max: float
    n: int
    log_norms: tuple = ()


def left_quarters(E: list, a: np.ndarray):
    """(Q1, Q4): the upper-left quarter of the frame, Q1[(left bond below, d), (top bond, r)],
    and the lower-left one, the upper-left quarter of the frame turned three times,
    Q4[(bottom bond, r), (left bond above, u)]. They meet at the left-side cut."""
    fr = frames(E, a)
    return quarter(*fr[0]), quarter(*fr[3])


def projectors(E: list, a: np.ndarray, chi: int):
    """Oblique projectors (P_a, P_b) of the left-side bonds, each [(bond, bulk leg), kept]."""
    Q1, Q4 = left_quarters(E, a)
    X = Q1.T @ Q4.T
    U, s, Vt = np.linalg.svd(X, full_matrices=False)
    keep = min(chi, int(np.count_nonzero(s > SV_CUTOFF * s[0])))
    r = 1.0 / np.sqrt(s[:keep])
    Pa = (Q4.T @ Vt[:keep].T) * r
    Pb = (Q1 @ U[:, :keep]) * r
    nxt = float(s[keep]) if keep < len(s) else 0.0
    gap = (float(s[keep - 1]) - nxt) / float(s[0]) if keep < len(s) else np.inf
    return Pa, Pb, MoveInfo(kept=s[:keep] / s[0], gap=gap, s_max=float(s[0]), n=len(s))


def left_move(E: list, a: np.ndarray, chi: int):
    """Absorb one column into the left side of the frame and truncate the left bonds to chi.

      C1 <- P_a^T (C1 T1),   T4 <- P_a^T (T4 a) P_b,   C4 <- (T3 C4) P_b,

    with P_a on the upper side of each left-side bond and P_b on its lower side.
    """
    C1, T1, C2, T2, C3, T3, C4, T4 = E
    Pa, Pb, info = projectors(E, a, chi)
    chiL, q = T4.shape[0], a.shape[0]
    Pa3 = Pa.reshape(chiL, q, -1)
    Pb3 = Pb.reshape(chiL, q, -1)
    # C1n[c, e] = Pa[(b, x), c] C1[b, g] T1[g, x, e]
    C1n = np.tensordot(Pa3, np.tensordot(C1, T1, axes=([1], [0])), axes=([0, 1], [0, 1]))
    # T4n[c, r, k] = Pa[(alpha, d), c] T4[alpha, x, beta] a[u, x, d, r] Pb[(beta, u), k]
    Y1 = np.tensordot(Pa3, T4, axes=([0], [0]))            # [d, c, x, beta]
    Y2 = np.tensordot(Y1, a, axes=([0, 2], [2, 1]))        # [c, beta, u, r]
    T4n = np.tensordot(Y2, Pb3, axes=([1, 2], [0, 1]))     # [c, r, k]
    # C4n[alpha, k] = T3[alpha, x, b] C4[b, g] Pb[(g, x), k]
    C4n = np.tensordot(np.tensordot(T3, C4, axes=([2], [0])), Pb3, axes=([2, 1], [0, 1]))
    nC1, nT4, nC4 = (float(np.abs(t).max()) for t in (C1n, T4n, C4n))
    info.log_norms = (np.log(nC1), np.log(nT4), np.log(nC4))
    return [C1n / nC1, T1, C2, T2, C3, T3, C4n / nC4, T4n / nT4], info


def sweep(E: list, a: np.ndarray, chi: int):
    """Left, top, right and bottom moves, each as a left move of its frame."""
    infos = []
    for _ in range(4):
        E, info = left_move(E, a, chi)
        infos.append(info)
        E, a = rotate(E, a)
    return E, infos


@dataclass
class Result:
    E: list
    infos: list = field(default_factory=list)

    @property
    def min_gap(self) -> float:
        g = [i.gap for i in self.infos if np.isfinite(i.gap)]
        return min(g) if g else np.inf


def run(a: np.ndarray, chi: int, sweeps: int) -> Result:
    """Traced-boundary initialisation followed by `sweeps` sweeps of four directional moves."""
    E = init_environment(a)
    res = Result(E)
    for _ in range(sweeps):
        E, infos = sweep(E, a, chi)
        res.infos.extend(infos)
    res.E = E
    return res


# ---- observables of the four-corner environment (Sec. III.A) -------------------------------

def one_site_environment(E: list) -> np.ndarray:
    """eps[u, l, d, r]: the boundary ring around one site, Fig. 1(d) with the centre removed."""
    C1, T1, C2, T2, C3, T3, C4, T4 = E
    top = np.tensordot(np.tensordot(C1, T1, axes=([1], [0])), C2, axes=([2], [0]))   # [a, u, e]
    top = np.tensordot(top, T2, axes=([2], [0]))                                    # [a, u, r, f]
    bot = np.tensordot(np.tensordot(C3, T3, axes=([1], [0])), C4, axes=([2], [0]))   # [f, d, i]
    ring = np.tensordot(top, bot, axes=([3], [0]))                                  # [a, u, r, d, i]
    eps = np.tensordot(ring, T4, axes=([4, 0], [0, 2]))                             # [u, r, d, l]
    return np.ascontiguousarray(eps.transpose(0, 3, 2, 1))


def one_site_rdm(E: list, A: np.ndarray) -> np.ndarray:
    """rho1[s, s'], not normalised: eps closed with A_s (x) conj(A_s')."""
    return np.einsum("stuldr,uldr->st", open_double_layer(A), one_site_environment(E), optimize=True)


def two_site_rdm_horizontal(E: list, A: np.ndarray) -> np.ndarray:
    """rho[(s1 s2), (s1' s2')] of a horizontal bond (site 1 left of site 2), not normalised.

        C1 T1 T1 C2
        T4 *1 *2 T2
        C4 T3 T3 C3
    """
    C1, T1, C2, T2, C3, T3, C4, T4 = E
    d = A.shape[0]
    ao = open_double_layer(A)                            # [s, s', u, l, d, r]
    # left half L[b, t, s1, s1', m] and right half R[t, b, s2, s2', m]: t the top bond between
    # the two T1, b the bottom bond between the two T3, m the bond between the sites
    top = np.tensordot(C1, T1, axes=([1], [0]))          # [a, u1, t]
    lft = np.tensordot(C4, T4, axes=([1], [0]))          # [h, l1, a]
    bot = np.tensordot(T3, lft, axes=([2], [0]))         # [b, d1, l1, a]
    L1 = np.tensordot(bot, top, axes=([3], [0]))         # [b, d1, l1, u1, t]
    L = np.tensordot(L1, ao, axes=([1, 2, 3], [4, 3, 2]))  # [b, t, s1, s1', m]
    rtop = np.tensordot(T1, C2, axes=([2], [0]))         # [t, u2, g]
    rgt = np.tensordot(T2, C3, axes=([2], [0]))          # [g, r2, f]
    rbot = np.tensordot(rgt, T3, axes=([2], [0]))        # [g, r2, d2, b]
    R1 = np.tensordot(rtop, rbot, axes=([2], [0]))       # [t, u2, r2, d2, b]
    R = np.tensordot(R1, ao, axes=([1, 2, 3], [2, 5, 4]))  # [t, b, s2, s2', m]
    rho = np.tensordot(L, R, axes=([0, 1, 4], [1, 0, 4]))  # [s1, s1', s2, s2']
    return rho.transpose(0, 2, 1, 3).reshape(d * d, d * d)


def rotate_site(A: np.ndarray) -> np.ndarray:
    """A[p, u, l, d, r] in the frame turned counter-clockwise (as rotate() turns a)."""
    return np.ascontiguousarray(A.transpose(0, 4, 1, 2, 3))


def two_site_rdm_vertical(E: list, A: np.ndarray) -> np.ndarray:
    """rho of a vertical bond, [(s_upper s_lower), (s_upper' s_lower')]: the horizontal RDM of
    the frame turned counter-clockwise, in which the upper site is the left one."""
    E1, _ = rotate(E, np.zeros((1, 1, 1, 1)))
    return two_site_rdm_horizontal(E1, rotate_site(A))


def log_kappa(E: list, a: np.ndarray) -> float:
    """ln kappa = ln(Z11 Z00 / (Z10 Z01)): the free energy per site, -beta f, of the norm network.

    Z11: the ring around a; Z00: the four corners alone (Tr C1 C2 C3 C4); Z10: the ring with
    the top and bottom edges joined through their bulk legs and no side edges; Z01 the same
    with the side edges. Invariant under rescaling any corner or edge.
    """
    C1, T1, C2, T2, C3, T3, C4, T4 = E
    Z11 = np.sum(one_site_environment(E) * a)
    Z00 = np.trace(C1 @ C2 @ C3 @ C4)
    Z10 = np.einsum("ab,bxc,ce,ef,fxg,ga->", C1, T1, C2, C3, T3, C4, optimize=True)
    Z01 = np.einsum("ab,bc,cxe,ef,fg,gxa->", C1, C2, T2, C3, C4, T4, optimize=True)
    return float(np.log(Z11 * Z00 / (Z10 * Z01)))
