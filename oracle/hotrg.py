"""Dense HOTRG (Sec. II.A, Ref. xie12) and its Hermitian-symmetry probe (Sec. III.A).

Test infrastructure only (see the package docstring).

A coarse-graining step stacks two tensors T[u, l, d, r] vertically,
M[u, (l1 l2), d, (r1 r2)] = sum_k T[u, l1, k, r1] T[k, l2, d, r2], and truncates
each fused horizontal leg to chi with the eigenvectors of the Gram matrix of
the fused left leg, G = M M^dagger (Sec. II.A: truncation to the chi most
relevant states from an eigenvalue decomposition). The right Gram matrix is
also formed and the side with the smaller discarded weight supplies the
isometry (Ref. xie12); ties go to the left. Steps alternate between the
vertical and the horizontal direction; a horizontal step is a vertical step on
the tensor rotated by 90 degrees.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rotate(T: np.ndarray) -> np.ndarray:
    """R[u, l, d, r] = T[l, d, r, u]: the tensor turned by 90 degrees."""
    return np.transpose(T, (3, 0, 1, 2))


def unrotate(T: np.ndarray) -> np.ndarray:
    """Inverse of rotate."""
    return np.transpose(T, (1, 2, 3, 0))


def stack_vertical(Ttop: np.ndarray, Tbot: np.ndarray) -> np.ndarray:
    """M[u, l1, l2, d, r1, r2] = sum_k Ttop[u, l1, k, r1] Tbot[k, l2, d, r2]."""
    M = np.tensordot(Ttop, Tbot, axes=([2], [0]))        # [u, l1, r1, l2, d, r2]
    return M.transpose(0, 1, 3, 4, 2, 5)


def isometry(M: np.ndarray, chi: int):
    """Top-chi eigenvectors of the left or right Gram matrix of M (whichever discards less).

    Returns (V, w, side): the kept eigenvectors as columns, the Gram matrix's
    eigenvalues in descending order, and side = 0 (left) or 1 (right).
    """
    u, l1, l2, d, r1, r2 = M.shape
    ML = M.transpose(1, 2, 0, 3, 4, 5).reshape(l1 * l2, -1)
    MR = M.transpose(4, 5, 0, 1, 2, 3).reshape(r1 * r2, -1)
    out = []
    for Mx in (ML, MR):
        G = Mx @ Mx.conj().T
        w, V = np.linalg.eigh(0.5 * (G + G.conj().T))
        order = np.argsort(-w, kind="stable")
        keep = min(chi, len(w))
        out.append((float(np.sum(w[order[keep:]])), V[:, order[:keep]], w[order]))
    (eL, VL, wL), (eR, VR, wR) = out
    return (VL, wL, 0) if eL <= eR else (VR, wR, 1)


def contract_step(M: np.ndarray, V: np.ndarray) -> np.ndarray:
    """T_new[u, L, d, R] = sum conj(V[(l1 l2), L]) M[u, (l1 l2), d, (r1 r2)] V[(r1 r2), R]."""
    u, l1, l2, d, r1, r2 = M.shape
    Mm = M.reshape(u, l1 * l2, d, r1 * r2)
    X = np.tensordot(np.conj(V), Mm, axes=([0], [1]))    # [L, u, d, (r1 r2)]
    Tn = np.tensordot(X, V, axes=([3], [0]))             # [L, u, d, R]
    return Tn.transpose(1, 0, 2, 3)


@dataclass
class HOTRGResult:
    T: np.ndarray
    log_norms: list = field(default_factory=list)
    impurity: np.ndarray | None = None
    impurity_abs: np.ndarray | None = None
    spectra: list = field(default_factory=list)
    sides: list = field(default_factory=list)


def run(a: np.ndarray, chi: int, steps: int, impurity=None, impurity_abs=None) -> HOTRGResult:
    """HOTRG from the double layer a; optionally carries impurity tensors along.

    Each step: vertical stacking on even steps, horizontal on odd steps. The
    pure tensor is divided by its largest modulus c_k after every step
    (log c_k recorded; c_0 normalises a itself). An impurity replaces the
    upper tensor of its pair and is renormalised with the same isometry and
    the same c_k, so ratios of impurity traces are unaffected by the scaling.
    """
    T = a / np.abs(a).max()
    res = HOTRGResult(T, [float(np.log(np.abs(a).max()))])
    imps = [x / np.abs(a).max() if x is not None else None for x in (impurity, impurity_abs)]
    for k in range(steps):
        horizontal = k % 2 == 1
        Tw = rotate(T) if horizontal else T
        impw = [rotate(x) if (x is not None and horizontal) else x for x in imps]
        M = stack_vertical(Tw, Tw)
        V, w, side = isometry(M, chi)
        res.spectra.append(w)
        res.sides.append(side)
        Tn = contract_step(M, V)
        c = np.abs(Tn).max()
        Tn = Tn / c
        new_imps = []
        for x in impw:
            if x is None:
                new_imps.append(None)
                continue
            xn = contract_step(stack_vertical(x, Tw), V) / c
            new_imps.append(xn)
        T = unrotate(Tn) if horizontal else Tn
        imps = [unrotate(x) if (x is not None and horizontal) else x for x in new_imps]
        res.log_norms.append(float(np.log(c)))
    res.T = T
    res.impurity, res.impurity_abs = imps
    return res


def trace(T: np.ndarray):
    """Periodic trace sum_{u, l} T[u, l, u, l]."""
    return np.einsum("ulul->", T)


def log_z_per_site(res: HOTRGResult) -> float:
    """ln Z / N after the recorded steps: ln c_0 + sum_k ln(c_k) / 2^k + ln Tr(T_n) / 2^n."""
    n = len(res.log_norms) - 1
    val = res.log_norms[0]
    for k in range(1, n + 1):
        val += res.log_norms[k] / 2.0 ** k
    val += np.log(np.real(trace(res.T))) / 2.0 ** n
    return float(val)


def b_tensor(D: int, absolute: bool = False) -> np.ndarray:
    """The probe b of Sec. III.A as a double-layer tensor of shape (D^2,)*4.

    As a D^4 x D^4 matrix from the ket indices (u, l, d, r) to the bra indices
    it has +1 above the diagonal, -1 below and 0 on it; absolute=True gives
    |b| (1 everywhere off the diagonal).
    """
    n = D ** 4
    I, J = np.indices((n, n))
    B = np.where(I < J, 1.0, np.where(I > J, (1.0 if absolute else -1.0), 0.0))
    b8 = B.reshape((D,) * 8)                             # [u, l, d, r, U, L, Dd, R]
    # combined index ket + D*bra: axis order (bra, ket) per leg
    b8 = b8.transpose(4, 0, 5, 1, 6, 2, 7, 3)
    return np.ascontiguousarray(b8.reshape(D * D, D * D, D * D, D * D))


def symmetry_error(a: np.ndarray, D: int, chi: int, steps: int) -> float:
    """|<b>| / <|b|>: HOTRG network with one a replaced by b, over the same with |b| (Sec. III.A)."""
    res = run(a, chi, steps, impurity=b_tensor(D), impurity_abs=b_tensor(D, absolute=True))
    return float(abs(trace(res.impurity)) / abs(trace(res.impurity_abs)))
