"""Independent references used to pin the oracle (test helpers, no oracle imports).

* Onsager's exact solution of the square-lattice Ising model.
* Brute-force row-by-row contraction of finite patches of double-layer
  tensors with a traced outer boundary.
"""
from __future__ import annotations

import numpy as np
from scipy.special import ellipk


def onsager_log_z(beta: float, n: int = 512) -> float:
    """-beta f per site: ln 2 + (1/8pi^2) int int ln[cosh^2 2b - sinh 2b (cos t1 + cos t2)].

    The integrand is smooth and periodic away from the critical point, so the
    midpoint rule on an n x n grid converges exponentially.
    """
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    t1, t2 = np.meshgrid(th, th)
    integrand = np.log(np.cosh(2 * beta) ** 2 - np.sinh(2 * beta) * (np.cos(t1) + np.cos(t2)))
    return float(np.log(2.0) + 0.5 * np.mean(integrand))


def onsager_nn(beta: float) -> float:
    """<s_i s_j> on a nearest-neighbour bond: -u/2 with Onsager's internal energy u."""
    k = 2 * np.sinh(2 * beta) / np.cosh(2 * beta) ** 2
    u = -(1 / np.tanh(2 * beta)) * (1 + 2 / np.pi * (2 * np.tanh(2 * beta) ** 2 - 1) * ellipk(k * k))
    return float(-u / 2)


def _onsager_grid(K1: float, K2: float, n: int):
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    c1, s1, c2, s2 = np.cosh(2 * K1), np.sinh(2 * K1), np.cosh(2 * K2), np.sinh(2 * K2)
    den = c1 * c2 - s1 * np.cos(t1) - s2 * np.cos(t2)
    return t1, t2, c1, s1, c2, s2, den


def onsager_log_z_aniso(K1: float, K2: float, n: int = 512) -> float:
    """-beta f per site with couplings K1 on one bond direction and K2 on the other:
    ln 2 + (1/8pi^2) int int ln[cosh 2K1 cosh 2K2 - sinh 2K1 cos t1 - sinh 2K2 cos t2]."""
    *_, den = _onsager_grid(K1, K2, n)
    return float(np.log(2.0) + 0.5 * np.mean(np.log(den)))


def onsager_nn_aniso(K1: float, K2: float, n: int = 512) -> float:
    """<s_i s_j> on a bond of coupling K1: d(-beta f)/dK1 (one such bond per site), the
    derivative of the integrand taken in closed form."""
    t1, _, c1, s1, c2, _, den = _onsager_grid(K1, K2, n)
    return float(0.5 * np.mean((2 * s1 * c2 - 2 * c1 * np.cos(t1)) / den))


def _traced(D: int) -> np.ndarray:
    v = np.zeros(D * D)
    for k in range(D):
        v[k + D * k] = 1.0
    return v


def contract_patch(site_tensor, rows: int, cols: int, D: int):
    """Contract a rows x cols patch with every outer leg closed by delta(i, ibar).

    site_tensor(r, c) returns either a 4-leg tensor t[u, l, d, r] (fully
    contracted into the patch) or a tuple ('open', t) with t[*extra, u, l, d, r]:
    its extra leading legs stay open in the result, in the order the sites are
    visited (row by row, left to right). Returns an array of all open legs.

    The state is psi[x_0, .., x_{cols-1}, h, *open]: the vertical bonds below
    the processed part, the running horizontal bond h, then the open legs.
    """
    v = _traced(D)
    q = D * D
    psi = v
    for _ in range(cols - 1):
        psi = np.multiply.outer(psi, v)
    psi = psi.reshape((q,) * cols)
    n_open = 0
    for r in range(rows):
        psi = np.tensordot(psi, v, axes=0)               # h from the left boundary, at axis cols
        psi = np.moveaxis(psi, psi.ndim - 1, cols)
        for c in range(cols):
            st = site_tensor(r, c)
            if isinstance(st, tuple):
                t = st[1]
                n_extra = t.ndim - 4
            else:
                t = st
                n_extra = 0
            # contract x_c (axis c) with u and h (axis cols) with l
            psi = np.tensordot(psi, t, axes=([c, cols], [n_extra + 0, n_extra + 1]))
            # psi axes: [x_0..x_{c-1}, x_{c+1}..x_{cols-1}, open(n_open), extra, d, r]
            nd = psi.ndim
            d_ax, r_ax = nd - 2, nd - 1
            # move d back to position c and r to position cols
            psi = np.moveaxis(psi, d_ax, c)
            psi = np.moveaxis(psi, psi.ndim - 1, cols)
            # extra legs sit just after the old open legs: already in order
            n_open += n_extra
        psi = np.tensordot(psi, v, axes=([cols], [0]))   # close h on the right
    for c in range(cols):
        psi = np.tensordot(v, psi, axes=([0], [0]))      # close bottom legs
    return psi


def contract_quadrant(a: np.ndarray, m: int, D: int) -> np.ndarray:
    """Q[(x_0..x_{m-1}), (y_0..y_{m-1})]: an m x m patch of double-layer tensors
    a[u, l, d, r] whose top and left outer legs are closed with delta(i, ibar)
    and whose bottom legs x_j and right legs y_i stay open (the upper-left
    corner of the lattice as a matrix between its two cuts).

    Built on contract_patch: a site on the bottom row (right column) gets its
    d (r) leg re-routed into an open leg and its boundary leg fed the dual of
    the traced vector, w = delta / D, so that closing it there contributes 1.
    """
    q = D * D
    w = _traced(D) / D

    def site(i, j):
        bottom, right = i == m - 1, j == m - 1
        if bottom and right:
            return ("open", np.einsum("ulxy,d,r->xyuldr", a, w, w))
        if bottom:
            return ("open", np.einsum("ulxr,d->xuldr", a, w))
        if right:
            return ("open", np.einsum("uldy,r->yuldr", a, w))
        return a

    out = contract_patch(site, m, m, D)
    # open legs in visiting order: y_0 .. y_{m-2}, x_0 .. x_{m-2}, x_{m-1}, y_{m-1}
    ys = list(range(m - 1)) + [2 * m - 1]
    xs = list(range(m - 1, 2 * m - 1))
    return out.transpose(xs + ys).reshape(q ** m, q ** m)
