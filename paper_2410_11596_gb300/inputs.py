"""Seeded synthetic inputs shared by the GPU path, the tests and the benchmark.

This module holds no step of the contraction method itself. It only draws and
prepares input tensors:

* random iPEPS tensors A[p, u, l, d, r] (one physical leg p of dimension d and
  four auxiliary legs up/left/down/right of dimension D, as in the ansatz of
  Sec. II.A, Fig. 1(a)), averaged over the eight point-group images of the
  square lattice because the CTMRG of Sec. II.A assumes a C4v-symmetric state;
* closed-form test states (a product state and the iPEPS whose norm is the
  classical 2D Ising partition function);
* the two-site Heisenberg coupling h = S.S used as the bond observable of
  Sec. III.

All arrays are numpy float64 / complex128, C-contiguous.
"""
from __future__ import annotations

import numpy as np

#: Seed base: workload k draws from ``numpy.random.default_rng(SEED_BASE + k)``.
SEED_BASE = 1159600

#: The eight permutations of the auxiliary legs (u, l, d, r) that form the
#: point group of the square lattice: four rotations, then the four mirrors
#: (left-right, up-down, main diagonal, anti-diagonal).
D4_LEG_PERMUTATIONS = (
    (0, 1, 2, 3), (1, 2, 3, 0), (2, 3, 0, 1), (3, 0, 1, 2),
    (0, 3, 2, 1), (2, 1, 0, 3), (1, 0, 3, 2), (3, 2, 1, 0),
)


def d4_symmetrize(A: np.ndarray) -> np.ndarray:
    """Average A[p, u, l, d, r] over the eight leg permutations of D4."""
    acc = np.zeros_like(A)
    for g in D4_LEG_PERMUTATIONS:
        acc += np.transpose(A, (0, 1 + g[0], 1 + g[1], 1 + g[2], 1 + g[3]))
    return acc / len(D4_LEG_PERMUTATIONS)


def random_ipeps(d: int, D: int, seed: int, complex_valued: bool = False) -> np.ndarray:
    """Seeded random C4v iPEPS tensor of shape (d, D, D, D, D), scaled to max|A| = 1.

    Real entries are N(0, 1). Complex entries have real and imaginary parts
    each N(0, 1/2), drawn as two full arrays (real first) from one generator.
    """
    rng = np.random.default_rng(seed)
    shape = (d, D, D, D, D)
    if complex_valued:
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        A = (re + 1j * im) * np.sqrt(0.5)
    else:
        A = rng.standard_normal(shape)
    A = d4_symmetrize(A)
    return np.ascontiguousarray(A / np.abs(A).max())


def lopsided_ipeps(D: int = 3, seed: int = 21, eps: float = 0.3) -> np.ndarray:
    """A tensor that is NOT mirror symmetric: A[p,u,l,d,r] = X[p,u,l,d] y[r] + eps N(0,1),
    so its right leg is close to rank one. X, y and the noise are N(0,1) from
    ``default_rng(seed)`` (X, then y, then the noise); scaled to max|A| = 1.
    Used to exercise the left/right choice of the HOTRG truncation."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((2, D, D, D))
    y = rng.standard_normal(D)
    A = np.einsum("puld,r->puldr", X, y) + eps * rng.standard_normal((2, D, D, D, D))
    return np.ascontiguousarray(A / np.abs(A).max())


def product_state_ipeps(phi: np.ndarray, D: int = 1) -> np.ndarray:
    """Product state |phi>^N embedded at bond dimension D: A[p, 0, 0, 0, 0] = phi[p]."""
    phi = np.asarray(phi)
    A = np.zeros((phi.shape[0], D, D, D, D), dtype=phi.dtype)
    A[:, 0, 0, 0, 0] = phi
    return A


def ising_ipeps(beta: float) -> np.ndarray:
    """Real iPEPS (d = D = 2) whose norm network is the 2D Ising partition function.

    A[p, u, l, d, r] = M[p, u] M[p, l] M[p, d] M[p, r] with M the symmetric
    square root of G = [[e^{b/2}, e^{-b/2}], [e^{-b/2}, e^{b/2}]]. Each bond of
    the double layer then carries G[p, p']^2 = exp(beta * s s'), s = +-1.
    """
    g = np.array([[np.exp(beta / 2), np.exp(-beta / 2)],
                  [np.exp(-beta / 2), np.exp(beta / 2)]])
    w, v = np.linalg.eigh(g)
    M = (v * np.sqrt(w)) @ v.T
    return np.einsum("pu,pl,pd,pr->puldr", M, M, M, M)


def anisotropic_ising_ipeps(beta_x: float, beta_y: float) -> np.ndarray:
    """As ising_ipeps, with coupling beta_x on the horizontal legs (l, r) and beta_y on the
    vertical legs (u, d): the norm network is the anisotropic 2D Ising partition function."""
    def root(beta):
        g = np.array([[np.exp(beta / 2), np.exp(-beta / 2)],
                      [np.exp(-beta / 2), np.exp(beta / 2)]])
        w, v = np.linalg.eigh(g)
        return (v * np.sqrt(w)) @ v.T
    Mx, My = root(beta_x), root(beta_y)
    return np.einsum("pu,pl,pd,pr->puldr", My, Mx, My, Mx)


def asymmetric_ipeps(d: int, D: int, seed: int) -> np.ndarray:
    """Seeded random real iPEPS tensor with no lattice symmetry: N(0, 1) entries from
    ``default_rng(seed)`` (not averaged over D4), scaled to max|A| = 1. Input of the
    directional CTMRG, which assumes no C4v symmetry."""
    A = np.random.default_rng(seed).standard_normal((d, D, D, D, D))
    return np.ascontiguousarray(A / np.abs(A).max())


def heisenberg_bond() -> np.ndarray:
    """Two-site h = S^x S^x + S^y S^y + S^z S^z (S = sigma/2, J = 1) as a real 4x4.

    Index order: h[(s1 s2), (s1' s2')] with s2 fastest. S^y (x) S^y is real.
    """
    sx = np.array([[0.0, 0.5], [0.5, 0.0]])
    sy_sy = np.kron(np.array([[0.0, -0.5j], [0.5j, 0.0]]), np.array([[0.0, -0.5j], [0.5j, 0.0]]))
    sz = np.array([[0.5, 0.0], [0.0, -0.5]])
    h = np.kron(sx, sx) + sy_sy.real + np.kron(sz, sz)
    assert np.abs(sy_sy.imag).max() == 0.0
    return np.ascontiguousarray(h)


def sz_sz_bond() -> np.ndarray:
    """Two-site sigma^z sigma^z (Pauli, not spin-1/2) as a real 4x4."""
    sz = np.diag([1.0, -1.0])
    return np.kron(sz, sz)


#: The benchmark workloads: (d, D, chi, moves, complex_valued).
WORKLOADS = {
    1: dict(d=2, D=2, chi=16, moves=30, complex_valued=False),
    2: dict(d=2, D=4, chi=64, moves=50, complex_valued=False),
    3: dict(d=2, D=6, chi=144, moves=50, complex_valued=False),
    5: dict(d=2, D=5, chi=100, moves=40, complex_valued=True),
    # small complex case for parity tests (the oracle finishes it in seconds)
    6: dict(d=2, D=3, chi=27, moves=30, complex_valued=True),
    # the largest shape of the batched workload (D=7: q=49 = 28 even + 21 odd,
    # chi = 4 D^2 = 196): its first D=7 instance (instance 1, seed SEED_BASE + 4001)
    7: dict(d=2, D=7, chi=196, moves=40, complex_valued=False, seed=SEED_BASE + 4001),
}


def batched_workload(n: int = 32, seed: int | None = None) -> list[tuple[int, int, np.ndarray]]:
    """n independent real iPEPS instances: D uniform in {3, ..., 7} from
    rng(SEED_BASE + 4), chi = 4 D^2, instance i seeded SEED_BASE + 4000 + i.
    Returns (D, chi, A) per instance."""
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    Ds = rng.integers(3, 8, size=n)
    return [(int(D), 4 * int(D) * int(D), random_ipeps(2, int(D), SEED_BASE + 4000 + i)) for i, D in enumerate(Ds)]


def workload_tensor(k: int) -> np.ndarray:
    """The seeded iPEPS tensor of workload k (seed SEED_BASE + k unless the workload names its own)."""
    w = WORKLOADS[k]
    return random_ipeps(w["d"], w["D"], w.get("seed", SEED_BASE + k), w["complex_valued"])
