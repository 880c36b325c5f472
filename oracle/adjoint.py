"""Gradient of the bond energy with the environment held fixed (test infrastructure).

E(A) = Re Tr(rho(A) h) / Tr rho(A), rho the two-site RDM of observables.two_site_rdm
with C and T fixed (real or complex A). The same network is written here in torch (float64, CPU)
so that torch.autograd supplies dE/dA; it is pinned against central finite
differences of the numpy oracle (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import torch


def _open_double_layer(A: torch.Tensor) -> torch.Tensor:
    """a[s, s', (u ubar), ...] = A[s, u, l, d, r] conj(A[s', ubar, ...]), combined index ket fastest."""
    d, D = A.shape[0], A.shape[1]
    q = D * D
    a = torch.einsum("suldr,tUVWX->stUuVlWdXr", A, A.conj())   # bra index (capital) before ket
    return a.reshape(d, d, q, q, q, q)


def energy_torch(C: torch.Tensor, T: torch.Tensor, A: torch.Tensor, h: torch.Tensor) -> torch.Tensor:
    """Bond energy of the network of observables.two_site_rdm (clockwise boundary ring), in torch."""
    d = A.shape[0]
    a_open = _open_double_layer(A)
    H = torch.tensordot(torch.tensordot(C, T, dims=([1], [0])), C, dims=([2], [0]))   # [a, x, b]
    L1 = torch.tensordot(T, H, dims=([2], [0]))                                       # [b, d1, l1, e]
    L2 = torch.tensordot(L1, T, dims=([3], [0]))                                      # [b, d1, l1, u1, t]
    LB = torch.tensordot(L2, a_open, dims=([1, 2, 3], [4, 3, 2]))                     # [b, t, s1, s1', m]
    RB = torch.tensordot(L2, a_open, dims=([1, 2, 3], [2, 5, 4]))                     # [t, b, s2, s2', m]
    rho = torch.tensordot(LB, RB, dims=([0, 1, 4], [1, 0, 4]))                        # [s1, s1', s2, s2']
    rho = rho.permute(0, 2, 1, 3).reshape(d * d, d * d)
    return torch.real(torch.trace(rho @ h.to(rho.dtype)) / torch.trace(rho))


def energy_gradient(C: np.ndarray, T: np.ndarray, A: np.ndarray, h: np.ndarray) -> np.ndarray:
    """dE/dA by torch.autograd on energy_torch; for complex A the result is
    dE/dRe A + i dE/dIm A."""
    At = torch.tensor(A, requires_grad=True)
    e = energy_torch(torch.tensor(C), torch.tensor(T), At, torch.tensor(h))
    e.backward()
    return At.grad.numpy()
