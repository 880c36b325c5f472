"""Gradient of the bond energy with the environment held fixed (test infrastructure).

E(A) = Tr(rho(A) h) / Tr rho(A), rho the two-site RDM of observables.two_site_rdm
with C and T fixed. The same network is written here in torch (float64, CPU)
so that torch.autograd supplies dE/dA; it is pinned against central finite
differences of the numpy oracle (tests/test_oracle_adjoint.py).
"""
from __future__ import annotations

import numpy as np
import torch


def _open_double_layer(A: torch.Tensor) -> torch.Tensor:
    d, D = A.shape[0], A.shape[1]
    q = D * D
    a = torch.einsum("suldr,tUVWX->stUuVlWdXr", A, A)   # bra index (capital) before ket
    return a.reshape(d, d, q, q, q, q)


def energy_torch(C: torch.Tensor, T: torch.Tensor, A: torch.Tensor, h: torch.Tensor) -> torch.Tensor:
    """Bond energy of the network of observables.two_site_rdm, in torch."""
    d = A.shape[0]
    a_open = _open_double_layer(A)
    E = torch.tensordot(torch.tensordot(C, T, dims=([1], [0])), C, dims=([2], [0]))   # [t, x, b]
    Z1 = torch.tensordot(E, T, dims=([0], [0]))                                         # [l, b, u, t']
    Z2 = torch.tensordot(Z1, T, dims=([1], [0]))                                        # [l, u, t', d, b']
    LB = torch.tensordot(Z2, a_open, dims=([0, 1, 3], [3, 2, 4]))                      # [t', b', s1, s1', m]
    Z1r = torch.tensordot(E, T, dims=([0], [2]))
    Z2r = torch.tensordot(Z1r, T, dims=([1], [2]))
    RB = torch.tensordot(Z2r, a_open, dims=([0, 2, 4], [5, 2, 4]))
    rho = torch.tensordot(LB, RB, dims=([0, 1, 4], [0, 1, 4]))                          # [s1, s1', s2, s2']
    rho = rho.permute(0, 2, 1, 3).reshape(d * d, d * d)
    return torch.trace(rho @ h) / torch.trace(rho)


def energy_gradient(C: np.ndarray, T: np.ndarray, A: np.ndarray, h: np.ndarray) -> np.ndarray:
    """dE/dA by torch.autograd on energy_torch (real A)."""
    At = torch.tensor(A, dtype=torch.float64, requires_grad=True)
    e = energy_torch(torch.tensor(C), torch.tensor(T), At, torch.tensor(h))
    e.backward()
    return At.grad.numpy()
