"""Python front end of libhs: allocates device buffers with torch and calls the C ABI.

No arithmetic of the method happens here; every step runs in the CUDA library.
"""
from __future__ import annotations

import functools

import numpy as np
import torch

from . import _lib as L

BASIS = {"dense": L.HS_BASIS_DENSE, "hermitian": L.HS_BASIS_HERMITIAN}
PRECISION = {"f64": L.HS_PREC_F64, "tf32x3": L.HS_PREC_TF32X3, "tf32": L.HS_PREC_TF32,
             "bf16x3": L.HS_PREC_BF16X3}
BACKEND = {"own": L.HS_GEMM_OWN, "cublas": L.HS_GEMM_CUBLAS}
EIG = {"f64": L.HS_EIG_F64, "f32p": L.HS_EIG_F32_PROJECTED, "subspace": L.HS_EIG_SUBSPACE,
       "adaptive": L.HS_EIG_SUBSPACE_ADAPTIVE}


class Context:
    """An hs_ctx bound to a CUDA device and the current torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        if not torch.cuda.is_available():
            raise L.HsError(-5, "no CUDA device: libhs has no CPU path")
        self.device = device
        self.stream = stream or torch.cuda.current_stream(device)
        self.handle = L.hs_create(device, self.stream.cuda_stream)

    def close(self) -> None:
        if self.handle:
            L.hs_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self) -> None:
        L.hs_sync(self.handle)


def _record(x, stream) -> None:
    if isinstance(x, torch.Tensor) and x.is_cuda:
        x.record_stream(stream)
    elif isinstance(x, (tuple, list)):
        for y in x:
            _record(y, stream)


def on_ctx_stream(fn):
    """Run a method of an object with a `ctx` on the context's stream: the
    context stream first waits for the caller's stream (inputs made there),
    torch work inside (allocations, copies) is issued on the context stream,
    and the caller's stream then waits for it (outputs handed back)."""
    @functools.wraps(fn)
    def wrapper(self, *args, **kwargs):
        s = self.ctx.stream
        caller = torch.cuda.current_stream(self.ctx.device)
        if s == caller:
            return fn(self, *args, **kwargs)
        s.wait_stream(caller)
        with torch.cuda.stream(s):
            out = fn(self, *args, **kwargs)
        caller.wait_stream(s)
        _record(out, caller)
        return out
    return wrapper


def to_device(A: np.ndarray, device: int = 0) -> torch.Tensor:
    """Copy a host iPEPS tensor to the device (complex as interleaved float64)."""
    A = np.ascontiguousarray(A)
    if np.iscomplexobj(A):
        A = A.astype(np.complex128).view(np.float64)
    return torch.from_numpy(A.astype(np.float64)).to(f"cuda:{device}")


class CTMRG:
    """C4v CTMRG of one iPEPS tensor on one GPU through the C ABI.

    A complex A (numpy complex array, or a torch tensor of interleaved float64
    with complex_valued=True) runs the graded path of Sec. II.C in the
    Hermitian basis; a real one the Z2 block path of Sec. II.B.
    """

    def __init__(self, ctx: Context, A: np.ndarray | torch.Tensor, chi: int, basis: str = "hermitian",
                 precision: str = "f64", backend: str = "own", eig: str = "f64", complex_valued: bool | None = None):
        self.ctx = ctx
        self._init(A, chi, basis, precision, backend, eig, complex_valued)

    @on_ctx_stream
    def _init(self, A, chi, basis, precision, backend, eig, complex_valued):
        ctx = self.ctx
        dev = f"cuda:{ctx.device}"
        if complex_valued is None:
            complex_valued = isinstance(A, np.ndarray) and np.iscomplexobj(A)
        self.complex = bool(complex_valued)
        self.dtype = L.HS_C128 if self.complex else L.HS_F64
        self.A = A if isinstance(A, torch.Tensor) else to_device(A, ctx.device)
        self.d, self.D = int(self.A.shape[0]), int(self.A.shape[1])
        self.chi = chi
        nbytes = L.hs_z2_tensor_bytes(self.D, BASIS[basis], self.dtype)
        self.a_buf = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
        self.a = L.hs_double_layer_hermitian(ctx.handle, self.A, self.d, self.D, self.dtype, BASIS[basis],
                                             self.a_buf)
        cb, tb = L.hs_env_bytes(self.D, chi)
        if self.complex and basis == "dense":      # complex environments of the plain basis: complex128
            cb, tb = 2 * cb, 2 * tb
        self.C_buf = torch.empty(cb // 8, dtype=torch.float64, device=dev)
        self.T_buf = torch.empty(tb // 8, dtype=torch.float64, device=dev)
        self.env = L.hs_ctmrg_init(ctx.handle, self.a, chi, PRECISION[precision], BACKEND[backend],
                                   self.C_buf, self.T_buf)
        self.env.eig_mode = EIG[eig]
        self.infos: list[dict] = []

    @on_ctx_stream
    def move(self) -> dict:
        info = L.hs_ctmrg_move(self.ctx.handle, self.a, self.env, self.chi).as_dict()
        self.infos.append(info)
        return info

    def run(self, moves: int) -> list[dict]:
        return [self.move() for _ in range(moves)]

    @property
    def chi_now(self) -> int:
        return self.env.chi_even + self.env.chi_odd

    @on_ctx_stream
    def corner_spectrum(self) -> torch.Tensor:
        """Singular values of C divided by the largest, descending (hs_corner_spectrum, on the GPU)."""
        out = torch.empty(self.chi_now, dtype=torch.float64, device=self.A.device)
        L.hs_corner_spectrum(self.ctx.handle, self.env, out)
        return out

    @on_ctx_stream
    def double_layer_dense(self) -> torch.Tensor:
        """The double layer back in the plain combined basis, a[u, l, d, r] (hs_from_hermitian_basis);
        complex128 for complex A. Hermitian basis only."""
        q = self.D * self.D
        if self.complex:
            a = torch.empty((q, q, q, q, 2), dtype=torch.float64, device=self.A.device)
            L.hs_from_hermitian_basis(self.ctx.handle, self.a, a)
            return torch.view_as_complex(a)
        a = torch.empty((q, q, q, q), dtype=torch.float64, device=self.A.device)
        L.hs_from_hermitian_basis(self.ctx.handle, self.a, a)
        return a

    @on_ctx_stream
    def rdm1(self, h1: np.ndarray | None = None):
        """(rho1, Tr rho1, Tr rho1 h1) of one site (HS_RDM_ONE_SITE); h1 a d x d real matrix.
        For complex A, rho1 is complex128 and the traces are complex."""
        dev = self.A.device
        d = self.d
        hd = None if h1 is None else torch.from_numpy(np.ascontiguousarray(np.real(h1), dtype=np.float64)).to(dev)
        if self.complex:
            rho = torch.empty((d, d, 2), dtype=torch.float64, device=dev)
            tr = torch.empty(4, dtype=torch.float64, device=dev)
            L.hs_rdm(self.ctx.handle, self.env, self.A, d, self.D, L.HS_C128, L.HS_RDM_ONE_SITE, hd, rho, tr)
            t = tr.cpu().numpy()
            return torch.view_as_complex(rho), complex(t[0], t[1]), complex(t[2], t[3])
        rho = torch.empty((d, d), dtype=torch.float64, device=dev)
        tr = torch.empty(2, dtype=torch.float64, device=dev)
        L.hs_rdm(self.ctx.handle, self.env, self.A, d, self.D, L.HS_F64, L.HS_RDM_ONE_SITE, hd, rho, tr)
        t = tr.cpu().numpy()
        return rho, float(t[0]), float(t[1])

    @on_ctx_stream
    def dense_env(self) -> tuple[torch.Tensor, torch.Tensor]:
        """(C[chi, chi], T[chi, D^2, chi]) in the plain combined basis (complex128 for complex A)."""
        chi, q = self.chi_now, self.D * self.D
        dev = self.A.device
        if self.complex:
            C = torch.empty((chi, chi, 2), dtype=torch.float64, device=dev)
            T = torch.empty((chi, q, chi, 2), dtype=torch.float64, device=dev)
            L.hs_env_to_dense(self.ctx.handle, self.env, C, T)
            return torch.view_as_complex(C), torch.view_as_complex(T)
        C = torch.empty((chi, chi), dtype=torch.float64, device=dev)
        T = torch.empty((chi, q, chi), dtype=torch.float64, device=dev)
        L.hs_env_to_dense(self.ctx.handle, self.env, C, T)
        return C, T

    @on_ctx_stream
    def rdm2(self, h: np.ndarray):
        """(rho, Tr rho, Tr rho h) of a horizontal bond; h a d^2 x d^2 real matrix.
        For complex A, rho is complex128 and the traces are complex."""
        dev = self.A.device
        n = self.d * self.d
        hd = torch.from_numpy(np.ascontiguousarray(np.real(h), dtype=np.float64)).to(dev)
        if self.complex:
            rho = torch.empty((n, n, 2), dtype=torch.float64, device=dev)
            tr = torch.empty(4, dtype=torch.float64, device=dev)
            L.hs_rdm(self.ctx.handle, self.env, self.A, self.d, self.D, L.HS_C128, L.HS_RDM_TWO_SITE, hd, rho, tr)
            t = tr.cpu().numpy()
            return torch.view_as_complex(rho), complex(t[0], t[1]), complex(t[2], t[3])
        rho = torch.empty((n, n), dtype=torch.float64, device=dev)
        tr = torch.empty(2, dtype=torch.float64, device=dev)
        L.hs_rdm(self.ctx.handle, self.env, self.A, self.d, self.D, L.HS_F64, L.HS_RDM_TWO_SITE, hd, rho, tr)
        t = tr.cpu().numpy()
        return rho, float(t[0]), float(t[1])

    def energy(self, h: np.ndarray) -> float:
        _, t0, t1 = self.rdm2(h)
        return float(np.real(t1 / t0))

    @on_ctx_stream
    def rdm2_of(self, A: torch.Tensor, h: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
        """(rho, [Tr rho, Tr rho h]) for another tensor A with this (fixed) environment.
        Complex A (a complex128 tensor) gives complex rho and traces."""
        n = self.d * self.d
        if self.complex:
            Ai = torch.view_as_real(A.to(torch.complex128)).contiguous()
            rho = torch.empty((n, n, 2), dtype=torch.float64, device=A.device)
            tr = torch.empty((2, 2), dtype=torch.float64, device=A.device)
            L.hs_rdm(self.ctx.handle, self.env, Ai, self.d, self.D, L.HS_C128, L.HS_RDM_TWO_SITE, h.contiguous(),
                     rho, tr)
            return torch.view_as_complex(rho), torch.view_as_complex(tr)
        rho = torch.empty((n, n), dtype=torch.float64, device=A.device)
        tr = torch.empty(2, dtype=torch.float64, device=A.device)
        L.hs_rdm(self.ctx.handle, self.env, A.contiguous(), self.d, self.D, L.HS_F64, L.HS_RDM_TWO_SITE,
                 h.contiguous(), rho, tr)
        return rho, tr

    @on_ctx_stream
    def rdm2_vjp(self, A: torch.Tensor, drho: torch.Tensor) -> torch.Tensor:
        """Adjoint of rdm2_of: drho (cotangent dE/dRe rho + i dE/dIm rho for complex A) -> dA."""
        if self.complex:
            Ai = torch.view_as_real(A.to(torch.complex128)).contiguous()
            dr = torch.view_as_real(drho.to(torch.complex128)).contiguous()
            dA = torch.empty_like(Ai)
            L.hs_rdm_vjp(self.ctx.handle, self.env, Ai, self.d, self.D, dr, dA, L.HS_C128)
            return torch.view_as_complex(dA)
        dA = torch.empty_like(A)
        L.hs_rdm_vjp(self.ctx.handle, self.env, A.contiguous(), self.d, self.D, drho.contiguous(), dA)
        return dA

    @on_ctx_stream
    def energy_vjp(self, A: torch.Tensor, h: torch.Tensor, dE: float) -> torch.Tensor:
        """dE * gradient of E = Re Tr(rho h) / Tr rho with respect to A, environment fixed (hs_energy_vjp)."""
        if self.complex:
            Ai = torch.view_as_real(A.to(torch.complex128)).contiguous()
            dA = torch.empty_like(Ai)
            L.hs_energy_vjp(self.ctx.handle, self.env, Ai, self.d, self.D, L.HS_C128, h.contiguous(), dE, dA)
            return torch.view_as_complex(dA)
        dA = torch.empty_like(A)
        L.hs_energy_vjp(self.ctx.handle, self.env, A.contiguous(), self.d, self.D, L.HS_F64, h.contiguous(), dE, dA)
        return dA

    def correlation_length(self, max_iter: int = 200, tol: float = 1e-12) -> float:
        """xi = -1/ln|lambda_2/lambda_1| of the column transfer matrix T-a-T (real A)."""
        return L.hs_correlation_length(self.ctx.handle, self.env, self.A, self.d, self.D, max_iter, tol)[2]

    @on_ctx_stream
    def one_site_env(self) -> torch.Tensor:
        """eps[u, l, d, r] in the plain combined basis (Eq. (4)); complex128 for complex A."""
        q = self.D * self.D
        if self.complex:
            eps = torch.empty((q, q, q, q, 2), dtype=torch.float64, device=self.A.device)
            L.hs_rdm(self.ctx.handle, self.env, self.A, self.d, self.D, L.HS_C128, L.HS_RDM_ENV_ONE_SITE,
                     None, eps, None)
            return torch.view_as_complex(eps)
        eps = torch.empty((q, q, q, q), dtype=torch.float64, device=self.A.device)
        L.hs_rdm(self.ctx.handle, self.env, self.A, self.d, self.D, L.HS_F64, L.HS_RDM_ENV_ONE_SITE,
                 None, eps, None)
        return eps


class DirectionalCTMRG:
    """CTMRG without lattice symmetry (four corners, four edges) of one real iPEPS tensor on one
    GPU through the C ABI: a sweep moves the left, top, right and bottom sides in turn."""

    def __init__(self, ctx: Context, A: np.ndarray | torch.Tensor, chi: int, basis: str = "hermitian",
                 svd: str = "jacobi"):
        self.ctx = ctx
        self._init(A, chi, basis, svd)

    @on_ctx_stream
    def _init(self, A, chi, basis, svd):
        ctx = self.ctx
        dev = f"cuda:{ctx.device}"
        self.A = A if isinstance(A, torch.Tensor) else to_device(A, ctx.device)
        self.d, self.D = int(self.A.shape[0]), int(self.A.shape[1])
        self.chi = chi
        nbytes = L.hs_z2_tensor_bytes(self.D, BASIS[basis], L.HS_F64)
        self.a_buf = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
        self.a = L.hs_double_layer_hermitian(ctx.handle, self.A, self.d, self.D, L.HS_F64, BASIS[basis], self.a_buf)
        cb, tb = L.hs_env_bytes(self.D, chi)
        self.C_bufs = [torch.empty(cb // 8, dtype=torch.float64, device=dev) for _ in range(4)]
        self.T_bufs = [torch.empty(tb // 8, dtype=torch.float64, device=dev) for _ in range(4)]
        self.env = L.hs_ctmrg4_init(ctx.handle, self.a, chi, self.C_bufs, self.T_bufs)
        self.env.svd = {"jacobi": L.HS_SVD_JACOBI, "polar": L.HS_SVD_POLAR}[svd]
        self.infos: list[dict] = []
        self.spectra: list[list] = []

    @on_ctx_stream
    def move(self, direction: int) -> dict:
        info, sv = L.hs_ctmrg4_move(self.ctx.handle, self.a, self.env, self.chi, direction)
        self.infos.append(info)
        self.spectra.append(sv)
        return info

    def sweep(self) -> list[dict]:
        return [self.move(k) for k in range(4)]

    def run(self, sweeps: int) -> list[dict]:
        for _ in range(sweeps):
            self.sweep()
        return self.infos

    def bond(self, b: int) -> int:
        return self.env.chi_even[b] + self.env.chi_odd[b]

    @on_ctx_stream
    def dense_env(self) -> list[torch.Tensor]:
        """[C1, T1, C2, T2, C3, T3, C4, T4] as dense FP64 device tensors in the plain basis."""
        q = self.D * self.D
        dev = self.A.device
        C = [torch.empty(self.bond((k + 3) % 4), self.bond(k), dtype=torch.float64, device=dev) for k in range(4)]
        T = [torch.empty(self.bond(k), q, self.bond(k), dtype=torch.float64, device=dev) for k in range(4)]
        L.hs_env4_to_dense(self.ctx.handle, self.env, C, T)
        return [x for k in range(4) for x in (C[k], T[k])]


class HOTRG:
    """HOTRG of one real iPEPS double layer on one GPU through the C ABI."""

    def __init__(self, ctx: Context, A: np.ndarray | torch.Tensor, chi: int, basis: str = "hermitian",
                 precision: str = "f64"):
        self.ctx = ctx
        self.precision = PRECISION[precision]
        self._init(A, chi, basis)

    @on_ctx_stream
    def _init(self, A, chi, basis):
        ctx = self.ctx
        dev = f"cuda:{ctx.device}"
        self.A = A if isinstance(A, torch.Tensor) else to_device(A, ctx.device)
        self.d, self.D = int(self.A.shape[0]), int(self.A.shape[1])
        self.chi = chi
        nbytes = L.hs_z2_tensor_bytes(self.D, BASIS[basis])
        self.a_buf = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
        self.a = L.hs_double_layer_hermitian(ctx.handle, self.A, self.d, self.D, L.HS_F64, BASIS[basis],
                                             self.a_buf)
        self.t_buf = torch.empty(L.hs_hotrg_tensor_bytes(self.D, chi) // 8, dtype=torch.float64, device=dev)
        self.t, ln0 = L.hs_hotrg_init(ctx.handle, self.a, self.t_buf)
        self.log_norms = [ln0]
        self.infos: list[dict] = []

    def step(self) -> dict:
        direction = len(self.infos) % 2          # vertical, horizontal, vertical, ...
        info = L.hs_hotrg_step(self.ctx.handle, self.t, self.chi, direction, self.precision)
        self.infos.append(info)
        self.log_norms.append(info["log_norm"])
        return info

    def run(self, steps: int) -> list[dict]:
        return [self.step() for _ in range(steps)]

    def log_z_per_site(self) -> float:
        """ln Z / N of the steps so far (hs_hotrg_log_z)."""
        return L.hs_hotrg_log_z(self.log_norms, self.infos[-1]["trace"] if self.infos else 0.0)


class BatchedCTMRG:
    """Many independent CTMRG instances (any mix of D, chi, real or complex) moved
    together by hs_ctmrg_move_batched: each instance has its own context and
    stream, and a pool of host threads drives them concurrently."""

    def __init__(self, tensors: list, chis: list, device: int = 0, precision: str = "tf32x3",
                 eig: str = "subspace", nthreads: int | None = None):
        self.members = []
        self.contexts = []
        for A, chi in zip(tensors, chis):
            ctx = Context(device, torch.cuda.Stream(device))
            self.contexts.append(ctx)
            self.members.append(CTMRG(ctx, A, chi, precision=precision, eig=eig))
        self.nthreads = nthreads or min(len(self.members), 32)
        self.latencies_ms: list[list[float]] = []
        self.mode = "concurrent per-instance moves (own streams, host thread pool)"

    def move(self) -> list[dict]:
        infos, ms = L.hs_ctmrg_move_batched([c.handle for c in self.contexts], [m.a for m in self.members],
                                            [m.env for m in self.members], [m.chi for m in self.members],
                                            self.nthreads)
        for m, i in zip(self.members, infos):
            m.infos.append(i)
        self.latencies_ms.append(ms)
        return infos

    def run(self, moves: int) -> None:
        for _ in range(moves):
            self.move()

    def close(self) -> None:
        for c in self.contexts:
            c.close()


class EnergyFn(torch.autograd.Function):
    """E(A) = Re Tr(rho(A) h) / Tr rho(A) with the environment of `ctm` held fixed.

    forward: hs_rdm; backward: hs_energy_vjp (the cotangent of rho and the
    hand-written adjoint, both in the library). For complex A the gradient is
    dE/dRe A + i dE/dIm A.
    """

    @staticmethod
    def forward(fctx, A: torch.Tensor, ctm: "CTMRG", h: torch.Tensor):
        rho, tr = ctm.rdm2_of(A.detach(), h)
        fctx.ctm = ctm
        fctx.save_for_backward(A.detach(), h)
        return torch.real(tr[1] / tr[0])

    @staticmethod
    def backward(fctx, g):
        A, h = fctx.saved_tensors
        return fctx.ctm.energy_vjp(A, h, float(g)), None, None


def bond_energy(ctm: CTMRG, A: torch.Tensor, h: np.ndarray | torch.Tensor) -> torch.Tensor:
    """Differentiable bond energy with the environment of ctm held fixed."""
    hd = h if isinstance(h, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64))
    return EnergyFn.apply(A, ctm, hd.to(A.device))


class CTMRGEnergyFn(torch.autograd.Function):
    """E(A): the bond energy after `moves` C4v CTMRG moves from the traced boundary (FP64,
    chi kept states), differentiated through every move (hs_ctmrg_energy_grad computes E and
    dE/dA together; the backward scales the stored gradient)."""

    @staticmethod
    def forward(fctx, A: torch.Tensor, ctx: Context, chi: int, moves: int, h: torch.Tensor, basis: str):
        s = ctx.stream
        caller = torch.cuda.current_stream(ctx.device)
        s.wait_stream(caller)
        with torch.cuda.stream(s):
            Ad = A.detach().contiguous()
            dA = torch.empty_like(Ad)
            e = L.hs_ctmrg_energy_grad(ctx.handle, Ad, int(A.shape[0]), int(A.shape[1]), BASIS[basis], chi, moves,
                                       h.contiguous(), dA)
        caller.wait_stream(s)
        dA.record_stream(caller)
        fctx.save_for_backward(dA)
        return torch.tensor(e, dtype=A.dtype, device=A.device)

    @staticmethod
    def backward(fctx, g):
        (dA,) = fctx.saved_tensors
        return g * dA, None, None, None, None, None


def ctmrg_energy(ctx: Context, A: torch.Tensor, chi: int, moves: int, h: np.ndarray | torch.Tensor,
                 basis: str = "hermitian") -> torch.Tensor:
    """Differentiable bond energy of a whole C4v CTMRG run (gradient through the iterations)."""
    hd = h if isinstance(h, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(h, dtype=np.float64))
    return CTMRGEnergyFn.apply(A, ctx, chi, moves, hd.to(A.device), basis)
