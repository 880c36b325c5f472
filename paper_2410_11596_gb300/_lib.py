"""ctypes binding of libhs (include/hs.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts between
torch device tensors / Python values and the C structs of the ABI. If the
library has not been built, loading fails with an error: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, c_double, c_int, c_size_t, c_uint, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "hs.h")

HS_OK = 0
STATUS_NAMES = {
    0: "HS_OK", -1: "HS_ERR_INVALID_ARG", -2: "HS_ERR_SHAPE", -3: "HS_ERR_DTYPE",
    -4: "HS_ERR_NOT_HERMITIAN", -5: "HS_ERR_CUDA", -6: "HS_ERR_SOLVER", -7: "HS_ERR_TIMEOUT",
    -8: "HS_ERR_NONFINITE", -9: "HS_ERR_WORKSPACE", -10: "HS_ERR_UNSUPPORTED",
}
HS_F64, HS_C128 = 0, 1
HS_PREC_F64, HS_PREC_TF32X3, HS_PREC_TF32, HS_PREC_BF16X3 = 0, 1, 2, 3
HS_BASIS_DENSE, HS_BASIS_HERMITIAN = 0, 1
HS_GEMM_OWN, HS_GEMM_CUBLAS = 0, 1
HS_RDM_TWO_SITE, HS_RDM_ENV_ONE_SITE, HS_RDM_ONE_SITE = 0, 1, 2
HS_EIG_F64, HS_EIG_F32_PROJECTED, HS_EIG_SUBSPACE, HS_EIG_SUBSPACE_ADAPTIVE = 0, 1, 2, 3
HS_SVD_JACOBI, HS_SVD_POLAR = 0, 1


class HsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Z2Tensor(ctypes.Structure):
    _fields_ = [("D", c_int), ("n_even", c_int), ("n_odd", c_int), ("basis", c_int), ("dtype", c_int),
                ("data", c_void_p), ("capacity_bytes", c_size_t), ("v_even", c_int), ("v_odd", c_int),
                ("h_even", c_int), ("h_odd", c_int)]


class HotrgInfo(ctypes.Structure):
    _fields_ = [("h_even", c_int), ("h_odd", c_int), ("side", c_int), ("discarded_left", c_double),
                ("discarded_right", c_double), ("log_norm", c_double), ("trace", c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Env(ctypes.Structure):
    _fields_ = [("D", c_int), ("chi_max", c_int), ("chi_even", c_int), ("chi_odd", c_int),
                ("q_even", c_int), ("q_odd", c_int), ("basis", c_int), ("precision", c_int),
                ("gemm_backend", c_int), ("moves", c_int), ("log_norm_C", c_double),
                ("log_norm_T", c_double), ("C", c_void_p), ("T", c_void_p), ("C_bytes", c_size_t),
                ("T_bytes", c_size_t), ("eig_mode", c_int), ("dtype", c_int)]


class MoveInfo(ctypes.Structure):
    _fields_ = [("chi_even", c_int), ("chi_odd", c_int), ("n_even", c_int), ("n_odd", c_int),
                ("lam_max", c_double), ("lam_cut", c_double), ("lam_next", c_double), ("gap", c_double),
                ("log_norm_C", c_double), ("log_norm_T", c_double), ("gemm_flops", c_double),
                ("flags", c_int), ("subspace_iters", c_int), ("subspace_reason", c_int),
                ("subspace_resid", c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class Env4(ctypes.Structure):
    _fields_ = [("D", c_int), ("chi_max", c_int), ("chi_even", c_int * 4), ("chi_odd", c_int * 4),
                ("q_even", c_int), ("q_odd", c_int), ("basis", c_int), ("moves", c_int),
                ("C", c_void_p * 4), ("T", c_void_p * 4), ("C_bytes", c_size_t), ("T_bytes", c_size_t),
                ("log_norm_C", c_double * 4), ("log_norm_T", c_double * 4), ("svd", c_int)]


class Move4Info(ctypes.Structure):
    _fields_ = [("direction", c_int), ("chi_even", c_int), ("chi_odd", c_int), ("m_even", c_int),
                ("m_odd", c_int), ("n_even", c_int), ("n_odd", c_int), ("s_max", c_double), ("s_cut", c_double),
                ("s_next", c_double), ("gap", c_double), ("gemm_flops", c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_PROTOS = {
    "hs_create": (c_int, [POINTER(c_void_p), c_int, c_void_p]),
    "hs_destroy": (c_int, [c_void_p]),
    "hs_last_error": (ctypes.c_char_p, []),
    "hs_sync": (c_int, [c_void_p]),
    "hs_abi_version": (c_int, []),
    "hs_make_double_layer": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p]),
    "hs_z2_tensor_bytes": (c_size_t, [c_int, c_int, c_int]),
    "hs_to_hermitian_basis": (c_int, [c_void_p, c_void_p, c_int, c_int, c_double, POINTER(Z2Tensor)]),
    "hs_double_layer_hermitian": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                          POINTER(Z2Tensor)]),
    "hs_env_bytes": (c_int, [c_int, c_int, POINTER(c_size_t), POINTER(c_size_t)]),
    "hs_ctmrg_init": (c_int, [c_void_p, POINTER(Z2Tensor), c_int, c_int, c_int, POINTER(Env)]),
    "hs_ctmrg_move": (c_int, [c_void_p, POINTER(Z2Tensor), POINTER(Env), c_int, POINTER(MoveInfo)]),
    "hs_ctmrg_move_batched": (c_int, [POINTER(c_void_p), c_int, POINTER(POINTER(Z2Tensor)), POINTER(POINTER(Env)),
                                      POINTER(c_int), POINTER(MoveInfo), POINTER(c_double), c_int]),
    "hs_env_to_dense": (c_int, [c_void_p, POINTER(Env), c_void_p, c_void_p]),
    "hs_corner_spectrum": (c_int, [c_void_p, POINTER(Env), c_void_p]),
    "hs_from_hermitian_basis": (c_int, [c_void_p, POINTER(Z2Tensor), c_void_p]),
    "hs_correlation_length": (c_int, [c_void_p, POINTER(Env), c_void_p, c_int, c_int, c_int, c_double,
                                      POINTER(c_double), POINTER(c_double)]),
    "hs_rdm": (c_int, [c_void_p, POINTER(Env), c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p,
                       c_void_p]),
    "hs_workspace_query": (c_int, [c_int, c_int, c_int, POINTER(c_size_t)]),
    "hs_profile_enable": (c_int, [c_void_p, c_int]),
    "hs_profile_phases": (c_int, [c_void_p, c_uint]),
    "hs_profile_read": (c_int, [c_void_p, POINTER(c_double), POINTER(c_double), c_int,
                                POINTER(ctypes.c_longlong)]),
    "hs_gemm": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int]),
    "hs_rdm_vjp": (c_int, [c_void_p, POINTER(Env), c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "hs_energy_vjp": (c_int, [c_void_p, POINTER(Env), c_void_p, c_int, c_int, c_int, c_void_p, c_double,
                              c_void_p]),
    "hs_ctmrg_energy_grad": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_int, c_void_p,
                                     POINTER(c_double), c_void_p]),
    "hs_ctmrg4_init": (c_int, [c_void_p, POINTER(Z2Tensor), c_int, POINTER(Env4)]),
    "hs_ctmrg4_move": (c_int, [c_void_p, POINTER(Z2Tensor), POINTER(Env4), c_int, c_int, POINTER(Move4Info),
                               POINTER(c_double)]),
    "hs_env4_to_dense": (c_int, [c_void_p, POINTER(Env4), POINTER(c_void_p), POINTER(c_void_p)]),
    "hs_selftest_bounded_wait": (c_int, [c_void_p, ctypes.c_longlong, POINTER(c_int)]),
    "hs_hotrg_tensor_bytes": (c_size_t, [c_int, c_int]),
    "hs_hotrg_init": (c_int, [c_void_p, POINTER(Z2Tensor), POINTER(Z2Tensor), POINTER(c_double)]),
    "hs_hotrg_step": (c_int, [c_void_p, POINTER(Z2Tensor), c_int, c_int, c_int, POINTER(HotrgInfo)]),
    "hs_hotrg_log_z": (c_int, [POINTER(c_double), c_int, c_double, POINTER(c_double)]),
    "hs_gemm_static": (c_int, [c_int, c_int, c_int, c_int, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int,
                               c_void_p, c_void_p]),
}

PHASES = ("gemm", "permute", "eig", "select", "normalize", "gemm_tc", "gemm_tc_split")

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/hs.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_[a-z0-9_]+)\s*\(", text)))


def load(path: str = LIB_PATH):
    """Load libhs.so (once) and declare the prototypes. Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise HsError(-5, f"{path} is missing: build it with paper_2410_11596_gb300/build.py "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _PROTOS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int) -> None:
    if status != HS_OK:
        raise HsError(status, load().hs_last_error().decode())


def ptr(t) -> int:
    """Device pointer of a contiguous torch tensor."""
    assert t.is_contiguous()
    return t.data_ptr()


# ---- thin wrappers with the C names -----------------------------------------


def hs_create(device: int = 0, stream: int | None = None) -> int:
    h = c_void_p()
    check(load().hs_create(ctypes.byref(h), device, stream))
    return h.value


def hs_destroy(ctx: int) -> None:
    check(load().hs_destroy(ctx))


def hs_sync(ctx: int) -> None:
    check(load().hs_sync(ctx))


def hs_z2_tensor_bytes(D: int, basis: int, dtype: int = HS_F64) -> int:
    return load().hs_z2_tensor_bytes(D, basis, dtype)


def hs_make_double_layer(ctx: int, A, d: int, D: int, dtype: int, a_out) -> None:
    check(load().hs_make_double_layer(ctx, ptr(A), d, D, dtype, ptr(a_out)))


def hs_to_hermitian_basis(ctx: int, a_dense, D: int, dtype: int, herm_tol: float, out_buf) -> Z2Tensor:
    t = Z2Tensor(data=ptr(out_buf), capacity_bytes=out_buf.numel() * out_buf.element_size())
    check(load().hs_to_hermitian_basis(ctx, ptr(a_dense), D, dtype, herm_tol, ctypes.byref(t)))
    return t


def hs_double_layer_hermitian(ctx: int, A, d: int, D: int, dtype: int, basis: int, out_buf) -> Z2Tensor:
    t = Z2Tensor(data=ptr(out_buf), capacity_bytes=out_buf.numel() * out_buf.element_size())
    check(load().hs_double_layer_hermitian(ctx, ptr(A), d, D, dtype, basis, ctypes.byref(t)))
    return t


def hs_env_bytes(D: int, chi_max: int) -> tuple[int, int]:
    cb, tb = c_size_t(), c_size_t()
    check(load().hs_env_bytes(D, chi_max, ctypes.byref(cb), ctypes.byref(tb)))
    return cb.value, tb.value


def hs_ctmrg_init(ctx: int, a: Z2Tensor, chi_max: int, precision: int, backend: int, C_buf, T_buf) -> Env:
    env = Env(C=ptr(C_buf), T=ptr(T_buf), C_bytes=C_buf.numel() * 8, T_bytes=T_buf.numel() * 8)
    check(load().hs_ctmrg_init(ctx, ctypes.byref(a), chi_max, precision, backend, ctypes.byref(env)))
    return env


def hs_ctmrg_move(ctx: int, a: Z2Tensor, env: Env, chi: int) -> MoveInfo:
    info = MoveInfo()
    check(load().hs_ctmrg_move(ctx, ctypes.byref(a), ctypes.byref(env), chi, ctypes.byref(info)))
    return info


def hs_ctmrg_move_batched(ctxs: list, a: list, env: list, chi: list, nthreads: int) -> tuple[list, list]:
    """One move of each instance, concurrently; returns (move records, wall-clock ms per instance)."""
    n = len(ctxs)
    c_ctx = (c_void_p * n)(*ctxs)
    c_a = (POINTER(Z2Tensor) * n)(*[ctypes.pointer(x) for x in a])
    c_env = (POINTER(Env) * n)(*[ctypes.pointer(x) for x in env])
    c_chi = (c_int * n)(*chi)
    info = (MoveInfo * n)()
    ms = (c_double * n)()
    check(load().hs_ctmrg_move_batched(c_ctx, n, c_a, c_env, c_chi, info, ms, nthreads))
    return [info[i].as_dict() for i in range(n)], [ms[i] for i in range(n)]


def hs_correlation_length(ctx: int, env: Env, A, d: int, D: int, max_iter: int = 200,
                          tol: float = 1e-12) -> tuple[float, float, float]:
    lam = (c_double * 2)()
    xi = c_double()
    check(load().hs_correlation_length(ctx, ctypes.byref(env), ptr(A), d, D, max_iter, tol, lam, ctypes.byref(xi)))
    return lam[0], lam[1], xi.value


def hs_env_to_dense(ctx: int, env: Env, C_dense, T_dense) -> None:
    check(load().hs_env_to_dense(ctx, ctypes.byref(env), ptr(C_dense), ptr(T_dense)))


def hs_ctmrg4_init(ctx: int, a: Z2Tensor, chi_max: int, C_bufs, T_bufs) -> Env4:
    env = Env4(C=(c_void_p * 4)(*[ptr(b) for b in C_bufs]), T=(c_void_p * 4)(*[ptr(b) for b in T_bufs]),
               C_bytes=min(b.numel() for b in C_bufs) * 8, T_bytes=min(b.numel() for b in T_bufs) * 8)
    check(load().hs_ctmrg4_init(ctx, ctypes.byref(a), chi_max, ctypes.byref(env)))
    return env


def hs_ctmrg4_move(ctx: int, a: Z2Tensor, env: Env4, chi: int, direction: int) -> tuple[dict, list]:
    """One directional move; returns (move record, kept singular values / largest)."""
    info = Move4Info()
    sv = (c_double * chi)()
    check(load().hs_ctmrg4_move(ctx, ctypes.byref(a), ctypes.byref(env), chi, direction, ctypes.byref(info), sv))
    d = info.as_dict()
    return d, [sv[i] for i in range(d["chi_even"] + d["chi_odd"])]


def hs_env4_to_dense(ctx: int, env: Env4, C_dense, T_dense) -> None:
    check(load().hs_env4_to_dense(ctx, ctypes.byref(env), (c_void_p * 4)(*[ptr(x) for x in C_dense]),
                                  (c_void_p * 4)(*[ptr(x) for x in T_dense])))


def hs_selftest_bounded_wait(ctx: int, limit: int) -> list[int]:
    out = (c_int * 7)()
    check(load().hs_selftest_bounded_wait(ctx, limit, out))
    return list(out)


def hs_corner_spectrum(ctx: int, env: Env, out) -> None:
    check(load().hs_corner_spectrum(ctx, ctypes.byref(env), ptr(out)))


def hs_from_hermitian_basis(ctx: int, t: Z2Tensor, a_dense) -> None:
    check(load().hs_from_hermitian_basis(ctx, ctypes.byref(t), ptr(a_dense)))


def hs_rdm(ctx: int, env: Env, A, d: int, D: int, dtype: int, kind: int, h, out, tr_out) -> None:
    check(load().hs_rdm(ctx, ctypes.byref(env), ptr(A), d, D, dtype, kind,
                        ptr(h) if h is not None else None, ptr(out),
                        ptr(tr_out) if tr_out is not None else None))


def hs_workspace_query(D: int, chi: int, precision: int) -> int:
    b = c_size_t()
    check(load().hs_workspace_query(D, chi, precision, ctypes.byref(b)))
    return b.value


def hs_profile_enable(ctx: int, enable: bool) -> None:
    check(load().hs_profile_enable(ctx, 1 if enable else 0))


def hs_profile_phases(ctx: int, phases=None) -> None:
    """Time only the named phases (None: all of them)."""
    mask = 0xFFFFFFFF if phases is None else sum(1 << PHASES.index(p) for p in phases)
    check(load().hs_profile_phases(ctx, mask))


def hs_profile_read(ctx: int) -> dict:
    ms = (c_double * len(PHASES))()
    fl = (c_double * len(PHASES))()
    n = ctypes.c_longlong()
    check(load().hs_profile_read(ctx, ms, fl, len(PHASES), ctypes.byref(n)))
    return {"phase_ms": dict(zip(PHASES, list(ms))), "phase_flops": dict(zip(PHASES, list(fl))),
            "launches": n.value}


def hs_gemm(ctx: int, precision: int, A, B, C) -> None:
    """C = A B^T for contiguous row-major FP64 device tensors."""
    M, K = A.shape
    N = B.shape[0]
    check(load().hs_gemm(ctx, precision, M, N, K, ptr(A), K, ptr(B), K, ptr(C), N))


def hs_gemm_static(precision: int, A, B, C, status, stream: int | None = None) -> None:
    """C = A B^T through the allocation-free entry point; status is a device int32 tensor."""
    M, K = A.shape
    N = B.shape[0]
    check(load().hs_gemm_static(precision, M, N, K, ptr(A), K, ptr(B), K, ptr(C), N, ptr(status), stream))


def hs_hotrg_tensor_bytes(D: int, chi: int) -> int:
    return load().hs_hotrg_tensor_bytes(D, chi)


def hs_hotrg_init(ctx: int, a: Z2Tensor, t_buf) -> tuple[Z2Tensor, float]:
    t = Z2Tensor(data=ptr(t_buf), capacity_bytes=t_buf.numel() * t_buf.element_size())
    ln = c_double()
    check(load().hs_hotrg_init(ctx, ctypes.byref(a), ctypes.byref(t), ctypes.byref(ln)))
    return t, ln.value


def hs_hotrg_step(ctx: int, t: Z2Tensor, chi: int, direction: int, precision: int = HS_PREC_F64) -> dict:
    info = HotrgInfo()
    check(load().hs_hotrg_step(ctx, ctypes.byref(t), chi, direction, precision, ctypes.byref(info)))
    return info.as_dict()


def hs_hotrg_log_z(log_norms, trace: float) -> float:
    """ln Z / N from the log norms of hs_hotrg_init and of every step, and the last step's trace."""
    n = len(log_norms)
    arr = (c_double * n)(*[float(x) for x in log_norms])
    out = c_double()
    check(load().hs_hotrg_log_z(arr, n - 1, float(trace), ctypes.byref(out)))
    return out.value


def hs_rdm_vjp(ctx: int, env: Env, A, d: int, D: int, drho, dA, dtype: int = HS_F64) -> None:
    check(load().hs_rdm_vjp(ctx, ctypes.byref(env), ptr(A), d, D, dtype, ptr(drho), ptr(dA)))


def hs_energy_vjp(ctx: int, env: Env, A, d: int, D: int, dtype: int, h, dE: float, dA) -> None:
    check(load().hs_energy_vjp(ctx, ctypes.byref(env), ptr(A), d, D, dtype, ptr(h), float(dE), ptr(dA)))


def hs_ctmrg_energy_grad(ctx: int, A, d: int, D: int, basis: int, chi: int, moves: int, h, dA) -> float:
    """E of a whole CTMRG run from A and dE/dA into dA (device)."""
    e = c_double()
    check(load().hs_ctmrg_energy_grad(ctx, ptr(A), d, D, basis, chi, moves, ptr(h), ctypes.byref(e), ptr(dA)))
    return e.value
