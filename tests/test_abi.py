"""The C-ABI library builds, loads and exports every entry point of include/hs.h (no GPU needed)."""
import ctypes
import os

import pytest

from paper_2410_11596_gb300 import _lib as L, build


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(L.LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(L.LIB_PATH) for s in build.sources()):
        build.build()
    return L.load()


def test_every_declared_function_is_exported(lib):
    names = L.header_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_header():
    assert set(L.header_functions()) == set(L._PROTOS)


def test_abi_version(lib):
    assert lib.hs_abi_version() == 5


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 6, 7])
def test_z2_tensor_bytes_closed_form(lib, D):
    """Stored entries of a~: q_e^4 + 6 q_e^2 q_o^2 + q_o^4 (even-total blocks only)."""
    qe, qo = D * (D + 1) // 2, D * (D - 1) // 2
    assert L.hs_z2_tensor_bytes(D, L.HS_BASIS_HERMITIAN) == 8 * (qe ** 4 + 6 * qe ** 2 * qo ** 2 + qo ** 4)
    assert L.hs_z2_tensor_bytes(D, L.HS_BASIS_DENSE) == 8 * D ** 8


def test_d6_storage_fraction(lib):
    """D = 6: 840456 of 1679616 entries stored (50.04%), the twofold memory saving of Sec. I."""
    assert L.hs_z2_tensor_bytes(6, L.HS_BASIS_HERMITIAN) // 8 == 840456


def test_env_bytes(lib):
    assert L.hs_env_bytes(6, 144) == (144 * 144 * 8, 144 * 36 * 144 * 8)
    assert L.hs_env_bytes(6, 8) == (36 * 36 * 8, 36 * 36 * 36 * 8)   # at least chi0 = D^2


def test_errors_are_reported_not_raised_in_c(lib):
    with pytest.raises(L.HsError) as e:
        L.hs_env_bytes(0, 10)
    assert e.value.status == -1
    assert "bad arguments" in str(e.value)
    assert lib.hs_destroy(None) == 0


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(L.HsError):
        saved = L._lib
        L._lib = None
        try:
            L.load(str(tmp_path / "nope.so"))
        finally:
            L._lib = saved


def test_struct_layouts_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the C compiler gives the
    struct of include/hs.h (tests/abi_layout.c, built with the host compiler)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    here = os.path.dirname(os.path.abspath(__file__))
    exe = str(tmp_path / "abi_layout")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(os.path.dirname(here), "include"),
                    os.path.join(here, "abi_layout.c"), "-o", exe], check=True)
    lines = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    c_side = {ln.split()[0]: [int(x) for x in ln.split()[1:]] for ln in lines if ln.strip()}
    structs = {"hs_z2_tensor": L.Z2Tensor, "hs_env": L.Env, "hs_move_info": L.MoveInfo,
               "hs_hotrg_info": L.HotrgInfo, "hs_env4": L.Env4, "hs_move4_info": L.Move4Info}
    for name, cls in structs.items():
        size, *offsets = c_side[name]
        assert ctypes.sizeof(cls) == size, name
        assert [getattr(cls, f).offset for f, _ in cls._fields_] == offsets, name


def _zero_args(argtypes):
    out = []
    for a in argtypes:
        if a in (ctypes.c_int, ctypes.c_uint, ctypes.c_long, ctypes.c_ulong):
            out.append(0)
        elif a is ctypes.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


def test_null_context_is_an_error_not_a_crash(lib):
    """Every call that takes a context, given a null context (and null buffers, zero sizes),
    returns HS_ERR_INVALID_ARG and leaves a message, before touching any device state; the calls
    without a context reject null output pointers and empty batches the same way."""
    taking_ctx = [n for n, (_, args) in L._PROTOS.items() if args and args[0] is ctypes.c_void_p
                  and n not in ("hs_destroy",)]
    assert len(taking_ctx) >= 24
    for name in taking_ctx:
        _, args = L._PROTOS[name]
        assert getattr(lib, name)(*_zero_args(args)) == -1, name
        assert "null context" in lib.hs_last_error().decode(), name
    for name, msg in (("hs_create", "null output pointer"), ("hs_ctmrg_move_batched", "bad arguments"),
                      ("hs_workspace_query", "bad arguments"), ("hs_env_bytes", "bad arguments")):
        assert getattr(lib, name)(*_zero_args(L._PROTOS[name][1])) == -1, name
        assert msg in lib.hs_last_error().decode(), name
    assert lib.hs_destroy(None) == 0


def test_byte_counts_of_invalid_sizes_are_zero(lib):
    assert L.hs_z2_tensor_bytes(0, L.HS_BASIS_HERMITIAN) == 0
    assert lib.hs_z2_tensor_bytes(3, L.HS_BASIS_HERMITIAN, 99) == 0
    assert lib.hs_hotrg_tensor_bytes(0, 16) == 0 and lib.hs_hotrg_tensor_bytes(2, 0) == 0
    assert lib.hs_hotrg_tensor_bytes(2, 16) == 16 ** 4 * 8 and lib.hs_hotrg_tensor_bytes(5, 16) == 25 ** 4 * 8


def test_hotrg_log_z(lib):
    """hs_hotrg_log_z (host only): ln Z / N from the normalisation logs of a run and the last trace,
    against the sum written out term by term (the factor of step k is shared by 2^k sites), and
    its error statuses."""
    import math
    ln = [0.7, 1.1, -2.3, 4.9]
    want = 0.7 + 1.1 / 2 - 2.3 / 4 + 4.9 / 8 + math.log(3.5) / 8
    assert L.hs_hotrg_log_z(ln, 3.5) == pytest.approx(want, rel=1e-15)
    assert L.hs_hotrg_log_z([0.2, 0.4], 2.0) == pytest.approx(0.2 + 0.2 + math.log(2.0) / 2, rel=1e-15)
    # thirty steps: the last trace weighs 2^-30
    ln30 = [0.5] + [0.25] * 30
    assert L.hs_hotrg_log_z(ln30, 7.0) == pytest.approx(0.5 + 0.25 * (1 - 2.0 ** -30) + math.log(7.0) * 2.0 ** -30,
                                                         rel=1e-15)
    for log_norms, trace, status in (([0.1], 1.0, -1), ([0.1, 0.2], 0.0, -8), ([0.1, 0.2], -1.0, -8),
                                     ([0.1, float("nan")], 1.0, -8), ([0.1, 0.2], float("inf"), -8)):
        with pytest.raises(L.HsError) as e:
            L.hs_hotrg_log_z(log_norms, trace)
        assert e.value.status == status, (log_norms, trace)


def test_workspace_query_is_the_stated_estimate(lib):
    """hs_workspace_query (host only): two (chi D^2)^2 ping-pong buffers and three chi^2 D^2 ones,
    chi at least D^2, in doubles."""
    for D, chi in ((2, 16), (6, 144), (7, 196), (3, 4)):
        q, c = D * D, max(chi, D * D)
        out = ctypes.c_size_t()
        assert lib.hs_workspace_query(D, chi, 0, ctypes.byref(out)) == 0
        assert out.value == 8 * (2 * (c * q) ** 2 + 3 * c * c * q)
