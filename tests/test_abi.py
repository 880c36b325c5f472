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
    assert lib.hs_abi_version() == 4


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
