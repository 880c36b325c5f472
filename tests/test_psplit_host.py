"""Host check of the destination map of the tensor-core GEMM's split epilogue
(the outputs X2, X3, Y, Z written as the next GEMM's permuted split operand)
against the permute plan of the same layouts (tests/psplit_map_check.cu)."""
import os
import shutil
import subprocess

import pytest

from paper_2410_11596_gb300 import _lib as L, build

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2410_11596_gb300", "csrc")


def test_psplit_destination_map(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("no nvcc")
    if not os.path.exists(L.LIB_PATH) or any(
            os.path.getmtime(s) > os.path.getmtime(L.LIB_PATH) for s in build.sources()):
        build.build()
    libdir = os.path.dirname(L.LIB_PATH)
    exe = tmp_path / "psplit_map_check"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, os.path.join(HERE, "psplit_map_check.cu"), "-o", str(exe),
                    "-L", libdir, "-lhs", "-Xlinker", "-rpath=" + libdir], check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
