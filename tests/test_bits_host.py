"""Host check of the bit-level helpers used by the CUDA kernels (hs_bits.cuh):
division by invariant integers for the permute index decode, the FP64 -> TF32/BF16
hi+lo operand split and the FP32 -> FP64 widening of the tensor-core epilogue,
each against an independent reference (tests/bits_check.cpp)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2410_11596_gb300", "csrc")


def test_bit_helpers(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "bits_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "bits_check.cpp"), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
