"""The register-resident Jacobi's pairing order, checked on the host: the
kernel's own index functions (csrc/jacobi_order.h) compiled with the host
compiler and driven through three sweeps for every c = 1..160 (every move a
permutation, every pair of columns once per sweep)."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


def test_jacobi_pairing_order_is_a_tournament(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = tmp_path / "jacobi_order_check"
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", str(ROOT / "paper_2302_07084_gb300" / "csrc"),
                    str(ROOT / "tests" / "cpp" / "jacobi_order_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip().endswith("ok")
