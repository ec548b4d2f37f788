"""df64::from_double (the integer-instruction FP64 -> FP32-pair split that
the FP32 / DF64 residual reads) compiled for the host and checked against its
documented bound: hi is the nearest FP32 value, |v - (hi + lo)| <= 2^-48 |v|
over the FP32 range, special cases as documented.  CPU only (nvcc compiles the
header's host path)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_integer_split_meets_its_bound(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "df64_split")
    src = os.path.join(ROOT, "tests", "host", "df64_split.cu")
    inc = os.path.join(ROOT, "paper_2402_02273_gb300", "csrc")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + inc, src, "-o", exe], check=True, capture_output=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
