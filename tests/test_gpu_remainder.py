"""Device check of the exact 64-by-32 remainder that hash_crc (Fig. 3) takes on 32-bit
positions: its reciprocal for every normalised divisor and the remainder on 2^32 random
pairs, against the integer division that defines them (tests/device/remainder_check.cu)."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_crc_remainder_reciprocal_exhaustive_and_remainder_on_random_pairs():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = os.path.join(ROOT, "tests", "device", "remainder_check.cu")
    out_dir = os.path.join(ROOT, "tests", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "remainder_check")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                    "-I", os.path.join(ROOT, "paper_1602_07106_gb300", "csrc"), "-o", exe, src],
                   check=True, capture_output=True, text=True)
    res = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "reciprocal mismatches 0" in res.stdout and "remainder mismatches 0" in res.stdout
