"""The product kernels' unit decoding on the host: multiply-high division by invariant divisors
(Granlund and Montgomery) against integer division, the 32-bit member orders against the 64-bit
member_tile, and the kept-A strips covering every (modulus, tile) once (tests/decode/decode_check.cu,
built host-only with nvcc)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"), reason="no nvcc")
def test_unit_decoding_helpers():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out_dir = os.path.join(HERE, "decode", "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "decode_check")
    src = os.path.join(HERE, "decode", "decode_check.cu")
    b = subprocess.run([nvcc, "-O2", "-std=c++17", src, "-o", exe], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:]
    assert "mismatches 0" in r.stdout
