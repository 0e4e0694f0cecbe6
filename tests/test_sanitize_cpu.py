"""Host-side AddressSanitizer / UndefinedBehaviorSanitizer runs (CPU only):

* the oracle's C code, driven by tests/sanitize/oracle_driver.c over every entry point on
  empty, single-element, ragged and padded shapes, both transposes and non-finite values;
* the C-ABI library's host code (all of csrc compiled with the sanitizers), driven by
  tests/sanitize/abi_driver.cpp over the paths that need no GPU: argument validation, null
  handles, handle creation failing cleanly without a device, the moduli planning call over
  its range, the tile-order queries and the status strings.

Any finding (out-of-bounds access, leak, overflow, invalid shift) fails the run.  Skipped
where the toolchain has no sanitizer runtime."""
import glob
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BUILD = os.path.join(ROOT, "tests", "sanitize", "_build")
# separate flags: nvcc's -Xcompiler takes a comma-separated list
SAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")


def _have(tool):
    return shutil.which(tool) is not None


def _run(cmd, **kw):
    return subprocess.run(cmd, capture_output=True, text=True, **kw)


@pytest.mark.skipif(not _have("gcc"), reason="no gcc")
def test_oracle_under_sanitizers():
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "oracle_driver")
    r = _run(["gcc", "-O1", "-g", "-ffp-contract=off", "-std=gnu11", *SAN,
              os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"), os.path.join(ROOT, "oracle", "momms_oracle.c"),
              "-lm", "-o", exe])
    if r.returncode != 0 and "asan" in (r.stderr + r.stdout).lower():
        pytest.skip("no sanitizer runtime: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr
    run = _run([exe], env=ENV, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "all calls clean" in run.stdout


@pytest.mark.skipif(not _have("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"), reason="no nvcc")
def test_abi_host_code_under_sanitizers():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    obj = os.path.join(BUILD, "obj")
    os.makedirs(obj, exist_ok=True)
    host = ["-Xcompiler", ",".join(["-fPIC", *SAN])]
    common = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-g", "-std=c++17", *host,
              "-I", os.path.join(ROOT, "include")]
    procs = []
    for src in sorted(glob.glob(os.path.join(ROOT, "paper_1904_05717_gb300", "csrc", "*.cu"))):
        out = os.path.join(obj, os.path.basename(src)[:-3] + ".o")
        procs.append((src, subprocess.Popen(common + ["-c", src, "-o", out], stdout=subprocess.PIPE,
                                            stderr=subprocess.PIPE, text=True)))
    for src, p in procs:
        _, err = p.communicate(timeout=600)
        assert p.returncode == 0, f"{src}: {err[-2000:]}"
    exe = os.path.join(BUILD, "abi_driver")
    r = _run(common + [os.path.join(ROOT, "tests", "sanitize", "abi_driver.cpp"),
                       *sorted(glob.glob(os.path.join(obj, "*.o"))), "-o", exe], timeout=600)
    if r.returncode != 0 and "asan" in (r.stderr + r.stdout).lower():
        pytest.skip("no sanitizer runtime: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-2000:]
    run = _run([exe], env=ENV, timeout=300)
    assert run.returncode == 0, run.stdout + run.stderr[-4000:]
    assert "all calls clean" in run.stdout
