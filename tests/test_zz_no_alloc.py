"""The allocation-free emulated product against the allocating one.

momms_gemm_emulated_noalloc exists for callers that cannot allocate device memory
(graph capture in progress, allocator-less runtimes, pools that forbid outside
allocations): it runs the emulated path with all scratch in the library's static
device array.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes on its own in a fresh
process."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import bound

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    import torch
    m, n, k, S = 300, 500, 333, 10  # phi = 1 inputs at this k need S >= 9 for the bound
    A = syn.matrix("phi", m, k, 9001, phi=1.0)
    B = syn.matrix("phi", k, n, 9002, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 9003)
    alpha, beta = 1.25, -0.5
    tol = bound(k, alpha, beta, oracle.dgemm_abs(A, B), C0)
    Cref = oracle.dgemm(A, B, C0.copy(order="F"), alpha, beta)

    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    h = M.Handle(mode=M.MODE_EMULATED, slices=S)
    dC = M.DeviceMatrix.from_numpy(C0)
    M.check(M.momms_gemm_ex(h, 0, 0, m, n, k, alpha, dA.ptr, dA.ld, dB.ptr, dB.ld, beta, dC.ptr, dC.ld), "ex")
    existing = dC.to_numpy()
    assert np.all(np.abs(existing - Cref) <= tol)

    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        dN = M.DeviceMatrix.from_numpy(C0)
        M.check(M.momms_gemm_emulated_noalloc(0, 0, m, n, k, S, alpha, dA.ptr, dA.ld, dB.ptr, dB.ld, beta,
                                              dN.ptr, dN.ld), f"noalloc call {call}")
        rc, status = M.momms_noalloc_status()  # waits for the stream; no bounded wait ran out
        assert rc == M.MOMMS_OK and status == M.MOMMS_OK, (rc, status)
        torch.cuda.synchronize()
        got = dN.to_numpy()
        assert np.all(np.abs(got - existing) <= tol), f"call {call}"
        assert np.all(np.abs(got - Cref) <= tol), f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    cap = M.momms_noalloc_scratch_bytes()
    assert cap == 64 << 20
    n = 8192  # 8192^2 digits in 8 slices need far more than the static array holds
    rc = M.momms_gemm_emulated_noalloc(0, 0, n, n, n, 8, 1.0, 1 << 40, n, 1 << 41, n, 0.0, 1 << 42, n)
    assert rc == M.MOMMS_ERR_WORKSPACE
    assert M.momms_gemm_emulated_noalloc(0, 0, 8, 8, 8, 0, 1.0, 1 << 40, 8, 1 << 41, 8, 0.0, 1 << 42, 8) == -6
    # sizes whose byte counts would wrap 64-bit arithmetic are rejected before any offset is formed
    big = 1 << 40
    rc = M.momms_gemm_emulated_noalloc(0, 0, 8, 8, big, 16, 1.0, 1 << 40, 8, 1 << 41, big, 0.0, 1 << 42, 8)
    assert rc == M.MOMMS_ERR_WORKSPACE
    rc = M.momms_gemm_emulated_noalloc(0, 0, (1 << 31) + 1, 8, 8, 1, 1.0, 1 << 40, (1 << 31) + 1, 1 << 41, 8, 0.0,
                                       1 << 42, (1 << 31) + 1)
    assert rc == M.MOMMS_ERR_WORKSPACE


def test_noalloc_timeout_is_reported_and_cleared():
    # the timeout test hook (one stage of CTA 0 left empty, so a bounded wait runs out) on the
    # allocation-free entry point: momms_noalloc_status reports it once, and the next call is correct
    m, n, k, S = 200, 300, 256, 8
    A = syn.matrix("uniform", m, k, 9101)
    B = syn.matrix("uniform", k, n, 9102)
    C0 = syn.matrix("uniform", m, n, 9103)
    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    tol = bound(k, 1.0, 1.0, oracle.dgemm_abs(A, B), C0)
    Cref = oracle.dgemm(A, B, C0.copy(order="F"), 1.0, 1.0)
    for call in range(2):
        if call == 0:
            M.momms_debug_withhold_load()
        dN = M.DeviceMatrix.from_numpy(C0)
        M.check(M.momms_gemm_emulated_noalloc(0, 0, m, n, k, S, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0,
                                              dN.ptr, dN.ld), f"noalloc call {call}")
        rc, status = M.momms_noalloc_status()
        assert rc == M.MOMMS_OK
        if call == 0:
            assert status == M.MOMMS_ERR_TIMEOUT
            assert M.momms_noalloc_status() == (M.MOMMS_OK, M.MOMMS_OK)  # cleared by the read
        else:
            assert status == M.MOMMS_OK
            assert np.all(np.abs(dN.to_numpy() - Cref) <= tol)
