"""Full-size workloads in the launch configuration the benchmark times, checked on
sampled rows and columns against the oracle (each sampled output computed by the
oracle from its own row/column of the inputs), plus Freivalds' check on all of C."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import bound

pytestmark = pytest.mark.gpu


def sample_ratio(A, B, C0, C, alpha, beta, nrows=24, ncols=24, seed=1):
    m, k = A.shape
    n = B.shape[1]
    rs = np.unique((syn.unit_uniform(seed, nrows) * m).astype(np.int64))
    cs = np.unique((syn.unit_uniform(seed + 1, ncols) * n).astype(np.int64))
    rs = np.unique(np.concatenate([rs, [0, m - 1]]))
    cs = np.unique(np.concatenate([cs, [0, n - 1]]))
    worst = 0.0
    Ar = np.asfortranarray(A[rs, :])
    C0r = np.asfortranarray(C0[rs, :])
    ref = oracle.dgemm(Ar, B, C0r.copy(order="F"), alpha, beta)
    N = oracle.dgemm_abs(Ar, B)
    worst = max(worst, float(np.max(np.abs(C[rs, :] - ref) / bound(k, alpha, beta, N, C0r))))
    Bc = np.asfortranarray(B[:, cs])
    C0c = np.asfortranarray(C0[:, cs])
    ref = oracle.dgemm(A, Bc, C0c.copy(order="F"), alpha, beta)
    N = oracle.dgemm_abs(A, Bc)
    worst = max(worst, float(np.max(np.abs(C[:, cs] - ref) / bound(k, alpha, beta, N, C0c))))
    return worst


def freivalds_ok(A, B, C0, C, alpha, beta, seed=7):
    """alpha*A(Bx) + beta*C0 x against Cx, with the bound propagated through |.|."""
    n = B.shape[1]
    k = A.shape[1]
    x = syn.uniform_pm1(seed, n)
    lhs = C @ x
    rhs = alpha * (A @ (B @ x)) + beta * (C0 @ x)
    mag = np.abs(alpha) * (np.abs(A) @ (np.abs(B) @ np.abs(x))) + abs(beta) * (np.abs(C0) @ np.abs(x))
    tol = 4.0 * (k + n) * 2.0 ** -53 * mag * 2.0 + 1e-300
    return bool(np.all(np.abs(lhs - rhs) <= tol))


def run(A, B, C0, mode, slices=0, alpha=1.0, beta=1.0, scheme=M.SCHEME_AUTO):
    h = M.Handle(mode=mode, slices=slices, scheme=scheme)
    dA, dB, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, alpha, beta, handle=h)
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    h.close()
    out = dC.to_numpy()
    del dA, dB, dC
    return out, rep


def test_square_8192_auto_as_benchmarked():
    # the benchmark's workload and launch configuration: AUTO plan (emulated, data-driven S)
    n = 8192
    A = syn.matrix("uniform", n, n, syn.workload_seed(1, "A"))
    B = syn.matrix("uniform", n, n, syn.workload_seed(1, "B"))
    C0 = syn.matrix("uniform", n, n, syn.workload_seed(1, "C"))
    C, rep = run(A, B, C0, M.MODE_AUTO)
    assert rep["mode"] == M.MODE_EMULATED and rep["moduli"] > 0
    assert sample_ratio(A, B, C0, C, 1.0, 1.0) <= 1.0
    assert freivalds_ok(A, B, C0, C, 1.0, 1.0)
    # sampled elements bit for bit against the definition of the modular result: the exact
    # product of the truncated rows and columns (their exponents span the whole k), rounded once
    rs = np.array([0, 4095, 8191])
    cs = np.array([0, 5000, 8191])
    Co, _ = oracle.modular_dgemm(np.asfortranarray(A[rs, :]), np.asfortranarray(B[:, cs]), rep["operand_bits"],
                                 np.asfortranarray(C0[np.ix_(rs, cs)]), 1.0, 1.0)
    assert np.array_equal(C[np.ix_(rs, cs)], Co)


def test_square_16384_auto_as_benchmarked():
    # the largest square of the shape sweep (bench --size 16384): AUTO plan as timed; 26 sampled rows
    # and columns against the oracle, Freivalds on all of C, sampled elements bit for bit against the
    # definition of the modular result
    n = 16384
    A = syn.matrix("uniform", n, n, syn.workload_seed(1, "A"))
    B = syn.matrix("uniform", n, n, syn.workload_seed(1, "B"))
    C0 = syn.matrix("uniform", n, n, syn.workload_seed(1, "C"))
    C, rep = run(A, B, C0, M.MODE_AUTO)
    assert rep["mode"] == M.MODE_EMULATED and rep["moduli"] > 0
    assert sample_ratio(A, B, C0, C, 1.0, 1.0) <= 1.0
    assert freivalds_ok(A, B, C0, C, 1.0, 1.0)
    rs = np.array([0, 127, 128, 9000, 16383])
    cs = np.array([0, 191, 192, 12345, 16383])
    Co, _ = oracle.modular_dgemm(np.asfortranarray(A[rs, :]), np.asfortranarray(B[:, cs]), rep["operand_bits"],
                                 np.asfortranarray(C0[np.ix_(rs, cs)]), 1.0, 1.0)
    assert np.array_equal(C[np.ix_(rs, cs)], Co)


def test_square_8192_slices():
    n = 8192
    A = syn.matrix("uniform", n, n, syn.workload_seed(1, "A"))
    B = syn.matrix("uniform", n, n, syn.workload_seed(1, "B"))
    C0 = syn.matrix("uniform", n, n, syn.workload_seed(1, "C"))
    C, rep = run(A, B, C0, M.MODE_EMULATED, scheme=M.SCHEME_SLICES)
    assert rep["moduli"] == 0
    assert sample_ratio(A, B, C0, C, 1.0, 1.0) <= 1.0
    assert freivalds_ok(A, B, C0, C, 1.0, 1.0)


def test_square_8192_native():
    n = 8192
    A = syn.matrix("uniform", n, n, syn.workload_seed(1, "A"))
    B = syn.matrix("uniform", n, n, syn.workload_seed(1, "B"))
    C0 = syn.matrix("uniform", n, n, syn.workload_seed(1, "C"))
    C, rep = run(A, B, C0, M.MODE_NATIVE)
    assert rep["mode"] == M.MODE_NATIVE
    assert sample_ratio(A, B, C0, C, 1.0, 1.0) <= 1.0


@pytest.mark.parametrize("phi", [0.0, 1.0, 4.0])
def test_phi_workload_8192_auto_slices(phi):
    # entries (u - 0.5) exp(phi g): the slice count chosen from the data must meet the bound
    n = 8192
    A = syn.matrix("phi", n, n, syn.workload_seed(3, "A"), phi=phi)
    B = syn.matrix("phi", n, n, syn.workload_seed(3, "B"), phi=phi)
    C0 = np.zeros((n, n), order="F")
    C, rep = run(A, B, C0, M.MODE_EMULATED, 0, 1.0, 0.0)
    assert 5 <= rep["slices"] <= 12
    assert sample_ratio(A, B, C0, C, 1.0, 0.0, 16, 16) <= 1.0


@pytest.mark.parametrize("shape", [(16384, 16384, 256), (16384, 256, 16384)])
@pytest.mark.parametrize("mode", [M.MODE_EMULATED, M.MODE_NATIVE])
def test_rank_k_and_panel_panel(shape, mode):
    m, n, k = shape
    A = syn.matrix("uniform", m, k, syn.workload_seed(1, "A") + m)
    B = syn.matrix("uniform", k, n, syn.workload_seed(1, "B") + n)
    C0 = syn.matrix("uniform", m, n, syn.workload_seed(1, "C") + k)
    C, _ = run(A, B, C0, mode)
    assert sample_ratio(A, B, C0, C, 1.0, 1.0, 16, 16) <= 1.0


def test_syrk_8192_as_benchmarked():
    # the benchmark's SYRK workload (C lower += A A^T, n = k = 8192, AUTO plan): the modular
    # encoding over the triangle's tiles; sampled lower-triangle elements bit for bit against the
    # definition of the modular result, the upper triangle untouched
    n = 8192
    A = syn.matrix("uniform", n, n, syn.workload_seed(6, "A"))
    C0 = syn.matrix("uniform", n, n, syn.workload_seed(6, "C"))
    h = M.Handle()
    dA, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(C0)
    M.check(M.momms_syrk(h, M.LOWER, M.OP_N, n, n, 1.0, dA.ptr, dA.ld, 1.0, dC.ptr, dC.ld), "syrk")
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    h.close()
    C = dC.to_numpy()
    del dA, dC
    assert rep["mode"] == M.MODE_EMULATED and rep["moduli"] > 0
    up = np.triu(np.ones((n, n), bool), 1)
    assert np.array_equal(C[up], C0[up])
    rs = np.array([0, 127, 128, 4095, 5000, 8191])
    cs = np.array([0, 127, 191, 192, 4095, 8191])
    Co, _ = oracle.modular_dgemm(np.asfortranarray(A[rs, :]), np.asfortranarray(A[cs, :].T), rep["operand_bits"],
                                 np.asfortranarray(C0[np.ix_(rs, cs)]), 1.0, 1.0)
    low = rs[:, None] >= cs[None, :]
    assert np.array_equal(C[np.ix_(rs, cs)][low], Co[low])
