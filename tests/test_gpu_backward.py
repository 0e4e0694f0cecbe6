"""Backward pass (dA = dC B^T, dB = A^T dC) through the autograd.Function and the C ABI:
central finite differences and the oracle's gradients."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("mode", [M.MODE_NATIVE, M.MODE_EMULATED])
def test_autograd_finite_differences(mode):
    # m = 64, k = 48, n = 32, h = 1e-6 on the bilinear loss L = <G, A B>
    import torch

    from paper_1904_05717_gb300.autograd import matmul
    m, k, n, h = 64, 48, 32, 1e-6
    A = _t(syn.matrix("normal", m, k, 201))
    B = _t(syn.matrix("normal", k, n, 202))
    G = _t(syn.matrix("normal", m, n, 203))
    A.requires_grad_(True)
    B.requires_grad_(True)
    L = (G * matmul(A, B, mode)).sum()
    L.backward()
    dA, dB = A.grad.detach().clone(), B.grad.detach().clone()
    with torch.no_grad():
        for X, dX, seed in ((A, dA, 204), (B, dB, 205)):
            V = _t(syn.matrix("normal", X.shape[0], X.shape[1], seed))
            Xp, Xm = X + h * V, X - h * V
            Lp = (G * (matmul(Xp, B, mode) if X is A else matmul(A, Xp, mode))).sum()
            Lm = (G * (matmul(Xm, B, mode) if X is A else matmul(A, Xm, mode))).sum()
            fd = float((Lp - Lm) / (2 * h))
            ana = float((dX * V).sum())
            assert abs(fd - ana) <= 1e-6 * (abs(ana) + 1.0), (fd, ana)
            # single entries as well
            for (i, j) in ((0, 0), (X.shape[0] - 1, X.shape[1] - 1), (5, 3)):
                E = torch.zeros_like(X)
                E[i, j] = 1.0
                Lp = (G * (matmul(X + h * E, B, mode) if X is A else matmul(A, X + h * E, mode))).sum()
                Lm = (G * (matmul(X - h * E, B, mode) if X is A else matmul(A, X - h * E, mode))).sum()
                fd = float((Lp - Lm) / (2 * h))
                assert abs(fd - float(dX[i, j])) <= 1e-6 * (abs(float(dX[i, j])) + 1.0)
    # and the analytical gradients equal the oracle's within the bound
    Ah, Bh, Gh = (np.asfortranarray(t.detach().cpu().numpy()) for t in (A, B, G))
    dA_ref = oracle.dgemm(Gh, Bh, transb=True)
    dB_ref = oracle.dgemm(Ah, Gh, transa=True)
    assert max_ratio(dA.cpu().numpy(), dA_ref, n, 1.0, 0.0, oracle.dgemm_abs(Gh, Bh, transb=True)) <= 1.0
    assert max_ratio(dB.cpu().numpy(), dB_ref, m, 1.0, 0.0, oracle.dgemm_abs(Ah, Gh, transa=True)) <= 1.0


@pytest.mark.parametrize("mode", [M.MODE_NATIVE, M.MODE_EMULATED])
def test_backward_config3_full_size(mode):
    # A 4096 x 2048, B 2048 x 4096, dC 4096 x 4096, standard normal; full oracle comparison
    m, k, n = 4096, 2048, 4096
    A = syn.matrix("normal", m, k, syn.workload_seed(2, "A"))
    B = syn.matrix("normal", k, n, syn.workload_seed(2, "B"))
    G = syn.matrix("normal", m, n, syn.workload_seed(2, "dC"))
    h = M.Handle(mode=mode)
    dA_, dB_, dG = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(G)
    gA, gB = M.DeviceMatrix(m, k), M.DeviceMatrix(k, n)
    M.check(M.momms_gemm_backward(h, m, n, k, dA_.ptr, dA_.ld, dB_.ptr, dB_.ld, dG.ptr, dG.ld,
                                  gA.ptr, gA.ld, gB.ptr, gB.ld), "backward")
    assert h.device_status() == M.MOMMS_OK
    dA_ref = oracle.dgemm(G, B, transb=True)
    dB_ref = oracle.dgemm(A, G, transa=True)
    assert max_ratio(gA.to_numpy(), dA_ref, n, 1.0, 0.0, oracle.dgemm_abs(G, B, transb=True)) <= 1.0
    assert max_ratio(gB.to_numpy(), dB_ref, m, 1.0, 0.0, oracle.dgemm_abs(A, G, transa=True)) <= 1.0


def test_backward_null_gradients_are_skipped():
    m, k, n = 50, 40, 30
    A = syn.matrix("normal", m, k, 211)
    B = syn.matrix("normal", k, n, 212)
    G = syn.matrix("normal", m, n, 213)
    h = M.Handle(mode=M.MODE_NATIVE)
    dA_, dB_, dG = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(G)
    gB = M.DeviceMatrix(k, n)
    M.check(M.momms_gemm_backward(h, m, n, k, dA_.ptr, dA_.ld, dB_.ptr, dB_.ld, dG.ptr, dG.ld, 0, m,
                                  gB.ptr, gB.ld), "backward dB only")
    dB_ref = oracle.dgemm(A, G, transa=True)
    assert max_ratio(gB.to_numpy(), dB_ref, m, 1.0, 0.0, oracle.dgemm_abs(A, G, transa=True)) <= 1.0
