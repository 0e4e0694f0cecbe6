"""torch.autograd.Function over the C ABI: C = A @ B with a hand-written backward.

Forward calls momms_gemm_ex, backward calls momms_gemm_backward, which computes
dA = dC B^T and dB = A^T dC through the transposed-operand paths of the kernels
(no transposed copies).  Tensors are ordinary row-major torch float64 CUDA
tensors; a row-major (r x c) tensor is the column-major (c x r) matrix of the
C ABI, so the product is issued as C^T = B^T A^T.
"""
from __future__ import annotations

import threading

import torch

from . import momms as M

_local = threading.local()


def _handle(mode):
    """The handle of this thread for (current device, mode): a handle holds per-call state (report,
    workspace, status word) and belongs to one thread and one device."""
    key = (torch.cuda.current_device(), mode)
    handles = getattr(_local, "handles", None)
    if handles is None:
        handles = _local.handles = {}
    h = handles.get(key)
    if h is None:
        h = M.Handle(mode=mode)
        handles[key] = h
    return h


def _check2d(t, name):
    if t.dim() != 2 or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a 2-D float64 CUDA tensor")
    return t.contiguous()


class MommsMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, mode=M.MODE_AUTO):
        A = _check2d(A, "A")
        B = _check2d(B, "B")
        m, k = A.shape
        k2, n = B.shape
        if k != k2:
            raise ValueError("inner dimensions differ")
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
        h = _handle(mode)
        # column-major view: C^T (n x m, ld n) = B^T (n x k, ld n) * A^T (k x m, ld k)
        M.check(M.momms_gemm_ex(h, M.OP_N, M.OP_N, n, m, k, 1.0, B.data_ptr(), max(n, 1), A.data_ptr(),
                                max(k, 1), 0.0, C.data_ptr(), max(n, 1)), "momms_gemm_ex")
        ctx.save_for_backward(A, B)
        ctx.mode = mode
        return C

    @staticmethod
    def backward(ctx, dC):
        A, B = ctx.saved_tensors
        dC = dC.contiguous()
        m, k = A.shape
        n = B.shape[1]
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dA = torch.empty_like(A) if need_a else None
        dB = torch.empty_like(B) if need_b else None
        h = _handle(ctx.mode)
        # In the column-major view the forward product is C' = A' B' with A' = B^T (n x k),
        # B' = A^T (k x m), C' = C^T; its gradients dA' = dC' B'^T = (dB)^T and
        # dB' = A'^T dC' = (dA)^T are exactly the memory of row-major dB and dA.
        M.check(M.momms_gemm_backward(h, n, m, k, B.data_ptr(), max(n, 1), A.data_ptr(), max(k, 1),
                                      dC.data_ptr(), max(n, 1),
                                      dB.data_ptr() if need_b else 0, max(n, 1),
                                      dA.data_ptr() if need_a else 0, max(k, 1)), "momms_gemm_backward")
        return dA, dB, None


def matmul(A, B, mode=M.MODE_AUTO):
    """C = A @ B (float64 CUDA tensors), differentiable."""
    return MommsMatmul.apply(A, B, mode)
