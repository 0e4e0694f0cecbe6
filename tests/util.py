"""Shared helpers of the test suite (host side)."""
import numpy as np

import oracle

U = 2.0 ** -53


def F(x):
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def bound(k, alpha, beta, N, C0=None):
    """Componentwise error bound of the product (the reading of the stated bound
    4k 2^-53 |A||B| extended to alpha, beta and the initial C):
        4 max(k,1) u (|alpha| N + |beta| |C0|) (1 + 4ku) + 2^-1021."""
    kk = max(int(k), 1)
    t = abs(alpha) * N
    if C0 is not None and beta != 0.0:
        t = t + abs(beta) * np.abs(C0)
    return 4.0 * kk * U * t * (1.0 + 4.0 * kk * U) + 2.0 ** -1021


def max_ratio(C, Cref, k, alpha, beta, N, C0=None):
    b = bound(k, alpha, beta, N, C0)
    return float(np.max(np.abs(C - Cref) / b)) if C.size else 0.0


def reference(A, B, C0=None, alpha=1.0, beta=0.0, transa=False, transb=False):
    """Oracle result, magnitude matrix N and the initial C."""
    Cref = oracle.dgemm(A, B, None if C0 is None else C0.copy(order="F"), alpha, beta, transa, transb)
    N = oracle.dgemm_abs(A, B, transa, transb)
    return Cref, N
