"""Triangular solve B := alpha op(A)^-1 B or alpha B op(A)^-1 against the oracle's
substitution: every side / uplo / trans / diag, native and emulated, blocks of 128 with a
ragged last block, the triangle's outside (and a unit diagonal) never read.

The check is the componentwise residual of the computed X in exact arithmetic terms,
|op(A) X - alpha B| <= c t 2^-53 (|op(A)| |X| + |alpha B|) with c = 16 (the GEMM updates'
bound is 4k 2^-53 |.||.|; the 128 x 128 diagonal blocks are applied through FP64 inverses of
well-conditioned triangles), plus closeness to the oracle's X."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import F

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def triangle(t, seed, lower, unit):
    """A well-conditioned triangle: off-diagonal uniform[-1,1] / sqrt(t), diagonal in [1, 2];
    NaN outside the triangle (and on a unit diagonal): those entries must not be read."""
    A = syn.matrix("uniform", t, t, seed) / np.sqrt(t)
    A[np.diag_indices(t)] = 1.0 + syn.unit_uniform(seed + 1, t)
    keep = np.tril(np.ones((t, t), bool)) if lower else np.triu(np.ones((t, t), bool))
    if unit:
        keep[np.diag_indices(t)] = False
    return F(np.where(keep, A, np.nan)), A


def explicit(A, lower, unit):
    T = np.tril(A) if lower else np.triu(A)
    if unit:
        T = T.copy()
        np.fill_diagonal(T, 1.0)
    return T


def solve(mode, side, uplo, trans, diag, A, B0, alpha, S=0):
    m, n = B0.shape
    h = M.Handle(mode=mode, slices=S)
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B0)
    M.check(M.momms_trsm(h, side, uplo, trans, diag, m, n, alpha, dA.ptr, dA.ld, dB.ptr, dB.ld), "trsm")
    st = h.device_status()
    rep = h.report()
    h.close()
    assert st == M.MOMMS_OK
    return dB.to_numpy(), rep


def residual_ratio(Top, X, B0, alpha, side):
    """max |op(A) X - alpha B| / (t 2^-53 (|op(A)| |X| + |alpha B|)), products in FP64 by the oracle
    (their own rounding is a few units of the same scale)."""
    if side == M.LEFT:
        R = oracle.dgemm(F(Top), F(X)) - alpha * B0
        N = oracle.dgemm(F(np.abs(Top)), F(np.abs(X))) + abs(alpha) * np.abs(B0)
    else:
        R = oracle.dgemm(F(X), F(Top)) - alpha * B0
        N = oracle.dgemm(F(np.abs(X)), F(np.abs(Top))) + abs(alpha) * np.abs(B0)
    t = Top.shape[0]
    return float(np.max(np.abs(R) / (t * U * N + 1e-300)))


@pytest.mark.parametrize("mode", [M.MODE_NATIVE, M.MODE_EMULATED])
@pytest.mark.parametrize("side", [M.LEFT, M.RIGHT])
@pytest.mark.parametrize("uplo", [M.LOWER, M.UPPER])
@pytest.mark.parametrize("trans,diag", [(M.OP_N, M.NON_UNIT), (M.OP_T, M.UNIT), (M.OP_T, M.NON_UNIT)])
def test_trsm_matches_oracle(mode, side, uplo, trans, diag):
    m, n = 300, 260                     # t = 300 (LEFT) or 260 (RIGHT): blocks 128, 128, ragged
    t = m if side == M.LEFT else n
    lower, unit = uplo == M.LOWER, diag == M.UNIT
    A_nan, A = triangle(t, 1401 + 10 * side + 3 * uplo, lower, unit)
    B0 = syn.matrix("uniform", m, n, 1402)
    X, rep = solve(mode, side, uplo, trans, diag, A_nan, B0, -1.5)
    T = explicit(A, lower, unit)
    Top = T.T if trans == M.OP_T else T
    assert residual_ratio(Top, X, B0, -1.5, side) <= 16.0
    Xo = oracle.trsm(A, B0, -1.5, "L" if side == M.LEFT else "R", lower, trans == M.OP_T, unit)
    assert np.max(np.abs(X - Xo)) <= 1e-11 * np.max(np.abs(Xo))
    assert rep["launches"] >= 3


def test_trsm_larger_emulated_updates_and_integer_exact():
    # t = 1024: the top update is a 512 x 512 x 512 product (emulated), eight leaf blocks
    m, n = 1024, 512
    A_nan, A = triangle(m, 1411, True, False)
    B0 = syn.matrix("uniform", m, n, 1412)
    X, _ = solve(M.MODE_AUTO, M.LEFT, M.LOWER, M.OP_N, M.NON_UNIT, A_nan, B0, 1.0)
    T = explicit(A, True, False)
    assert residual_ratio(T, X, B0, 1.0, M.LEFT) <= 16.0
    # unit triangle of small integers with an integer solution, built so that every step is
    # exact: random {-1, 0, 1} between the 128-blocks (the GEMM updates), a {-1, 1} subdiagonal
    # inside them (their inverses have entries in {-1, 0, 1})
    t, r = 384, 200
    rng = np.random.default_rng(1413)
    blk = np.arange(t) // 128
    Ai = np.where(blk[:, None] > blk[None, :], rng.integers(-1, 2, (t, t)), 0).astype(np.float64)
    sub = np.arange(1, t)
    inside = blk[sub] == blk[sub - 1]
    Ai[sub[inside], sub[inside] - 1] = rng.choice([-1.0, 1.0], inside.sum())
    Ai = F(Ai + np.eye(t))
    Xi = F(rng.integers(-2, 3, (t, r)).astype(np.float64))
    Bi = F(Ai @ Xi)
    assert np.max(np.abs(Bi)) < 2 ** 40
    for mode, S in ((M.MODE_NATIVE, 0), (M.MODE_EMULATED, 7)):
        got, _ = solve(mode, M.LEFT, M.LOWER, M.OP_N, M.UNIT, Ai, Bi, 1.0, S)
        assert np.array_equal(got, Xi), mode


def test_trsm_alpha_zero_and_errors():
    m, n = 130, 70
    A_nan, _ = triangle(m, 1421, True, False)
    B0 = syn.matrix("uniform", m, n, 1422)
    X, _ = solve(M.MODE_NATIVE, M.LEFT, M.LOWER, M.OP_N, M.NON_UNIT, A_nan, B0, 0.0)
    assert np.array_equal(X, np.zeros_like(B0))
    h = M.Handle()
    assert M.momms_trsm(h, 2, 0, 0, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -2
    assert M.momms_trsm(h, 0, 2, 0, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -3
    assert M.momms_trsm(h, 0, 0, 2, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -4
    assert M.momms_trsm(h, 0, 0, 0, 2, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -5
    assert M.momms_trsm(h, 1, 0, 0, 0, 4, 8, 1.0, 1 << 40, 7, 1 << 41, 4) == -10
    assert M.momms_trsm(h, 0, 0, 0, 0, 8, 4, 1.0, 1 << 40, 8, 1 << 41, 7) == -12
    h.close()
