"""Triangular product B := alpha op(A) B or alpha B op(A), A triangular: against the oracle's
product with the explicit triangle (the other triangle zero, a unit diagonal as ones), native
and emulated, every side / uplo / trans / diag."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import F, max_ratio, reference

pytestmark = pytest.mark.gpu


def explicit(A, uplo, diag):
    T = np.tril(A) if uplo == M.LOWER else np.triu(A)
    if diag == M.UNIT:
        np.fill_diagonal(T, 1.0)
    return F(T)


def trmm(mode, S, side, uplo, trans, diag, A, B0, alpha, scheme=M.SCHEME_AUTO, tile_n=0):
    m, n = B0.shape
    h = M.Handle(mode=mode, slices=S, scheme=scheme)
    if tile_n:
        h.set_tile_n(tile_n)
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B0)
    M.check(M.momms_trmm(h, side, uplo, trans, diag, m, n, alpha, dA.ptr, dA.ld, dB.ptr, dB.ld), "trmm")
    st = h.device_status()
    rep = h.report()
    h.close()
    assert st == M.MOMMS_OK
    return dB.to_numpy(), rep


@pytest.mark.parametrize("mode,S", [(M.MODE_NATIVE, 0), (M.MODE_EMULATED, 0)])
@pytest.mark.parametrize("side", [M.LEFT, M.RIGHT])
@pytest.mark.parametrize("uplo", [M.LOWER, M.UPPER])
@pytest.mark.parametrize("trans,diag", [(M.OP_N, M.NON_UNIT), (M.OP_T, M.UNIT)])
def test_trmm_matches_oracle(mode, S, side, uplo, trans, diag):
    m, n = 300, 260
    t = m if side == M.LEFT else n
    # the triangle's outside and (for a unit diagonal) its diagonal hold NaN: they must not be read
    A = syn.matrix("uniform", t, t, 1301)
    keep = np.tril(np.ones((t, t), bool)) if uplo == M.LOWER else np.triu(np.ones((t, t), bool))
    if diag == M.UNIT:
        np.fill_diagonal(keep, False)
    A_nan = F(np.where(keep, A, np.nan))
    B0 = syn.matrix("uniform", m, n, 1302)
    out, rep = trmm(mode, S, side, uplo, trans, diag, A_nan, B0, -1.5)
    assert rep["mode"] == mode
    T = explicit(A, uplo, diag)
    if side == M.LEFT:
        Cref, N = reference(T, B0, None, -1.5, 0.0, transa=(trans == M.OP_T))
        k = m
    else:
        Cref, N = reference(B0, T, None, -1.5, 0.0, transb=(trans == M.OP_T))
        k = n
    assert max_ratio(out, Cref, k, 1.5, 0.0, N) <= 1.0


def test_trmm_integer_exact_alpha_zero_and_errors():
    m, n = 200, 150
    A = syn.matrix("int", m, m, 1311)
    B0 = syn.matrix("int", m, n, 1312)
    exact = np.tril(A) @ B0
    for mode, S in ((M.MODE_NATIVE, 0), (M.MODE_EMULATED, 2)):
        out, _ = trmm(mode, S, M.LEFT, M.LOWER, M.OP_N, M.NON_UNIT, A, B0, 1.0)
        assert np.array_equal(out, exact)
    out, _ = trmm(M.MODE_EMULATED, 2, M.LEFT, M.LOWER, M.OP_N, M.NON_UNIT, A, B0, 0.0)
    assert np.array_equal(out, np.zeros_like(B0))
    h = M.Handle()
    assert M.momms_trmm(h, 2, 0, 0, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -2
    assert M.momms_trmm(h, 0, 2, 0, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -3
    assert M.momms_trmm(h, 0, 0, 0, 2, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4) == -5
    assert M.momms_trmm(h, 1, 0, 0, 0, 4, 8, 1.0, 1 << 40, 7, 1 << 41, 4) == -10
    assert M.momms_trmm(h, 0, 0, 0, 0, 8, 4, 1.0, 1 << 40, 8, 1 << 41, 7) == -12
    h.close()


@pytest.mark.parametrize("side", [M.LEFT, M.RIGHT])
@pytest.mark.parametrize("uplo", [M.LOWER, M.UPPER])
@pytest.mark.parametrize("trans", [M.OP_N, M.OP_T])
def test_trmm_moduli_skip_zero_k_bitwise(side, uplo, trans):
    # modular encoding: every tile's residue products skip the k range where op(A) is zero; the
    # skipped products are exact zeros, so B is bit for bit the oracle's modular result for the
    # explicit triangle (t = 200: a ragged second tile row of 72 and, right side, a ragged tile
    # column of 8 (192) or of 8 after two of 96)
    t, r = 200, 64
    m, n = (t, r) if side == M.LEFT else (r, t)
    A = syn.matrix("normal", t, t, 1331 + 4 * uplo + 2 * trans + side)
    B0 = syn.matrix("uniform", m, n, 1332)
    T = explicit(A, uplo, M.NON_UNIT)
    opT = F(T.T if trans == M.OP_T else T)
    if side == M.LEFT:
        want, _ = oracle.modular_dgemm(opT, B0, 42, None, 0.75, 0.0)
    else:
        want, _ = oracle.modular_dgemm(B0, opT, 42, None, 0.75, 0.0)
    for tile_n in (96, 192):
        out, rep = trmm(M.MODE_EMULATED, 6, side, uplo, trans, M.NON_UNIT, A, B0, 0.75, M.SCHEME_MODULI, tile_n)
        assert rep["moduli"] == 12 and rep["tile_n"] == tile_n
        assert np.array_equal(out, want), tile_n
