"""Symmetric rank-k update C := alpha op(A) op(A)^T + beta C on one triangle: the
referenced triangle against the oracle's product within the bound, the other triangle
untouched bit for bit, native and emulated (one split serving both operands; the slice
encoding's batched triangle and the modular encoding's triangle of residue products, the
latter bit for bit against the oracle's definition of the modular result)."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio, reference

pytestmark = pytest.mark.gpu


def syrk(mode, S, uplo, trans, A, C0, alpha, beta, scheme=M.SCHEME_AUTO, tile_n=0):
    n = C0.shape[0]
    k = A.shape[1] if trans == M.OP_N else A.shape[0]
    h = M.Handle(mode=mode, slices=S, scheme=scheme)
    if tile_n:
        h.set_tile_n(tile_n)
    dA = M.DeviceMatrix.from_numpy(A)
    dC = M.DeviceMatrix.from_numpy(C0)
    M.check(M.momms_syrk(h, uplo, trans, n, k, alpha, dA.ptr, dA.ld, beta, dC.ptr, dC.ld), "syrk")
    st = h.device_status()
    rep = h.report()
    h.close()
    assert st == M.MOMMS_OK
    return dC.to_numpy(), rep


def check(C, C0, A, trans, uplo, alpha, beta):
    n = C0.shape[0]
    k = A.shape[1] if trans == M.OP_N else A.shape[0]
    op = A if trans == M.OP_N else A.T
    Cref, N = reference(np.asfortranarray(op), np.asfortranarray(op.T), C0, alpha, beta)
    tri = np.tril(np.ones((n, n), bool)) if uplo == M.LOWER else np.triu(np.ones((n, n), bool))
    # the other triangle is neither read nor written
    assert np.array_equal(C[~tri], C0[~tri], equal_nan=True)
    Cm, Rm, Nm, C0m = (np.where(tri, X, 0.0) for X in (C, Cref, N, np.nan_to_num(C0)))
    assert max_ratio(np.asfortranarray(Cm), np.asfortranarray(Rm), k, abs(alpha), abs(beta),
                     np.asfortranarray(Nm), np.asfortranarray(C0m)) <= 1.0


@pytest.mark.parametrize("mode,S,scheme", [(M.MODE_NATIVE, 0, M.SCHEME_AUTO), (M.MODE_EMULATED, 8, M.SCHEME_AUTO),
                                           (M.MODE_EMULATED, 0, M.SCHEME_AUTO), (M.MODE_EMULATED, 8, M.SCHEME_SLICES)])
@pytest.mark.parametrize("uplo", [M.LOWER, M.UPPER])
@pytest.mark.parametrize("trans", [M.OP_N, M.OP_T])
def test_syrk_matches_oracle_on_its_triangle(mode, S, scheme, uplo, trans):
    n, k = 333, 275   # ragged: 3 row blocks of 128, 2 column tiles of 192
    A = syn.matrix("uniform", n, k, 1201) if trans == M.OP_N else syn.matrix("uniform", k, n, 1202)
    C0 = syn.matrix("uniform", n, n, 1203)
    C, rep = syrk(mode, S, uplo, trans, A, C0, 0.75, -1.25, scheme)
    assert rep["mode"] == mode
    if S == 8 and scheme == M.SCHEME_AUTO:
        assert rep["moduli"] == 16        # 56-bit operands: AUTO takes 16 moduli for 36 digit pairs
    if scheme == M.SCHEME_SLICES:
        assert rep["moduli"] == 0
    check(C, C0, A, trans, uplo, 0.75, -1.25)


@pytest.mark.parametrize("trans", [M.OP_N, M.OP_T])
def test_syrk_moduli_triangle_bitwise(trans):
    # n = 300: 3 tile rows of 128 (the last one 44 rows), 2 tile columns of 192 or 4 of 96, the
    # reconstruction four rows per thread; n = 299 (op T): one row per thread
    n, k = (300, 40) if trans == M.OP_N else (299, 40)
    A = syn.matrix("normal", n, k, 1231) if trans == M.OP_N else syn.matrix("normal", k, n, 1232)
    C0 = syn.matrix("uniform", n, n, 1233)
    op = np.asfortranarray(A if trans == M.OP_N else A.T)
    Co, _ = oracle.modular_dgemm(op, np.asfortranarray(op.T), 42, C0.copy(order="F"), 0.75, -1.25)
    for uplo in (M.LOWER, M.UPPER):
        tri = np.tril(np.ones((n, n), bool)) if uplo == M.LOWER else np.triu(np.ones((n, n), bool))
        for tile_n in (96, 192):
            C, rep = syrk(M.MODE_EMULATED, 6, uplo, trans, A, C0, 0.75, -1.25, M.SCHEME_MODULI, tile_n)
            assert rep["moduli"] == 12 and rep["operand_bits"] == 42 and rep["tile_n"] == tile_n
            assert np.array_equal(C[tri], Co[tri]), (uplo, tile_n)
            assert np.array_equal(C[~tri], C0[~tri]), (uplo, tile_n)


def test_syrk_moduli_beta_zero_nan_outside_and_one_tile():
    # beta = 0 writes the triangle only (NaN stays outside); n = 100 is a single diagonal tile
    for n in (100, 1):
        A = syn.matrix("uniform", n, 70, 1241)
        C0 = np.full((n, n), np.nan, order="F")
        Co, _ = oracle.modular_dgemm(A, np.asfortranarray(A.T), 42, None, 2.0, 0.0)
        C, rep = syrk(M.MODE_EMULATED, 6, M.UPPER, M.OP_N, A, C0, 2.0, 0.0, M.SCHEME_MODULI)
        up = np.triu(np.ones((n, n), bool))
        assert rep["moduli"] == 12
        assert np.array_equal(C[up], Co[up]) and np.isnan(C[~up]).all()


def test_syrk_beta_zero_leaves_nan_in_the_other_triangle_and_k_passes():
    # beta = 0: the referenced triangle is write-only; NaN in the other one stays; S = 16 forces
    # two k passes (8320 + 128)
    n, k = 200, 8448
    A = syn.matrix("uniform", n, k, 1211)
    C0 = np.full((n, n), np.nan, order="F")
    C, rep = syrk(M.MODE_EMULATED, 16, M.LOWER, M.OP_N, A, C0, 1.0, 0.0)
    assert rep["k_passes"] == 2
    Cref, N = reference(A, np.asfortranarray(A.T))
    low = np.tril(np.ones((n, n), bool))
    assert np.isnan(C[~low]).all()
    assert max_ratio(np.asfortranarray(np.where(low, C, 0.0)), np.asfortranarray(np.where(low, Cref, 0.0)),
                     k, 1.0, 0.0, np.asfortranarray(np.where(low, N, 0.0))) <= 1.0


def test_syrk_integer_inputs_exact_and_alpha_zero_scales_the_triangle():
    n, k = 260, 130
    A = syn.matrix("int", n, k, 1221)
    C0 = syn.matrix("int", n, n, 1222)
    exact = A @ A.T + C0
    for mode, S in ((M.MODE_NATIVE, 0), (M.MODE_EMULATED, 2)):
        C, _ = syrk(mode, S, M.UPPER, M.OP_N, A, C0, 1.0, 1.0)
        up = np.triu(np.ones((n, n), bool))
        assert np.array_equal(C[up], exact[up]) and np.array_equal(C[~up], C0[~up])
    C, _ = syrk(M.MODE_EMULATED, 4, M.LOWER, M.OP_N, A, C0, 0.0, 2.0)
    low = np.tril(np.ones((n, n), bool))
    assert np.array_equal(C[low], 2.0 * C0[low]) and np.array_equal(C[~low], C0[~low])


def test_syrk_argument_errors():
    h = M.Handle()
    assert M.momms_syrk(h, 2, 0, 4, 4, 1.0, 1 << 40, 4, 0.0, 1 << 41, 4) == -2
    assert M.momms_syrk(h, 0, 2, 4, 4, 1.0, 1 << 40, 4, 0.0, 1 << 41, 4) == -3
    assert M.momms_syrk(h, 0, 0, -1, 4, 1.0, 1 << 40, 4, 0.0, 1 << 41, 4) == -4
    assert M.momms_syrk(h, 0, 1, 8, 4, 1.0, 1 << 40, 3, 0.0, 1 << 41, 8) == -8
    assert M.momms_syrk(h, 0, 0, 8, 4, 1.0, 1 << 40, 8, 0.0, 1 << 41, 7) == -11
    h.close()
