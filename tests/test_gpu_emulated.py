"""Emulated FP64 path (integer digit slices on the tcgen05 tensor cores) against the oracle.

Integer / byte work is compared bit for bit (exponents, flags, digits, exact
integer products); floating-point results against the componentwise bound."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import F, U, max_ratio, reference

pytestmark = pytest.mark.gpu

BETA = 7


def torch_mod():
    import torch
    return torch


def stored(which, op, rows, inner, seed, kind="phi", phi=1.0):
    """The stored matrix X whose op(.) has `rows` vectors of length `inner`."""
    if which == 0:
        shape = (inner, rows) if op else (rows, inner)
    else:
        shape = (rows, inner) if op else (inner, rows)
    return syn.matrix(kind, shape[0], shape[1], seed, phi=phi)


@pytest.mark.parametrize("which,op", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_scale_bitwise(which, op):
    torch = torch_mod()
    rows, inner = 301, 257
    X = stored(which, op, rows, inner, 7 + 2 * which + op, phi=4.0)
    # an all-zero vector, a vector with Inf, one with NaN, one with a subnormal maximum
    def vec_set(r, vals):
        for q, v in enumerate(vals):
            if which == 0:
                X[(q, r) if op else (r, q)] = v
            else:
                X[(r, q) if op else (q, r)] = v
    vec_set(3, [0.0] * inner)
    vec_set(5, [np.inf] + [1.0] * (inner - 1))
    vec_set(8, [np.nan] * inner)
    vec_set(9, [2.0 ** -1070] + [0.0] * (inner - 1))
    dX = M.DeviceMatrix.from_numpy(X)
    e = torch.empty(rows, dtype=torch.int32, device="cuda")
    fl = torch.empty(rows, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(which, op, rows, inner, dX.ptr, dX.ld, e.data_ptr(), fl.data_ptr()), "scale")
    eo, flo = oracle.exponents(X, "rows" if which == 0 else "cols", bool(op))
    assert np.array_equal(e.cpu().numpy(), eo)
    assert np.array_equal(fl.cpu().numpy(), flo)


@pytest.mark.parametrize("which,op", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("S,beta", [(5, 7), (9, 7), (12, 7), (3, 8)])
def test_split_bitwise(which, op, S, beta):
    torch = torch_mod()
    rows, inner = 200, 100
    X = stored(which, op, rows, inner, 17 + which + 3 * op, phi=4.0)
    rows_pad, inner_pad = 256, 128
    dX = M.DeviceMatrix.from_numpy(X)
    e = torch.empty(rows, dtype=torch.int32, device="cuda")
    fl = torch.empty(rows, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(which, op, rows, inner, dX.ptr, dX.ld, e.data_ptr(), fl.data_ptr()), "scale")
    dg = torch.full((S, rows_pad, inner_pad), 99.0, dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_split(which, op, rows, inner, dX.ptr, dX.ld, e.data_ptr(), fl.data_ptr(), S, beta,
                              dg.data_ptr(), rows_pad, inner_pad), "split")
    got = dg.cpu().numpy().astype(np.float64)
    eo, flo = oracle.exponents(X, "rows" if which == 0 else "cols", bool(op))
    want = oracle.split(X, "rows" if which == 0 else "cols", eo, flo, S, beta, bool(op))
    assert np.array_equal(got[:, :rows, :inner], want.astype(np.float64))
    assert not np.any(got[:, rows:, :]) and not np.any(got[:, :, inner:])  # zero padding


def emulated(A, B, C0, alpha, beta, S, opa=0, opb=0, member=M.MEMBER_AUTO, ldc=None, ctas=0,
             scheme=M.SCHEME_SLICES):
    # the digit-slice encoding unless a test asks otherwise (test_gpu_moduli covers the other)
    h = M.Handle(mode=M.MODE_EMULATED, member=member, slices=S, scheme=scheme)
    h.set_max_ctas(ctas)
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B)
    dC = M.DeviceMatrix.from_numpy(C0, ld=ldc)
    M.gemm(dA, dB, dC, alpha, beta, opa, opb, handle=h)
    st = h.device_status()
    rep = h.report()
    h.close()
    assert st == M.MOMMS_OK, f"device status {st}"
    return dC.to_numpy(), rep, dC


@pytest.mark.parametrize("S", [1, 2, 4])
def test_emulated_integer_inputs_bitwise(S):
    m, n, k = 150, 300, 200
    A = syn.matrix("int", m, k, 31)
    B = syn.matrix("int", k, n, 32)
    C0 = syn.matrix("int", m, n, 33)
    Cref, _ = reference(A, B, C0, 1.0, 1.0)
    C, rep, _ = emulated(A, B, C0, 1.0, 1.0, S)
    assert rep["mode"] == M.MODE_EMULATED and rep["slices"] == S
    assert np.array_equal(C, Cref)


def test_fp32_tensor_memory_accumulation_is_exact():
    # every digit at its maximum 127: each 1024-product chunk sums to 127^2 * 1024 < 2^24,
    # the largest value the FP32 accumulator must hold exactly; signs alternate to mix cancellation
    m, n, k = 128, 256, 4096
    rs = np.where((np.arange(m)[:, None] + np.arange(k)[None, :]) % 3 == 0, -1.0, 1.0)
    A = F(rs * (127.0 / 128.0))
    B = F(np.ones((k, n)) * (127.0 / 128.0))
    B[:, 1::2] *= -1.0
    Cref, _ = reference(A, B)
    C, rep, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, 1)
    assert np.array_equal(C, Cref)
    A2 = F(np.full((m, k), 127.0 / 128.0))
    C2, _, _ = emulated(A2, B, F(np.zeros((m, n))), 1.0, 0.0, 1)
    assert np.array_equal(C2, reference(A2, B)[0])


@pytest.mark.parametrize("kind,phi,S", [("uniform", 0.0, 7), ("phi", 1.0, 9), ("phi", 4.0, 12)])
@pytest.mark.parametrize("m,n,k", [(130, 270, 333), (256, 512, 1024)])
@pytest.mark.parametrize("scheme", [M.SCHEME_SLICES, M.SCHEME_AUTO])
def test_emulated_within_bound(kind, phi, S, m, n, k, scheme):
    A = syn.matrix(kind, m, k, 41, phi=phi)
    B = syn.matrix(kind, k, n, 42, phi=phi)
    C0 = syn.matrix("uniform", m, n, 43)
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    C, _, _ = emulated(A, B, C0, 1.0, 1.0, S, scheme=scheme)
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0


def test_emulated_matches_oracle_emulation():
    # same digits, same pair set: only the FP64 rounding of the recombination differs
    m, n, k, S = 100, 90, 300, 11  # several int64 groups: FP64 folds between them
    A = syn.matrix("phi", m, k, 51, phi=1.0)
    B = syn.matrix("phi", k, n, 52, phi=1.0)
    Co, _ = oracle.emulated_dgemm(A, B, S, BETA)
    C, _, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, S)
    N = oracle.dgemm_abs(A, B)
    assert np.all(np.abs(C - Co) <= 4 * (S + 2) * U * N + 2.0 ** -1021)


@pytest.mark.parametrize("S", [4, 6])
def test_emulated_single_group_bitwise_vs_oracle_emulation(S):
    # With S <= 6 and k <= 8192 every diagonal sum fits one exact int64 group, so the
    # kernel's recombination is the exact digit expansion rounded once -- the oracle's.
    m, n, k = 200, 300, 1000
    A = syn.matrix("phi", m, k, 55, phi=1.0)
    B = syn.matrix("phi", k, n, 56, phi=1.0)
    Co, _ = oracle.emulated_dgemm(A, B, S, BETA)
    C, _, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, S)
    assert np.array_equal(C, Co)


@pytest.mark.parametrize("scale", [-510, -520, 512])
def test_emulated_rounding_at_the_ends_of_the_exponent_range(scale):
    # products scaled into the subnormal range (the 53-bit rounding, then the subnormal grid, as the
    # oracle does it) and beyond the largest double (infinities): one exact group, so bit for bit
    m, n, k, S = 130, 200, 120, 6
    A = syn.matrix("phi", m, k, 53, phi=1.0) * 2.0 ** scale
    B = syn.matrix("phi", k, n, 54, phi=1.0) * 2.0 ** scale
    Co, _ = oracle.emulated_dgemm(A, B, S, BETA)
    C, _, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, S)
    if scale < 0:  # -510: normal and subnormal results mixed, -520: all subnormal
        assert np.any((Co != 0) & (np.abs(Co) < np.finfo(np.float64).tiny))
    else:
        assert np.any(np.isinf(Co)) and np.any(np.isfinite(Co))
    assert np.array_equal(C, Co)


@pytest.mark.parametrize("opa,opb", [(1, 0), (0, 1), (1, 1)])
def test_emulated_transposes(opa, opb):
    m, n, k = 140, 260, 150
    A = syn.matrix("normal", k if opa else m, m if opa else k, 61)
    B = syn.matrix("normal", n if opb else k, k if opb else n, 62)
    C0 = syn.matrix("normal", m, n, 63)
    Cref, N = reference(A, B, C0, 0.75, -1.5, bool(opa), bool(opb))
    C, _, _ = emulated(A, B, C0, 0.75, -1.5, 8, opa, opb)
    assert max_ratio(C, Cref, k, 0.75, -1.5, N, C0) <= 1.0


def test_emulated_members_bitwise_identical():
    m, n, k = 300, 600, 200
    A = syn.matrix("uniform", m, k, 71)
    B = syn.matrix("uniform", k, n, 72)
    C0 = syn.matrix("uniform", m, n, 73)
    outs = [emulated(A, B, C0, 1.0, 1.0, 6, member=mem)[0]
            for mem in (M.MEMBER_C2, M.MEMBER_A2, M.MEMBER_B2, M.MEMBER_A1)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("ctas", [1, 5, 1000])
def test_emulated_capped_grid_bitwise_identical(ctas):
    # fewer persistent CTAs (or a cap above the SM count, clamped) change only which CTA
    # computes a tile: 3 x 4 tiles of 128 x 192 with ragged edges
    m, n, k = 300, 650, 200
    A = syn.matrix("uniform", m, k, 81)
    B = syn.matrix("uniform", k, n, 82)
    C0 = syn.matrix("uniform", m, n, 83)
    base = emulated(A, B, C0, 1.0, 1.0, 6)[0]
    for mem in (M.MEMBER_C2, M.MEMBER_A2, M.MEMBER_B2, M.MEMBER_A1):
        assert np.array_equal(emulated(A, B, C0, 1.0, 1.0, 6, member=mem, ctas=ctas)[0], base)


def test_emulated_beta_zero_nan_and_padded_ldc():
    m, n, k = 77, 99, 64
    A = syn.matrix("uniform", m, k, 81)
    B = syn.matrix("uniform", k, n, 82)
    C0 = F(np.full((m, n), np.nan))
    Cref, N = reference(A, B)
    C, _, dC = emulated(A, B, C0, 1.0, 0.0, 7, ldc=m + 5)
    assert np.all(np.isfinite(C))
    assert max_ratio(C, Cref, k, 1.0, 0.0, N) <= 1.0
    assert np.all(np.isnan(dC.padding_numpy()))


def test_emulated_nonfinite_rows_give_nan():
    m, n, k = 64, 64, 64
    A = syn.matrix("uniform", m, k, 91)
    A[5, 7] = np.inf
    B = syn.matrix("uniform", k, n, 92)
    B[3, 9] = np.nan
    C, _, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, 6)
    assert np.all(np.isnan(C[5, :])) and np.all(np.isnan(C[:, 9]))
    mask = np.ones((m, n), bool)
    mask[5, :] = False
    mask[:, 9] = False
    assert np.all(np.isfinite(C[mask]))


@pytest.mark.parametrize("phi", [0.0, 1.0, 4.0])
@pytest.mark.parametrize("scheme", [M.SCHEME_SLICES, M.SCHEME_AUTO])
def test_emulated_auto_slices_meet_bound(phi, scheme):
    m, n, k = 200, 300, 1024
    A = syn.matrix("phi", m, k, 101, phi=phi)
    B = syn.matrix("phi", k, n, 102, phi=phi)
    Cref, N = reference(A, B)
    C, rep, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, 0, scheme=scheme)
    assert 3 <= rep["slices"] <= 14
    assert max_ratio(C, Cref, k, 1.0, 0.0, N) <= 1.0


def test_slice_gemm_entry_point_and_k_passes():
    torch = torch_mod()
    # k above one pass for S = 16 (8320) so that the kernel runs two passes
    m, n, k, S = 128, 256, 8448, 16
    A = syn.matrix("uniform", m, k, 111)
    B = syn.matrix("uniform", k, n, 112)
    Cref, N = reference(A, B)
    C, rep, _ = emulated(A, B, F(np.zeros((m, n))), 1.0, 0.0, S)
    assert rep["k_passes"] == 2
    assert max_ratio(C, Cref, k, 1.0, 0.0, N) <= 1.0
    # the step-level entry points give the same bits as the pipeline
    m_pad, n_pad, k_pad = 128, 256, 8448
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B)
    e = torch.empty(m, dtype=torch.int32, device="cuda"); ef = torch.empty(m, dtype=torch.uint8, device="cuda")
    f = torch.empty(n, dtype=torch.int32, device="cuda"); ff = torch.empty(n, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr()), "scale A")
    M.check(M.momms_emu_scale(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr()), "scale B")
    Ad = torch.empty((S, m_pad, k_pad), dtype=torch.float16, device="cuda")
    Bd = torch.empty((S, n_pad, k_pad), dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_split(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), S, BETA, Ad.data_ptr(), m_pad, k_pad), "split A")
    M.check(M.momms_emu_split(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), S, BETA, Bd.data_ptr(), n_pad, k_pad), "split B")
    nbytes = M.momms_emu_scratch_bytes()
    scratch = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dC = M.DeviceMatrix(m, n)
    M.check(M.momms_emu_slice_gemm(m, n, k, S, BETA, Ad.data_ptr(), Bd.data_ptr(), m_pad, n_pad, k_pad,
                                   e.data_ptr(), ef.data_ptr(), f.data_ptr(), ff.data_ptr(), 1.0, 0.0,
                                   dC.ptr, dC.ld, M.MEMBER_C2, scratch.data_ptr(), nbytes,
                                   status.data_ptr()), "slice gemm")
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(dC.to_numpy(), C)


def _slice_products(torch, A, B, S, nbytes):
    """Scale, split and one slice-product call through the step entry points, with `nbytes`
    of recombination scratch; returns C (beta = 0) and the device status word."""
    m, k = A.shape
    n = B.shape[1]
    k_pad = -(-k // 64) * 64
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B)
    e = torch.empty(m, dtype=torch.int32, device="cuda"); ef = torch.empty(m, dtype=torch.uint8, device="cuda")
    f = torch.empty(n, dtype=torch.int32, device="cuda"); ff = torch.empty(n, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr()), "scale A")
    M.check(M.momms_emu_scale(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr()), "scale B")
    Ad = torch.empty((S, m, k_pad), dtype=torch.float16, device="cuda")
    Bd = torch.empty((S, n, k_pad), dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_split(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), S, BETA, Ad.data_ptr(), m, k_pad),
            "split A")
    M.check(M.momms_emu_split(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), S, BETA, Bd.data_ptr(), n, k_pad),
            "split B")
    scratch = torch.full((nbytes // 8,), 7.0, dtype=torch.float64, device="cuda")  # not zero on purpose
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    dC = M.DeviceMatrix(m, n)
    M.check(M.momms_emu_slice_gemm(m, n, k, S, BETA, Ad.data_ptr(), Bd.data_ptr(), m, n, k_pad, e.data_ptr(),
                                   ef.data_ptr(), f.data_ptr(), ff.data_ptr(), 1.0, 0.0, dC.ptr, dC.ld, M.MEMBER_C2,
                                   scratch.data_ptr(), nbytes, status.data_ptr()), "slice gemm")
    torch.cuda.synchronize()
    return dC.to_numpy(), int(status.item())


@pytest.mark.parametrize("m,n,k,S", [
    (1280, 3072, 3000, 6),    # 10 x 16 = 160 tiles: 8 left over for 152 CTAs, 19 k parts each
    (1300, 3000, 2000, 9),    # 11 x 16 = 176 tiles: 24 left over, 6 parts each, ragged edges
    (1280, 3072, 8832, 16),   # two k passes (the second of 8 slabs: 8 parts), S = 16
])
def test_tail_split_bitwise_identical_to_whole_tiles(m, n, k, S):
    # Given the larger scratch, the slice-product call cuts the tiles of its last, partial round
    # of CTAs along k; the parts' int32 sums add up exactly, so C must not change by one bit.
    torch = torch_mod()
    A = syn.matrix("uniform", m, k, 5000 + m)
    B = syn.matrix("uniform", k, n, 6000 + n)
    base, big = M.momms_emu_scratch_bytes(), M.momms_emu_scratch_bytes_for(m, n, k, S)
    assert big > base  # the tail split is on for these shapes on a 152-SM GB300
    whole, st0 = _slice_products(torch, A, B, S, base)
    split, st1 = _slice_products(torch, A, B, S, big)
    assert st0 == 0 and st1 == 0
    assert np.array_equal(split, whole)
    rows = np.array([0, 1, m // 2, m - 1])
    Cref, N = reference(F(A[rows, :]), B)
    assert max_ratio(split[rows, :], Cref, k, 1.0, 0.0, N) <= 1.0
    # every tile of the split round in full: the last tiles % ctas tiles of the C2 order
    from paper_1904_05717_gb300 import iomodel as I
    ctas = torch.cuda.get_device_properties(0).multi_processor_count
    tiles_m, tiles_n = -(-m // 128), -(-n // 192)
    total = tiles_m * tiles_n
    for t in range(total // ctas * ctas, total):
        tm, tn = I.member_tile(M.MEMBER_C2, 0, t % ctas, ctas, t // ctas, tiles_m, tiles_n)
        r = np.arange(tm * 128, min(m, tm * 128 + 128))
        c = np.arange(tn * 192, min(n, tn * 192 + 192))
        Cref, N = reference(F(A[r, :]), F(B[:, c]))
        assert max_ratio(split[np.ix_(r, c)], Cref, k, 1.0, 0.0, N) <= 1.0


def test_scratch_for_any_shape_covers_the_step_entry_minimum():
    # momms_emu_slice_gemm requires at least momms_emu_scratch_bytes(); the size for a given
    # problem only adds the tail split's partial sums, even when the grid has fewer CTAs than SMs
    base = M.momms_emu_scratch_bytes()
    for m, n, k, S in [(100, 100, 100, 4), (1024, 1024, 1024, 6), (8192, 8192, 8192, 6), (1, 1, 1, 1)]:
        assert M.momms_emu_scratch_bytes_for(m, n, k, S) >= base


@pytest.mark.parametrize("m,n,k,S,opa,opb", [
    (300, 650, 200, 8, 0, 0),     # ragged in m and n, one group
    (257, 200, 1500, 9, 1, 0),    # two int64 groups (FP64 fold between them), op(A) = A^T
    (130, 97, 64, 12, 0, 1),      # one k slab, op(B) = B^T, many groups
    (700, 400, 3000, 7, 1, 1),    # both transposed
])
def test_emulated_tile_widths_bitwise_identical(m, n, k, S, opa, opb):
    # the narrow tile (96 columns, group sums in tensor memory) and the wide one (192, group sums
    # in a global scratch block) do the same exact integer sums and the same FP64 operations
    A = syn.matrix("uniform", k if opa else m, m if opa else k, 1401)
    B = syn.matrix("uniform", n if opb else k, k if opb else n, 1402)
    C0 = syn.matrix("uniform", m, n, 1403)
    outs = []
    for tn in (96, 192):
        h = M.Handle(mode=M.MODE_EMULATED, slices=S)
        h.set_tile_n(tn)
        dA, dB, dC = (M.DeviceMatrix.from_numpy(X) for X in (A, B, C0))
        M.gemm(dA, dB, dC, 0.5, -1.0, opa, opb, handle=h)
        assert h.device_status() == M.MOMMS_OK
        assert h.report()["tile_n"] == tn
        outs.append(dC.to_numpy())
        h.close()
    assert np.array_equal(outs[0], outs[1])
    Cref, N = reference(A, B, C0, 0.5, -1.0, bool(opa), bool(opb))
    assert max_ratio(outs[0], Cref, k, 0.5, -1.0, N, C0) <= 1.0
