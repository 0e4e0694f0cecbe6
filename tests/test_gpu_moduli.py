"""Modular (Chinese remainder) encoding of the emulated product against the oracle.

The residues of the truncated operands are compared bit for bit; the product is the exact
integer product of the truncated operands rounded once, so C is compared bit for bit with
the oracle's definition (Python integers), and against the componentwise FP64 bound."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import F, max_ratio, reference

pytestmark = pytest.mark.gpu


def stored(which, op, rows, inner, seed, kind="phi", phi=1.0):
    if which == 0:
        shape = (inner, rows) if op else (rows, inner)
    else:
        shape = (rows, inner) if op else (inner, rows)
    return syn.matrix(kind, shape[0], shape[1], seed, phi=phi)


@pytest.mark.parametrize("which,op", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("bits,k", [(21, 64), (39, 8192), (42, 1000), (49, 1000)])
def test_residue_split_bitwise(which, op, bits, k):
    import torch
    rows, inner = 150, 200
    X = stored(which, op, rows, inner, 301 + 2 * which + op, phi=3.0)
    # a vector with Inf (flagged: zero residues) and an all-zero one
    if which == 0:
        X[(0, 7) if op else (7, 0)] = np.inf
    else:
        X[(7, 0) if op else (0, 7)] = np.inf
    rows_pad, inner_pad = 160, 256
    mods = M.momms_crt_moduli(bits, k)
    assert mods == oracle.greedy_moduli(16)[:len(mods)] and oracle.moduli_suffice(mods, bits, k, margin=2)
    dX = M.DeviceMatrix.from_numpy(X)
    e = torch.empty(rows, dtype=torch.int32, device="cuda")
    fl = torch.empty(rows, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(which, op, rows, inner, dX.ptr, dX.ld, e.data_ptr(), fl.data_ptr()), "scale")
    planes = torch.full((len(mods), rows_pad, inner_pad), 99.0, dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_residues(which, op, rows, inner, dX.ptr, dX.ld, e.data_ptr(), fl.data_ptr(), bits, k,
                                 planes.data_ptr(), rows_pad, inner_pad), "residues")
    got = planes.cpu().numpy().astype(np.float64)
    name = "rows" if which == 0 else "cols"
    eo, flo = oracle.exponents(X, name, bool(op))
    want = oracle.centred_residues(oracle.truncated_integers(X, name, eo, flo, bits, bool(op)), mods)
    assert flo[7] == 1
    assert np.array_equal(got[:, :rows, :inner], want.astype(np.float64))
    assert not np.any(got[:, rows:, :]) and not np.any(got[:, :, inner:])


def modular(A, B, C0, alpha, beta, S=0, opa=0, opb=0, scheme=M.SCHEME_MODULI, tile_n=0, ctas=0, fusion=0, pairs=0,
            plan_on_device=1):
    h = M.Handle(mode=M.MODE_EMULATED, slices=S, scheme=scheme)
    h.set_plan_on_device(plan_on_device)
    h.set_tile_n(tile_n)
    h.set_max_ctas(ctas)
    h.set_crt_fusion(fusion)
    h.set_cta_pairs(pairs)
    dA = M.DeviceMatrix.from_numpy(A)
    dB = M.DeviceMatrix.from_numpy(B)
    dC = M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, alpha, beta, opa, opb, handle=h)
    st = h.device_status()
    rep = h.report()
    h.close()
    assert st == M.MOMMS_OK, f"device status {st}"
    return dC.to_numpy(), rep


@pytest.mark.parametrize("S,alpha,beta", [(6, 1.0, 1.0), (5, -0.75, 2.5), (3, 1.5, 0.0)])
@pytest.mark.parametrize("fusion", [1, 2])
def test_modular_product_bitwise_vs_oracle(S, alpha, beta, fusion):
    # ragged in every dimension: 2 x 2 tiles of 128 x 192 with partial edges, 3 k slabs; the
    # reconstruction as its own launch and fused into the last modulus's epilogue
    m, n, k = 150, 200, 150
    A = syn.matrix("phi", m, k, 311, phi=1.0)
    B = syn.matrix("phi", k, n, 312, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 313)
    C, rep = modular(A, B, C0, alpha, beta, S, fusion=fusion)
    assert rep["crt_fused"] == (fusion == 2)
    assert rep["moduli"] == len(M.momms_crt_moduli(7 * S, k)) and rep["operand_bits"] == 7 * S
    Co, _ = oracle.modular_dgemm(A, B, 7 * S, C0.copy(order="F"), alpha, beta)
    assert np.array_equal(C, Co)


@pytest.mark.parametrize("opa,opb", [(1, 0), (0, 1), (1, 1)])
def test_modular_transposes_bitwise(opa, opb):
    m, n, k = 70, 90, 130
    A = syn.matrix("phi", k if opa else m, m if opa else k, 321 + opa, phi=2.0)
    B = syn.matrix("phi", n if opb else k, k if opb else n, 323 + opb, phi=2.0)
    C0 = syn.matrix("uniform", m, n, 325)
    C, rep = modular(A, B, C0, 1.0, -1.0, 6, opa, opb)
    assert rep["moduli"] > 0
    Co, _ = oracle.modular_dgemm(A, B, 42, C0.copy(order="F"), 1.0, -1.0, bool(opa), bool(opb))
    assert np.array_equal(C, Co)


def test_modular_auto_width_bitwise_and_within_bound():
    # automatic slice count: the rule's width in whole bits (report.operand_bits)
    m, n, k = 130, 100, 700
    A = syn.matrix("uniform", m, k, 331)
    B = syn.matrix("uniform", k, n, 332)
    C0 = syn.matrix("uniform", m, n, 333)
    C, rep = modular(A, B, C0, 1.0, 1.0, 0, scheme=M.SCHEME_AUTO)
    assert rep["moduli"] > 0 and 7 * rep["slices"] - 6 <= rep["operand_bits"] <= 7 * rep["slices"]
    Co, _ = oracle.modular_dgemm(A, B, rep["operand_bits"], C0.copy(order="F"), 1.0, 1.0)
    assert np.array_equal(C, Co)
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0


def test_modular_tile_widths_and_capped_grid_bitwise_identical():
    m, n, k = 300, 500, 260
    A = syn.matrix("phi", m, k, 341, phi=1.0)
    B = syn.matrix("phi", k, n, 342, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 343)
    runs = [modular(A, B, C0, 1.0, 1.0, 6, tile_n=t, ctas=c) for t, c in ((192, 0), (96, 0), (192, 5), (96, 3))]
    assert [r["tile_n"] for _, r in runs] == [192, 96, 192, 96]
    for C, _ in runs[1:]:
        assert np.array_equal(C, runs[0][0])


def test_modular_integer_inputs_exact_nonfinite_and_beta_zero():
    m, n, k = 140, 210, 90
    A = syn.matrix("int", m, k, 351)
    B = syn.matrix("int", k, n, 352)
    C0 = syn.matrix("int", m, n, 353)
    C, rep = modular(A, B, C0, 1.0, 1.0, 3)
    assert rep["moduli"] > 0 and np.array_equal(C, A @ B + C0)
    A2 = A.copy(order="F")
    A2[5, 11] = np.nan
    B2 = B.copy(order="F")
    B2[3, 17] = -np.inf
    Cn = np.full((m, n), np.nan, order="F")       # beta = 0: C is write-only
    C, _ = modular(A2, B2, Cn, 2.0, 0.0, 3)
    assert np.all(np.isnan(C[5, :])) and np.all(np.isnan(C[:, 17]))
    keep = np.ones((m, n), bool)
    keep[5, :] = False
    keep[:, 17] = False
    assert np.array_equal(C[keep], (2.0 * (A @ B))[keep])


def test_scheme_choice_and_fallbacks():
    m, n, k = 256, 256, 512
    A = syn.matrix("uniform", m, k, 361)
    B = syn.matrix("uniform", k, n, 362)
    C0 = syn.matrix("uniform", m, n, 363)
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    # AUTO: 3 slices take 6 pairs, 21-bit operands 7 moduli -- not two fewer: slices
    assert len(M.momms_crt_moduli(21, k)) == 7
    C, rep = modular(A, B, C0, 1.0, 1.0, 3, scheme=M.SCHEME_AUTO)
    assert rep["moduli"] == 0
    # AUTO with 6 slices: 13 moduli (42-bit operands, k = 512) against 21 pairs
    C, rep = modular(A, B, C0, 1.0, 1.0, 6, scheme=M.SCHEME_AUTO)
    assert rep["moduli"] == len(M.momms_crt_moduli(42, k)) == 13
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0
    # MODULI requested where 17 moduli would be needed (56-bit operands, k = 8192): slices
    k2 = 8192
    A2 = syn.matrix("uniform", 128, k2, 364)
    B2 = syn.matrix("uniform", k2, 192, 365)
    C2 = syn.matrix("uniform", 128, 192, 366)
    C, rep = modular(A2, B2, C2, 1.0, 1.0, 8)
    assert rep["moduli"] == 0 and rep["slices"] == 8
    Cref2, N2 = reference(A2, B2, C2, 1.0, 1.0)
    assert max_ratio(C, Cref2, k2, 1.0, 1.0, N2, C2) <= 1.0
    # SLICES requested: never moduli
    C, rep = modular(A, B, C0, 1.0, 1.0, 6, scheme=M.SCHEME_SLICES)
    assert rep["moduli"] == 0
    h = M.Handle()
    with pytest.raises(M.MommsError):
        h.set_scheme(3)
    h.close()


def test_modular_workspace_query_covers_the_call():
    import torch
    m, n, k = 400, 300, 500
    A = syn.matrix("uniform", m, k, 371)
    B = syn.matrix("uniform", k, n, 372)
    for S in (0, 6):
        h = M.Handle(mode=M.MODE_EMULATED, slices=S, scheme=M.SCHEME_MODULI)
        need = h.workspace_size(m, n, k)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        h.set_workspace(ws.data_ptr(), need)
        dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
        dC = M.DeviceMatrix(m, n)
        M.gemm(dA, dB, dC, 1.0, 0.0, handle=h)
        assert h.device_status() == M.MOMMS_OK and h.report()["moduli"] > 0
        Cref, N = reference(A, B)
        assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 0.0, N) <= 1.0
        h.set_workspace(ws.data_ptr(), need - 256)
        with pytest.raises(M.MommsError):
            M.gemm(dA, dB, dC, 1.0, 0.0, handle=h)
        h.set_workspace(0, 0)
        h.close()


def test_residue_products_and_reconstruction_pieces_bitwise():
    # the two kernels of the modular product on their own: the residue bytes of the exact
    # integer product, then C from them
    import torch
    m, n, k, bits = 200, 230, 190, 40
    A = syn.matrix("phi", m, k, 381, phi=1.0)
    B = syn.matrix("phi", k, n, 382, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 383)
    mods = M.momms_crt_moduli(bits, k)
    N, k_pad = len(mods), 192
    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    e = torch.empty(m, dtype=torch.int32, device="cuda"); ef = torch.empty(m, dtype=torch.uint8, device="cuda")
    f = torch.empty(n, dtype=torch.int32, device="cuda"); ff = torch.empty(n, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr()), "scale")
    M.check(M.momms_emu_scale(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr()), "scale")
    Ar = torch.empty((N, m, k_pad), dtype=torch.float16, device="cuda")
    Br = torch.empty((N, n, k_pad), dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_residues(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), bits, k, Ar.data_ptr(),
                                 m, k_pad), "residues")
    M.check(M.momms_emu_residues(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), bits, k, Br.data_ptr(),
                                 n, k_pad), "residues")
    res = torch.full((N, n, m), 255, dtype=torch.uint8, device="cuda")
    nbytes = M.momms_emu_scratch_bytes()
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    M.check(M.momms_emu_residue_gemm(m, n, k, bits, Ar.data_ptr(), Br.data_ptr(), m, n, k_pad, 0, res.data_ptr(),
                                     scratch.data_ptr(), nbytes, st.data_ptr()), "residue gemm")
    Co, det = oracle.modular_dgemm(A, B, bits, C0.copy(order="F"), 0.5, -2.0)
    Z = det["Z"]
    want = np.zeros((N, n, m), dtype=np.uint8)
    for l, p in enumerate(mods):
        for j in range(n):
            for i in range(m):
                want[l, j, i] = int(Z[i, j]) % p
    assert int(st.item()) == 0
    assert np.array_equal(res.cpu().numpy(), want)
    dC = M.DeviceMatrix.from_numpy(C0)
    M.check(M.momms_crt_reconstruct(m, n, k, bits, res.data_ptr(), e.data_ptr(), ef.data_ptr(), f.data_ptr(),
                                    ff.data_ptr(), 0.5, -2.0, dC.ptr, dC.ld), "crt")
    assert np.array_equal(dC.to_numpy(), Co)


def test_sixteen_moduli_product_bitwise():
    # 50-bit operands, k = 65536: all 16 moduli (P ~ 2^125, arithmetic modulo 2^128)
    m, n, k = 20, 12, 65536
    assert len(M.momms_crt_moduli(50, k)) == 16
    A = syn.matrix("phi", m, k, 391, phi=1.0)
    B = syn.matrix("phi", k, n, 392, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 393)
    dA, dB, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C0)
    # 50 bits is not a whole number of digits: drive the pieces through the ABI
    import torch
    e = torch.empty(m, dtype=torch.int32, device="cuda"); ef = torch.empty(m, dtype=torch.uint8, device="cuda")
    f = torch.empty(n, dtype=torch.int32, device="cuda"); ff = torch.empty(n, dtype=torch.uint8, device="cuda")
    M.check(M.momms_emu_scale(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr()), "scale")
    M.check(M.momms_emu_scale(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr()), "scale")
    Ar = torch.empty((16, m, k), dtype=torch.float16, device="cuda")
    Br = torch.empty((16, n, k), dtype=torch.float16, device="cuda")
    M.check(M.momms_emu_residues(0, 0, m, k, dA.ptr, dA.ld, e.data_ptr(), ef.data_ptr(), 50, k, Ar.data_ptr(), m, k),
            "residues")
    M.check(M.momms_emu_residues(1, 0, n, k, dB.ptr, dB.ld, f.data_ptr(), ff.data_ptr(), 50, k, Br.data_ptr(), n, k),
            "residues")
    res = torch.empty((16, n, m), dtype=torch.uint8, device="cuda")
    nbytes = M.momms_emu_scratch_bytes()
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    M.check(M.momms_emu_residue_gemm(m, n, k, 50, Ar.data_ptr(), Br.data_ptr(), m, n, k, 0, res.data_ptr(),
                                     scratch.data_ptr(), nbytes, st.data_ptr()), "residue gemm")
    M.check(M.momms_crt_reconstruct(m, n, k, 50, res.data_ptr(), e.data_ptr(), ef.data_ptr(), f.data_ptr(),
                                    ff.data_ptr(), 1.0, 1.0, dC.ptr, dC.ld), "crt")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    Co, _ = oracle.modular_dgemm(A, B, 50, C0.copy(order="F"), 1.0, 1.0)
    assert np.array_equal(dC.to_numpy(), Co)


def test_residue_products_exact_at_the_chunk_edge():
    # residue planes at the largest magnitude (127): every 1024-product FP32 chunk reaches
    # 1024 * 127^2 = 16,516,096 < 2^24 and the int32 sums k * 127^2 (k = 65536: 1.06e9) stay exact
    import torch
    m, n, k, bits = 130, 200, 65536, 30
    mods = M.momms_crt_moduli(bits, k)
    N = len(mods)
    sa = np.where((np.arange(m)[:, None] + np.arange(k)[None, :]) % 5 == 0, -1.0, 1.0)
    sa[:64] = 1.0                                  # rows whose every product is +127^2
    sb = np.where((np.arange(n)[:, None] * 3 + np.arange(k)[None, :]) % 7 == 0, -1.0, 1.0)
    sb[:96] = 1.0
    Ar = torch.from_numpy(np.ascontiguousarray(np.broadcast_to((127.0 * sa).astype(np.float16), (N, m, k)))).cuda()
    Br = torch.from_numpy(np.ascontiguousarray(np.broadcast_to((127.0 * sb).astype(np.float16), (N, n, k)))).cuda()
    res = torch.full((N, n, m), 255, dtype=torch.uint8, device="cuda")
    nbytes = M.momms_emu_scratch_bytes()
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    M.check(M.momms_emu_residue_gemm(m, n, k, bits, Ar.data_ptr(), Br.data_ptr(), m, n, k, 0, res.data_ptr(),
                                     scratch.data_ptr(), nbytes, st.data_ptr()), "residue gemm")
    # integer sums below 2^53: the FP64 product of the sign patterns is exact
    Z = np.rint((127.0 * sa) @ (127.0 * sb).T).astype(np.int64)
    assert Z.max() == k * 127 * 127
    want = np.stack([np.mod(Z.T, p) for p in mods])                      # [l][j][i]
    assert int(st.item()) == 0
    assert np.array_equal(res.cpu().numpy().astype(np.int64), want)


@pytest.mark.parametrize("m,n,k", [(2000, 2000, 2100), (300, 1000, 2048), (1030, 770, 4096)])
def test_fused_reconstruction_bitwise_equal_to_separate(m, n, k):
    # fused: groups of four waves' tiles keep a tile's moduli on one CTA, the last, partial group
    # spreads them over several CTAs (published through the tile counters); tiles above and below
    # the grid size
    A = syn.matrix("uniform", m, k, 401)
    B = syn.matrix("normal", k, n, 402)
    C0 = syn.matrix("uniform", m, n, 403)
    # data-driven width (S = 0): the bound holds; both runs take the same width from the same data
    # (the fused form chooses its width on the host: compare launch counts with the host plan)
    Cs, rs = modular(A, B, C0, -1.25, 0.5, 0, fusion=0, plan_on_device=0)
    Cf, rf = modular(A, B, C0, -1.25, 0.5, 0, fusion=2)
    assert rs["moduli"] > 0 and rs["crt_fused"] == 0
    assert rf["crt_fused"] == 1 and rf["launches"] == rs["launches"] - 1
    assert np.array_equal(Cf, Cs)
    Cref, N = reference(A, B, C0, -1.25, 0.5)
    assert max_ratio(Cf, Cref, k, 1.25, 0.5, N, C0) <= 1.0


@pytest.mark.parametrize("m,n,k,opa,opb,ctas", [(300, 1000, 520, 0, 0, 0), (200, 700, 300, 1, 0, 0),
                                                (2000, 900, 1100, 0, 1, 0), (1024, 1152, 640, 1, 1, 0),
                                                (700, 450, 2000, 0, 0, 6)])
def test_cta_pairs_bitwise_identical(m, n, k, opa, opb, ctas):
    # the residue product on CTA pairs (one MMA over two SMs, 256 x 192 tiles, each CTA staging
    # its own rows of A and half of B) against single CTAs: ragged pair rows (the second half of the
    # last pair row past m: zero operands, nothing stored), one pair row, transposes, a capped grid
    A = syn.matrix("phi", k if opa else m, m if opa else k, 431, phi=1.0)
    B = syn.matrix("phi", n if opb else k, k if opb else n, 432, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 433)
    C1, r1 = modular(A, B, C0, 1.5, -0.5, 6, opa, opb, tile_n=192, ctas=ctas, pairs=1)
    C2, r2 = modular(A, B, C0, 1.5, -0.5, 6, opa, opb, tile_n=192, ctas=ctas, pairs=2)
    assert r1["moduli"] > 0 and r2["moduli"] == r1["moduli"]
    assert r2["ctas"] % 2 == 0
    assert np.array_equal(C1, C2)
    # sampled elements at the pair tile's seams bit for bit against the definition of the result
    rs = np.unique([0, 127, 128, min(255, m - 1), min(256, m - 1), m - 1])
    cs = np.unique([0, 95, 96, min(191, n - 1), min(192, n - 1), n - 1])
    As = np.asfortranarray(A[:, rs] if opa else A[rs, :])
    Bs = np.asfortranarray(B[cs, :] if opb else B[:, cs])
    Co, _ = oracle.modular_dgemm(As, Bs, 42, np.asfortranarray(C0[np.ix_(rs, cs)]), 1.5, -0.5, bool(opa), bool(opb))
    assert np.array_equal(C2[np.ix_(rs, cs)], Co)


def test_cta_pairs_timeout_path():
    # the timeout test hook on the pair kernel: the leader of the first pair leaves a stage empty,
    # both CTAs' bounded waits run out, the status reads MOMMS_ERR_TIMEOUT, the next call is exact
    m, n, k = 600, 800, 512
    A = syn.matrix("uniform", m, k, 441)
    B = syn.matrix("uniform", k, n, 442)
    C0 = syn.matrix("uniform", m, n, 443)
    h = M.Handle(mode=M.MODE_EMULATED, slices=6, scheme=M.SCHEME_MODULI)
    h.set_tile_n(192)
    h.set_cta_pairs(2)
    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    M.momms_debug_withhold_load()
    dC = M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)
    assert h.device_status() == M.MOMMS_ERR_TIMEOUT
    dC = M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)
    assert h.device_status() == M.MOMMS_OK
    rs, cs = np.array([0, 255, 256, 599]), np.array([0, 96, 191, 192, 799])
    Co, _ = oracle.modular_dgemm(np.asfortranarray(A[rs, :]), np.asfortranarray(B[:, cs]), 42,
                                 np.asfortranarray(C0[np.ix_(rs, cs)]), 1.0, 1.0)
    assert np.array_equal(dC.to_numpy()[np.ix_(rs, cs)], Co)
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 1.0, N, C0) <= 1.0
    h.close()


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 5, 70), (129, 1, 300), (1, 300, 64)])
def test_modular_tiny_and_single_vector_shapes_bitwise(m, n, k):
    # one element, ragged rows below the 4-row vector path of the reconstruction, one column
    A = syn.matrix("phi", m, k, 421, phi=1.0)
    B = syn.matrix("phi", k, n, 422, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 423)
    C, rep = modular(A, B, C0, 2.0, -1.0, 5)
    assert rep["moduli"] > 0
    Co, _ = oracle.modular_dgemm(A, B, 35, C0.copy(order="F"), 2.0, -1.0)
    assert np.array_equal(C, Co)


def test_modular_odd_leading_dimension_bitwise():
    # ldc odd: the reconstruction cannot pair C elements into 16-byte words
    m, n, k = 64, 50, 200
    A = syn.matrix("uniform", m, k, 431)
    B = syn.matrix("uniform", k, n, 432)
    C0 = syn.matrix("uniform", m, n, 433)
    h = M.Handle(mode=M.MODE_EMULATED, slices=6, scheme=M.SCHEME_MODULI)
    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    dC = M.DeviceMatrix.from_numpy(C0, ld=m + 1)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)
    assert h.device_status() == M.MOMMS_OK and h.report()["moduli"] > 0
    h.close()
    Co, _ = oracle.modular_dgemm(A, B, 42, C0.copy(order="F"), 1.0, 1.0)
    assert np.array_equal(dC.to_numpy(), Co)
    assert np.all(np.isnan(dC.padding_numpy()))          # the row of padding is never written


@pytest.mark.parametrize("m,n,k,opa,opb", [(300, 500, 130, 0, 0), (260, 620, 64, 1, 0), (388, 400, 256, 0, 1),
                                           (200, 900, 200, 1, 1), (390, 400, 256, 0, 0)])
def test_kept_a_short_k_bitwise(m, n, k, opa, opb):
    # k <= 256: each CTA keeps its A tile in shared memory over a strip of tiles (at least as many
    # tiles as CTAs, m a multiple of 4) and stores its residues straight from the accumulator; a
    # grid of 5 CTAs over 6-15 tiles gives strips that end inside and at the end of a tile row,
    # several moduli per strip; 40 CTAs (more than the tiles) and m = 390 take the ring kernel
    A = syn.matrix("phi", k if opa else m, m if opa else k, 451, phi=1.0)
    B = syn.matrix("phi", n if opb else k, k if opb else n, 452, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 453)
    Ck, rk = modular(A, B, C0, -1.5, 0.5, 6, opa, opb, tile_n=192, ctas=5)
    Cr, rr = modular(A, B, C0, -1.5, 0.5, 6, opa, opb, tile_n=192, ctas=40)
    assert rk["moduli"] > 0 and rk["ctas"] == 5 and rr["ctas"] > 5
    assert np.array_equal(Ck, Cr)
    # rows and columns at the tile seams bit for bit against the definition of the result
    rs = np.unique([0, 1, 127, 128, 129, min(255, m - 1), min(256, m - 1), m - 1])
    cs = np.unique([0, 1, 191, 192, 193, min(383, n - 1), min(384, n - 1), n - 1])
    As = np.asfortranarray(A[:, rs] if opa else A[rs, :])
    Bs = np.asfortranarray(B[cs, :] if opb else B[:, cs])
    Co, _ = oracle.modular_dgemm(As, Bs, 42, np.asfortranarray(C0[np.ix_(rs, cs)]), -1.5, 0.5, bool(opa), bool(opb))
    assert np.array_equal(Ck[np.ix_(rs, cs)], Co)


def test_kept_a_full_grid_bitwise_at_tile_seams():
    # every SM's CTA on the kept-A kernel: 17 x 9 = 153 tiles (at least one per CTA), ragged m, n
    # and k (4 slabs, the last partial); elements at the tile seams bit for bit against the definition
    m, n, k = 2084, 1700, 200
    A = syn.matrix("phi", m, k, 461, phi=1.0)
    B = syn.matrix("phi", k, n, 462, phi=1.0)
    C0 = syn.matrix("uniform", m, n, 463)
    C, rep = modular(A, B, C0, 1.0, 1.0, 6, tile_n=192)
    assert rep["moduli"] > 0
    rs = np.unique([0, 127, 128, 1023, 1024, 2047, 2048, m - 1])
    cs = np.unique([0, 191, 192, 767, 768, 1535, 1536, n - 1])
    Co, _ = oracle.modular_dgemm(np.asfortranarray(A[rs, :]), np.asfortranarray(B[:, cs]), 42,
                                 np.asfortranarray(C0[np.ix_(rs, cs)]), 1.0, 1.0)
    assert np.array_equal(C[np.ix_(rs, cs)], Co)
