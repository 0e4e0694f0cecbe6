"""Native FP64 (DMMA) path against the CPU oracle, through the C ABI."""
import numpy as np
import pytest

from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import F, max_ratio, reference

pytestmark = pytest.mark.gpu


def run(A, B, C0, alpha, beta, opa=M.OP_N, opb=M.OP_N, member=M.MEMBER_AUTO, lds=(None, None, None), ctas=0):
    h = M.Handle(mode=M.MODE_NATIVE, member=member)
    h.set_max_ctas(ctas)
    dA = M.DeviceMatrix.from_numpy(A, ld=lds[0])
    dB = M.DeviceMatrix.from_numpy(B, ld=lds[1])
    dC = M.DeviceMatrix.from_numpy(C0, ld=lds[2])
    M.gemm(dA, dB, dC, alpha, beta, opa, opb, handle=h)
    out = dC.to_numpy()
    pad = dC.padding_numpy()
    rep = h.report()
    h.close()
    return out, pad, rep


SHAPES = [(1, 1, 1), (7, 5, 3), (33, 17, 65), (64, 64, 16), (129, 67, 200), (65, 130, 1), (300, 260, 190)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_native_matches_oracle(m, n, k):
    A = syn.matrix("uniform", m, k, 1 + m)
    B = syn.matrix("uniform", k, n, 2 + n)
    C0 = syn.matrix("uniform", m, n, 3 + k)
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    C, _, rep = run(A, B, C0, 1.0, 1.0)
    assert rep["mode"] == M.MODE_NATIVE
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0


@pytest.mark.parametrize("opa,opb", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_native_transposes(opa, opb):
    m, n, k = 70, 45, 99
    A = syn.matrix("normal", k if opa else m, m if opa else k, 11)
    B = syn.matrix("normal", n if opb else k, k if opb else n, 12)
    C0 = syn.matrix("normal", m, n, 13)
    Cref, N = reference(A, B, C0, -0.5, 2.0, bool(opa), bool(opb))
    C, _, _ = run(A, B, C0, -0.5, 2.0, opa, opb)
    assert max_ratio(C, Cref, k, -0.5, 2.0, N, C0) <= 1.0


def test_native_integer_inputs_bitwise():
    m, n, k = 96, 80, 64
    A = syn.matrix("int", m, k, 21)
    B = syn.matrix("int", k, n, 22)
    C0 = syn.matrix("int", m, n, 23)
    Cref, _ = reference(A, B, C0, 1.0, 1.0)
    C, _, _ = run(A, B, C0, 1.0, 1.0)
    assert np.array_equal(C, Cref)


def test_native_padded_ld_canaries_and_beta_zero_nan():
    m, n, k = 37, 29, 41
    A = syn.matrix("uniform", m, k, 31)
    B = syn.matrix("uniform", k, n, 32)
    C0 = F(np.full((m, n), np.nan))
    Cref, N = reference(A, B)
    C, pad, _ = run(A, B, C0, 1.0, 0.0, lds=(m + 3, k + 5, m + 7))
    assert np.all(np.isfinite(C))  # beta = 0: NaNs in C do not propagate; NaN padding of A/B never read
    assert max_ratio(C, Cref, k, 1.0, 0.0, N) <= 1.0
    assert np.all(np.isnan(pad))   # rows between m and ldc untouched


def test_native_alpha_zero_and_k_zero():
    m, n = 20, 30
    C0 = syn.matrix("uniform", m, n, 41)
    A = syn.matrix("uniform", m, 8, 42)
    B = syn.matrix("uniform", 8, n, 43)
    C, _, _ = run(A, B, C0, 0.0, 3.0)
    assert np.array_equal(C, 3.0 * C0)
    h = M.Handle(mode=M.MODE_NATIVE)
    dC = M.DeviceMatrix.from_numpy(C0)
    M.check(M.momms_gemm_ex(h, 0, 0, m, n, 0, 1.0, 0, m, 0, 1, -1.0, dC.ptr, dC.ld), "k=0")
    assert np.array_equal(dC.to_numpy(), -C0)


def test_native_members_bitwise_identical_and_deterministic():
    m, n, k = 200, 333, 150
    A = syn.matrix("uniform", m, k, 51)
    B = syn.matrix("uniform", k, n, 52)
    C0 = syn.matrix("uniform", m, n, 53)
    outs = [run(A, B, C0, 1.0, 1.0, member=mem)[0] for mem in (M.MEMBER_C2, M.MEMBER_A2, M.MEMBER_B2, M.MEMBER_A1)]
    outs.append(run(A, B, C0, 1.0, 1.0, member=M.MEMBER_C2)[0])
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("ctas", [1, 7, 152])
def test_native_capped_grid_loops_over_member_tiles(ctas):
    # a capped grid makes each CTA loop over its share of tiles in member order; every
    # member must still cover every tile once (ragged 300 x 333: 5 x 6 tiles of 64)
    m, n, k = 300, 333, 97
    A = syn.matrix("uniform", m, k, 61)
    B = syn.matrix("uniform", k, n, 62)
    C0 = syn.matrix("uniform", m, n, 63)
    base = run(A, B, C0, 1.0, 1.0)[0]
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(base, Cref, k, 1.0, 1.0, N, C0) <= 1.0
    for mem in (M.MEMBER_C2, M.MEMBER_A2, M.MEMBER_B2, M.MEMBER_A1):
        assert np.array_equal(run(A, B, C0, 1.0, 1.0, member=mem, ctas=ctas)[0], base)


def test_native_config1_512_cube():
    # workload 1: m = n = k = 512, C += A B (alpha = beta = 1), uniform[-1, 1]
    m = n = k = 512
    A = syn.matrix("uniform", m, k, syn.workload_seed(0, "A"))
    B = syn.matrix("uniform", k, n, syn.workload_seed(0, "B"))
    C0 = syn.matrix("uniform", m, n, syn.workload_seed(0, "C"))
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    C, _, _ = run(A, B, C0, 1.0, 1.0)
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0
