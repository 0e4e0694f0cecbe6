"""Out-of-core product (host memory as the slow level, HBM as the fast one): results
against the oracle, and the host<->device bytes against the Resident C closed forms
(Sec. 2.2.1) that the CPU counting oracle pins."""
import numpy as np
import pytest

from paper_1904_05717_gb300 import iomodel as I
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio, reference

pytestmark = pytest.mark.gpu


def pinned(X):
    """A pinned host copy of the column-major matrix X (torch tensor of shape (cols, rows))."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    return t


def run_host(h, A, B, C0, alpha, beta, block=0, device_bytes=0, pin=True):
    m, k = A.shape
    n = B.shape[1]
    import torch
    if pin:
        tA, tB, tC = pinned(A), pinned(B), pinned(C0)
        pa, pb, pc = tA.data_ptr(), tB.data_ptr(), tC.data_ptr()
    else:
        tA, tB, tC = (np.asfortranarray(X) for X in (A, B, C0.copy()))
        pa, pb, pc = tA.ctypes.data, tB.ctypes.data, tC.ctypes.data
    s = torch.cuda.current_stream()
    M.check(M.momms_gemm_host(h, m, n, k, alpha, pa, m, pb, k, beta, pc, m, device_bytes, block, s), "gemm_host")
    torch.cuda.synchronize()
    out = tC.numpy().T.copy(order="F") if pin else np.array(tC, order="F")
    return out, h.report()


def closed_form_bytes(m, n, k, b, beta_nonzero):
    w = I.resident_c_words(m, n, k, b, b, c_read=beta_nonzero)
    return 8 * (w["a_reads"] + w["b_reads"] + w["c_reads"]), 8 * w["c_writes"]


@pytest.mark.parametrize("mode,S", [(M.MODE_NATIVE, 0), (M.MODE_EMULATED, 8), (M.MODE_EMULATED, 0)])
@pytest.mark.parametrize("pin", [True, False])
def test_host_product_matches_oracle_and_closed_form_io(mode, S, pin):
    m, n, k, b = 700, 530, 900, 256   # ragged in every dimension: 3 x 3 C blocks, 4 k blocks
    A = syn.matrix("uniform", m, k, 901)
    B = syn.matrix("uniform", k, n, 902)
    C0 = syn.matrix("uniform", m, n, 903)
    h = M.Handle(mode=mode, slices=S)
    C, rep = run_host(h, A, B, C0, 1.0, 1.0, block=b, pin=pin)
    assert h.device_status() == M.MOMMS_OK
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0
    h2d, d2h = closed_form_bytes(m, n, k, b, True)
    assert (rep["ooc_block"], rep["h2d_bytes"], rep["d2h_bytes"]) == (b, h2d, d2h)
    h.close()


def test_host_product_beta_zero_reads_no_c_and_alpha_zero_scales():
    m, n, k, b = 300, 600, 520, 256
    A = syn.matrix("uniform", m, k, 911)
    B = syn.matrix("uniform", k, n, 912)
    C0 = np.full((m, n), np.nan, order="F")
    h = M.Handle(mode=M.MODE_EMULATED, slices=8)
    C, rep = run_host(h, A, B, C0, -2.0, 0.0, block=b)
    Cref, N = reference(A, B, None, -2.0, 0.0)
    assert max_ratio(C, Cref, k, 2.0, 0.0, N) <= 1.0
    h2d, d2h = closed_form_bytes(m, n, k, b, False)
    assert (rep["h2d_bytes"], rep["d2h_bytes"]) == (h2d, d2h)
    C1 = syn.matrix("uniform", m, n, 913)
    C, rep = run_host(h, A, B, C1, 0.0, 3.0, block=b)
    assert np.array_equal(C, 3.0 * C1)
    assert rep["h2d_bytes"] == 8 * m * n and rep["d2h_bytes"] == 8 * m * n
    h.close()


def test_host_product_block_from_budget_and_argument_errors():
    m, n, k = 640, 640, 640
    A = syn.matrix("uniform", m, k, 921)
    B = syn.matrix("uniform", k, n, 922)
    C0 = syn.matrix("uniform", m, n, 923)
    h = M.Handle(mode=M.MODE_NATIVE)
    # six 256 x 256 FP64 buffers fit in 4 MB, six 512 x 512 ones do not
    C, rep = run_host(h, A, B, C0, 1.0, 1.0, device_bytes=4 << 20)
    assert rep["ooc_block"] == 256
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(C, Cref, k, 1.0, 1.0, N, C0) <= 1.0
    assert M.momms_gemm_host(h, m, n, k, 1.0, 1 << 40, m, 1 << 41, k, 1.0, 1 << 42, m, 0, 300) == -14
    assert M.momms_gemm_host(h, m, n, k, 1.0, 1 << 40, m - 1, 1 << 41, k, 1.0, 1 << 42, m, 0, 256) == -7
    h.close()


@pytest.mark.parametrize("shape", [(700, 530, 900), (600, 1100, 256), (300, 200, 700)])
@pytest.mark.parametrize("member", [M.MEMBER_C2, M.MEMBER_A1])
@pytest.mark.parametrize("beta", [1.0, 0.0])
def test_four_level_members_resident_a_and_c_at_the_hbm_level(shape, member, beta):
    # the four-level composition: the HBM-level member (Resident C or Resident A over host memory)
    # times the L2-level member of each block product (C2 blocked, or A1: L2 not blocked for, the
    # paper's skipped level, Sec. 4.3).  Host<->device bytes equal the closed forms of the
    # HBM-level member exactly, the report names both members, and C meets the bound
    m, n, k = shape
    b = 256
    A = syn.matrix("uniform", m, k, 931)
    B = syn.matrix("uniform", k, n, 932)
    C0 = syn.matrix("uniform", m, n, 933) if beta else np.full((m, n), np.nan, order="F")
    for resident in (0, 1):
        h = M.Handle(mode=M.MODE_EMULATED, member=member)
        h.set_host_resident(resident)
        C, rep = run_host(h, A, B, C0, 1.0, beta, block=b)
        assert h.device_status() == M.MOMMS_OK
        Cref, N = reference(A, B, C0 if beta else None, 1.0, beta)
        assert max_ratio(C, Cref, k, 1.0, beta, N, C0 if beta else None) <= 1.0
        if resident:
            w = I.resident_a_words(m, n, k, b, b, c_read=beta != 0.0)
        else:
            w = I.resident_c_words(m, n, k, b, b, c_read=beta != 0.0)
        h2d = 8 * (w["a_reads"] + w["b_reads"] + w["c_reads"])
        assert (rep["ooc_resident"], rep["h2d_bytes"], rep["d2h_bytes"]) == (resident, h2d, 8 * w["c_writes"])
        assert rep["member"] == member
        h.close()
