"""The timeout path of the tcgen05 product kernel, made to run on purpose without a fault.

momms_debug_withhold_load() makes the next slice- or residue-product launch leave the first
shared-memory stage of CTA 0 empty (its bytes are announced, no copy is issued).  The MMA
thread's bounded wait on that stage runs out after about 2 s; the CTA raises its abort flag,
waits (bounded) for its issued copies and MMAs, frees its tensor memory and writes
MOMMS_ERR_TIMEOUT to the launch's status word.  The tests read that status back and then
check that the next product on the same handle is correct (the context, TMEM and the
handle's status word are usable again)."""
import numpy as np
import pytest

from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio, reference

pytestmark = pytest.mark.gpu


def inputs(m, n, k, seed):
    A = syn.matrix("uniform", m, k, seed)
    B = syn.matrix("uniform", k, n, seed + 1)
    C0 = syn.matrix("uniform", m, n, seed + 2)
    return A, B, C0


@pytest.mark.parametrize("scheme,slices", [(M.SCHEME_MODULI, 6), (M.SCHEME_SLICES, 8), (M.SCHEME_AUTO, 0)])
def test_withheld_stage_times_out_and_the_next_product_is_correct(scheme, slices):
    m, n, k = 700, 900, 640
    A, B, C0 = inputs(m, n, k, 5100)
    h = M.Handle(mode=M.MODE_EMULATED, slices=slices, scheme=scheme)
    dA, dB = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B)
    assert h.device_status() == M.MOMMS_OK

    M.momms_debug_withhold_load()
    dC = M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)  # enqueues; the launch itself succeeds
    assert h.device_status() == M.MOMMS_ERR_TIMEOUT
    assert h.device_status() == M.MOMMS_OK  # reading the status cleared it

    # the same handle, right after: every SM's tensor memory was freed, C is correct
    dC = M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)
    assert h.device_status() == M.MOMMS_OK
    Cref, N = reference(A, B, C0, 1.0, 1.0)
    assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 1.0, N, C0) <= 1.0
    h.close()


def test_withheld_stage_in_a_batched_call():
    # the batched residue-product launch takes the hook too; the call after it is correct
    sizes = [(130, 200, 300), (64, 64, 64), (257, 100, 513)]
    probs = [inputs(m, n, k, 5200 + 10 * i) for i, (m, n, k) in enumerate(sizes)]
    h = M.Handle(mode=M.MODE_EMULATED, slices=8, scheme=M.SCHEME_MODULI)
    dA = [M.DeviceMatrix.from_numpy(A) for A, _, _ in probs]
    dB = [M.DeviceMatrix.from_numpy(B) for _, B, _ in probs]
    for attempt in range(2):
        if attempt == 0:
            M.momms_debug_withhold_load()
        dC = [M.DeviceMatrix.from_numpy(C0) for _, _, C0 in probs]
        M.check(M.momms_gemm_batched(
            h, m=[s[0] for s in sizes], n=[s[1] for s in sizes], k=[s[2] for s in sizes], alpha=[1.0] * 3,
            A=[d.ptr for d in dA], lda=[d.ld for d in dA], B=[d.ptr for d in dB], ldb=[d.ld for d in dB],
            beta=[1.0] * 3, C=[d.ptr for d in dC], ldc=[d.ld for d in dC]), "batched")
        st = h.device_status()
        if attempt == 0:
            assert st == M.MOMMS_ERR_TIMEOUT
            continue
        assert st == M.MOMMS_OK
        for (A, B, C0), d, (m, n, k) in zip(probs, dC, sizes):
            Cref, N = reference(A, B, C0, 1.0, 1.0)
            assert max_ratio(d.to_numpy(), Cref, k, 1.0, 1.0, N, C0) <= 1.0
    h.close()
