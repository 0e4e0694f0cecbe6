"""The data-driven slice count chosen on the device (momms_set_plan_on_device).

With the default device plan an AUTO / EMULATED product with slices = 0 reads nothing back: a
one-thread kernel turns the measured spreads into S, the operand width and the encoding, and the
split, product and reconstruction kernels read that plan when they start.  The tests check that
the device plan and the host plan (spreads read back) give the same plan and the same C bit for
bit, that the result meets the bound against the oracle, and that such a call captured once in a
CUDA graph replays correctly on new data whose plan differs (moduli for uniform data, digit
slices for the wide-exponent phi = 4 family, whose width exceeds what 16 moduli cover)."""
import numpy as np
import pytest

from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio, reference

pytestmark = pytest.mark.gpu


def product(A, B, C0, alpha, beta, on_device, opa=0, opb=0, mode=M.MODE_EMULATED):
    h = M.Handle(mode=mode)
    h.set_plan_on_device(on_device)
    dA, dB, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, alpha, beta, opa, opb, handle=h)
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    h.close()
    return dC.to_numpy(), rep


@pytest.mark.parametrize("kind,phi,m,n,k,opa,opb", [
    ("uniform", 0.0, 700, 900, 640, 0, 0),
    ("normal", 0.0, 513, 260, 1100, 1, 0),
    ("phi", 1.0, 300, 1000, 520, 0, 1),
    ("phi", 4.0, 640, 500, 700, 1, 1),   # wide exponent range: more bits than 16 moduli cover -> slices
    ("uniform", 0.0, 2048, 2048, 2048, 0, 0),
])
def test_device_plan_equals_host_plan(kind, phi, m, n, k, opa, opb):
    A = syn.matrix(kind, k if opa else m, m if opa else k, 6100, phi=phi)
    B = syn.matrix(kind, n if opb else k, k if opb else n, 6101, phi=phi)
    C0 = syn.matrix("uniform", m, n, 6102)
    Cd, rd = product(A, B, C0, 1.25, -0.5, 1, opa, opb)
    Ch, rh = product(A, B, C0, 1.25, -0.5, 0, opa, opb)
    for key in ("slices", "moduli", "operand_bits"):
        assert rd[key] == rh[key], (key, rd[key], rh[key])
    assert np.array_equal(Cd, Ch)
    Cref, N = reference(A, B, C0, 1.25, -0.5, bool(opa), bool(opb))
    assert max_ratio(Cd, Cref, k, 1.25, 0.5, N, C0) <= 1.0
    if kind == "phi" and phi == 4.0:
        assert rd["moduli"] == 0 and rd["slices"] >= 9
    if kind == "uniform":
        assert rd["moduli"] > 0


def test_auto_product_captured_in_a_graph_replays_on_new_data():
    import torch
    m, n, k = 1000, 1100, 900
    h = M.Handle()  # AUTO: emulated at this size, data-driven S, plan on the device
    dA, dB, dC = M.DeviceMatrix(m, k), M.DeviceMatrix(k, n), M.DeviceMatrix(m, n)
    first = [syn.matrix("uniform", m, k, 6200), syn.matrix("uniform", k, n, 6201), syn.matrix("uniform", m, n, 6202)]
    for d, x in zip((dA, dB, dC), first):
        d.storage.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        M.check(M.momms_gemm_ex(h, 0, 0, m, n, k, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0, dC.ptr, dC.ld, s),
                "warm-up")  # sizes the workspace: the captured call allocates nothing
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_ex(h, 0, 0, m, n, k, 1.0, dA.ptr, dA.ld, dB.ptr, dB.ld, 1.0, dC.ptr, dC.ld, s),
                "capture")
    plans = []
    for kind, phi, seed in (("uniform", 0.0, 6300), ("phi", 4.0, 6400), ("normal", 0.0, 6500)):
        A = syn.matrix(kind, m, k, seed, phi=phi)
        B = syn.matrix(kind, k, n, seed + 1, phi=phi)
        C0 = syn.matrix("uniform", m, n, seed + 2)
        for d, x in zip((dA, dB, dC), (A, B, C0)):
            d.storage.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert h.device_status() == M.MOMMS_OK
        rep = h.report()  # the plan the replay used, read from the device
        plans.append((rep["slices"], rep["moduli"], rep["operand_bits"]))
        Cref, N = reference(A, B, C0, 1.0, 1.0)
        assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 1.0, N, C0) <= 1.0, (kind, rep)
    assert plans[0][1] > 0 and plans[1][1] == 0  # moduli for uniform data, digit slices for phi = 4
    assert plans[1][0] > plans[0][0]
    h.close()
