"""Batched uneven products: one persistent launch over a device tile table (native),
the emulated pipeline per problem (digit slices or the modular encoding, chosen per problem),
and CUDA-graph capture and replay."""
import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio

pytestmark = pytest.mark.gpu


def make_problems(count, lo, hi, seed):
    sizes = syn.log_uniform_sizes(seed, count, lo, hi)
    probs = []
    for i, (m, n, k) in enumerate(sizes):
        A = syn.matrix("uniform", int(m), int(k), seed + 10 * i + 1)
        B = syn.matrix("uniform", int(k), int(n), seed + 10 * i + 2)
        C = syn.matrix("uniform", int(m), int(n), seed + 10 * i + 3)
        probs.append((int(m), int(n), int(k), A, B, C))
    return probs


def run_batched(h, probs, alpha=1.0, beta=1.0):
    dev = [(M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C))
           for (_, _, _, A, B, C) in probs]
    cnt = len(probs)
    args = dict(
        m=[p[0] for p in probs], n=[p[1] for p in probs], k=[p[2] for p in probs],
        alpha=[alpha] * cnt, A=[d[0].ptr for d in dev], lda=[d[0].ld for d in dev],
        B=[d[1].ptr for d in dev], ldb=[d[1].ld for d in dev], beta=[beta] * cnt,
        C=[d[2].ptr for d in dev], ldc=[d[2].ld for d in dev])
    M.check(M.momms_gemm_batched(h, **args), "batched")
    return dev, args


def check_all(probs, dev, alpha=1.0, beta=1.0):
    worst = 0.0
    for (m, n, k, A, B, C), d in zip(probs, dev):
        Cref = oracle.dgemm(A, B, C.copy(order="F"), alpha, beta)
        N = oracle.dgemm_abs(A, B)
        worst = max(worst, max_ratio(d[2].to_numpy(), Cref, k, alpha, beta, N, C))
    return worst


def test_batched_native_one_launch():
    probs = make_problems(60, 32, 400, 3000)
    h = M.Handle(mode=M.MODE_NATIVE)
    dev, _ = run_batched(h, probs)
    rep = h.report()
    assert rep["launches"] == 1
    assert check_all(probs, dev) <= 1.0


def test_batched_emulated():
    probs = make_problems(12, 64, 700, 4000)
    h = M.Handle(mode=M.MODE_EMULATED)
    dev, _ = run_batched(h, probs)
    assert h.device_status() == M.MOMMS_OK
    assert check_all(probs, dev) <= 1.0


def test_batched_with_empty_and_k_zero_problems():
    probs = make_problems(5, 32, 100, 5000)
    probs.append((0, 7, 3, np.zeros((0, 3), order="F"), syn.matrix("uniform", 3, 7, 1), np.zeros((0, 7), order="F")))
    C0 = syn.matrix("uniform", 9, 4, 2)
    probs.append((9, 4, 0, np.zeros((9, 0), order="F"), np.zeros((0, 4), order="F"), C0))
    h = M.Handle(mode=M.MODE_NATIVE)
    dev, _ = run_batched(h, probs, 1.0, 2.0)
    assert np.array_equal(dev[-1][2].to_numpy(), 2.0 * C0)
    assert check_all(probs[:5], dev[:5], 1.0, 2.0) <= 1.0


def test_batched_native_cuda_graph_replay():
    import torch
    probs = make_problems(40, 32, 300, 6000)
    h = M.Handle(mode=M.MODE_NATIVE)
    dev, args = run_batched(h, probs, 1.0, 0.0)  # eager call uploads the tile table
    torch.cuda.synchronize()
    eager = [d[2].to_numpy() for d in dev]
    for d in dev:
        d[2].storage.fill_(float("nan"))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_batched(h, stream=s, **args), "capture")
    g.replay()
    torch.cuda.synchronize()
    for d, e in zip(dev, eager):
        assert np.array_equal(d[2].to_numpy(), e)


def test_batched_2000_uneven_problems_native_one_launch():
    # the batched workload: 2000 problems, m, n, k log-uniform in [32, 2048], uniform[-1, 1];
    # one persistent launch; every 10th problem checked against the oracle in full
    import torch
    count = 2000
    sizes = syn.log_uniform_sizes(syn.workload_seed(4, "A"), count, 32, 2048)
    h = M.Handle(mode=M.MODE_NATIVE)
    dev, hosts = [], []
    for i, (m, n, k) in enumerate(sizes):
        m, n, k = int(m), int(n), int(k)
        A = syn.matrix("uniform", m, k, 100000 + 3 * i)
        B = syn.matrix("uniform", k, n, 100001 + 3 * i)
        C = syn.matrix("uniform", m, n, 100002 + 3 * i)
        dev.append((M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C)))
        hosts.append((m, n, k, A, B, C) if i % 10 == 0 else None)
    args = dict(m=[int(s[0]) for s in sizes], n=[int(s[1]) for s in sizes], k=[int(s[2]) for s in sizes],
                alpha=[1.0] * count, A=[d[0].ptr for d in dev], lda=[d[0].ld for d in dev],
                B=[d[1].ptr for d in dev], ldb=[d[1].ld for d in dev], beta=[1.0] * count,
                C=[d[2].ptr for d in dev], ldc=[d[2].ld for d in dev])
    M.check(M.momms_gemm_batched(h, **args), "batched 2000")
    torch.cuda.synchronize()
    assert h.report()["launches"] == 1
    worst = 0.0
    for hst, d in zip(hosts, dev):
        if hst is None:
            continue
        m, n, k, A, B, C = hst
        Cref = oracle.dgemm(A, B, C.copy(order="F"), 1.0, 1.0)
        worst = max(worst, max_ratio(d[2].to_numpy(), Cref, k, 1.0, 1.0, oracle.dgemm_abs(A, B), C))
    assert worst <= 1.0


def test_batched_emulated_one_slice_launch_and_graph_replay():
    # fixed slice count: 2 scale + 2 split + ONE slice-product launch, and a captured graph replays it
    import torch
    probs = make_problems(30, 48, 600, 7000)
    h = M.Handle(mode=M.MODE_EMULATED, slices=9)
    dev, args = run_batched(h, probs, 1.0, 0.0)
    torch.cuda.synchronize()
    assert h.report()["launches"] == 5
    assert h.device_status() == M.MOMMS_OK
    assert check_all(probs, dev, 1.0, 0.0) <= 1.0
    eager = [d[2].to_numpy() for d in dev]
    for d in dev:
        d[2].storage.fill_(float("nan"))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_batched(h, stream=s, **args), "capture")
    g.replay()
    torch.cuda.synchronize()
    for d, e in zip(dev, eager):
        assert np.array_equal(d[2].to_numpy(), e)


def test_batched_2000_uneven_problems_emulated():
    # the batched workload in emulated mode (data-driven slice count per problem)
    import torch
    count = 2000
    sizes = syn.log_uniform_sizes(syn.workload_seed(4, "A"), count, 32, 2048)
    h = M.Handle(mode=M.MODE_EMULATED)
    dev, hosts = [], []
    for i, (m, n, k) in enumerate(sizes):
        m, n, k = int(m), int(n), int(k)
        A = syn.matrix("uniform", m, k, 100000 + 3 * i)
        B = syn.matrix("uniform", k, n, 100001 + 3 * i)
        C = syn.matrix("uniform", m, n, 100002 + 3 * i)
        dev.append((M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C)))
        hosts.append((m, n, k, A, B, C) if i % 20 == 0 else None)
    args = dict(m=[int(s[0]) for s in sizes], n=[int(s[1]) for s in sizes], k=[int(s[2]) for s in sizes],
                alpha=[1.0] * count, A=[d[0].ptr for d in dev], lda=[d[0].ld for d in dev],
                B=[d[1].ptr for d in dev], ldb=[d[1].ld for d in dev], beta=[1.0] * count,
                C=[d[2].ptr for d in dev], ldc=[d[2].ld for d in dev])
    M.check(M.momms_gemm_batched(h, **args), "batched 2000 emulated")
    torch.cuda.synchronize()
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    # short k needs more than 56 bits (digit slices), long k takes the moduli: 2 scale, the device
    # plan, 2 split, 2 residue split, the slice-product and residue-product launches and the
    # reconstruction
    assert rep["slices"] > 0 and rep["moduli"] > 0 and rep["launches"] == 10
    worst = 0.0
    for hst, d in zip(hosts, dev):
        if hst is None:
            continue
        m, n, k, A, B, C = hst
        Cref = oracle.dgemm(A, B, C.copy(order="F"), 1.0, 1.0)
        worst = max(worst, max_ratio(d[2].to_numpy(), Cref, k, 1.0, 1.0, oracle.dgemm_abs(A, B), C))
    assert worst <= 1.0


def test_batched_emulated_same_handle_new_problems_reuses_table_memory():
    # two calls on one handle with the same problem count: the second call's tensor maps are
    # uploaded to the same device table as the first call's and must be the ones used
    h = M.Handle(mode=M.MODE_EMULATED, slices=9)
    for seed in (8100, 8200):
        probs = make_problems(6, 64, 500, seed)
        dev, _ = run_batched(h, probs)
        assert h.device_status() == M.MOMMS_OK
        assert check_all(probs, dev) <= 1.0
    h.close()


def test_batched_auto_picks_emulation_by_total_work():
    # AUTO: the emulated pipeline once the batch holds >= 2e9 flops (here ~2.2e9), native below
    big = []
    for i in range(8):
        A = syn.matrix("uniform", 520, 512, 2000 + 3 * i)
        B = syn.matrix("uniform", 512, 530, 2001 + 3 * i)
        C = syn.matrix("uniform", 520, 530, 2002 + 3 * i)
        big.append((520, 530, 512, A, B, C))
    h = M.Handle()
    dev, _ = run_batched(h, big)
    assert h.report()["mode"] == M.MODE_EMULATED
    assert h.device_status() == M.MOMMS_OK
    assert check_all(big, dev) <= 1.0
    small = make_problems(6, 32, 200, 2100)
    dev, _ = run_batched(h, small)
    assert h.report()["mode"] == M.MODE_NATIVE
    assert check_all(small, dev) <= 1.0
    h.close()


def test_batched_moduli_bitwise_and_graph_replay():
    # fixed S = 6 with the modular encoding: every problem's C bit for bit against the oracle's
    # modular result (42-bit operands; 11 moduli at k = 1, 12 at the others), ragged tiles, m not a
    # multiple of four, single rows and columns; then a captured graph replays the call
    import torch
    shapes = [(130, 200, 70), (1, 5, 3), (37, 1, 129), (257, 64, 1), (64, 193, 64), (100, 100, 100)]
    probs = []
    for i, (m, n, k) in enumerate(shapes):
        A = syn.matrix("normal", m, k, 9100 + 3 * i)
        B = syn.matrix("uniform", k, n, 9101 + 3 * i)
        C = syn.matrix("uniform", m, n, 9102 + 3 * i)
        probs.append((m, n, k, A, B, C))
    h = M.Handle(mode=M.MODE_EMULATED, slices=6, scheme=M.SCHEME_MODULI)
    dev, args = run_batched(h, probs, 0.5, -2.0)
    torch.cuda.synchronize()
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    assert rep["moduli"] == 12 and rep["slices"] == 0
    assert rep["launches"] == 6   # 2 scale, 2 residue split, residue products, reconstruction
    eager = []
    for (m, n, k, A, B, C), d in zip(probs, dev):
        Co, _ = oracle.modular_dgemm(A, B, 42, C.copy(order="F"), 0.5, -2.0)
        got = d[2].to_numpy()
        assert np.array_equal(got, Co), (m, n, k)
        eager.append(got)
    for d, (_, _, _, _, _, C) in zip(dev, probs):
        d[2].storage[: C.shape[1], : C.shape[0]].copy_(torch.from_numpy(np.ascontiguousarray(C.T)))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_batched(h, stream=s, **args), "capture")
    for d, (_, _, _, _, _, C) in zip(dev, probs):
        d[2].storage[: C.shape[1], : C.shape[0]].copy_(torch.from_numpy(np.ascontiguousarray(C.T)))
    g.replay()
    torch.cuda.synchronize()
    for d, e in zip(dev, eager):
        assert np.array_equal(d[2].to_numpy(), e)
    h.close()


def test_batched_mixed_encodings_within_the_bound():
    # data-driven S: k = 40 needs more than 56 bits (digit slices), k = 2048 and 3000 take the moduli
    # (their reconstruction is paid for); one call runs both product launches
    probs = []
    for i, (m, n, k) in enumerate([(300, 260, 40), (200, 330, 2048), (129, 97, 33), (256, 256, 3000)]):
        A = syn.matrix("uniform", m, k, 9200 + 3 * i)
        B = syn.matrix("uniform", k, n, 9201 + 3 * i)
        C = syn.matrix("uniform", m, n, 9202 + 3 * i)
        probs.append((m, n, k, A, B, C))
    h = M.Handle(mode=M.MODE_EMULATED)
    dev, _ = run_batched(h, probs, 1.0, 1.0)
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    assert rep["slices"] > 0 and rep["moduli"] > 0 and rep["launches"] == 10  # (with the device plan kernel)
    assert check_all(probs, dev) <= 1.0
    h.close()


def test_batched_auto_device_plan_equals_host_plan_and_replays_from_a_graph():
    # AUTO batched call with the slice count of every problem chosen on the device (nothing read
    # back): bit for bit the host plan's result, within the bound against the oracle, and the same
    # call captured in a CUDA graph replays it exactly
    import torch
    probs = make_problems(200, 32, 1024, 8000)
    hd = M.Handle(mode=M.MODE_EMULATED)
    hh = M.Handle(mode=M.MODE_EMULATED)
    hh.set_plan_on_device(0)
    dev_d, args_d = run_batched(hd, probs, 1.0, 1.0)
    dev_h, _ = run_batched(hh, probs, 1.0, 1.0)
    torch.cuda.synchronize()
    assert hd.device_status() == M.MOMMS_OK and hh.device_status() == M.MOMMS_OK
    rd, rh = hd.report(), hh.report()
    assert (rd["slices"], rd["moduli"]) == (rh["slices"], rh["moduli"])
    for a, b in zip(dev_d, dev_h):
        assert np.array_equal(a[2].to_numpy(), b[2].to_numpy())
    assert check_all(probs, dev_d, 1.0, 1.0) <= 1.0
    eager = [d[2].to_numpy() for d in dev_d]
    for d, p in zip(dev_d, probs):
        d[2].storage.copy_(torch.from_numpy(np.ascontiguousarray(p[5].T)))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_batched(hd, stream=s, **args_d), "capture")
    g.replay()
    torch.cuda.synchronize()
    assert hd.device_status() == M.MOMMS_OK
    for d, e in zip(dev_d, eager):
        assert np.array_equal(d[2].to_numpy(), e)


def test_batched_2000_auto_graph_capture():
    # the batched workload (2000 problems, m, n, k log-uniform in [32, 2048]) in AUTO mode captured in
    # a CUDA graph after one eager call: the replay equals the eager result bit for bit; every 20th
    # problem against the oracle
    import torch
    count = 2000
    sizes = syn.log_uniform_sizes(syn.workload_seed(4, "A"), count, 32, 2048)
    h = M.Handle()
    dev, hosts = [], []
    for i, (m, n, k) in enumerate(sizes):
        m, n, k = int(m), int(n), int(k)
        A = syn.matrix("uniform", m, k, 100000 + 3 * i)
        B = syn.matrix("uniform", k, n, 100001 + 3 * i)
        C = syn.matrix("uniform", m, n, 100002 + 3 * i)
        dev.append((M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C)))
        hosts.append((m, n, k, A, B, C) if i % 20 == 0 else (None, None, None, None, None, C))
    args = dict(m=[int(s_[0]) for s_ in sizes], n=[int(s_[1]) for s_ in sizes], k=[int(s_[2]) for s_ in sizes],
                alpha=[1.0] * count, A=[d[0].ptr for d in dev], lda=[d[0].ld for d in dev],
                B=[d[1].ptr for d in dev], ldb=[d[1].ld for d in dev], beta=[1.0] * count,
                C=[d[2].ptr for d in dev], ldc=[d[2].ld for d in dev])
    M.check(M.momms_gemm_batched(h, **args), "eager")
    torch.cuda.synchronize()
    assert h.device_status() == M.MOMMS_OK
    assert h.report()["mode"] == M.MODE_EMULATED
    eager = [d[2].to_numpy() for d in dev]
    for d, hst in zip(dev, hosts):
        d[2].storage.copy_(torch.from_numpy(np.ascontiguousarray(hst[5].T)))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        M.check(M.momms_gemm_batched(h, stream=s, **args), "capture")
    g.replay()
    torch.cuda.synchronize()
    assert h.device_status() == M.MOMMS_OK
    worst = 0.0
    for d, e, hst in zip(dev, eager, hosts):
        got = d[2].to_numpy()
        assert np.array_equal(got, e)
        if hst[0] is not None:
            m, n, k, A, B, C = hst
            Cref = oracle.dgemm(A, B, C.copy(order="F"), 1.0, 1.0)
            worst = max(worst, max_ratio(got, Cref, k, 1.0, 1.0, oracle.dgemm_abs(A, B), C))
    assert worst <= 1.0
