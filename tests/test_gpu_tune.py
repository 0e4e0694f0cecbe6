"""Plan cache: momms_tune times the candidate plans per size bucket, persists them, and a
fresh handle loading the file uses them; a file written for another device is ignored."""
import os

import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import momms as M
from paper_1904_05717_gb300 import synthetic as syn
from util import max_ratio

pytestmark = pytest.mark.gpu


def test_tune_persist_reload(tmp_path):
    path = str(tmp_path / "plans.txt")
    shapes = [(512, 512, 512), (2048, 2048, 256), (1024, 768, 2048, M.OP_T, M.OP_N)]
    h = M.Handle()
    log = tmp_path / "tune.log"
    os.environ["MOMMS_TUNE_LOG"] = str(log)
    try:
        h.tune(shapes, path)
    finally:
        del os.environ["MOMMS_TUNE_LOG"]
    assert os.path.exists(path)
    lines = open(path).read().strip().splitlines()
    assert lines[0].startswith("momms-plan v2 ")
    assert len(lines) == 1 + len(shapes)
    for ln in lines[1:]:
        key, mode, member, slices, tile_n, scheme, pairs = (int(x) for x in ln.split())
        assert mode in (M.MODE_NATIVE, M.MODE_EMULATED) and member in (1, 2, 3, 4) and slices >= 0
        assert tile_n in (0, 96, 192) and scheme in (0, 1, 2) and pairs in (0, 1, 2)
    # every candidate was timed: native + 4 members x (2 widths x 2 encodings + pairs on the wide moduli)
    timed = log.read_text().strip().splitlines()
    assert len(timed) == len(shapes) * (1 + 4 * 5)
    # the transposed bucket is its own; its untransposed neighbour is untuned
    assert h.plan(1024, 768, 2048, M.OP_T, M.OP_N)["tuned"] == 1
    assert h.plan(1024, 768, 2048)["tuned"] == 0
    # a fresh handle loads the plans and still computes the right product
    h2 = M.Handle()
    assert h2.load_plans(path) == M.MOMMS_OK
    m, n, k = shapes[0]
    A = syn.matrix("uniform", m, k, 301)
    B = syn.matrix("uniform", k, n, 302)
    dA, dB, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix(m, n)
    M.gemm(dA, dB, dC, 1.0, 0.0, handle=h2)
    Cref = oracle.dgemm(A, B)
    assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 0.0, oracle.dgemm_abs(A, B)) <= 1.0
    # the call ran the tuned plan
    plan, rep = h2.plan(m, n, k), h2.report()
    assert plan["tuned"] == 1 and rep["mode"] == plan["mode"] and rep["member"] == plan["member"]


@pytest.mark.parametrize("mode,member,tile_n,scheme,pairs", [
    (M.MODE_EMULATED, 2, 96, M.SCHEME_SLICES, 1),
    (M.MODE_EMULATED, 3, 192, M.SCHEME_MODULI, 2),
    (M.MODE_EMULATED, 4, 192, M.SCHEME_MODULI, 1),
    (M.MODE_NATIVE, 1, 0, M.SCHEME_AUTO, 0),
])
def test_the_plan_in_the_file_is_what_runs(tmp_path, mode, member, tile_n, scheme, pairs):
    # a plan file written by hand for one bucket: the call of that bucket runs exactly that plan
    m, n, k = 1500, 1300, 700
    h0 = M.Handle()
    h0.tune([(64, 64, 64)], str(tmp_path / "hdr.txt"))
    header = open(tmp_path / "hdr.txt").read().splitlines()[0]
    key = (11 | (11 << 8) | (10 << 16))  # ceil log2 of 1500, 1300, 700; op N, N
    path = tmp_path / "plan.txt"
    path.write_text(f"{header}\n{key} {mode} {member} 0 {tile_n} {scheme} {pairs}\n")
    h = M.Handle()
    assert h.load_plans(str(path)) == M.MOMMS_OK
    assert h.plan(m, n, k) == {"tuned": 1, "mode": mode, "member": member, "slices": 0, "tile_n": tile_n,
                               "scheme": scheme, "cta_pairs": pairs}
    A = syn.matrix("uniform", m, k, 311)
    B = syn.matrix("uniform", k, n, 312)
    C0 = syn.matrix("uniform", m, n, 313)
    dA, dB, dC = M.DeviceMatrix.from_numpy(A), M.DeviceMatrix.from_numpy(B), M.DeviceMatrix.from_numpy(C0)
    M.gemm(dA, dB, dC, 1.0, 1.0, handle=h)
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    assert rep["mode"] == mode and rep["member"] == member
    if mode == M.MODE_EMULATED:
        assert rep["tile_n"] == tile_n
        assert (rep["moduli"] > 0) == (scheme == M.SCHEME_MODULI)
        assert rep["cta_pairs"] == (1 if pairs == 2 else 0)
    Cref = oracle.dgemm(A, B, C0.copy(order="F"), 1.0, 1.0)
    assert max_ratio(dC.to_numpy(), Cref, k, 1.0, 1.0, oracle.dgemm_abs(A, B), C0) <= 1.0


def test_stale_plan_file_is_ignored(tmp_path):
    path = tmp_path / "stale.txt"
    path.write_text("momms-plan v2 SomeOtherGPU sms=1 l2=1\n1 2 1 8 0 0 0\n")
    h = M.Handle()
    assert h.load_plans(str(path)) == M.MOMMS_ERR_IO
    path.write_text("garbage\n")
    assert h.load_plans(str(path)) == M.MOMMS_ERR_IO


def test_batched_call_takes_each_problems_plan(tmp_path):
    # plans for two buckets: (300, 200, 150) native, (700, 600, 500) emulated on moduli.  Without
    # plans this batch (1.3e9 flops) runs natively as a whole; with them each problem takes its
    # bucket's engine (one native launch beside the emulated pipeline) and all stay within the bound
    h0 = M.Handle()
    h0.tune([(64, 64, 64)], str(tmp_path / "hdr.txt"))
    header = open(tmp_path / "hdr.txt").read().splitlines()[0]
    key_nat = 9 | (8 << 8) | (8 << 16)
    key_emu = 10 | (10 << 8) | (9 << 16)
    path = tmp_path / "plan.txt"
    path.write_text(f"{header}\n{key_nat} {M.MODE_NATIVE} 1 0 0 0 0\n"
                    f"{key_emu} {M.MODE_EMULATED} 1 0 192 {M.SCHEME_MODULI} 1\n")
    sizes = [(300, 200, 150), (700, 600, 500), (290, 210, 140), (650, 620, 480), (257, 129, 200), (513, 600, 300)]
    probs = []
    for i, (m, n, k) in enumerate(sizes):
        probs.append((syn.matrix("uniform", m, k, 321 + 3 * i), syn.matrix("uniform", k, n, 322 + 3 * i),
                      syn.matrix("uniform", m, n, 323 + 3 * i)))
    dev = [tuple(M.DeviceMatrix.from_numpy(x) for x in p) for p in probs]
    cnt = len(sizes)
    args = dict(m=[s_[0] for s_ in sizes], n=[s_[1] for s_ in sizes], k=[s_[2] for s_ in sizes],
                alpha=[1.0] * cnt, A=[d[0].ptr for d in dev], lda=[d[0].ld for d in dev],
                B=[d[1].ptr for d in dev], ldb=[d[1].ld for d in dev], beta=[1.0] * cnt,
                C=[d[2].ptr for d in dev], ldc=[d[2].ld for d in dev])
    h = M.Handle()
    assert h.load_plans(str(path)) == M.MOMMS_OK
    M.check(M.momms_gemm_batched(h, **args), "batched")
    assert h.device_status() == M.MOMMS_OK
    rep = h.report()
    assert rep["mode"] == M.MODE_EMULATED and rep["moduli"] > 0
    for (m, n, k), (A, B, C0), d in zip(sizes, probs, dev):
        Cref = oracle.dgemm(A, B, C0.copy(order="F"), 1.0, 1.0)
        assert max_ratio(d[2].to_numpy(), Cref, k, 1.0, 1.0, oracle.dgemm_abs(A, B), C0) <= 1.0
    # the same batch without plans: one native launch for all
    dev2 = [(dev[i][0], dev[i][1], M.DeviceMatrix.from_numpy(probs[i][2])) for i in range(cnt)]
    args2 = dict(args, C=[d[2].ptr for d in dev2])
    h2 = M.Handle()
    M.check(M.momms_gemm_batched(h2, **args2), "batched")
    assert h2.report()["mode"] == M.MODE_NATIVE and h2.report()["launches"] == 1
