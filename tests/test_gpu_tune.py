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
    shapes = [(512, 512, 512), (2048, 2048, 256)]
    h = M.Handle()
    h.tune(shapes, path)
    assert os.path.exists(path)
    lines = open(path).read().strip().splitlines()
    assert lines[0].startswith("momms-plan v1 ")
    assert len(lines) == 1 + len(shapes)
    for ln in lines[1:]:
        key, mode, member, slices = (int(x) for x in ln.split())
        assert mode in (M.MODE_NATIVE, M.MODE_EMULATED) and member in (1, 2, 3, 4) and slices >= 0
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


def test_stale_plan_file_is_ignored(tmp_path):
    path = tmp_path / "stale.txt"
    path.write_text("momms-plan v1 SomeOtherGPU sms=1 l2=1\n1 2 1 8\n")
    h = M.Handle()
    assert h.load_plans(str(path)) == M.MOMMS_ERR_IO
    path.write_text("garbage\n")
    assert h.load_plans(str(path)) == M.MOMMS_ERR_IO
