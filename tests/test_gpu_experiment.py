"""Bandwidth-ratio sweep (the paper's varying-bandwidth experiment on one GPU): the
background copy is correct, the handle knobs it uses are honoured, and a product
computed beside the background traffic is bit-identical to the same product alone."""
import numpy as np
import pytest

from paper_1904_05717_gb300 import experiments as E
from paper_1904_05717_gb300 import momms as M

pytestmark = pytest.mark.gpu


def test_stream_copy_copies_every_word():
    import torch
    n = (3 << 20) + 5  # not a multiple of the grid stride: exercises the tail loop
    src = torch.randn(2 * n, dtype=torch.float64, device="cuda")
    dst = torch.zeros_like(src)
    assert M.momms_stream_copy(dst.data_ptr(), src.data_ptr(), src.numel() * 8, 7, 2) == 0
    torch.cuda.synchronize()
    assert torch.equal(dst, src)
    assert M.momms_stream_copy(dst.data_ptr(), src.data_ptr(), src.numel() * 8, 0, 1) == 0
    torch.cuda.synchronize()
    assert torch.equal(dst, src)


def test_handle_knobs_are_reported():
    h = M.Handle(mode=M.MODE_EMULATED, slices=4)
    with pytest.raises(M.MommsError):
        h.set_max_ctas(-1)
    with pytest.raises(M.MommsError):
        h.set_raster_group(-1)
    h.set_max_ctas(9)
    h.set_raster_group(3)
    A = M.DeviceMatrix.from_numpy(np.ones((700, 64), order="F"))
    B = M.DeviceMatrix.from_numpy(np.ones((64, 900), order="F"))
    C = M.DeviceMatrix(700, 900)
    M.gemm(A, B, C, 1.0, 0.0, handle=h)
    rep = h.report()
    assert rep["ctas"] == 9 and rep["group"] == 3
    assert np.array_equal(C.to_numpy(), np.full((700, 900), 64.0))
    h.set_max_ctas(0)
    h.set_raster_group(0)
    M.gemm(A, B, C, 1.0, 0.0, handle=h)
    rep = h.report()
    import torch
    # one unit per tile (digit slices) or per tile and modulus (modular encoding)
    units = -(-700 // 128) * -(-900 // rep["tile_n"]) * max(1, rep["moduli"])
    assert rep["ctas"] == min(torch.cuda.get_device_properties(0).multi_processor_count, units)
    assert rep["group"] >= 1
    h.close()


def test_small_sweep_results_unchanged_beside_background_traffic():
    rows = E.run(size=1024, members=("C2", "A1"), points=((38, 0), (38, 38)), reps=2, native_size=512,
                 check_results=True)
    assert len(rows) == 2 * 2 * 2
    for r in rows:
        assert r["ms"] > 0.0
        assert r["bitwise_equal_to_alone"], r
        if r["engine"] == "emulated":
            assert r["product_ctas"] == 38 and r["model_slice_dram_gb"] > 0.0
    assert "| emulated | 1024 | 38 | 38 | A1 |" in E.table(rows)
