"""The C-ABI library builds, loads and exports every symbol include/momms.h declares,
and rejects invalid arguments (BLAS-style index) before touching a GPU.  CPU only."""
import ctypes

import pytest

from paper_1904_05717_gb300 import momms as M


@pytest.fixture(scope="module")
def L():
    return M.lib(build_if_missing=True)


def test_every_declared_symbol_is_exported(L):
    syms = M.header_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing
    # and the binding marshals every one of them
    assert set(syms) == set(M._SIGS)


def test_status_strings(L):
    assert M.status_string(0) == "ok"
    assert "timeout" in M.status_string(M.MOMMS_ERR_TIMEOUT) or "wait" in M.status_string(M.MOMMS_ERR_TIMEOUT)
    assert M.status_string(-3) == "invalid argument"


@pytest.mark.parametrize("args,expect", [
    ((-1, 2, 3, 1.0, 8, 1, 8, 3, 0.0, 8, 1), -1),       # m < 0
    ((2, -2, 3, 1.0, 8, 2, 8, 3, 0.0, 8, 2), -2),       # n < 0
    ((2, 2, -3, 1.0, 8, 2, 8, 3, 0.0, 8, 2), -3),       # k < 0
    ((4, 2, 3, 1.0, 8, 3, 8, 3, 0.0, 8, 4), -6),        # lda < m
    ((4, 2, 3, 1.0, 8, 4, 8, 2, 0.0, 8, 4), -8),        # ldb < k
    ((4, 2, 3, 1.0, 8, 4, 8, 3, 0.0, 8, 3), -11),       # ldc < m
    ((4, 2, 3, 1.0, 0, 4, 8, 3, 0.0, 8, 4), -5),        # A null with work to do
    ((4, 2, 3, 1.0, 8, 4, 0, 3, 0.0, 8, 4), -7),        # B null
    ((4, 2, 3, 1.0, 8, 4, 8, 3, 0.0, 0, 4), -10),       # C null
])
def test_gemm_argument_errors(L, args, expect):
    m, n, k, alpha, A, lda, B, ldb, beta, C, ldc = args
    # pointers here are fake non-null addresses: validation fails before any CUDA call
    big = 1 << 40
    p = lambda v: 0 if v == 0 else big + v * (1 << 30)
    rc = M.momms_gemm(m, n, k, alpha, p(A), lda, p(B), ldb, beta, p(C), ldc, 0)
    assert rc == expect


def test_overlapping_c_is_rejected(L):
    base = 1 << 40
    # C aliases A
    rc = M.momms_gemm(8, 8, 8, 1.0, base, 8, base + (1 << 30), 8, 0.0, base + 64, 8, 0)
    assert rc == -10


def test_step_entry_points_validate(L):
    assert M.momms_emu_scale(2, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 0) == -1
    assert M.momms_emu_scale(0, 3, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 0) == -2
    assert M.momms_emu_scale(0, 0, 4, 4, 1 << 40, 3, 1 << 41, 1 << 42, 0) == -6
    # rows_pad must hold every row
    assert M.momms_emu_split(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 5, 7, 1 << 43, 3, 64, 0) == -12
    assert M.momms_emu_split(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 0, 7, 1 << 43, 128, 64, 0) == -9
    assert M.momms_emu_split(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 5, 11, 1 << 43, 128, 64, 0) == -10


def test_null_handle_is_rejected(L):
    assert L.momms_set_mode(None, 1) == M.MOMMS_ERR_HANDLE
    assert L.momms_gemm_ex(None, 0, 0, 1, 1, 1, 1.0, None, 1, None, 1, 0.0, None, 1, None) == M.MOMMS_ERR_HANDLE
    r = M.Report()
    assert L.momms_get_last_report(None, ctypes.byref(r)) == M.MOMMS_ERR_HANDLE
    assert L.momms_set_max_ctas(None, 4) == M.MOMMS_ERR_HANDLE
    assert L.momms_set_raster_group(None, 4) == M.MOMMS_ERR_HANDLE
    assert M.momms_gemm_host(None, 4, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4, 0.0, 1 << 42, 4, stream=0) == \
        M.MOMMS_ERR_HANDLE
    assert M.momms_syrk(None, 0, 0, 4, 4, 1.0, 1 << 40, 4, 0.0, 1 << 41, 4, stream=0) == M.MOMMS_ERR_HANDLE
    assert M.momms_trmm(None, 0, 0, 0, 0, 4, 4, 1.0, 1 << 40, 4, 1 << 41, 4, stream=0) == M.MOMMS_ERR_HANDLE


def test_stream_copy_validates_before_launch(L):
    base = 1 << 40

    def copy(dst, src, nbytes, ctas=0, repeats=1):
        return M.momms_stream_copy(dst, src, nbytes, ctas, repeats, stream=0)
    assert copy(base + 8, base + (1 << 30), 64) == -1       # dst not 16-byte aligned
    assert copy(base, base + (1 << 30) + 4, 64) == -2       # src not 16-byte aligned
    assert copy(base, base + (1 << 30), 63) == -3           # not a multiple of 16
    assert copy(base, base + (1 << 30), 64, ctas=-1) == -4
    assert copy(base, base + (1 << 30), 64, repeats=-1) == -5
    assert copy(base, base + 32, 64) == -1                  # overlapping ranges
    assert copy(base, base + (1 << 30), 0) == 0             # nothing to copy


def test_default_group_minimises_wave_rows():
    # the library's default C2 group (momms_member_tile with group 0) is the candidate with the
    # fewest operand rows over all waves; brute force over every group here
    from paper_1904_05717_gb300 import iomodel as I
    for tiles_m, tiles_n, ctas in [(64, 43, 152), (32, 22, 152), (128, 86, 152), (10, 7, 38), (64, 43, 76)]:
        def cost(g):
            return sum(r * 128 + c * 192 for r, c in I.waves(M.MEMBER_C2, tiles_m, tiles_n, ctas, g))
        default = cost(0)
        assert default == min(cost(g) for g in range(1, tiles_m + 1))


def test_crt_moduli_are_the_fewest_greedy_moduli(L):
    # host-only planning call: the library's moduli are the oracle's greedy coprime moduli,
    # as few as the range argument with a factor-2 margin allows (|product| <= P / 4)
    import oracle
    ref = oracle.greedy_moduli(16)
    for bits, k in [(7, 1), (21, 64), (35, 1024), (39, 8192), (42, 8192), (42, 65536), (49, 2048), (49, 133120),
                    (56, 1), (56, 4096)]:
        need = [n for n in range(1, 17) if oracle.moduli_suffice(ref[:n], bits, k, margin=2)]
        if not need:
            with pytest.raises(M.MommsError):
                M.momms_crt_moduli(bits, k)
            continue
        assert M.momms_crt_moduli(bits, k) == ref[:need[0]], (bits, k)
    with pytest.raises(M.MommsError):
        M.momms_crt_moduli(56, 8192)       # would take 17 moduli
    with pytest.raises(M.MommsError):
        M.momms_crt_moduli(7, 200000)      # the int32 residue sums would overflow
    buf = (ctypes.c_uint32 * 16)()
    cnt = ctypes.c_int(0)
    assert L.momms_crt_moduli(0, 4, ctypes.byref(cnt), buf) == -1
    assert L.momms_crt_moduli(10, 0, ctypes.byref(cnt), buf) == -2
    # the residue split validates before any launch
    assert M.momms_emu_residues(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 0, 4, 1 << 43, 128, 64, 0) == -9
    assert M.momms_emu_residues(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 21, 4, 1 << 43, 3, 64, 0) == -12
    assert M.momms_emu_residues(0, 0, 4, 4, 1 << 40, 4, 1 << 41, 1 << 42, 56, 8192, 1 << 43, 128, 64, 0) == \
        M.MOMMS_ERR_UNSUPPORTED
    assert L.momms_set_scheme(None, 1) == M.MOMMS_ERR_HANDLE
    # the residue product and the reconstruction validate before any launch
    assert M.momms_emu_residue_gemm(4, 4, 0, 21, 1 << 40, 1 << 41, 4, 4, 64, 0, 1 << 42, 1 << 43, 1 << 20,
                                    1 << 44, stream=0) == -3
    assert M.momms_emu_residue_gemm(4, 4, 4, 21, 1 << 40, 1 << 41, 4, 4, 60, 0, 1 << 42, 1 << 43, 1 << 20,
                                    1 << 44, stream=0) == -9
    assert M.momms_emu_residue_gemm(4, 4, 4, 21, 1 << 40, 1 << 41, 4, 4, 64, 7, 1 << 42, 1 << 43, 1 << 20,
                                    1 << 44, stream=0) == -10
    assert M.momms_crt_reconstruct(4, 4, 4, 57, 1 << 40, 1 << 41, 1 << 42, 1 << 43, 1 << 44, 1.0, 0.0,
                                   1 << 45, 4, stream=0) == -4
    assert M.momms_crt_reconstruct(4, 4, 4, 21, 1 << 40, 1 << 41, 1 << 42, 1 << 43, 1 << 44, 1.0, 0.0,
                                   1 << 45, 3, stream=0) == -13
    assert M.momms_crt_reconstruct(4, 4, 8192, 56, 1 << 40, 1 << 41, 1 << 42, 1 << 43, 1 << 44, 1.0, 0.0,
                                   1 << 45, 4, stream=0) == M.MOMMS_ERR_UNSUPPORTED
