"""Python binding of libmomms (the C ABI in include/momms.h).

Argument marshalling only: every step of the product runs in the library's CUDA
kernels.  The functions keep the C names (``momms_gemm``, ``momms_gemm_ex`` ...)
and take device pointers as Python ints; ``DeviceMatrix`` and ``matmul`` are
conveniences that hold column-major matrices in torch CUDA memory.  There is no
CPU fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

MOMMS_OK = 0
MOMMS_ERR_CUDA = 1001
MOMMS_ERR_TIMEOUT = 1002
MOMMS_ERR_NONFINITE = 1003
MOMMS_ERR_WORKSPACE = 1004
MOMMS_ERR_UNSUPPORTED = 1005
MOMMS_ERR_ALLOC = 1006
MOMMS_ERR_HANDLE = 1007
MOMMS_ERR_IO = 1008

OP_N, OP_T = 0, 1
LOWER, UPPER = 0, 1
LEFT, RIGHT = 0, 1
NON_UNIT, UNIT = 0, 1
MODE_AUTO, MODE_NATIVE, MODE_EMULATED = 0, 1, 2
SCHEME_AUTO, SCHEME_SLICES, SCHEME_MODULI = 0, 1, 2
MEMBER_AUTO, MEMBER_C2, MEMBER_A2, MEMBER_B2, MEMBER_A1 = 0, 1, 2, 3, 4
MEMBER_NAMES = {MEMBER_C2: "C2", MEMBER_A2: "A2", MEMBER_B2: "B2", MEMBER_A1: "A1"}
MAX_SLICES = 16


class MommsError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: status {status} ({status_string(status)})")


class Report(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("member", ctypes.c_int), ("slices", ctypes.c_int),
                ("digit_bits", ctypes.c_int), ("k_passes", ctypes.c_int), ("tile_m", ctypes.c_int),
                ("tile_n", ctypes.c_int), ("ctas", ctypes.c_int), ("group", ctypes.c_int),
                ("launches", ctypes.c_int64), ("est_err_ratio", ctypes.c_double),
                ("ooc_block", ctypes.c_int64), ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64),
                ("moduli", ctypes.c_int), ("operand_bits", ctypes.c_int), ("crt_fused", ctypes.c_int),
                ("cta_pairs", ctypes.c_int), ("ooc_resident", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanT(ctypes.Structure):
    _fields_ = [("tuned", ctypes.c_int), ("mode", ctypes.c_int), ("member", ctypes.c_int), ("slices", ctypes.c_int),
                ("tile_n", ctypes.c_int), ("scheme", ctypes.c_int), ("cta_pairs", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

_I64, _I32, _DBL, _VP, _SZ = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
_SIGS = {
    "momms_create": ([ctypes.POINTER(_VP)], _I32),
    "momms_destroy": ([_VP], _I32),
    "momms_set_mode": ([_VP, _I32], _I32),
    "momms_set_member": ([_VP, _I32], _I32),
    "momms_set_slices": ([_VP, _I32], _I32),
    "momms_set_max_ctas": ([_VP, _I32], _I32),
    "momms_set_raster_group": ([_VP, _I32], _I32),
    "momms_set_tile_n": ([_VP, _I32], _I32),
    "momms_set_scheme": ([_VP, _I32], _I32),
    "momms_set_plan_on_device": ([_VP, _I32], _I32),
    "momms_set_host_resident": ([_VP, _I32], _I32),
    "momms_set_cta_pairs": ([_VP, _I32], _I32),
    "momms_set_crt_fusion": ([_VP, _I32], _I32),
    "momms_trsm": ([_VP, _I32, _I32, _I32, _I32, _I64, _I64, _DBL, _VP, _I64, _VP, _I64, _VP], _I32),
    "momms_crt_moduli": ([_I32, _I64, _VP, _VP], _I32),
    "momms_emu_residue_gemm": ([_I64, _I64, _I64, _I32, _VP, _VP, _I64, _I64, _I64, _I32, _VP, _VP, _SZ, _VP, _VP],
                               _I32),
    "momms_crt_reconstruct": ([_I64, _I64, _I64, _I32, _VP, _VP, _VP, _VP, _VP, _DBL, _DBL, _VP, _I64, _VP], _I32),
    "momms_emu_residues": ([_I32, _I32, _I64, _I64, _VP, _I64, _VP, _VP, _I32, _I64, _VP, _I64, _I64, _VP], _I32),
    "momms_get_last_report": ([_VP, ctypes.POINTER(Report)], _I32),
    "momms_check_device_status": ([_VP, _VP], _I32),
    "momms_status_string": ([_I32], ctypes.c_char_p),
    "momms_workspace_size": ([_VP, _I32, _I32, _I64, _I64, _I64, ctypes.POINTER(_SZ)], _I32),
    "momms_set_workspace": ([_VP, _VP, _SZ], _I32),
    "momms_gemm": ([_I64, _I64, _I64, _DBL, _VP, _I64, _VP, _I64, _DBL, _VP, _I64, _VP], _I32),
    "momms_gemm_ex": ([_VP, _I32, _I32, _I64, _I64, _I64, _DBL, _VP, _I64, _VP, _I64, _DBL, _VP, _I64, _VP], _I32),
    "momms_gemm_host": ([_VP, _I64, _I64, _I64, _DBL, _VP, _I64, _VP, _I64, _DBL, _VP, _I64, _SZ, _I64, _VP], _I32),
    "momms_syrk": ([_VP, _I32, _I32, _I64, _I64, _DBL, _VP, _I64, _DBL, _VP, _I64, _VP], _I32),
    "momms_trmm": ([_VP, _I32, _I32, _I32, _I32, _I64, _I64, _DBL, _VP, _I64, _VP, _I64, _VP], _I32),
    "momms_gemm_backward": ([_VP, _I64, _I64, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _VP, _I64, _VP], _I32),
    "momms_gemm_batched": ([_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _I32),
    "momms_emu_scale": ([_I32, _I32, _I64, _I64, _VP, _I64, _VP, _VP, _VP], _I32),
    "momms_emu_split": ([_I32, _I32, _I64, _I64, _VP, _I64, _VP, _VP, _I32, _I32, _VP, _I64, _I64, _VP], _I32),
    "momms_emu_slice_gemm": ([_I64, _I64, _I64, _I32, _I32, _VP, _VP, _I64, _I64, _I64, _VP, _VP, _VP, _VP,
                              _DBL, _DBL, _VP, _I64, _I32, _VP, _SZ, _VP, _VP], _I32),
    "momms_emu_scratch_bytes": ([], _SZ),
    "momms_emu_scratch_bytes_for": ([_I64, _I64, _I64, _I32], _SZ),
    "momms_tune": ([_VP, ctypes.c_char_p, _I64, _VP, _VP, _VP, _VP], _I32),
    "momms_load_plans": ([_VP, ctypes.c_char_p], _I32),
    "momms_tune_ex": ([_VP, ctypes.c_char_p, _I64, _VP, _VP, _VP, _VP, _VP, _VP], _I32),
    "momms_get_plan": ([_VP, _I32, _I32, _I64, _I64, _I64, _VP], _I32),
    "momms_probe_peak": ([_I32, ctypes.POINTER(_DBL), _VP], _I32),
    "momms_stream_copy": ([_VP, _VP, _SZ, _I32, _I32, _VP], _I32),
    "momms_gemm_emulated_noalloc": ([_I32, _I32, _I64, _I64, _I64, _I32, _DBL, _VP, _I64, _VP, _I64, _DBL, _VP,
                                     _I64, _VP], _I32),
    "momms_noalloc_scratch_bytes": ([], _SZ),
    "momms_noalloc_status": ([_VP, ctypes.POINTER(_I32)], _I32),
    "momms_debug_withhold_load": ([], None),
    "momms_set_kernel_timing": ([_VP, _I32], _I32),
    "momms_kernel_timing": ([_VP, ctypes.POINTER(_DBL), ctypes.POINTER(_I64)], _I32),
    "momms_member_tile": ([_I32, _I32, _I64, _I64, _I64, _I32, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)],
                          _I32),
    "momms_tri_tile": ([_I32, _I32, _I64, _I64, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64)],
                       _I32),
}


def header_symbols():
    """Every function the public header declares (``momms_*(``)."""
    hdr = os.path.join(_build.INCLUDE, "momms.h")
    text = open(hdr).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(momms_[a-z0-9_]+)\s*\(", text)))


def lib(build_if_missing: bool = True):
    """Load libmomms.so (building it first if allowed); raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"libmomms is not built ({path})")
                path = _build.build()
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib(False).momms_status_string(int(status)).decode()
    except Exception:
        return "?"


def check(status: int, where: str = "momms"):
    if status != MOMMS_OK:
        raise MommsError(status, where)
    return status


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ---------------------------------------------------------------- raw C-ABI calls (same names)
def momms_gemm(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    return lib().momms_gemm(m, n, k, alpha, _VP(A), lda, _VP(B), ldb, beta, _VP(C), ldc, _stream(stream))


def momms_gemm_ex(handle, op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    return lib().momms_gemm_ex(_h(handle), op_a, op_b, m, n, k, alpha, _VP(A), lda, _VP(B), ldb, beta,
                               _VP(C), ldc, _stream(stream))


def momms_gemm_host(handle, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, device_bytes=0, block=0, stream=None):
    """A, B, C: host addresses (ints), e.g. of pinned torch tensors or numpy arrays."""
    return lib().momms_gemm_host(_h(handle), m, n, k, alpha, _VP(A), lda, _VP(B), ldb, beta, _VP(C), ldc,
                                 device_bytes, block, _stream(stream))


def momms_syrk(handle, uplo, trans, n, k, alpha, A, lda, beta, C, ldc, stream=None):
    return lib().momms_syrk(_h(handle), uplo, trans, n, k, alpha, _VP(A), lda, beta, _VP(C), ldc, _stream(stream))


def momms_trmm(handle, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=None):
    return lib().momms_trmm(_h(handle), side, uplo, trans, diag, m, n, alpha, _VP(A), lda, _VP(B), ldb,
                            _stream(stream))


def momms_trsm(handle, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=None):
    return lib().momms_trsm(_h(handle), side, uplo, trans, diag, m, n, alpha, _VP(A), lda, _VP(B), ldb,
                            _stream(stream))


def momms_gemm_backward(handle, m, n, k, A, lda, B, ldb, dC, lddc, dA, ldda, dB, lddb, stream=None):
    return lib().momms_gemm_backward(_h(handle), m, n, k, _VP(A), lda, _VP(B), ldb, _VP(dC), lddc,
                                     _VP(dA), ldda, _VP(dB), lddb, _stream(stream))


def momms_gemm_batched(handle, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """All arguments after the handle are equal-length Python sequences (pointers as ints)."""
    cnt = len(m)
    a64 = lambda v: np.ascontiguousarray(v, dtype=np.int64)
    af = lambda v: np.ascontiguousarray(v, dtype=np.float64)
    au = lambda v: np.ascontiguousarray(v, dtype=np.uint64)
    arrs = [a64(m), a64(n), a64(k), af(alpha), au(A), a64(lda), au(B), a64(ldb), af(beta), au(C), a64(ldc)]
    ptrs = [_VP(x.ctypes.data) for x in arrs]
    rc = lib().momms_gemm_batched(_h(handle), cnt, *ptrs, _stream(stream))
    return rc


def momms_emu_scale(which, op, rows, inner, X, ldx, exps, flags, stream=None):
    return lib().momms_emu_scale(which, op, rows, inner, _VP(X), ldx, _VP(exps), _VP(flags), _stream(stream))


def momms_emu_split(which, op, rows, inner, X, ldx, exps, flags, slices, digit_bits, digits, rows_pad,
                    inner_pad, stream=None):
    return lib().momms_emu_split(which, op, rows, inner, _VP(X), ldx, _VP(exps), _VP(flags), slices,
                                 digit_bits, _VP(digits), rows_pad, inner_pad, _stream(stream))


def momms_crt_moduli(bits, k):
    """The moduli the modular encoding uses for `bits`-bit operands and contraction length k
    (a list), or raises MommsError when they do not exist."""
    count = ctypes.c_int(0)
    buf = (ctypes.c_uint32 * 16)()
    check(lib().momms_crt_moduli(bits, k, ctypes.byref(count), buf), "momms_crt_moduli")
    return [int(buf[i]) for i in range(count.value)]


def momms_emu_residues(which, op, rows, inner, X, ldx, exps, flags, bits, k, planes, rows_pad, inner_pad,
                       stream=None):
    return lib().momms_emu_residues(which, op, rows, inner, _VP(X), ldx, _VP(exps), _VP(flags), bits, k,
                                    _VP(planes), rows_pad, inner_pad, _stream(stream))


def momms_emu_residue_gemm(m, n, k, bits, Ar, Br, m_pad, n_pad, k_pad, member, res, scratch, scratch_bytes, status,
                           stream=None):
    return lib().momms_emu_residue_gemm(m, n, k, bits, _VP(Ar), _VP(Br), m_pad, n_pad, k_pad, member, _VP(res),
                                        _VP(scratch), scratch_bytes, _VP(status), _stream(stream))


def momms_crt_reconstruct(m, n, k, bits, res, e, ef, f, ff, alpha, beta, C, ldc, stream=None):
    return lib().momms_crt_reconstruct(m, n, k, bits, _VP(res), _VP(e), _VP(ef), _VP(f), _VP(ff), alpha, beta,
                                       _VP(C), ldc, _stream(stream))


def momms_emu_slice_gemm(m, n, k, slices, digit_bits, Ad, Bd, m_pad, n_pad, k_pad, e, ef, f, ff, alpha,
                         beta, C, ldc, member, scratch, scratch_bytes, status, stream=None):
    return lib().momms_emu_slice_gemm(m, n, k, slices, digit_bits, _VP(Ad), _VP(Bd), m_pad, n_pad, k_pad,
                                      _VP(e), _VP(ef), _VP(f), _VP(ff), alpha, beta, _VP(C), ldc, member,
                                      _VP(scratch), scratch_bytes, _VP(status), _stream(stream))


def momms_emu_scratch_bytes():
    return int(lib().momms_emu_scratch_bytes())


def momms_emu_scratch_bytes_for(m, n, k, slices):
    return int(lib().momms_emu_scratch_bytes_for(m, n, k, slices))


def momms_gemm_emulated_noalloc(op_a, op_b, m, n, k, slices, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    """The allocation-free emulated product (scratch in the library's static device array)."""
    return lib().momms_gemm_emulated_noalloc(op_a, op_b, m, n, k, slices, alpha, _VP(A), lda, _VP(B), ldb, beta,
                                             _VP(C), ldc, _stream(stream))


def momms_noalloc_scratch_bytes():
    return int(lib().momms_noalloc_scratch_bytes())


def momms_debug_withhold_load():
    """Test hook: the next slice-product launch leaves one stage empty, so its bounded wait runs out."""
    lib().momms_debug_withhold_load()


def momms_noalloc_status(stream=None):
    """(return code, status word) of the allocation-free calls on the current device; clears the word."""
    st = _I32(0)
    rc = lib().momms_noalloc_status(_stream(stream), ctypes.byref(st))
    return int(rc), int(st.value)


def momms_probe_peak(kind, stream=None):
    out = _DBL(0.0)
    check(lib().momms_probe_peak(kind, ctypes.byref(out), _stream(stream)), "momms_probe_peak")
    return out.value


def momms_stream_copy(dst, src, nbytes, ctas=0, repeats=1, stream=None):
    return lib().momms_stream_copy(_VP(dst), _VP(src), nbytes, ctas, repeats, _stream(stream))


def _h(handle):
    return handle.ptr if isinstance(handle, Handle) else _VP(handle)


class Handle:
    """Owns a momms_handle_t."""

    def __init__(self, mode=MODE_AUTO, member=MEMBER_AUTO, slices=0, scheme=SCHEME_AUTO):
        self.ptr = _VP()
        check(lib().momms_create(ctypes.byref(self.ptr)), "momms_create")
        self.set_mode(mode)
        self.set_member(member)
        self.set_slices(slices)
        if scheme != SCHEME_AUTO:
            self.set_scheme(scheme)

    def close(self):
        if self.ptr:
            lib().momms_destroy(self.ptr)
            self.ptr = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode):
        check(lib().momms_set_mode(self.ptr, mode), "momms_set_mode")

    def set_member(self, member):
        check(lib().momms_set_member(self.ptr, member), "momms_set_member")

    def set_slices(self, slices):
        check(lib().momms_set_slices(self.ptr, slices), "momms_set_slices")

    def set_max_ctas(self, ctas):
        check(lib().momms_set_max_ctas(self.ptr, ctas), "momms_set_max_ctas")

    def set_raster_group(self, group):
        check(lib().momms_set_raster_group(self.ptr, group), "momms_set_raster_group")

    def set_tile_n(self, tile_n):
        check(lib().momms_set_tile_n(self.ptr, tile_n), "momms_set_tile_n")

    def set_scheme(self, scheme):
        check(lib().momms_set_scheme(self.ptr, scheme), "momms_set_scheme")

    def set_host_resident(self, resident):
        check(lib().momms_set_host_resident(self.ptr, resident), "momms_set_host_resident")

    def set_plan_on_device(self, on):
        check(lib().momms_set_plan_on_device(self.ptr, on), "momms_set_plan_on_device")

    def set_cta_pairs(self, mode):
        check(lib().momms_set_cta_pairs(self.ptr, mode), "momms_set_cta_pairs")

    def set_crt_fusion(self, mode):
        check(lib().momms_set_crt_fusion(self.ptr, mode), "momms_set_crt_fusion")


    def report(self):
        r = Report()
        check(lib().momms_get_last_report(self.ptr, ctypes.byref(r)), "momms_get_last_report")
        return r.as_dict()

    def device_status(self, stream=None):
        return lib().momms_check_device_status(self.ptr, _stream(stream))

    def set_kernel_timing(self, max_launches):
        check(lib().momms_set_kernel_timing(self.ptr, max_launches), "momms_set_kernel_timing")

    def kernel_timing(self):
        """(total ms, launches) of the product launches timed since the last read."""
        t, c = _DBL(0.0), _I64(0)
        check(lib().momms_kernel_timing(self.ptr, ctypes.byref(t), ctypes.byref(c)), "momms_kernel_timing")
        return float(t.value), int(c.value)

    def workspace_size(self, m, n, k, op_a=OP_N, op_b=OP_N):
        out = _SZ(0)
        check(lib().momms_workspace_size(self.ptr, op_a, op_b, m, n, k, ctypes.byref(out)),
              "momms_workspace_size")
        return out.value

    def set_workspace(self, ptr, nbytes):
        check(lib().momms_set_workspace(self.ptr, _VP(ptr), nbytes), "momms_set_workspace")

    def tune(self, shapes, path=None, stream=None):
        """shapes: (m, n, k) or (m, n, k, op_a, op_b) tuples."""
        m = np.ascontiguousarray([s[0] for s in shapes], dtype=np.int64)
        n = np.ascontiguousarray([s[1] for s in shapes], dtype=np.int64)
        k = np.ascontiguousarray([s[2] for s in shapes], dtype=np.int64)
        oa = np.ascontiguousarray([s[3] if len(s) > 3 else OP_N for s in shapes], dtype=np.int32)
        ob = np.ascontiguousarray([s[4] if len(s) > 4 else OP_N for s in shapes], dtype=np.int32)
        check(lib().momms_tune_ex(self.ptr, path.encode() if path else None, len(shapes), _VP(m.ctypes.data),
                                  _VP(n.ctypes.data), _VP(k.ctypes.data), _VP(oa.ctypes.data), _VP(ob.ctypes.data),
                                  _stream(stream)), "momms_tune_ex")

    def plan(self, m, n, k, op_a=OP_N, op_b=OP_N):
        """The plan of the bucket of (op_a, op_b, m, n, k) as a dict (tuned = 0: the built-in default)."""
        p = PlanT()
        check(lib().momms_get_plan(self.ptr, op_a, op_b, m, n, k, ctypes.byref(p)), "momms_get_plan")
        return {f: getattr(p, f) for f, _ in PlanT._fields_}

    def load_plans(self, path):
        return lib().momms_load_plans(self.ptr, path.encode())


# ---------------------------------------------------------------- torch conveniences
class DeviceMatrix:
    """A column-major FP64 matrix (rows x cols, leading dimension ld) in torch CUDA memory.

    The storage is a (cols, ld) row-major torch tensor: element (i, j) sits at
    offset i + j*ld, exactly the column-major layout of the C ABI."""

    def __init__(self, rows, cols, ld=None, device="cuda", fill=None):
        import torch
        self.rows, self.cols = int(rows), int(cols)
        self.ld = int(ld) if ld is not None else max(1, self.rows)
        if self.ld < max(1, self.rows):
            raise ValueError("ld < rows")
        self.storage = torch.empty((max(self.cols, 1), self.ld), dtype=torch.float64, device=device)
        if fill is not None:
            self.storage.fill_(fill)

    @classmethod
    def from_numpy(cls, X, ld=None, device="cuda", pad_value=float("nan")):
        import torch
        X = np.asarray(X, dtype=np.float64)
        rows, cols = X.shape
        dm = cls(rows, cols, ld, device, fill=pad_value if (ld or rows) > rows else None)
        if rows and cols:
            host = torch.from_numpy(np.ascontiguousarray(X.T))  # (cols, rows) row-major == column-major X
            dm.storage[:cols, :rows].copy_(host)
        return dm

    @property
    def ptr(self) -> int:
        return self.storage.data_ptr()

    def to_numpy(self):
        if self.rows == 0 or self.cols == 0:
            return np.zeros((self.rows, self.cols), order="F")
        return np.asfortranarray(self.storage[: self.cols, : self.rows].cpu().numpy().T)

    def padding_numpy(self):
        """The rows between `rows` and `ld` of every column (canary region)."""
        return self.storage[: self.cols, self.rows:].cpu().numpy()


def gemm(A: DeviceMatrix, B: DeviceMatrix, C: DeviceMatrix, alpha=1.0, beta=0.0, op_a=OP_N, op_b=OP_N,
         handle: Handle | None = None, stream=None):
    """C := alpha*op(A)*op(B) + beta*C through momms_gemm_ex (or momms_gemm without a handle)."""
    m = C.rows
    n = C.cols
    k = A.cols if op_a == OP_N else A.rows
    if handle is None and op_a == OP_N and op_b == OP_N:
        rc = momms_gemm(m, n, k, alpha, A.ptr, A.ld, B.ptr, B.ld, beta, C.ptr, C.ld, stream)
        check(rc, "momms_gemm")
    else:
        h = handle or Handle()
        rc = momms_gemm_ex(h, op_a, op_b, m, n, k, alpha, A.ptr, A.ld, B.ptr, B.ld, beta, C.ptr, C.ld, stream)
        check(rc, "momms_gemm_ex")
    return C
