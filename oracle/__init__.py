"""CPU oracle for the MOMMS hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 reference written from the paper
(Smith & van de Geijn, "The MOMMS Family of Matrix Multiplication Algorithms",
SC19): the product definition of the Sec. 2.1 footnote and Sec. 2.2.1, the
resident-block I/O counts of Sec. 2.2, and the integer-slice emulation steps
(truncation splitting, exact slice products, exact recombination).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_1904_05717_gb300``) and neither imports the other.

Parity status of each function (what pins it, see ``tests/test_oracle_pins.py``):
  dgemm              pinned: exact integer brute force, rank-1 closed form,
                     identity/permutation, transpose identity, exact-rational
                     error bound
  dgemm_abs          pinned: closed forms on sign-flipped inputs
  exponents / split  pinned: hand-worked digits, error-free reconstruction,
                     bit-field identity of truncation digits
  slice_products     pinned: Python big-integer brute force
  recombine          pinned: exact rational value of the digit expansion
  count_member       pinned: the paper's closed-form I/O counts (Sec. 2.2) and
                     printed intensities (Sec. 5.2: 23.26 and 64 flops/byte)
  truncated_integers pinned: the digit expansion of `split`, truncation identity
  greedy_moduli,     pinned: pairwise coprimality, hand-listed factorisations,
  moduli_suffice     the range argument written out
  centred_residues,  pinned: reconstruction by sympy's CRT, round trip
  crt_reconstruct
  modular_dgemm      pinned: integer inputs exact, the one-slice emulation bit for
                     bit, the FP64 componentwise bound at 56 bits, fma semantics
  trsm               pinned: exact integer recovery, scipy.linalg.solve_triangular,
                     the identity
The modular encoding is not in the paper: it is the alternative integer encoding of
the emulated product (Ozaki, Uchino & Imamura, "Ozaki Scheme II", 2025); its oracle is
the definition of what it computes (the exact product of the truncated operands).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "momms_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libmomms_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, OpenMP if present)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=gnu11",
            "-shared", "-fPIC", _SRC, "-lm"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp])
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class IOCounts(ctypes.Structure):
    _fields_ = [("a_reads", ctypes.c_int64), ("b_reads", ctypes.c_int64),
                ("c_reads", ctypes.c_int64), ("c_writes", ctypes.c_int64),
                ("flops", ctypes.c_int64), ("fast_words", ctypes.c_int64)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, dbl, vp, ci = ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int
            L.oracle_dgemm.argtypes = [ci, ci, i64, i64, i64, dbl, vp, i64, vp, i64, dbl, vp, i64, ci]
            L.oracle_dgemm_abs.argtypes = [ci, ci, i64, i64, i64, vp, i64, vp, i64, vp, i64, ci]
            L.oracle_exponents.argtypes = [ci, ci, i64, i64, vp, i64, vp, vp]
            L.oracle_split.argtypes = [ci, ci, i64, i64, vp, i64, vp, vp, ci, ci, vp]
            L.oracle_slice_products.argtypes = [i64, i64, i64, ci, vp, vp, vp, ci]
            L.oracle_recombine.argtypes = [i64, i64, ci, ci, vp, vp, vp, vp, vp, dbl, dbl, vp, i64]
            L.oracle_count_member.argtypes = [ci, i64, i64, i64, i64, i64, i64, ci, vp, i64, vp, i64,
                                              vp, i64, ctypes.POINTER(IOCounts)]
            L.oracle_max_threads.argtypes = []
            for fn in ("oracle_dgemm", "oracle_dgemm_abs", "oracle_exponents", "oracle_split",
                       "oracle_slice_products", "oracle_recombine", "oracle_count_member",
                       "oracle_max_threads"):
                getattr(L, fn).restype = ci
            _lib = L
    return _lib


def _f64(x):
    x = np.asarray(x)
    if x.dtype != np.float64:
        raise TypeError("oracle expects float64 arrays")
    return x


def _ld(x):
    """Leading dimension of a Fortran-ordered 2-D float64 array (or a column slice of one)."""
    if x.ndim != 2:
        raise ValueError("expected a 2-D array")
    if x.size == 0:
        return max(1, x.shape[0])
    if x.strides[0] != 8 and x.shape[0] > 1:
        raise ValueError("expected column-major (Fortran-ordered) storage")
    return max(1, x.strides[1] // 8) if x.shape[1] > 1 else max(1, x.shape[0])


def _ptr(x):
    return ctypes.c_void_p(x.ctypes.data)


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def dgemm(A, B, C=None, alpha=1.0, beta=0.0, transa=False, transb=False, nthreads=0):
    """C := alpha*op(A)*op(B) + beta*C in plain FP64 (p ascending, no FMA).

    A, B (and C) are Fortran-ordered float64 arrays.  Returns C (a new array
    when C is None, else C updated in place)."""
    A = _f64(A); B = _f64(B)
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    kb = B.shape[1] if transb else B.shape[0]
    n = B.shape[0] if transb else B.shape[1]
    if k != kb:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = np.zeros((m, n), dtype=np.float64, order="F")
        beta = 0.0
    C = _f64(C)
    if C.shape != (m, n):
        raise ValueError("C has the wrong shape")
    rc = lib().oracle_dgemm(int(transa), int(transb), m, n, k, float(alpha), _ptr(A), _ld(A),
                            _ptr(B), _ld(B), float(beta), _ptr(C), _ld(C), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_dgemm failed ({rc})")
    return C


def dgemm_abs(A, B, transa=False, transb=False, nthreads=0):
    """N := |op(A)| * |op(B)| (the magnitude matrix of the error bound)."""
    A = _f64(A); B = _f64(B)
    m = A.shape[1] if transa else A.shape[0]
    k = A.shape[0] if transa else A.shape[1]
    n = B.shape[0] if transb else B.shape[1]
    N = np.zeros((m, n), dtype=np.float64, order="F")
    rc = lib().oracle_dgemm_abs(int(transa), int(transb), m, n, k, _ptr(A), _ld(A), _ptr(B), _ld(B),
                                _ptr(N), _ld(N), int(nthreads))
    if rc != 0:
        raise RuntimeError("oracle_dgemm_abs failed")
    return N


def exponents(X, which, trans=False):
    """Scaling exponents: which='rows' -> rows of op(X)=op(A); 'cols' -> columns of op(X)=op(B).

    Returns (exps int32, flags uint8)."""
    X = _f64(X)
    if which == "rows":
        rows = X.shape[1] if trans else X.shape[0]
        inner = X.shape[0] if trans else X.shape[1]
        w = 0
    else:
        rows = X.shape[0] if trans else X.shape[1]
        inner = X.shape[1] if trans else X.shape[0]
        w = 1
    e = np.zeros(rows, dtype=np.int32)
    fl = np.zeros(rows, dtype=np.uint8)
    lib().oracle_exponents(w, int(trans), rows, inner, _ptr(X), _ld(X), _ptr(e), _ptr(fl))
    return e, fl


def split(X, which, exps, flags, S, beta, trans=False):
    """Truncation digits: int16 array [S, rows, inner] (slice s+1 at index s)."""
    X = _f64(X)
    if which == "rows":
        rows = X.shape[1] if trans else X.shape[0]
        inner = X.shape[0] if trans else X.shape[1]
        w = 0
    else:
        rows = X.shape[0] if trans else X.shape[1]
        inner = X.shape[1] if trans else X.shape[0]
        w = 1
    exps = np.ascontiguousarray(exps, dtype=np.int32)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    D = np.zeros((S, rows, inner), dtype=np.int16)
    rc = lib().oracle_split(w, int(trans), rows, inner, _ptr(X), _ld(X), _ptr(exps), _ptr(flags),
                            int(S), int(beta), _ptr(D))
    if rc != 0:
        raise RuntimeError("oracle_split failed")
    return D


def slice_products(Ad, Bd, nthreads=0):
    """P[d-2] = sum_{s+t=d} A_s B_t (exact int64), d = 2..S+1; each m x n column-major."""
    Ad = np.ascontiguousarray(Ad, dtype=np.int16)
    Bd = np.ascontiguousarray(Bd, dtype=np.int16)
    S, m, k = Ad.shape
    S2, n, k2 = Bd.shape
    if S != S2 or k != k2:
        raise ValueError("slice stacks disagree")
    P = np.zeros((S, n, m), dtype=np.int64)  # [d][j][i] -> column-major m x n per diagonal
    lib().oracle_slice_products(m, n, k, S, _ptr(Ad), _ptr(Bd), _ptr(P), int(nthreads))
    return np.transpose(P, (0, 2, 1))  # view [d][i][j]


def recombine(P, e, eflag, f, fflag, S, beta, alpha=1.0, beta_c=0.0, C=None):
    """Exact recombination of the slice products, rounded once to FP64."""
    P = np.asarray(P)
    S_, m, n = P.shape
    Pc = np.ascontiguousarray(np.transpose(P, (0, 2, 1)), dtype=np.int64)
    if C is None:
        C = np.zeros((m, n), dtype=np.float64, order="F")
        beta_c = 0.0
    rc = lib().oracle_recombine(m, n, int(S), int(beta), _ptr(Pc),
                                _ptr(np.ascontiguousarray(e, dtype=np.int32)),
                                _ptr(np.ascontiguousarray(eflag, dtype=np.uint8)),
                                _ptr(np.ascontiguousarray(f, dtype=np.int32)),
                                _ptr(np.ascontiguousarray(fflag, dtype=np.uint8)),
                                float(alpha), float(beta_c), _ptr(C), _ld(C))
    if rc != 0:
        raise RuntimeError("oracle_recombine failed")
    return C


def emulated_dgemm(A, B, S, beta_bits, C=None, alpha=1.0, beta=0.0, transa=False, transb=False):
    """The whole integer-slice emulation on the CPU: scale, split, exact slice
    products, exact recombination.  Returns (C, details dict)."""
    e, ef = exponents(A, "rows", transa)
    f, ff = exponents(B, "cols", transb)
    Ad = split(A, "rows", e, ef, S, beta_bits, transa)
    Bd = split(B, "cols", f, ff, S, beta_bits, transb)
    P = slice_products(Ad, Bd)
    C = recombine(P, e, ef, f, ff, S, beta_bits, alpha, beta, C)
    return C, {"e": e, "eflag": ef, "f": f, "fflag": ff, "Ad": Ad, "Bd": Bd, "P": P}


MEMBERS = {"resident_c": 0, "resident_a": 1, "resident_b": 2, "goto": 3}


def count_member(member, A, B, C, b1, b2, b3=0, c_read=True):
    """Run a blocked member on an explicit two-level memory; C is updated in
    place with C += A*B.  Returns the word counts as a dict."""
    A = _f64(A); B = _f64(B); C = _f64(C)
    m, k = A.shape
    n = B.shape[1]
    out = IOCounts()
    rc = lib().oracle_count_member(MEMBERS[member], m, n, k, int(b1), int(b2), int(b3), int(bool(c_read)),
                                   _ptr(A), _ld(A), _ptr(B), _ld(B), _ptr(C), _ld(C),
                                   ctypes.byref(out))
    if rc != 0:
        raise RuntimeError("oracle_count_member failed")
    return out.as_dict()


# ---------------------------------------------------------------------------------------------
# Modular (Chinese remainder) encoding of the emulated product.  Its result has a plain
# definition -- the exact integer product of the operands truncated to `bits`-bit integers,
# rounded once to FP64 and scaled -- so the oracle is that definition (Python integers), plus
# the two pieces the CUDA path exposes on their own: the centred residues of the truncated
# operands and the choice of moduli.
#   truncated_integers  pinned: digit expansion of `split`, truncation identity
#   centred_residues    pinned: reconstruction by the library CRT (sympy)
#   crt_reconstruct     pinned: round trip on random integers, sympy
#   greedy_moduli       pinned: pairwise coprimality, hand-listed factorisations
#   modular_dgemm       pinned: integer inputs exact, S = 1 slice emulation (every digit pair
#                       kept) bit for bit, FP64 error bound at 53 bits
# ---------------------------------------------------------------------------------------------

def _op_vectors(X, which, trans):
    """The vectors the scaling runs along: rows of op(A) ('rows') or columns of op(B) ('cols'),
    as a 2-D float64 array [vector, inner]."""
    X = np.asarray(X, dtype=np.float64)
    op = X.T if trans else X
    return op if which == "rows" else op.T


def truncated_integers(X, which, exps, flags, bits, trans=False):
    """X^ = sign(x) trunc(|x| 2^(bits - e)) for each element x of op(X) (exponent e of its row
    of op(A) or column of op(B), from `exponents`), as Python ints in an object array
    [vector, inner]; flagged vectors give zeros.  |x| < 2^e makes |X^| < 2^bits."""
    import math
    V = _op_vectors(X, which, trans)
    out = np.zeros(V.shape, dtype=object)
    for r in range(V.shape[0]):
        if flags[r]:
            continue
        for q in range(V.shape[1]):
            out[r, q] = int(math.trunc(math.ldexp(float(V[r, q]), int(bits) - int(exps[r]))))
    return out


def greedy_moduli(count):
    """The first `count` numbers taken walking down from 255 that are coprime to every number
    taken before: pairwise coprime moduli whose centred residues fit in 8-bit digits."""
    import math
    taken = []
    p = 255
    while len(taken) < count and p >= 2:
        if all(math.gcd(p, q) == 1 for q in taken):
            taken.append(p)
        p -= 1
    return taken


def moduli_suffice(moduli, bits, k, margin=1):
    """True when the product P of the moduli exceeds margin * 2 k (2^bits - 1)^2; margin 1: the
    width of the range of a k-term dot product of `bits`-bit integers, so that its centred
    residue mod P is the product itself (margin 2 leaves |product| <= P / 4)."""
    P = 1
    for p in moduli:
        P *= int(p)
    return P > int(margin) * 2 * int(k) * (2 ** int(bits) - 1) ** 2


def centred_residues(Xhat, moduli):
    """r_l = X^ mod p_l moved into [-floor(p/2), floor((p-1)/2)]; int16 array [N, ...]."""
    out = np.zeros((len(moduli),) + Xhat.shape, dtype=np.int16)
    for l, p in enumerate(moduli):
        p = int(p)
        for idx, v in np.ndenumerate(Xhat):
            r = int(v) % p          # Python: in [0, p) for either sign
            if r > (p - 1) // 2:
                r -= p
            out[(l,) + idx] = r
    return out


def crt_reconstruct(residues, moduli):
    """The integer x with |x| < P/2 and x = r_l (mod p_l) for every l (Chinese remainder
    theorem, x = sum_l r_l M_l (M_l^-1 mod p_l) mod P, M_l = P / p_l, then centred)."""
    P = 1
    for p in moduli:
        P *= int(p)
    x = 0
    for r, p in zip(residues, moduli):
        p = int(p)
        Ml = P // p
        x += int(r) * Ml * pow(Ml % p, -1, p)
    x %= P
    return x - P if x > P // 2 else x


def _fma(a, b, c):
    """a * b + c rounded once (exact rationals), as the device fma does."""
    from fractions import Fraction
    import math
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        return a * b + c
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def modular_dgemm(A, B, bits, C=None, alpha=1.0, beta=0.0, transa=False, transb=False):
    """C := alpha 2^(e_i + f_j - 2 bits) (A^ B^)_ij + beta C with A^, B^ the `bits`-bit truncated
    integer operands and (A^ B^)_ij their exact dot product (Python integers), rounded once to
    FP64 (ties to even) before the exact power-of-two scaling; alpha times it is rounded, then
    fma(beta, C, that).  NaN in the rows of op(A) / columns of op(B) that hold Inf or NaN.
    Small inputs only (pure Python).  Returns (C, details dict)."""
    import math
    e, ef = exponents(A, "rows", transa)
    f, ff = exponents(B, "cols", transb)
    Ah = truncated_integers(A, "rows", e, ef, bits, transa)
    Bh = truncated_integers(B, "cols", f, ff, bits, transb)
    m, n = Ah.shape[0], Bh.shape[0]
    Z = np.zeros((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            Z[i, j] = sum(int(a) * int(b) for a, b in zip(Ah[i], Bh[j]))
    out = np.zeros((m, n), dtype=np.float64, order="F")
    for i in range(m):
        for j in range(n):
            if ef[i] or ff[j]:
                y = float("nan")
            else:
                y = math.ldexp(float(Z[i, j]), int(e[i]) + int(f[j]) - 2 * int(bits))
            ay = float(alpha) * y
            out[i, j] = ay if (C is None or beta == 0.0) else _fma(float(beta), float(C[i, j]), ay)
    return out, {"e": e, "eflag": ef, "f": f, "fflag": ff, "Ahat": Ah, "Bhat": Bh, "Z": Z}


# ---------------------------------------------------------------------------------------------
# Triangular solve (BLAS dtrsm semantics).  Plain substitution, row by row, in FP64.
#   trsm   pinned: exact integer recovery (unit triangle, integer solution), agreement with
#          scipy.linalg.solve_triangular, identity
# ---------------------------------------------------------------------------------------------

def trsm(A, B, alpha=1.0, side="L", lower=True, trans=False, unit=False):
    """X with op(A) X = alpha B (side 'L') or X op(A) = alpha B (side 'R'), A triangular (only
    the `lower` / upper triangle read; `unit`: ones on the diagonal, not read), by forward or
    back substitution: x_i = (r_i - sum_{k before i} M_ik x_k) / M_ii along the rows of
    M = op(A) (side 'R' solves M^T X^T = alpha B^T the same way)."""
    A = np.asarray(A, dtype=np.float64)
    T = np.tril(A) if lower else np.triu(A)
    if unit:
        T = T.copy()
        np.fill_diagonal(T, 1.0)
    M = T.T if trans else T
    R = float(alpha) * np.asarray(B, dtype=np.float64)
    if side == "R":
        M = M.T
        R = R.T
    is_lower = np.array_equal(M, np.tril(M))
    t = M.shape[0]
    X = np.zeros_like(R)
    order = range(t) if is_lower else range(t - 1, -1, -1)
    for i in order:
        if is_lower:
            acc = R[i] - M[i, :i] @ X[:i]
        else:
            acc = R[i] - M[i, i + 1:] @ X[i + 1:]
        X[i] = acc / M[i, i]
    return np.asfortranarray(X.T if side == "R" else X)
