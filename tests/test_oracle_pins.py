"""Pins of the CPU oracle to facts other than itself (CPU only).

Each test checks the oracle against something the paper or the mathematics
fixes: exact integer arithmetic, exact rational arithmetic (Python fractions),
closed forms (rank-1 products, identity and permutation matrices, transposes),
Python big-integer brute force for the digit-slice products, and the paper's
closed-form I/O counts and printed intensities (Sec. 2.2, Sec. 5.2, Sec. 5.4).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1904_05717_gb300 import synthetic as syn

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def F(x):
    return np.asfortranarray(np.asarray(x, dtype=np.float64))


def exact_product(A, B, transa=False, transb=False):
    """Exact rational op(A) op(B) as a nested list of Fractions."""
    Aop = A.T if transa else A
    Bop = B.T if transb else B
    m, k = Aop.shape
    n = Bop.shape[1]
    fa = [[Fraction(float(Aop[i, p])) for p in range(k)] for i in range(m)]
    fb = [[Fraction(float(Bop[p, j])) for j in range(n)] for p in range(k)]
    return [[sum((fa[i][p] * fb[p][j] for p in range(k)), Fraction(0)) for j in range(n)] for i in range(m)]


# --------------------------------------------------------------------------- product
@pytest.mark.parametrize("transa,transb", [(False, False), (True, False), (False, True), (True, True)])
def test_dgemm_integer_bruteforce_exact(transa, transb):
    # integer entries in [-8, 8], k <= 64: every partial sum < 2^53, so FP64 is exact
    rng_seed = 11 + 2 * transa + transb
    m, n, k = 13, 9, 64
    A = syn.matrix("int", k if transa else m, m if transa else k, rng_seed)
    B = syn.matrix("int", n if transb else k, k if transb else n, rng_seed + 100)
    C0 = syn.matrix("int", m, n, rng_seed + 200)
    Aop = A.T if transa else A
    Bop = B.T if transb else B
    ref = [[2 * sum(int(Aop[i, p]) * int(Bop[p, j]) for p in range(k)) - 3 * int(C0[i, j])
            for j in range(n)] for i in range(m)]
    C = oracle.dgemm(A, B, C0.copy(order="F"), alpha=2.0, beta=-3.0, transa=transa, transb=transb)
    assert np.array_equal(C, np.array(ref, dtype=np.float64))


def test_dgemm_rank1_closed_form():
    # (u v^T)(w z^T) = (v . w) u z^T; dyadic entries keep everything exact
    u = np.arange(1, 8, dtype=np.float64) / 4.0
    v = np.array([1, -2, 3, 0.5, -0.25], dtype=np.float64)
    w = np.array([2, 1, -1, 4, 8], dtype=np.float64)
    z = np.arange(-3, 3, dtype=np.float64) / 2.0
    A = F(np.outer(u, v))
    B = F(np.outer(w, z))
    C = oracle.dgemm(A, B)
    assert np.array_equal(C, float(np.dot(v, w)) * np.outer(u, z))


def test_dgemm_identity_and_permutation():
    m = 37
    B = syn.matrix("uniform", m, 21, 5)
    I = F(np.eye(m))
    assert np.array_equal(oracle.dgemm(I, B), B)
    perm = (np.arange(m) * 7 + 3) % m
    P = F(np.eye(m)[perm])
    assert np.array_equal(oracle.dgemm(P, B), B[perm])
    A = syn.matrix("uniform", 19, m, 6)
    assert np.array_equal(oracle.dgemm(A, I), A)


def test_dgemm_transpose_identity_bitwise():
    A = syn.matrix("uniform", 23, 41, 7)
    B = syn.matrix("uniform", 41, 17, 8)
    C = oracle.dgemm(A, B)
    Ct = oracle.dgemm(F(B.T), F(A.T))
    assert np.array_equal(C, Ct.T)
    # the op(.) flags read the same numbers as explicit transposes
    assert np.array_equal(oracle.dgemm(F(A.T), B, transa=True), C)
    assert np.array_equal(oracle.dgemm(A, F(B.T), transb=True), C)


def test_dgemm_error_within_gamma_k_of_exact():
    # |fl(sum) - sum| <= gamma_k * sum |a||b|, gamma_k = k u / (1 - k u)  (Higham, Thm 3.5)
    m, n, k = 6, 5, 57
    A = syn.matrix("uniform", m, k, 21)
    B = syn.matrix("uniform", k, n, 22)
    C = oracle.dgemm(A, B)
    N = oracle.dgemm_abs(A, B)
    ex = exact_product(A, B)
    exabs = exact_product(np.abs(A), np.abs(B))
    gk = k * U / (1 - k * U)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(float(C[i, j])) - ex[i][j])
            assert err <= Fraction(gk) * exabs[i][j]
            # N itself is within gamma_k of the exact sum of magnitudes
            assert abs(Fraction(float(N[i, j])) - exabs[i][j]) <= Fraction(gk) * exabs[i][j]


def test_dgemm_alpha_beta_semantics_and_beta_zero_nan():
    m, n, k = 8, 7, 5
    A = syn.matrix("int", m, k, 31)
    B = syn.matrix("int", k, n, 32)
    C0 = F(np.full((m, n), np.nan))
    C = oracle.dgemm(A, B, C0, alpha=0.5, beta=0.0)  # beta = 0: C is write-only
    ex = exact_product(A, B)
    assert np.array_equal(C, np.array([[float(x / 2) for x in r] for r in ex]))
    # k = 0: C := beta * C
    Ce = F(np.arange(m * n, dtype=np.float64).reshape(m, n))
    out = oracle.dgemm(F(np.zeros((m, 0))), F(np.zeros((0, n))), Ce.copy(order="F"), alpha=3.0, beta=2.0)
    assert np.array_equal(out, 2.0 * Ce)


def test_dgemm_abs_sign_invariance():
    A = syn.matrix("uniform", 9, 33, 41)
    B = syn.matrix("uniform", 33, 11, 42)
    N = oracle.dgemm_abs(A, B)
    sa = F(np.where(syn.unit_uniform(43, A.size).reshape(A.shape) < 0.5, -1.0, 1.0))
    assert np.array_equal(N, oracle.dgemm_abs(F(A * sa), B))
    assert np.all(N >= np.abs(oracle.dgemm(A, B)) * (1 - 40 * U))


def test_dgemm_threads_do_not_change_bits():
    A = syn.matrix("uniform", 65, 70, 51)
    B = syn.matrix("uniform", 70, 33, 52)
    assert np.array_equal(oracle.dgemm(A, B, nthreads=1), oracle.dgemm(A, B, nthreads=4))


# --------------------------------------------------------------------------- emulation steps
def test_exponents_hand_cases():
    X = F([[0.75, -0.1, 0.0], [1.0, 0.0, 0.0], [3.0, -5.0, 0.5], [0.0, 0.0, 0.0],
           [np.inf, 1.0, 0.0], [2.0 ** -1074, 0.0, 0.0], [-2.0 ** 1000, 1.0, 0.0]])
    e, fl = oracle.exponents(X, "rows")
    # e = floor(log2 max|x|) + 1: 0.75 -> 0, 1 -> 1, 5 -> 3, zero row -> 0, inf -> flagged
    assert list(e) == [0, 1, 3, 0, 0, -1073, 1001]
    assert list(fl) == [0, 0, 0, 0, 1, 0, 0]
    ec, flc = oracle.exponents(F(X.T), "cols")
    assert list(ec) == list(e) and list(flc) == list(fl)
    et, flt = oracle.exponents(F(X.T), "rows", trans=True)
    assert list(et) == list(e)


def digits_by_bitfield(x, e, S, beta):
    """Truncation digits from the exact rational value: X = floor(|x| 2^(beta S - e)),
    digit s = the s-th base-2^beta field of X from the top, carrying the sign of x."""
    fx = Fraction(x) * Fraction(2) ** (beta * S - e)
    X = abs(fx.numerator) // fx.denominator
    sg = -1 if x < 0 else 1
    return [sg * ((X >> (beta * (S - s))) & ((1 << beta) - 1)) for s in range(1, S + 1)]


def test_split_hand_worked_example():
    # 0.75 * 2^7 = 96 exactly; -0.1 has an infinite binary expansion
    X = F([[0.75, -0.1]])
    e, fl = oracle.exponents(X, "rows")
    D = oracle.split(X, "rows", e, fl, S=3, beta=7)
    assert list(D[:, 0, 0]) == [96, 0, 0]
    assert list(D[:, 0, 1]) == digits_by_bitfield(-0.1, 0, 3, 7)
    assert D[0, 0, 1] == -12  # trunc(-0.1 * 128) = trunc(-12.8)


@pytest.mark.parametrize("kind,phi", [("uniform", 0.0), ("phi", 1.0), ("phi", 4.0), ("normal", 0.0)])
@pytest.mark.parametrize("beta,S", [(7, 5), (7, 9), (8, 8), (6, 4)])
def test_split_matches_bitfields_and_bounds(kind, phi, beta, S):
    X = syn.matrix(kind, 6, 40, 61, phi=phi)
    e, fl = oracle.exponents(X, "rows")
    D = oracle.split(X, "rows", e, fl, S=S, beta=beta)
    assert np.abs(D).max() <= 2 ** beta - 1
    for i in range(X.shape[0]):
        for q in range(X.shape[1]):
            x = float(X[i, q])
            assert list(D[:, i, q]) == digits_by_bitfield(x, int(e[i]), S, beta)
            # truncation error below one unit of the last slice
            approx = sum(Fraction(int(D[s, i, q])) * Fraction(2) ** (-beta * (s + 1)) for s in range(S))
            err = Fraction(x) * Fraction(2) ** (-int(e[i])) - approx
            assert abs(err) < Fraction(2) ** (-beta * S)
            assert err == 0 or (err > 0) == (x > 0)


def test_split_error_free_when_enough_slices():
    # 53-bit significands inside one binade of the row maximum need ceil(54/beta) slices
    X = syn.matrix("uniform", 4, 30, 71)
    e, fl = oracle.exponents(X, "rows")
    S = 12
    D = oracle.split(X, "rows", e, fl, S=S, beta=7)
    for i in range(4):
        for q in range(30):
            x = float(X[i, q])
            if abs(x) < 2.0 ** (int(e[i]) - 30):
                continue
            rec = sum(Fraction(int(D[s, i, q])) * Fraction(2) ** (-7 * (s + 1)) for s in range(S))
            assert rec * Fraction(2) ** int(e[i]) == Fraction(x)


def test_split_transposed_and_columns_agree():
    A = syn.matrix("phi", 7, 19, 81, phi=1.0)
    e1, f1 = oracle.exponents(A, "rows")
    e2, f2 = oracle.exponents(F(A.T), "rows", trans=True)
    e3, f3 = oracle.exponents(F(A.T), "cols")
    assert np.array_equal(e1, e2) and np.array_equal(e1, e3)
    D1 = oracle.split(A, "rows", e1, f1, 6, 7)
    D2 = oracle.split(F(A.T), "rows", e2, f2, 6, 7, trans=True)
    D3 = oracle.split(F(A.T), "cols", e3, f3, 6, 7)
    assert np.array_equal(D1, D2) and np.array_equal(D1, D3)


def test_slice_products_bigint_bruteforce():
    S, m, n, k = 4, 3, 5, 11
    A = syn.matrix("uniform", m, k, 91)
    B = syn.matrix("uniform", k, n, 92)
    e, ef = oracle.exponents(A, "rows")
    f, ff = oracle.exponents(B, "cols")
    Ad = oracle.split(A, "rows", e, ef, S, 7)
    Bd = oracle.split(B, "cols", f, ff, S, 7)
    P = oracle.slice_products(Ad, Bd)
    for d in range(2, S + 2):
        for i in range(m):
            for j in range(n):
                want = 0
                for s in range(1, d):
                    t = d - s
                    want += sum(int(Ad[s - 1, i, p]) * int(Bd[t - 1, j, p]) for p in range(k))
                assert int(P[d - 2, i, j]) == want


@pytest.mark.parametrize("S,beta", [(5, 7), (11, 7), (10, 8)])
def test_recombine_is_exact_rational_rounded_once(S, beta):
    m, n, k = 4, 3, 9
    A = syn.matrix("phi", m, k, 101, phi=1.0)
    B = syn.matrix("phi", k, n, 102, phi=1.0)
    C, det = oracle.emulated_dgemm(A, B, S, beta)
    Ad, Bd, e, f = det["Ad"], det["Bd"], det["e"], det["f"]
    for i in range(m):
        for j in range(n):
            val = Fraction(0)
            for p in range(k):
                for s in range(1, S + 1):
                    for t in range(1, S + 2 - s):
                        val += (Fraction(int(Ad[s - 1, i, p]) * int(Bd[t - 1, j, p]))
                                * Fraction(2) ** (int(e[i]) + int(f[j]) - beta * (s + t)))
            assert C[i, j] == float(val)  # Fraction -> float rounds to nearest


def test_emulated_integer_inputs_exact():
    m, n, k = 17, 12, 40
    A = syn.matrix("int", m, k, 111)
    B = syn.matrix("int", k, n, 112)
    C0 = syn.matrix("int", m, n, 113)
    C, _ = oracle.emulated_dgemm(A, B, S=2, beta_bits=7, C=C0.copy(order="F"), alpha=1.0, beta=1.0)
    assert np.array_equal(C, oracle.dgemm(A, B, C0.copy(order="F"), alpha=1.0, beta=1.0))


@pytest.mark.parametrize("phi,S", [(0.0, 7), (1.0, 8), (4.0, 11)])
def test_emulated_within_componentwise_bound(phi, S):
    m, n, k = 12, 10, 96
    A = syn.matrix("phi", m, k, 121, phi=phi)
    B = syn.matrix("phi", k, n, 122, phi=phi)
    C, _ = oracle.emulated_dgemm(A, B, S=S, beta_bits=7)
    ex = exact_product(A, B)
    N = oracle.dgemm_abs(A, B)
    for i in range(m):
        for j in range(n):
            assert abs(Fraction(float(C[i, j])) - ex[i][j]) <= Fraction(4 * k * U) * Fraction(float(N[i, j]))


def test_emulated_nonfinite_rows_flagged_nan():
    A = syn.matrix("uniform", 5, 8, 131)
    A[2, 3] = np.inf
    B = syn.matrix("uniform", 8, 4, 132)
    B[1, 2] = np.nan
    C, det = oracle.emulated_dgemm(A, B, S=6, beta_bits=7)
    assert det["eflag"][2] == 1 and det["fflag"][2] == 1
    assert np.all(np.isnan(C[2, :])) and np.all(np.isnan(C[:, 2]))
    mask = np.ones_like(C, dtype=bool)
    mask[2, :] = False
    mask[:, 2] = False
    assert np.all(np.isfinite(C[mask]))


# --------------------------------------------------------------------------- modular encoding
def test_truncated_integers_are_the_digit_expansion():
    # bits = 7 S: X^ is the first S truncation digits read as one integer (the C split's digits)
    for which, trans in (("rows", False), ("cols", False), ("rows", True)):
        X = syn.matrix("phi", 9, 23, 141, phi=2.0)
        e, fl = oracle.exponents(X, which, trans)
        for S in (1, 3, 6):
            D = oracle.split(X, which, e, fl, S, 7, trans)
            Xh = oracle.truncated_integers(X, which, e, fl, 7 * S, trans)
            expansion = sum(D[s].astype(object) * (2 ** (7 * (S - 1 - s))) for s in range(S))
            assert np.array_equal(Xh, expansion)


def test_truncated_integers_truncation_identity():
    # any width: 0 <= |x| 2^(bits - e) - |X^| < 1, same sign, |X^| < 2^bits
    X = syn.matrix("phi", 7, 31, 142, phi=3.0)
    e, fl = oracle.exponents(X, "rows")
    for bits in (5, 20, 39, 56):
        Xh = oracle.truncated_integers(X, "rows", e, fl, bits)
        for i in range(7):
            for q in range(31):
                scaled = Fraction(float(X[i, q])) * Fraction(2) ** (bits - int(e[i]))
                h = int(Xh[i, q])
                assert abs(h) < 2 ** bits and 0 <= abs(scaled) - abs(h) < 1
                assert h == 0 or (h > 0) == (X[i, q] > 0)
    assert int(oracle.truncated_integers(F([[0.75]]), "rows", np.array([0]), np.array([0]), 3)[0, 0]) == 6


def test_greedy_moduli_are_pairwise_coprime_and_hand_listed():
    mods = oracle.greedy_moduli(14)
    assert all(math.gcd(a, b) == 1 for i, a in enumerate(mods) for b in mods[i + 1:])
    # 252 = 2^2 3^2 7 and 250 = 2 5^3 share factors with 255 = 3 5 17 / 254 = 2 127; 217 = 7 31
    # is the first composite taken after 247 = 13 19; 221 = 13 17 and 209 = 11 19 are skipped
    assert mods == [255, 254, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199]
    assert all(abs(p // 2) <= 127 for p in mods)


def test_centred_residues_reconstruct_through_library_crt():
    sympy_crt = pytest.importorskip("sympy.ntheory.modular").crt
    mods = oracle.greedy_moduli(13)
    rng = np.random.default_rng(143)
    vals = np.array([int(v) for v in rng.integers(-2 ** 62, 2 ** 62, 40)] + [0, 1, -1, 127, -128, 2 ** 80, -(2 ** 80) + 7],
                    dtype=object).reshape(47, 1)
    R = oracle.centred_residues(vals, mods)
    for l, p in enumerate(mods):
        assert R[l].min() >= -(p // 2) and R[l].max() <= (p - 1) // 2
    P = math.prod(mods)
    for t in range(vals.shape[0]):
        x, _ = sympy_crt(mods, [int(R[l, t, 0]) % p for l, p in enumerate(mods)])
        x = int(x)
        assert (x - P if x > P // 2 else x) == int(vals[t, 0])
        assert oracle.crt_reconstruct([int(R[l, t, 0]) for l in range(len(mods))], mods) == int(vals[t, 0])


def test_moduli_suffice_matches_the_range_argument():
    mods = oracle.greedy_moduli(13)
    P = math.prod(mods)
    # 42-bit operands, k = 8192: |sum| <= k (2^42 - 1)^2 < 2^97 < P / 2
    assert oracle.moduli_suffice(mods, 42, 8192) and P > 2 * 8192 * (2 ** 42 - 1) ** 2
    assert not oracle.moduli_suffice(mods[:12], 42, 8192)
    assert not oracle.moduli_suffice(oracle.greedy_moduli(14), 49, 8192)


def test_modular_dgemm_integer_inputs_exact():
    m, n, k = 11, 9, 30
    A = syn.matrix("int", m, k, 144)
    B = syn.matrix("int", k, n, 145)
    C0 = syn.matrix("int", m, n, 146)
    C, _ = oracle.modular_dgemm(A, B, 21, C0.copy(order="F"), 1.0, 1.0)
    assert np.array_equal(C, A @ B + C0)


def test_modular_dgemm_equals_one_slice_emulation_bitwise():
    # bits = 7: the one-slice emulation keeps its only digit pair, so both compute the same exact
    # integer product, rounded once
    A = syn.matrix("phi", 8, 40, 147, phi=1.0)
    B = syn.matrix("phi", 40, 6, 148, phi=1.0)
    C1, _ = oracle.emulated_dgemm(A, B, S=1, beta_bits=7)
    C2, _ = oracle.modular_dgemm(A, B, 7)
    assert np.array_equal(C1, C2)


@pytest.mark.parametrize("transa,transb", [(False, False), (True, True)])
def test_modular_dgemm_within_bound_at_full_width(transa, transb):
    m, n, k = 7, 6, 50
    A = syn.matrix("phi", k if transa else m, m if transa else k, 149, phi=1.0)
    B = syn.matrix("phi", n if transb else k, k if transb else n, 150, phi=1.0)
    C, _ = oracle.modular_dgemm(A, B, 56, transa=transa, transb=transb)
    ex = exact_product(A, B, transa, transb)
    N = oracle.dgemm_abs(A, B, transa, transb)
    for i in range(m):
        for j in range(n):
            assert abs(Fraction(float(C[i, j])) - ex[i][j]) <= Fraction(4 * k * U) * Fraction(float(N[i, j]))


def test_modular_dgemm_alpha_beta_fma_and_nan():
    A = syn.matrix("uniform", 4, 10, 151)
    A[1, 3] = np.nan
    B = syn.matrix("uniform", 10, 3, 152)
    C0 = syn.matrix("uniform", 4, 3, 153)
    C, det = oracle.modular_dgemm(A, B, 30, C0.copy(order="F"), -0.5, 3.0)
    assert np.all(np.isnan(C[1, :])) and det["eflag"][1] == 1
    for i in (0, 2, 3):
        for j in range(3):
            y = math.ldexp(float(det["Z"][i, j]), int(det["e"][i]) + int(det["f"][j]) - 60)
            exact = Fraction(3.0) * Fraction(float(C0[i, j])) + Fraction(-0.5 * y)
            assert C[i, j] == float(exact)


# --------------------------------------------------------------------------- triangular solve
@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("trans", [False, True])
def test_trsm_integer_recovery_exact(side, lower, trans):
    # unit triangle of small integers, integer solution: every substitution step is exact
    t, r = 12, 5
    rng = np.random.default_rng(161)
    A = rng.integers(-2, 3, (t, t)).astype(np.float64)
    A[np.diag_indices(t)] = np.nan                     # unit diagonal: never read
    T = np.tril(A, -1) if lower else np.triu(A, 1)
    T = T + np.eye(t)
    M = T.T if trans else T
    X = rng.integers(-3, 4, (t, r) if side == "L" else (r, t)).astype(np.float64)
    B = M @ X if side == "L" else X @ M
    got = oracle.trsm(A, B, 1.0, side, lower, trans, unit=True)
    assert np.array_equal(got, X)


@pytest.mark.parametrize("side", ["L", "R"])
@pytest.mark.parametrize("lower,trans", [(True, False), (False, True), (False, False)])
def test_trsm_agrees_with_scipy(side, lower, trans):
    sl = pytest.importorskip("scipy.linalg")
    t, r = 40, 7
    A = syn.matrix("uniform", t, t, 162) / t + np.diag(1.0 + syn.unit_uniform(163, t))
    B = syn.matrix("uniform", t, r, 164) if side == "L" else syn.matrix("uniform", r, t, 165)
    got = oracle.trsm(A, B, -2.0, side, lower, trans)
    if side == "L":
        want = sl.solve_triangular(A, -2.0 * B, lower=lower, trans=1 if trans else 0)
    else:   # X op(A) = B  <=>  op(A)^T X^T = B^T
        want = sl.solve_triangular(A, -2.0 * B.T, lower=lower, trans=0 if trans else 1).T
    assert np.allclose(got, want, rtol=1e-13, atol=1e-13)
    I = np.eye(t)
    assert np.array_equal(oracle.trsm(I, B, 3.0, side, lower, trans), 3.0 * B)


# --------------------------------------------------------------------------- I/O counts
def closed_form(member, m, n, k, b1, b2, c_read):
    """The paper's resident-algorithm I/O counts in margin (ceiling) form, Sec. 2.2."""
    cdiv = lambda a, b: -(-a // b)
    if member == "resident_c":      # Sec. 2.2.1: mn reads + mn writes of C
        mc, nc = b1, b2
        return dict(a_reads=m * k * cdiv(n, nc), b_reads=k * n * cdiv(m, mc),
                    c_reads=m * n if c_read else 0, c_writes=m * n)
    if member == "resident_a":      # Sec. 2.2.2: A read once, C per k_c block
        mc, kc = b1, b2
        nk = cdiv(k, kc)
        return dict(a_reads=m * k, b_reads=k * n * cdiv(m, mc),
                    c_reads=m * n * (nk - 1 + int(c_read)), c_writes=m * n * nk)
    if member == "resident_b":      # mirror of Resident A
        kc, nc = b1, b2
        nk = cdiv(k, kc)
        return dict(a_reads=m * k * cdiv(n, nc), b_reads=k * n,
                    c_reads=m * n * (nk - 1 + int(c_read)), c_writes=m * n * nk)
    if member == "goto":            # A2C0: A per n_c panel, B once, C per k_c block
        nc, kc = b1, b2
        nk = cdiv(k, kc)
        return dict(a_reads=m * k * cdiv(n, nc), b_reads=k * n,
                    c_reads=m * n * (nk - 1 + int(c_read)), c_writes=m * n * nk)
    raise ValueError(member)


@pytest.mark.parametrize("member,b1,b2,b3", [("resident_c", 8, 6, 0), ("resident_a", 8, 5, 0),
                                             ("resident_b", 5, 6, 0), ("goto", 6, 5, 4)])
@pytest.mark.parametrize("shape", [(37, 29, 41), (32, 30, 40), (1, 7, 3)])
@pytest.mark.parametrize("c_read", [True, False])
def test_counting_oracle_equals_closed_forms(member, b1, b2, b3, shape, c_read):
    m, n, k = shape
    A = syn.matrix("int", m, k, 141)
    B = syn.matrix("int", k, n, 142)
    C0 = syn.matrix("int", m, n, 143) if c_read else F(np.zeros((m, n)))
    C = C0.copy(order="F")
    cnt = oracle.count_member(member, A, B, C, b1, b2, b3, c_read=c_read)
    want = closed_form(member, m, n, k, b1, b2, c_read)
    for key, val in want.items():
        assert cnt[key] == val, (key, cnt[key], val)
    assert cnt["flops"] == 2 * m * n * k
    # integer inputs: any summation order is exact, so C must be C0 + A B exactly
    assert np.array_equal(C, oracle.dgemm(A, B, C0.copy(order="F"), 1.0, 1.0))


def lower_bound_reads(m, n, k, M):
    return 2 * m * n * k / math.sqrt(M) - 2 * M


@pytest.mark.parametrize("member,b1,b2,b3", [("resident_c", 8, 8, 0), ("resident_a", 8, 8, 0),
                                             ("resident_b", 8, 8, 0), ("goto", 16, 4, 4)])
def test_counting_oracle_respects_io_lower_bound(member, b1, b2, b3):
    # Sec. 2.1: any algorithm reads at least 2mnk/sqrt(M) - 2M words into a fast memory of M words
    m, n, k = 48, 40, 56
    A = syn.matrix("int", m, k, 151)
    B = syn.matrix("int", k, n, 152)
    C = syn.matrix("int", m, n, 153)
    cnt = oracle.count_member(member, A, B, C, b1, b2, b3)
    reads = cnt["a_reads"] + cnt["b_reads"] + cnt["c_reads"]
    assert reads >= lower_bound_reads(m, n, k, cnt["fast_words"])
    # and writes at least mn - M
    assert cnt["c_writes"] >= m * n - cnt["fast_words"]


def _limit_flops_per_byte(member, b1, b2):
    """Intensity 2mnk / (8 * words) of the closed forms as m = n = k = L grows."""
    vals = []
    for L in (10 ** 6, 10 ** 7):
        L = L - L % (b1 * b2)
        c = closed_form(member, L, L, L, b1, b2, True)
        words = sum(c.values())
        vals.append(2 * L ** 3 / (8 * words))
    return vals[-1]


def test_paper_printed_intensities():
    g = json.load(open(os.path.join(GOLDEN, "paper_intensities.json")))
    goto = g["goto_intensity"]
    val = _limit_flops_per_byte("goto", goto["n_c"], goto["k_c"])
    # the paper's own formula (1/k_c + 1/(2 n_c))^-1 flops per element
    formula = 1.0 / (1.0 / goto["k_c"] + 1.0 / (2 * goto["n_c"])) / 8.0
    assert round(val, goto["digits"]) == goto["flops_per_byte"]
    assert round(formula, goto["digits"]) == goto["flops_per_byte"]
    b3 = g["b3a2c0_intensity"]
    val = _limit_flops_per_byte("resident_b", b3["k_c"], b3["n_c"])
    assert round(val, b3["digits"]) == b3["flops_per_byte"]


def test_paper_wrong_member_and_goto_claims():
    g = json.load(open(os.path.join(GOLDEN, "paper_intensities.json")))
    b = 768
    L = 768 * 4000
    reads = lambda c: c["a_reads"] + c["b_reads"] + c["c_reads"]
    # m = n = sqrt(M), k large: Resident C is right, Resident A costs 50% more reads
    right = reads(closed_form("resident_c", b, b, L, b, b, True))
    wrong = reads(closed_form("resident_a", b, b, L, b, b, True))
    assert abs(wrong / right - g["wrong_member_penalty"]["ratio"]) < 0.01
    # Goto (n_c = 3000, k_c = 192) vs B3A2C0 (768 x 768 block of B): about twice the reads
    L = 3000 * 768 * 8
    goto = reads(closed_form("goto", L, L, L, 3000, 192, True))
    opt = reads(closed_form("resident_b", L, L, L, 768, 768, True))
    gv = g["goto_vs_optimal"]
    assert abs(goto / opt - gv["approx_ratio"]) < gv["tolerance"]
