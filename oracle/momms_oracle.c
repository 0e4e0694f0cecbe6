/*
 * momms_oracle.c -- plain, slow, obviously correct CPU reference for the
 * MOMMS hot path (Smith & van de Geijn, "The MOMMS Family of Matrix
 * Multiplication Algorithms", SC19).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no source with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC
 * (-ffp-contract=off keeps every multiply and add separately rounded, which is
 * what the definitions below state.)
 *
 * Contents
 *   1. oracle_dgemm       C := alpha*op(A)*op(B) + beta*C, the plain definition
 *                         (Sec. 2.1 footnote: gamma_ij = sum_p alpha_ip beta_pj;
 *                         Sec. 2.2.1: C += AB), p ascending from 0.0.
 *   2. oracle_dgemm_abs   N := |op(A)|*|op(B)|, the magnitude matrix of the
 *                         componentwise error bound.
 *   3. Emulated-FP64 steps (integer-slice splitting; no counterpart in the
 *      paper, written from the definition of truncation splitting):
 *        oracle_exponents  per-row / per-column scaling exponents
 *        oracle_split      signed beta-bit digit slices, in FP64 arithmetic
 *        oracle_slice_products  P_d = sum_{s+t=d} A_s B_t in exact int64
 *        oracle_recombine  C := alpha * 2^(e_i+f_j) * sum_d 2^(-beta d) P_d
 *                          + beta*C, summed exactly (multi-word) then rounded once
 *   4. oracle_count_member  a blocked two-level-memory simulation of each
 *      resident algorithm (Sec. 2.2, Sec. 4.3 for Goto's A2C0) that copies
 *      blocks between "slow" and "fast" buffers explicitly and counts every
 *      word moved, for comparison with the closed-form I/O counts.
 *
 * Layout: every matrix is column-major with a leading dimension, as in BLAS.
 * op(X) = X (trans = 0) or X^T (trans = 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

/* element (i, p) of op(A) where op(A) is m x k */
static inline double opget(const double* X, i64 ld, int trans, i64 r, i64 c) {
    return trans ? X[c + r * ld] : X[r + c * ld];
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 1. The plain product.                                                     */
/*    t_ij = sum_{p=0}^{k-1} a_ip * b_pj   (p ascending, starting from 0.0)   */
/*    C_ij = alpha*t_ij + beta*C_ij        (beta == 0: C is write-only)       */
/* Loop order j -> p -> i over a temporary column; per element this is the    */
/* same sequence of roundings as a p-ascending dot product.  The parallel     */
/* loop is over j only, so the result does not depend on the thread count.   */
/* ------------------------------------------------------------------------ */
int oracle_dgemm(int transa, int transb, i64 m, i64 n, i64 k, double alpha,
                 const double* A, i64 lda, const double* B, i64 ldb,
                 double beta, double* C, i64 ldc, int nthreads) {
    if (m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    set_threads(nthreads);
    int err = 0;
#pragma omp parallel
    {
        double* t = (double*)malloc((size_t)m * sizeof(double));
        if (!t) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(static)
        for (i64 j = 0; j < n; ++j) {
            if (!t) continue;
            for (i64 i = 0; i < m; ++i) t[i] = 0.0;
            for (i64 p = 0; p < k; ++p) {
                double b = opget(B, ldb, transb, p, j);
                if (!transa) {
                    const double* a = A + p * lda;
                    for (i64 i = 0; i < m; ++i) t[i] = t[i] + a[i] * b;
                } else {
                    for (i64 i = 0; i < m; ++i) t[i] = t[i] + A[p + i * lda] * b;
                }
            }
            double* c = C + j * ldc;
            if (beta == 0.0) {
                for (i64 i = 0; i < m; ++i) c[i] = alpha * t[i];
            } else {
                for (i64 i = 0; i < m; ++i) c[i] = alpha * t[i] + beta * c[i];
            }
        }
        free(t);
    }
    return err;
}

/* N_ij = sum_p |a_ip| * |b_pj|, same loop order. */
int oracle_dgemm_abs(int transa, int transb, i64 m, i64 n, i64 k,
                     const double* A, i64 lda, const double* B, i64 ldb,
                     double* N, i64 ldn, int nthreads) {
    if (m < 0 || n < 0 || k < 0) return -1;
    if (m == 0 || n == 0) return 0;
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (i64 j = 0; j < n; ++j) {
        double* t = N + j * ldn;
        for (i64 i = 0; i < m; ++i) t[i] = 0.0;
        for (i64 p = 0; p < k; ++p) {
            double b = fabs(opget(B, ldb, transb, p, j));
            for (i64 i = 0; i < m; ++i) t[i] = t[i] + fabs(opget(A, lda, transa, i, p)) * b;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 3. Emulated FP64 by signed integer digit slices.                          */
/*                                                                          */
/* Scaling exponent of a vector x (a row of op(A) or a column of op(B)):     */
/*   e = floor(log2(max |x|)) + 1, i.e. the frexp exponent of max|x|, so     */
/*   that every |x| * 2^-e < 1.  An all-zero vector gets e = 0.  A vector    */
/*   holding Inf or NaN is flagged (flag = 1) and gets e = 0.                */
/* ------------------------------------------------------------------------ */
static int vec_exponent(const double* x, i64 n, i64 stride, int* flag) {
    double mx = 0.0;
    *flag = 0;
    for (i64 i = 0; i < n; ++i) {
        double v = x[i * stride];
        if (!isfinite(v)) { *flag = 1; continue; }
        double a = fabs(v);
        if (a > mx) mx = a;
    }
    if (*flag || mx == 0.0) return 0;
    int e;
    (void)frexp(mx, &e); /* mx = f * 2^e, f in [0.5, 1) */
    return e;
}

/* which = 0: rows of op(A) (op(A) is rows x inner); which = 1: columns of
 * op(B) (op(B) is inner x rows).  exps[r], flags[r] for r < rows. */
int oracle_exponents(int which, int trans, i64 rows, i64 inner,
                     const double* X, i64 ld, int32_t* exps, uint8_t* flags) {
    for (i64 r = 0; r < rows; ++r) {
        int fl;
        int e;
        /* element q of vector r */
        if (which == 0) {
            /* row r of op(A): op(A)(r, q) */
            if (!trans) e = vec_exponent(X + r, inner, ld, &fl);
            else        e = vec_exponent(X + r * ld, inner, 1, &fl);
        } else {
            /* column r of op(B): op(B)(q, r) */
            if (!trans) e = vec_exponent(X + r * ld, inner, 1, &fl);
            else        e = vec_exponent(X + r, inner, ld, &fl);
        }
        exps[r] = e;
        flags[r] = (uint8_t)fl;
    }
    return 0;
}

/* Truncation splitting, in FP64 arithmetic (every step below is exact):
 *   x' = x * 2^-e                       (|x'| < 1)
 *   for s = 1..S:  t = x' * 2^beta;  d_s = trunc(t);  x' = t - d_s
 * so that x * 2^-e = sum_s d_s 2^(-beta s) + 2^(-beta S) * x'_S with every
 * |d_s| <= 2^beta - 1 and every d_s carrying the sign of x.
 * Output digits[(s * rows + r) * inner + q] for s = 0..S-1 (slice s+1),
 * i.e. each slice is a rows x inner matrix stored inner-contiguous.
 * Flagged (non-finite) vectors produce zero digits. */
int oracle_split(int which, int trans, i64 rows, i64 inner, const double* X, i64 ld,
                 const int32_t* exps, const uint8_t* flags, int S, int beta,
                 int16_t* digits) {
    if (S < 1 || beta < 1 || beta > 14) return -1;
    const double radix = ldexp(1.0, beta);
    for (i64 r = 0; r < rows; ++r) {
        for (i64 q = 0; q < inner; ++q) {
            double x;
            if (which == 0) x = opget(X, ld, trans, r, q);
            else            x = opget(X, ld, trans, q, r);
            if (flags[r]) x = 0.0;
            double xs = ldexp(x, -exps[r]);
            for (int s = 0; s < S; ++s) {
                double t = xs * radix;
                double d = trunc(t);
                xs = t - d;
                digits[((i64)s * rows + r) * inner + q] = (int16_t)d;
            }
        }
    }
    return 0;
}

/* P_d = sum_{s+t=d} A_s * B_t over slices s,t >= 1 with s + t <= S + 1
 * (the triangular pair set), for d = 2..S+1, in exact 64-bit integers.
 * Ad: S slices of m x k (k-contiguous), Bd: S slices of n x k (k-contiguous).
 * P[(d-2) * m * n + i + j * m]  (each diagonal column-major m x n). */
int oracle_slice_products(i64 m, i64 n, i64 k, int S, const int16_t* Ad,
                          const int16_t* Bd, int64_t* P, int nthreads) {
    set_threads(nthreads);
    for (int d = 2; d <= S + 1; ++d) {
        int64_t* Pd = P + (i64)(d - 2) * m * n;
#pragma omp parallel for schedule(static)
        for (i64 j = 0; j < n; ++j) {
            for (i64 i = 0; i < m; ++i) {
                int64_t acc = 0;
                for (int s = 1; s <= d - 1; ++s) {
                    int t = d - s;
                    const int16_t* a = Ad + ((i64)(s - 1) * m + i) * k;
                    const int16_t* b = Bd + ((i64)(t - 1) * n + j) * k;
                    for (i64 p = 0; p < k; ++p) acc += (int64_t)a[p] * (int64_t)b[p];
                }
                Pd[i + j * m] = acc;
            }
        }
    }
    return 0;
}

/* Exact signed sum of shifted 64-bit integers, rounded once to double.
 * The value is held in two's complement as NLIMB 32-bit limbs kept in int64
 * (carries are propagated on conversion), so any S with beta*(S-1) + 64 below
 * 32*NLIMB - 1 bits is exact. */
#define NLIMB 10
typedef struct { int64_t l[NLIMB]; } bigacc;

static void big_add_shifted(bigacc* a, int64_t v, int shift) {
    /* a += v * 2^shift, v split into 32-bit pieces with sign carried by the top one */
    int limb = shift / 32, off = shift % 32;
    __int128 w = (__int128)v * ((__int128)1 << off); /* |w| < 2^95 */
    for (int t = 0; t < 4 && limb + t < NLIMB; ++t) {
        int64_t piece = (int64_t)(w & 0xFFFFFFFF);
        if (t == 3) piece = (int64_t)w; /* remaining signed part */
        a->l[limb + t] += piece;
        w = (w - piece) / ((__int128)1 << 32);
        if (w == 0) break;
    }
}

static double big_to_double(bigacc* a, int exp2) {
    /* normalise limbs to [0, 2^32) with a signed carry out of the top */
    int64_t carry = 0;
    uint32_t limb[NLIMB];
    for (int t = 0; t < NLIMB; ++t) {
        int64_t v = a->l[t] + carry;
        int64_t lo = v & 0xFFFFFFFF;
        carry = (v - lo) / ((int64_t)1 << 32);
        limb[t] = (uint32_t)lo;
    }
    int neg = carry < 0; /* carry is 0 or -1 for values that fit */
    if (neg) { /* magnitude = two's complement negation */
        uint64_t c = 1;
        for (int t = 0; t < NLIMB; ++t) {
            uint64_t v = (uint64_t)(uint32_t)~limb[t] + c;
            limb[t] = (uint32_t)v;
            c = v >> 32;
        }
    }
    int top = -1;
    for (int t = NLIMB - 1; t >= 0; --t) if (limb[t]) { top = t; break; }
    if (top < 0) return neg ? -0.0 : 0.0;
    /* bit position of the leading one */
    int lead = 31;
    while (!((limb[top] >> lead) & 1u)) --lead;
    int msb = top * 32 + lead;
    /* take the 64 bits [msb-63, msb] and a sticky bit for everything below:
       rounding the 64-bit value to odd and then to double is the correctly
       rounded result (64 >= 53 + 2). */
    uint64_t T = 0;
    int sticky = 0;
    for (int b = msb; b >= 0; --b) {
        int bit = (limb[b / 32] >> (b % 32)) & 1u;
        if (msb - b < 64) T = (T << 1) | (uint64_t)bit;
        else if (bit) { sticky = 1; break; }
    }
    int low = msb - 63; /* exponent of T's last bit; < 0 means T is shorter than 64 bits */
    if (low < 0) low = 0;
    if (sticky) T |= 1u;
    double x = ldexp((double)T, low + exp2);
    return neg ? -x : x;
}

/* Recombination: the emulated product, computed exactly and rounded once.
 *   Q_ij = sum_{d=2}^{S+1} 2^(beta (S+1-d)) P_d,ij        (exact)
 *   x_ij = round_to_double(Q_ij * 2^(e_i + f_j - beta (S+1)))
 *   C_ij = alpha * x_ij + beta_c * C_ij   (beta_c == 0: C not read)
 * Rows / columns flagged non-finite give NaN. */
int oracle_recombine(i64 m, i64 n, int S, int beta, const int64_t* P,
                     const int32_t* e, const uint8_t* eflag, const int32_t* f,
                     const uint8_t* fflag, double alpha, double beta_c,
                     double* C, i64 ldc) {
    if (beta * (S - 1) + 100 >= 32 * NLIMB) return -1;
    for (i64 j = 0; j < n; ++j) {
        for (i64 i = 0; i < m; ++i) {
            double x;
            if (eflag[i] || fflag[j]) {
                x = NAN;
            } else {
                bigacc q;
                memset(&q, 0, sizeof(q));
                for (int d = 2; d <= S + 1; ++d)
                    big_add_shifted(&q, P[(i64)(d - 2) * m * n + i + j * m], beta * (S + 1 - d));
                x = big_to_double(&q, e[i] + f[j] - beta * (S + 1));
            }
            double* c = C + i + j * ldc;
            if (beta_c == 0.0) *c = alpha * x;
            else               *c = alpha * x + beta_c * *c;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 4. Counting oracle: blocked algorithms on an explicit two-level memory.   */
/*                                                                          */
/* Slow memory = the caller's A, B, C.  Fast memory = buffers below.  Every  */
/* word copied slow->fast counts as a read of that operand, every word       */
/* copied fast->slow as a write.  Arithmetic happens only on fast buffers.   */
/* The computed operation is the paper's C += A*B (Sec. 2.2), with the flag  */
/* c_read saying whether C's initial contents must be read (c_read = 0 is    */
/* BLAS beta = 0: C is overwritten and its first read is skipped).           */
/*                                                                          */
/* member 0: Resident C  (b1 = m_c, b2 = n_c)   Sec. 2.2.1                   */
/* member 1: Resident A  (b1 = m_c, b2 = k_c)   Sec. 2.2.2                   */
/* member 2: Resident B  (b1 = k_c, b2 = n_c)   Sec. 2.2.2 (mirror of A)     */
/* member 3: Goto A2C0   (b1 = n_c, b2 = k_c, b3 = m_c)   Sec. 4.3, Sec. 5.2 */
/*           a k_c x n_c panel of B (L3 guest) and an m_c x k_c block of A    */
/*           (L2 resident) in fast memory, C streamed per k_c block.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t a_reads, b_reads, c_reads, c_writes, flops, fast_words;
} oracle_io_counts;

static i64 imin(i64 a, i64 b) { return a < b ? a : b; }

int oracle_count_member(int member, i64 m, i64 n, i64 k, i64 b1, i64 b2, i64 b3,
                        int c_read, const double* A, i64 lda, const double* B,
                        i64 ldb, double* C, i64 ldc, oracle_io_counts* out) {
    memset(out, 0, sizeof(*out));
    if (b1 <= 0 || b2 <= 0) return -1;
    if (member == 0) {
        const i64 mc = b1, nc = b2;
        double* Cf = (double*)malloc((size_t)(mc * nc) * sizeof(double));
        double* af = (double*)malloc((size_t)mc * sizeof(double));
        double* bf = (double*)malloc((size_t)nc * sizeof(double));
        out->fast_words = mc * nc + mc + nc;
        for (i64 jb = 0; jb < n; jb += nc) {
            i64 nb = imin(nc, n - jb);
            for (i64 ib = 0; ib < m; ib += mc) {
                i64 mb = imin(mc, m - ib);
                for (i64 j = 0; j < nb; ++j)
                    for (i64 i = 0; i < mb; ++i)
                        Cf[i + j * mb] = c_read ? C[(ib + i) + (jb + j) * ldc] : 0.0;
                if (c_read) out->c_reads += mb * nb;
                for (i64 p = 0; p < k; ++p) {
                    for (i64 i = 0; i < mb; ++i) af[i] = A[(ib + i) + p * lda];
                    for (i64 j = 0; j < nb; ++j) bf[j] = B[p + (jb + j) * ldb];
                    out->a_reads += mb;
                    out->b_reads += nb;
                    for (i64 j = 0; j < nb; ++j)
                        for (i64 i = 0; i < mb; ++i)
                            Cf[i + j * mb] = Cf[i + j * mb] + af[i] * bf[j];
                    out->flops += 2 * mb * nb;
                }
                for (i64 j = 0; j < nb; ++j)
                    for (i64 i = 0; i < mb; ++i) C[(ib + i) + (jb + j) * ldc] = Cf[i + j * mb];
                out->c_writes += mb * nb;
            }
        }
        free(Cf); free(af); free(bf);
        return 0;
    }
    if (member == 1) {
        const i64 mc = b1, kc = b2;
        double* Af = (double*)malloc((size_t)(mc * kc) * sizeof(double));
        double* cf = (double*)malloc((size_t)mc * sizeof(double));
        double* bf = (double*)malloc((size_t)kc * sizeof(double));
        out->fast_words = mc * kc + mc + kc;
        for (i64 pb = 0; pb < k; pb += kc) {
            i64 kb = imin(kc, k - pb);
            for (i64 ib = 0; ib < m; ib += mc) {
                i64 mb = imin(mc, m - ib);
                for (i64 p = 0; p < kb; ++p)
                    for (i64 i = 0; i < mb; ++i) Af[i + p * mb] = A[(ib + i) + (pb + p) * lda];
                out->a_reads += mb * kb;
                for (i64 j = 0; j < n; ++j) {
                    int first = (pb == 0);
                    for (i64 i = 0; i < mb; ++i)
                        cf[i] = (first && !c_read) ? 0.0 : C[(ib + i) + j * ldc];
                    if (!(first && !c_read)) out->c_reads += mb;
                    for (i64 p = 0; p < kb; ++p) bf[p] = B[(pb + p) + j * ldb];
                    out->b_reads += kb;
                    for (i64 p = 0; p < kb; ++p)
                        for (i64 i = 0; i < mb; ++i) cf[i] = cf[i] + Af[i + p * mb] * bf[p];
                    out->flops += 2 * mb * kb;
                    for (i64 i = 0; i < mb; ++i) C[(ib + i) + j * ldc] = cf[i];
                    out->c_writes += mb;
                }
            }
        }
        free(Af); free(cf); free(bf);
        return 0;
    }
    if (member == 2) {
        const i64 kc = b1, nc = b2;
        double* Bf = (double*)malloc((size_t)(kc * nc) * sizeof(double));
        double* cf = (double*)malloc((size_t)nc * sizeof(double));
        double* af = (double*)malloc((size_t)kc * sizeof(double));
        out->fast_words = kc * nc + nc + kc;
        for (i64 pb = 0; pb < k; pb += kc) {
            i64 kb = imin(kc, k - pb);
            for (i64 jb = 0; jb < n; jb += nc) {
                i64 nb = imin(nc, n - jb);
                for (i64 j = 0; j < nb; ++j)
                    for (i64 p = 0; p < kb; ++p) Bf[p + j * kb] = B[(pb + p) + (jb + j) * ldb];
                out->b_reads += kb * nb;
                for (i64 i = 0; i < m; ++i) {
                    int first = (pb == 0);
                    for (i64 j = 0; j < nb; ++j)
                        cf[j] = (first && !c_read) ? 0.0 : C[i + (jb + j) * ldc];
                    if (!(first && !c_read)) out->c_reads += nb;
                    for (i64 p = 0; p < kb; ++p) af[p] = A[i + (pb + p) * lda];
                    out->a_reads += kb;
                    for (i64 j = 0; j < nb; ++j)
                        for (i64 p = 0; p < kb; ++p) cf[j] = cf[j] + af[p] * Bf[p + j * kb];
                    out->flops += 2 * nb * kb;
                    for (i64 j = 0; j < nb; ++j) C[i + (jb + j) * ldc] = cf[j];
                    out->c_writes += nb;
                }
            }
        }
        free(Bf); free(cf); free(af);
        return 0;
    }
    if (member == 3) {
        const i64 nc = b1, kc = b2, mc = b3 > 0 ? b3 : 1;
        double* Bp = (double*)malloc((size_t)(kc * nc) * sizeof(double));
        double* Af = (double*)malloc((size_t)(mc * kc) * sizeof(double));
        double* cf = (double*)malloc((size_t)mc * sizeof(double));
        out->fast_words = kc * nc + mc * kc + mc;
        for (i64 jb = 0; jb < n; jb += nc) {
            i64 nb = imin(nc, n - jb);
            for (i64 pb = 0; pb < k; pb += kc) {
                i64 kb = imin(kc, k - pb);
                for (i64 j = 0; j < nb; ++j)
                    for (i64 p = 0; p < kb; ++p) Bp[p + j * kb] = B[(pb + p) + (jb + j) * ldb];
                out->b_reads += kb * nb;
                for (i64 ib = 0; ib < m; ib += mc) {
                    i64 mb = imin(mc, m - ib);
                    for (i64 p = 0; p < kb; ++p)
                        for (i64 i = 0; i < mb; ++i) Af[i + p * mb] = A[(ib + i) + (pb + p) * lda];
                    out->a_reads += mb * kb;
                    for (i64 j = 0; j < nb; ++j) {
                        int first = (pb == 0);
                        for (i64 i = 0; i < mb; ++i)
                            cf[i] = (first && !c_read) ? 0.0 : C[(ib + i) + (jb + j) * ldc];
                        if (!(first && !c_read)) out->c_reads += mb;
                        for (i64 p = 0; p < kb; ++p)
                            for (i64 i = 0; i < mb; ++i) cf[i] = cf[i] + Af[i + p * mb] * Bp[p + j * kb];
                        out->flops += 2 * mb * kb;
                        for (i64 i = 0; i < mb; ++i) C[(ib + i) + (jb + j) * ldc] = cf[i];
                        out->c_writes += mb;
                    }
                }
            }
        }
        free(Bp); free(Af); free(cf);
        return 0;
    }
    return -1;
}
