/* Drives every entry point of the oracle's C code on small shapes (empty, single element,
 * ragged, padded leading dimensions, both transposes, non-finite values) with buffers of the
 * exact size each call may touch, so that an AddressSanitizer / UndefinedBehaviorSanitizer
 * build reports any out-of-bounds access, overflow or invalid shift.  Test infrastructure:
 * built and run by tests/test_sanitize_cpu.py. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;
typedef struct {
    i64 a_reads, b_reads, c_reads, c_writes, flops, fast_words;
} io_counts;

int oracle_dgemm(int, int, i64, i64, i64, double, const double*, i64, const double*, i64, double, double*, i64, int);
int oracle_dgemm_abs(int, int, i64, i64, i64, const double*, i64, const double*, i64, double*, i64, int);
int oracle_exponents(int, int, i64, i64, const double*, i64, int32_t*, uint8_t*);
int oracle_split(int, int, i64, i64, const double*, i64, const int32_t*, const uint8_t*, int, int, int16_t*);
int oracle_slice_products(i64, i64, i64, int, const int16_t*, const int16_t*, int64_t*, int);
int oracle_recombine(i64, i64, int, int, const int64_t*, const int32_t*, const uint8_t*, const int32_t*,
                     const uint8_t*, double, double, double*, i64);
int oracle_count_member(int, i64, i64, i64, i64, i64, i64, int, const double*, i64, const double*, i64, double*,
                        i64, io_counts*);

static uint64_t state = 0x9E3779B97F4A7C15ull;
static double next_uniform(void) {
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(state >> 11) * 0x1.0p-53 * 2.0 - 1.0;
}

/* a rows x cols column-major matrix with leading dimension ld: exactly ld * (cols - 1) + rows
 * elements (none for an empty matrix) */
static double* matrix(i64 rows, i64 cols, i64 ld) {
    const i64 count = (rows > 0 && cols > 0) ? ld * (cols - 1) + rows : 0;
    double* x = malloc((size_t)(count > 0 ? count : 1) * sizeof(double));
    for (i64 i = 0; i < count; ++i) x[i] = next_uniform();
    return x;
}

static int fails = 0;
#define CHECK(cond)                                                          \
    do {                                                                     \
        if (!(cond)) {                                                       \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            ++fails;                                                         \
        }                                                                    \
    } while (0)

static void one_shape(i64 m, i64 n, i64 k, int ta, int tb, i64 pad, int nonfinite) {
    const i64 ar = ta ? k : m, ac = ta ? m : k, br = tb ? n : k, bc = tb ? k : n;
    const i64 lda = (ar > 0 ? ar : 1) + pad, ldb = (br > 0 ? br : 1) + pad, ldc = (m > 0 ? m : 1) + pad;
    double* A = matrix(ar, ac, lda);
    double* B = matrix(br, bc, ldb);
    double* C = matrix(m, n, ldc);
    double* N = matrix(m, n, ldc);
    if (nonfinite && ar > 0 && ac > 0) A[0] = NAN;
    if (nonfinite && br > 0 && bc > 0) B[ldb * (bc - 1)] = INFINITY;
    CHECK(oracle_dgemm(ta, tb, m, n, k, 0.5, A, lda, B, ldb, -1.0, C, ldc, 2) == 0);
    CHECK(oracle_dgemm(ta, tb, m, n, k, 1.0, A, lda, B, ldb, 0.0, C, ldc, 1) == 0);
    CHECK(oracle_dgemm_abs(ta, tb, m, n, k, A, lda, B, ldb, N, ldc, 2) == 0);

    /* emulated steps: exponents, digits (S = 3 of 7 bits), slice products, recombination */
    const int S = 3, beta = 7;
    const i64 mm = m > 0 ? m : 1, nn = n > 0 ? n : 1, kk = k > 0 ? k : 1;
    int32_t* e = malloc(sizeof(int32_t) * (size_t)mm);
    int32_t* f = malloc(sizeof(int32_t) * (size_t)nn);
    uint8_t* ef = malloc((size_t)mm);
    uint8_t* ff = malloc((size_t)nn);
    CHECK(oracle_exponents(0, ta, m, k, A, lda, e, ef) == 0);
    CHECK(oracle_exponents(1, tb, n, k, B, ldb, f, ff) == 0);
    int16_t* Ad = malloc(sizeof(int16_t) * (size_t)(S * mm * kk));
    int16_t* Bd = malloc(sizeof(int16_t) * (size_t)(S * nn * kk));
    CHECK(oracle_split(0, ta, m, k, A, lda, e, ef, S, beta, Ad) == 0);
    CHECK(oracle_split(1, tb, n, k, B, ldb, f, ff, S, beta, Bd) == 0);
    int64_t* P = malloc(sizeof(int64_t) * (size_t)(S * mm * nn));
    CHECK(oracle_slice_products(m, n, k, S, Ad, Bd, P, 2) == 0);
    CHECK(oracle_recombine(m, n, S, beta, P, e, ef, f, ff, 1.0, 1.0, C, ldc) == 0);
    CHECK(oracle_recombine(m, n, S, beta, P, e, ef, f, ff, 2.0, 0.0, C, ldc) == 0);
    free(e); free(f); free(ef); free(ff); free(Ad); free(Bd); free(P);
    free(A); free(B); free(C); free(N);
}

static void one_count(int member, i64 m, i64 n, i64 k, i64 b1, i64 b2, i64 b3) {
    double* A = matrix(m, k, m);
    double* B = matrix(k, n, k);
    double* C = matrix(m, n, m);
    io_counts io;
    CHECK(oracle_count_member(member, m, n, k, b1, b2, b3, 1, A, m, B, k, C, m, &io) == 0);
    CHECK(io.flops == 2 * m * n * k);
    free(A); free(B); free(C);
}

int main(void) {
    const i64 shapes[][3] = {{1, 1, 1}, {3, 5, 7}, {17, 9, 33}, {0, 4, 4}, {4, 0, 4}, {4, 4, 0}, {2, 64, 3}};
    for (size_t s = 0; s < sizeof(shapes) / sizeof(shapes[0]); ++s)
        for (int ta = 0; ta < 2; ++ta)
            for (int tb = 0; tb < 2; ++tb)
                for (i64 pad = 0; pad < 2; ++pad)
                    one_shape(shapes[s][0], shapes[s][1], shapes[s][2], ta, tb, 3 * pad, (int)(s & 1));
    for (int member = 0; member < 4; ++member) {
        one_count(member, 13, 11, 9, 4, 3, 5);
        one_count(member, 8, 8, 8, 8, 8, 8);
    }
    if (fails) {
        fprintf(stderr, "%d checks failed\n", fails);
        return 1;
    }
    printf("oracle driver: all calls clean\n");
    return 0;
}
