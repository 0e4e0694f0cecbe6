// emu_crt.cu -- the modular (Chinese remainder) encoding of the emulated FP64 product:
// the choice of moduli and the reconstruction of C from the residues of the product.
//
// The operands are truncated to `bits`-bit integers A^ = trunc(A 2^(bits - e)) (row exponent
// e), B^ likewise; their exact product is known modulo each of N pairwise coprime moduli
// p_l <= 255 (one tensor product of residues per modulus, emu_slice_gemm.cu), and as
// |A^ B^| <= k (2^bits - 1)^2 < P / 4 with P = prod p_l, the Chinese remainder theorem gives
// it exactly:  A^B^ = sum_l c_l w_l mod P, centred, with w_l = (P / p_l) ((P / p_l)^-1 mod p_l).
// Then C := alpha 2^(e_i + f_j - 2 bits) A^B^ + beta C, rounded once to FP64 (plus the
// scaling).  The error is the truncation of A and B to `bits` bits -- that of the slice
// encoding with bits / 7 slices without its dropped digit pairs.
#include "crt.cuh"
#include "internal.h"
#include "ptx.cuh"

namespace momms {

namespace {

// The moduli: walking down from 255, every number coprime to all those already taken
// (255 = 3 5 17, 254 = 2 127, 253 = 11 23, 247 = 13 19, 217 = 7 31, the rest prime); their
// centred residues, |r| <= 127, are exact fp16 digits.
constexpr uint32_t kModuli[kCrtMaxModuli] = {255, 254, 253, 251, 247, 241, 239, 233,
                                             229, 227, 223, 217, 211, 199, 197, 193};

uint32_t inverse_mod(uint32_t a, uint32_t p) {  // a^-1 mod p (gcd(a, p) = 1)
    long long t = 0, nt = 1, r = p, nr = a % p;
    while (nr != 0) {
        const long long q = r / nr;
        long long tmp = t - q * nt;
        t = nt;
        nt = tmp;
        tmp = r - q * nr;
        r = nr;
        nr = tmp;
    }
    if (t < 0) t += p;
    return static_cast<uint32_t>(t);
}


// Moduli whose residues one thread loads at once (kGroup of crt_columns): eight (measured: the
// rank-k 16384^2 x 256 call 0.8 ms faster than one at a time, 8192^3 0.1 ms), but one for a
// triangle (SYRK n = k = 8192: 0.2 ms slower with four or eight -- 80 registers against 60).
constexpr int kGroupPlan = 8;
constexpr int kGroup = 8;  // (the batched reconstruction)

// C from the residue bytes res[l][j][i] (m n per modulus).  Per element, with S = sum_l c_l w_l
// (so S = Z mod P, and S / P = q + Z / P with |Z / P| <= 1/4 by the choice of moduli):
//   q  = round(sum_l c_l F_l / 2^19), F_l = round(2^19 w_l / P): one 32-bit multiply-add per
//        modulus (sum < 16 * 255 * 2^19 < 2^32), error below 16 * 255 * 2^-20 = 2^-8, far inside
//        the 1/4 margin,
//   Z  = S - q P computed modulo 2^(32 L) (|Z| < P / 2 <= 2^(32 L - 1): the wrap-around is exact),
// so no 128-bit division, comparison or reduction is needed: L limb sums of wide multiply-adds,
// one borrow chain, then the rounding of |Z| into the double's fields.  Blocks stride over the
// columns, threads over the rows of a column; with V = 4 (m a multiple of 4) a thread takes four
// consecutive rows and loads one 32-bit word per modulus, and with CV (16-byte aligned pairs of
// C) reads and writes C as two double2.  L = 3 when P < 2^96, else 4.  The modulus loop keeps
// few registers live, so that many warps hide the load latency.
template <int V, bool CV, int L, int kGroup>
__device__ __forceinline__ void crt_columns(int64_t m, int64_t n, const uint8_t* __restrict__ res, const CrtRecon& r,
                                            int bits, const int32_t* __restrict__ e, const uint8_t* __restrict__ ef,
                                            const int32_t* __restrict__ f, const uint8_t* __restrict__ ff,
                                            double alpha, double beta, double* __restrict__ C, int64_t ldc, int tri) {
    const int64_t mn = m * n;
    const int64_t groups = m / V;
    const bool unit_alpha = alpha == 1.0, beta_zero = beta == 0.0;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        const int Ej = f[j] - 2 * bits;
        const bool fj = ff[j] != 0;
        // a triangle (m = n): rows i >= j (lower) or i <= j (upper) of column j; the groups of V
        // rows that hold the diagonal element are written element by element
        const int64_t g_lo = tri == 1 ? j / V : 0, g_hi = tri == 2 ? min(groups, j / V + 1) : groups;
        for (int64_t g = g_lo + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < g_hi;
             g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
            const int64_t i0 = g * V;
            unsigned long long s[V][L];
            uint32_t qs[V];
#pragma unroll
            for (int t = 0; t < V; ++t) {
                qs[t] = 0u;
#pragma unroll
                for (int q = 0; q < L; ++q) s[t][q] = 0;
            }
            const uint8_t* src = res + j * m + i0;
            // the moduli eight at a time: their loads in flight together (one load per modulus
            // in turn left every modulus a full memory latency)
            for (int l0 = 0; l0 < r.N; l0 += kGroup) {
                uint32_t word[kGroup][V > 4 ? 2 : 1];
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    const int l = l0 + q;
                    if constexpr (V == 8) {
                        uint2 w2 = make_uint2(0u, 0u);
                        if (l < r.N) w2 = __ldcs(reinterpret_cast<const uint2*>(src + l * mn));
                        word[q][0] = w2.x;
                        word[q][V > 4 ? 1 : 0] = w2.y;
                    } else if constexpr (V == 4) {
                        word[q][0] = l < r.N ? __ldcs(reinterpret_cast<const unsigned int*>(src + l * mn)) : 0u;
                    } else {
                        word[q][0] = l < r.N ? src[l * mn] : 0u;
                    }
                }
#pragma unroll
                for (int q = 0; q < kGroup; ++q) {
                    const int l = l0 + q;
                    if (l >= r.N) break;
                    const uint32_t fl = r.frac[l];
#pragma unroll
                    for (int t = 0; t < V; ++t)
                        crt_accumulate<L>(s[t], qs[t], (word[q][t >> 2] >> (8 * (t & 3))) & 0xFFu, r.w[l], fl);
                }
            }
            double y[V];
#pragma unroll
            for (int t = 0; t < V; ++t) {
                const int64_t i = i0 + t;
                y[t] = (fj || ef[i] != 0) ? qnan : crt_value<L>(s[t], qs[t], r.Pw, e[i] + Ej);
                if (!unit_alpha) y[t] *= alpha;
            }
            double* cp = C + i0 + j * ldc;
            if (tri != 0 && j >= i0 && j < i0 + V) {
#pragma unroll
                for (int t = 0; t < V; ++t)
                    if (tri == 1 ? i0 + t >= j : i0 + t <= j) cp[t] = beta_zero ? y[t] : fma(beta, cp[t], y[t]);
            } else if constexpr (CV) {
                double2* c2 = reinterpret_cast<double2*>(cp);
#pragma unroll
                for (int h2 = 0; h2 < V / 2; ++h2) {
                    double2 a;
                    if (beta_zero) {
                        a = make_double2(y[2 * h2], y[2 * h2 + 1]);
                    } else {
                        a = __ldcs(c2 + h2);
                        a.x = fma(beta, a.x, y[2 * h2]);
                        a.y = fma(beta, a.y, y[2 * h2 + 1]);
                    }
                    __stcs(c2 + h2, a);
                }
            } else {
#pragma unroll
                for (int t = 0; t < V; ++t) cp[t] = beta_zero ? y[t] : fma(beta, cp[t], y[t]);
            }
        }
    }
}

// Four blocks of 256 threads resident per SM (at most 64 registers a thread): the kernel is bound
// by the issue of its wide multiply-adds and by load latency, and two resident blocks (98
// registers) left it short of warps -- rank-k 16384^2 with 15 moduli 4.80 -> 4.05 ms, 8192^2 with
// 12 moduli 1.04 -> 0.79 ms, the same bits (a few bytes of spills cost less than the lost warps).
constexpr int kCrtMinBlocks = 4;

template <int V, bool CV, int L, int G>
__global__ void __launch_bounds__(256, kCrtMinBlocks) crt_kernel(int64_t m, int64_t n, const uint8_t* __restrict__ res,
                                                  const __grid_constant__ CrtRecon r,
                                                  const int32_t* __restrict__ e, const uint8_t* __restrict__ ef,
                                                  const int32_t* __restrict__ f, const uint8_t* __restrict__ ff,
                                                  double alpha, double beta, double* __restrict__ C, int64_t ldc,
                                                  int tri) {
    crt_columns<V, CV, L, G>(m, n, res, r, r.bits, e, ef, f, ff, alpha, beta, C, ldc, tri);
}

// The same with the moduli count and the operand width from the device plan (the constants of
// every count in `set`); returns at once when the plan chose digit slices.
template <int V, bool CV>
__global__ void __launch_bounds__(256, kCrtMinBlocks) crt_plan_kernel(int64_t m, int64_t n, const uint8_t* __restrict__ res,
                                                       const __grid_constant__ CrtReconSet set,
                                                       const EmuPlan* __restrict__ plan,
                                                       const int32_t* __restrict__ e, const uint8_t* __restrict__ ef,
                                                       const int32_t* __restrict__ f, const uint8_t* __restrict__ ff,
                                                       double alpha, double beta, double* __restrict__ C,
                                                       int64_t ldc) {
    const int N = plan->N;
    if (N < 1 || N > kCrtMaxModuli) return;
    const CrtRecon& r = set.by_n[N];
    if (r.Pw[3] == 0) crt_columns<V, CV, 3, kGroupPlan>(m, n, res, r, plan->bits, e, ef, f, ff, alpha, beta, C, ldc, 0);
    else crt_columns<V, CV, 4, kGroupPlan>(m, n, res, r, plan->bits, e, ef, f, ff, alpha, beta, C, ldc, 0);
}

// One column of one problem of a batch: the warp's lanes take its rows 32 apart, one element
// each (byte loads, 32 consecutive bytes per warp and modulus), the arithmetic of crt_kernel.
template <int L>
__device__ __forceinline__ void crt_batch_column(const CrtBatchProblem& pr, const CrtRecon& r, int64_t j, int lane) {
    const int64_t m = pr.m, mn = m * pr.n;
    const int Ej = pr.f[j] - 2 * pr.bits;
    const bool fj = pr.ff[j] != 0;
    const bool unit_alpha = pr.alpha == 1.0, beta_zero = pr.beta == 0.0;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = lane; i < m; i += 32) {
        unsigned long long s[L];
        uint32_t qs = 0u;
#pragma unroll
        for (int q = 0; q < L; ++q) s[q] = 0;
        const uint8_t* src = pr.res + j * m + i;
        for (int l0 = 0; l0 < r.N; l0 += kGroup) {  // kGroup loads in flight at a time, as in crt_columns
            uint32_t c[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) c[q] = l0 + q < r.N ? src[(l0 + q) * mn] : 0u;
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (l0 + q >= r.N) break;
                crt_accumulate<L>(s, qs, c[q], r.w[l0 + q], r.frac[l0 + q]);
            }
        }
        double y = (fj || pr.ef[i] != 0) ? qnan : crt_value<L>(s, qs, r.Pw, pr.e[i] + Ej);
        if (!unit_alpha) y *= pr.alpha;
        double* cp = pr.C + i + j * pr.ldc;
        *cp = beta_zero ? y : fma(pr.beta, *cp, y);
    }
}

__global__ void __launch_bounds__(256, kCrtMinBlocks) crt_batch_kernel(const CrtBatchProblem* __restrict__ probs,
                                                        const int2* __restrict__ items,
                                                        const __grid_constant__ CrtReconSet set) {
    const int2 it = items[blockIdx.x];
    const CrtBatchProblem& pr = probs[it.x];
    const int64_t j = static_cast<int64_t>(it.y) * 8 + (threadIdx.x >> 5);
    if (j >= pr.n || pr.N < 1 || pr.N > kCrtMaxModuli) return;
    const CrtRecon& r = set.by_n[pr.N];
    if (r.Pw[3] == 0) crt_batch_column<3>(pr, r, j, threadIdx.x & 31);
    else crt_batch_column<4>(pr, r, j, threadIdx.x & 31);
}

}  // namespace

cudaError_t launch_crt_reconstruct_batched(const CrtBatchProblem* probs, const int2* items, int n_items,
                                           const CrtReconSet& set, cudaStream_t stream) {
    if (n_items <= 0) return cudaSuccess;
    crt_batch_kernel<<<static_cast<unsigned>(n_items), 256, 0, stream>>>(probs, items, set);
    return cudaGetLastError();
}

cudaError_t launch_crt_reconstruct_plan(int64_t m, int64_t n, const uint8_t* res, const CrtReconSet& set,
                                        const EmuPlan* plan, const int32_t* e, const uint8_t* ef, const int32_t* f,
                                        const uint8_t* ff, double alpha, double beta, double* C, int64_t ldc,
                                        cudaStream_t stream) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const bool vec = m % 4 == 0 && reinterpret_cast<uintptr_t>(res) % 4 == 0;
    const bool cvec = vec && ldc % 2 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0;
    const int64_t groups = vec ? m / 4 : m;
    int64_t bx = (groups + 255) / 256;
    if (bx > 64) bx = 64;
    const int64_t want = static_cast<int64_t>(device_sm_count()) * 16;
    int64_t by = (want + bx - 1) / bx;
    if (by > n) by = n;
    if (by > 65535) by = 65535;
    const dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(by));
    if (cvec)
        crt_plan_kernel<4, true><<<grid, 256, 0, stream>>>(m, n, res, set, plan, e, ef, f, ff, alpha, beta, C, ldc);
    else if (vec)
        crt_plan_kernel<4, false><<<grid, 256, 0, stream>>>(m, n, res, set, plan, e, ef, f, ff, alpha, beta, C, ldc);
    else
        crt_plan_kernel<1, false><<<grid, 256, 0, stream>>>(m, n, res, set, plan, e, ef, f, ff, alpha, beta, C, ldc);
    return cudaGetLastError();
}

int64_t crt_max_k() { return kCrtMaxK; }

bool crt_plan(int bits, int64_t k, CrtConsts* c, CrtRecon* r) {
    if (bits < 1 || bits > 56 || k < 1 || k > crt_max_k()) return false;
    int lk = 0;
    while ((int64_t(1) << lk) < k) ++lk;
    if (2 * bits + lk + 2 > 126) return false;
    // P > 4 k (2^bits - 1)^2: twice the range the centred residue needs, so that |Z / P| <= 1/4
    // and the reconstruction's fixed-point quotient estimate has a margin of 1/4
    const u128 v = (static_cast<u128>(1) << bits) - 1;
    const u128 need = static_cast<u128>(4) * static_cast<u128>(k) * v * v;
    u128 P = 1;
    int N = 0;
    while (N < kCrtMaxModuli && P <= need) P *= kModuli[N++];
    if (P <= need) return false;
    crt_consts(N, bits, c, r);
    return true;
}

void crt_consts(int N, int bits, CrtConsts* c, CrtRecon* r) {
    *c = CrtConsts{};
    *r = CrtRecon{};
    if (N < 1 || N > kCrtMaxModuli) return;
    u128 P = 1;
    for (int l = 0; l < N; ++l) P *= kModuli[l];
    c->N = r->N = N;
    c->bits = r->bits = bits;
    const long double Pl = static_cast<long double>(static_cast<unsigned long long>(P >> 64)) * 18446744073709551616.0L +
                           static_cast<long double>(static_cast<unsigned long long>(P));
    for (int l = 0; l < N; ++l) {
        const uint32_t p = kModuli[l];
        c->p[l] = p;
        c->magic[l] = static_cast<uint32_t>((1ull << 32) / p + 1);
        c->c16[l] = static_cast<uint32_t>((1ull << 16) % p);
        c->c32[l] = static_cast<uint32_t>((1ull << 32) % p);
        for (int j = 0; j < 3; ++j) c->kf[l][j] = static_cast<float>((1ull << (14 * (j + 1))) % p);
        c->pf[l] = static_cast<float>(p);
        c->invf[l] = 1.0f / static_cast<float>(p);
        c->lof[l] = -static_cast<float>(p / 2);
        c->hif[l] = static_cast<float>((p - 1) / 2);
        const u128 Ml = P / p;
        const uint32_t inv = inverse_mod(static_cast<uint32_t>(Ml % p), p);
        const u128 w = Ml * inv;  // < P
        for (int q = 0; q < 4; ++q) r->w[l][q] = static_cast<uint32_t>(w >> (32 * q));
        const long double wl = static_cast<long double>(static_cast<unsigned long long>(w >> 64)) *
                                   18446744073709551616.0L +
                               static_cast<long double>(static_cast<unsigned long long>(w));
        r->frac[l] = static_cast<uint32_t>(wl / Pl * 524288.0L + 0.5L);  // round(2^19 w_l / P)
    }
    for (int q = 0; q < 4; ++q) r->Pw[q] = static_cast<uint32_t>(P >> (32 * q));
}

cudaError_t launch_crt_reconstruct(int64_t m, int64_t n, const uint8_t* res, const CrtRecon& r, const int32_t* e,
                                   const uint8_t* ef, const int32_t* f, const uint8_t* ff, double alpha,
                                   double beta, double* C, int64_t ldc, cudaStream_t stream, int tri) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (tri != 0 && (m != n || tri < 0 || tri > 2)) return cudaErrorInvalidValue;
    // four rows per thread: eight (96-104 registers, a quarter of the warps resident) measured
    // 300 against 186 us at 4096^2
    const bool vec = m % 4 == 0 && reinterpret_cast<uintptr_t>(res) % 4 == 0;
    const bool cvec = vec && ldc % 2 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0;
    const bool three = r.Pw[3] == 0;  // P < 2^96: |Z| < 2^95, arithmetic modulo 2^96
    const int64_t groups = vec ? m / 4 : m;
    int64_t bx = (groups + 255) / 256;
    if (bx > 64) bx = 64;
    const int64_t want = static_cast<int64_t>(device_sm_count()) * 16;  // resident blocks to fill the chip
    int64_t by = (want + bx - 1) / bx;
    if (by > n) by = n;
    if (by > 65535) by = 65535;
    const dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(by));
#define MOMMS_CRT_LAUNCH(V, CV, L)                                                                    \
    do {                                                                                              \
        if (tri) crt_kernel<V, CV, L, 1><<<grid, 256, 0, stream>>>(m, n, res, r, e, ef, f, ff, alpha, beta, C, ldc, tri); \
        else crt_kernel<V, CV, L, kGroupPlan><<<grid, 256, 0, stream>>>(m, n, res, r, e, ef, f, ff, alpha, beta, C, ldc, tri); \
    } while (0)
    if (cvec) {
        if (three) MOMMS_CRT_LAUNCH(4, true, 3);
        else MOMMS_CRT_LAUNCH(4, true, 4);
    } else if (vec) {
        if (three) MOMMS_CRT_LAUNCH(4, false, 3);
        else MOMMS_CRT_LAUNCH(4, false, 4);
    } else {
        MOMMS_CRT_LAUNCH(1, false, 4);
    }
#undef MOMMS_CRT_LAUNCH
    return cudaGetLastError();
}

}  // namespace momms
