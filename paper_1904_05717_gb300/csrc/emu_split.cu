// emu_split.cu -- scaling exponents and truncation digits of the emulated path.
//
// Both steps are HBM-bound streaming passes on the CUDA cores; neither needs a
// floating-point operation: the exponent and the digits come from integer
// operations on the IEEE-754 bit pattern.
//
// Scaling (per row of op(A), per column of op(B)):
//     e = floor(log2 max |x|) + 1   (the frexp exponent of max|x|; 0 for an
//                                    all-zero vector; Inf/NaN -> flag)
// Digits (truncation splitting): with |x| = m * 2^e2 (m the integer significand),
//     d_s = sign(x) * ( floor(m * 2^(e2 - e + beta*s)) mod 2^beta ),  s = 1..S,
// which is the s-th base-2^beta digit of |x| * 2^-e truncated toward zero, so
//     x * 2^-e = sum_s d_s 2^(-beta s) + (remainder < 2^(-beta S)).
// Digits are written as fp16 (exact: |d_s| <= 2^beta - 1 <= 1023), each slice a
// rows_pad x inner_pad matrix stored inner-contiguous (K-major), zero-padded --
// the layout the tcgen05 kernel stages with TMA.  This pass is the GPU form of
// the paper's "pack on first residency" (Sec. 5.3): the operand is reorganised
// once, into the layout the inner kernel streams.
#include <cuda_fp16.h>

#include <climits>

#include "internal.h"

namespace momms {
namespace split {

constexpr int kNoExp = INT_MIN;
// cudaMemsetAsync(..., 0x80, ...) pattern: below every finite exponent (-1074..1024)
constexpr int kSentinel = static_cast<int>(0x80808080u);

// frexp exponent of |x| from its bits; kNoExp for zero; *nonfinite set for Inf/NaN.
__device__ __forceinline__ int elem_exponent(double x, int* nonfinite) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7FFFFFFFFFFFFFFFull;
    const int ef = static_cast<int>(b >> 52);
    const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
    if (ef == 0x7FF) {
        *nonfinite = 1;
        return kNoExp;
    }
    if (ef == 0) {
        if (mant == 0) return kNoExp;
        return 64 - __clzll(static_cast<long long>(mant)) - 1074;  // subnormal
    }
    return ef - 1022;
}

// Rows contiguous in memory (X[r + q*ld]): one thread per row over a slice of q,
// combined with atomicMax into exps (pre-set to a sentinel).
__global__ void scale_rows_contig(const double* __restrict__ X, int64_t ld, int64_t rows,
                                  int64_t inner, int64_t qchunk, int32_t* exps, uint8_t* flags,
                                  float* l1) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int64_t q0 = static_cast<int64_t>(blockIdx.y) * qchunk;
    int64_t q1 = q0 + qchunk;
    if (q1 > inner) q1 = inner;
    int emax = kNoExp, nf = 0;
    float sum = 0.f;
    int64_t q = q0;
    for (; q + 4 <= q1; q += 4) {  // four independent loads in flight per thread
        double x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = X[r + (q + t) * ld];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = elem_exponent(x[t], &nf);
            emax = e > emax ? e : emax;
            if (e != kNoExp) sum += static_cast<float>(fabs(x[t]));
        }
    }
    for (; q < q1; ++q) {
        const double x = X[r + q * ld];
        const int e = elem_exponent(x, &nf);
        emax = e > emax ? e : emax;
        if (e != kNoExp) sum += static_cast<float>(fabs(x));
    }
    if (emax != kNoExp) atomicMax(&exps[r], emax);
    if (nf) flags[r] = 1;
    if (l1 && sum != 0.f) atomicAdd(&l1[r], sum);
}

__global__ void scale_finalize(int64_t rows, int32_t* exps, uint8_t* flags) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    if (flags[r] || exps[r] == kSentinel) exps[r] = 0;
}

// Inner dimension contiguous (X[q + r*ld]): one warp per row.
__global__ void scale_inner_contig(const double* __restrict__ X, int64_t ld, int64_t rows,
                                   int64_t inner, int32_t* exps, uint8_t* flags, float* l1) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    int emax = kNoExp, nf = 0;
    float sum = 0.f;
    const double* x = X + r * ld;
    int64_t q = lane;
    for (; q + 96 < inner; q += 128) {  // four independent loads in flight per lane
        double v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = x[q + 32 * t];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = elem_exponent(v[t], &nf);
            emax = e > emax ? e : emax;
            if (e != kNoExp) sum += static_cast<float>(fabs(v[t]));
        }
    }
    for (; q < inner; q += 32) {
        const int e = elem_exponent(x[q], &nf);
        emax = e > emax ? e : emax;
        if (e != kNoExp) sum += static_cast<float>(fabs(x[q]));
    }
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    nf = __reduce_or_sync(0xFFFFFFFFu, nf);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    if (lane == 0) {
        exps[r] = (nf || emax == kNoExp) ? 0 : emax;
        flags[r] = static_cast<uint8_t>(nf != 0);
        if (l1) l1[r] = sum;
    }
}

// spread = max over vectors r of log2(2^e_r * inner / l1_r)  (>= 0 up to rounding):
// how far the vector maximum sits above the mean magnitude, in bits; written as
// ceil(16 * spread) with atomicMax into *out (pre-set to 0).
__global__ void spread_kernel(int64_t rows, int64_t inner, const int32_t* __restrict__ exps,
                              const uint8_t* __restrict__ flags, const float* __restrict__ l1,
                              int* out) {
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int v = 0;
    if (r < rows && !flags[r] && l1[r] > 0.f) {
        const float mean_log2 = log2f(l1[r]) - log2f(static_cast<float>(inner));
        const float sp = static_cast<float>(exps[r]) - mean_log2;
        v = sp > 0.f ? static_cast<int>(ceilf(16.f * sp)) : 0;
    }
    v = __reduce_max_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(out, v);
}

// The device plan of one product (EmuPlanTable): the slice-count rule on the spreads, then the
// encoding.  Every quantity is formed by the same IEEE operations, in the same order, as the host
// form of the rule, so both give the same S and width for the same spreads.
__global__ void plan_kernel(const int* __restrict__ spreads, const __grid_constant__ EmuPlanTable t, EmuPlan* out) {
    if (threadIdx.x != 0) return;
    const double sa = spreads[0] / 16.0;
    const double sb = t.tri ? sa : spreads[1] / 16.0;
    const double bits = t.c0 + 1.25 * (sa + sb);
    int S = static_cast<int>(ceil(bits / 7.0));
    S = S < 3 ? 3 : (S > t.smax ? t.smax : S);
    const int cb = static_cast<int>(ceil(bits));
    int w = cb > 7 * S - 6 ? cb : 7 * S - 6;
    w = w < 7 * S ? w : 7 * S;
    const int N = w <= kPlanMaxBits ? t.ntab[w] : 0;
    const bool mod = N > 0 && N <= t.n_alloc && (t.scheme_moduli || N + 2 <= S * (S + 1) / 2);
    EmuPlan p;
    p.S = S;
    p.bits = mod ? w : 7 * S;
    p.N = mod ? N : 0;
    p.pad = 0;
    p.est = 0.1 * exp2(bits - static_cast<double>(p.bits));  // the rule keeps a 10x margin
    *out = p;
}

// The batched device plan (EmuBatchPlanArgs), one block: per problem (threads in parallel) the
// rule of plan_kernel on its spreads and, for its width w, the fewest moduli whose product exceeds
// 4 k (2^w - 1)^2 (exact 128-bit arithmetic, as the host's choice of moduli); moduli when the
// problem's rule takes them (SLICES: never; MODULI: whenever they cover the width; AUTO: when they
// save two or more products and their per-element passes are paid for, N (k + 650) <= 0.9
// S (S + 1) / 2 k, as the host rule); then the units of both launches are laid out problem by problem.
__global__ void batch_plan_kernel(const __grid_constant__ EmuBatchPlanArgs a) {
    using u128 = unsigned __int128;
    __shared__ int smax_s, nmax_s, bmax_s;
    if (threadIdx.x == 0) {
        smax_s = 0;
        nmax_s = 0;
        bmax_s = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.count; i += blockDim.x) {
        EmuBatchPrep& q = a.prep[i];
        const double sa = q.spread[0] / 16.0, sb = q.spread[1] / 16.0;
        const double bits = q.c0 + 1.25 * (sa + sb);
        int S = static_cast<int>(ceil(bits / 7.0));
        S = S < 3 ? 3 : (S > a.smax ? a.smax : S);
        const int cb = static_cast<int>(ceil(bits));
        int w = cb > 7 * S - 6 ? cb : 7 * S - 6;
        w = w < 7 * S ? w : 7 * S;
        int N = 0;
        const bool range = q.scheme != 1 && w <= 56 && static_cast<int64_t>(q.k_pad) <= kCrtMaxK;
        if (range) {
            const u128 v = (static_cast<u128>(1) << w) - 1;
            const u128 need = static_cast<u128>(4) * static_cast<u128>(q.k) * v * v;
            for (int c = 1; c <= kCrtMaxModuli && N == 0; ++c) {
                const u128 P = (static_cast<u128>(a.P[c][1]) << 64) | a.P[c][0];
                if (P > need) N = c;
            }
        }
        const int pairs = S * (S + 1) / 2;
        const double kk = static_cast<double>(q.k);
        bool mod = N > 0;
        if (mod && q.scheme == 0)  // AUTO
            mod = N + 2 <= pairs && N * (kk + 650.0) <= 0.9 * pairs * kk;
        q.enc = mod ? 1 : 0;
        q.S = mod ? N : S;
        q.bits = mod ? w : 7 * S;
        a.slices[i].S = S;
        a.slices[i].group_end = emu_group_ends(S, 7, q.k_pad);
        a.moduli[i].S = mod ? N : 0;
        a.crt[i].N = mod ? N : 0;
        a.crt[i].bits = w;
        if (mod) {
            atomicMax(&nmax_s, N);
            atomicMax(&bmax_s, w);
        } else {
            atomicMax(&smax_s, S);
        }
    }
    __syncthreads();
    // unit offsets of both launches, problem by problem: a block-wide exclusive scan per chunk of
    // blockDim.x problems (two running totals carried from chunk to chunk)
    __shared__ long long scan_s[1024], scan_m[1024];
    __shared__ long long carry_s, carry_m;
    if (threadIdx.x == 0) {
        carry_s = 0;
        carry_m = 0;
    }
    __syncthreads();
    for (int c0 = 0; c0 < a.count; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        long long us = 0, um = 0;
        if (i < a.count) {
            const EmuBatchPrep& q = a.prep[i];
            const long long tiles = static_cast<long long>((q.m + kEmuBM - 1) / kEmuBM) * a.slices[i].tiles_n;
            if (q.enc) um = tiles * q.S;
            else us = tiles;
        }
        scan_s[threadIdx.x] = us;
        scan_m[threadIdx.x] = um;
        __syncthreads();
        for (int off = 1; off < static_cast<int>(blockDim.x); off <<= 1) {  // inclusive Hillis-Steele scan
            const long long vs = threadIdx.x >= off ? scan_s[threadIdx.x - off] : 0;
            const long long vm = threadIdx.x >= off ? scan_m[threadIdx.x - off] : 0;
            __syncthreads();
            scan_s[threadIdx.x] += vs;
            scan_m[threadIdx.x] += vm;
            __syncthreads();
        }
        if (i < a.count) {
            a.slices[i].tile0 = carry_s + scan_s[threadIdx.x] - us;
            a.moduli[i].tile0 = carry_m + scan_m[threadIdx.x] - um;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_s += scan_s[blockDim.x - 1];
            carry_m += scan_m[blockDim.x - 1];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    a.totals[0] = carry_s;
    a.totals[1] = carry_m;
    EmuPlan sm;
    sm.S = smax_s;
    sm.N = nmax_s;
    sm.bits = bmax_s > 7 * smax_s ? bmax_s : 7 * smax_s;
    sm.pad = 0;
    sm.est = 0.0;
    *a.summary = sm;
}

// Decompose x into (integer significand, binary exponent e2, sign); zero / non-finite -> mag 0.
__device__ __forceinline__ void decompose(double x, unsigned long long* mag, int* e2, bool* neg) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    *neg = (b >> 63) != 0;
    const int ef = static_cast<int>((b >> 52) & 0x7FF);
    unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    if (ef == 0x7FF) {
        m = 0;
        *e2 = 0;
    } else if (ef == 0) {
        *e2 = -1074;
    } else {
        m |= 1ull << 52;
        *e2 = ef - 1075;
    }
    *mag = m;
}

// Magnitude of digit s: bits [rs, rs + beta) of the significand m = hi:lo, rs = (e - e2) - beta*s
// (negative rs: the digit's low bits lie below the significand and are zero).
__device__ __forceinline__ uint32_t digit_bits(uint32_t lo, uint32_t hi, int rs, uint32_t mask) {
    if (rs >= 32) return rs >= 64 ? 0u : (hi >> (rs - 32)) & mask;
    if (rs >= 0) return __funnelshift_r(lo, hi, rs) & mask;
    return rs > -32 ? (lo << (-rs)) & mask : 0u;
}

// Two digit magnitudes u0, u1 < 1024 with signs as an fp16 pair: 1024 + u is exact in fp16
// (bits 0x6400 | u), subtracting 1024 leaves u exactly, the sign bit is set afterwards.
__device__ __forceinline__ uint32_t digits_to_half2(uint32_t u0, uint32_t u1, uint32_t s0, uint32_t s1) {
    const uint32_t biased = (0x6400u | u0) | ((0x6400u | u1) << 16);
    const __half2 v = __hsub2(*reinterpret_cast<const __half2*>(&biased), __half2half2(__ushort_as_half(0x6400)));
    return *reinterpret_cast<const uint32_t*>(&v) ^ (s0 | (s1 << 16));
}

// Four consecutive digits of one slice packed for one 8-byte store.
__device__ __forceinline__ uint2 pack4(__half h0, __half h1, __half h2, __half h3) {
    uint2 v;
    v.x = static_cast<uint32_t>(__half_as_ushort(h0)) | (static_cast<uint32_t>(__half_as_ushort(h1)) << 16);
    v.y = static_cast<uint32_t>(__half_as_ushort(h2)) | (static_cast<uint32_t>(__half_as_ushort(h3)) << 16);
    return v;
}

// Digits of four consecutive elements (same row) into the S slices at element offset `off`.
// Per element: significand words, the exponent distance t = e - e2, and the fp16 sign bit.
__device__ __forceinline__ void digit_source(double x, bool valid, int e, uint32_t* lo, uint32_t* hi, int* t,
                                             uint32_t* sgn) {
    unsigned long long mag = 0;
    int e2 = 0;
    bool neg = false;
    if (valid) decompose(x, &mag, &e2, &neg);
    *lo = static_cast<uint32_t>(mag);
    *hi = static_cast<uint32_t>(mag >> 32);
    *t = mag ? e - e2 : 1 << 20;  // zero: every digit shift runs past the significand
    *sgn = neg ? 0x8000u : 0u;
}

// 7-bit digits (the width the library uses) with shifts known at compile time.  |x| 2^-e is
// formed once per element as a 128-bit fixed-point fraction F = fh:fl (bit 127 worth 2^-1):
// F = m 2^(128 + e2 - e), truncated below 2^-128, i.e. past the 18th digit.  |x| < 2^e keeps F
// below 2^128.  Digit s (1-based) is then bits [128 - 7s, 135 - 7s) of F: with s unrolled every
// shift is a constant, two or three instructions a digit.
constexpr int kFastBeta = 7, kFastMaxS = 16;

__device__ __forceinline__ void fraction128(double x, bool valid, int e, unsigned long long* fh,
                                            unsigned long long* fl, uint32_t* sgn) {
    unsigned long long m = 0;
    int e2 = 0;
    bool neg = false;
    if (valid) decompose(x, &m, &e2, &neg);
    const int sh = 128 + e2 - e;
    *sgn = neg ? 0x8000u : 0u;
    if (m == 0 || sh <= -64) {
        *fh = 0;
        *fl = 0;
    } else if (sh >= 64) {
        *fh = m << (sh - 64);
        *fl = 0;
    } else if (sh > 0) {
        *fh = m >> (64 - sh);
        *fl = m << sh;
    } else {
        *fh = 0;
        *fl = m >> (-sh);
    }
}

__device__ __forceinline__ uint32_t digit7(unsigned long long fh, unsigned long long fl, int s) {
    const int lo = 128 - kFastBeta * s;  // lowest bit of digit s
    if (lo >= 64) return static_cast<uint32_t>(fh >> (lo - 64)) & 0x7Fu;
    if (lo + kFastBeta <= 64) return static_cast<uint32_t>(fl >> lo) & 0x7Fu;
    return static_cast<uint32_t>((fl >> lo) | (fh << (64 - lo))) & 0x7Fu;
}

template <int N>
__device__ __forceinline__ void write_digits_fast(const double (&x)[N], bool valid_row, int e, int S,
                                                  __half* __restrict__ digits, int64_t plane, int64_t off,
                                                  int s_first) {
    unsigned long long fh[N], fl[N];
    uint32_t sg[N];
#pragma unroll
    for (int i = 0; i < N; ++i) fraction128(x[i], valid_row, e, &fh[i], &fl[i], &sg[i]);
#pragma unroll
    for (int s = 1; s <= kFastMaxS; ++s) {
        if (s > S) break;
        if (s <= s_first) continue;
        uint32_t w[N / 2];
#pragma unroll
        for (int i = 0; i < N; i += 2)
            w[i / 2] = digits_to_half2(digit7(fh[i], fl[i], s), digit7(fh[i + 1], fl[i + 1], s), sg[i], sg[i + 1]);
        if constexpr (N == 8)
            *reinterpret_cast<uint4*>(digits + (s - 1) * plane + off) = make_uint4(w[0], w[1], w[2], w[3]);
        else
            *reinterpret_cast<uint2*>(digits + (s - 1) * plane + off) = make_uint2(w[0], w[1]);
    }
}

// Writes the digits of slices s_first+1 .. S (1-based); the digit of slice s does not depend on S.
__device__ __forceinline__ void write_digits4(const double (&x)[4], bool valid_row, int e, int S, int beta,
                                              __half* __restrict__ digits, int64_t plane, int64_t off,
                                              int s_first = 0) {
    if (beta == kFastBeta && S <= kFastMaxS) {
        write_digits_fast<4>(x, valid_row, e, S, digits, plane, off, s_first);
        return;
    }
    uint32_t lo[4], hi[4], sg[4];
    int t[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) digit_source(x[i], valid_row, e, &lo[i], &hi[i], &t[i], &sg[i]);
    const uint32_t mask = (1u << beta) - 1u;
    for (int s = s_first + 1; s <= S; ++s) {
        uint32_t u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) u[i] = digit_bits(lo[i], hi[i], t[i] - beta * s, mask);
        uint2 v;
        v.x = digits_to_half2(u[0], u[1], sg[0], sg[1]);
        v.y = digits_to_half2(u[2], u[3], sg[2], sg[3]);
        *reinterpret_cast<uint2*>(digits + (s - 1) * plane + off) = v;
    }
}

// Eight consecutive digits of each slice s_first+1 .. S with one 16-byte store per slice.
__device__ __forceinline__ void write_digits8(const double (&x)[8], bool valid_row, int e, int S, int beta,
                                              __half* __restrict__ digits, int64_t plane, int64_t off,
                                              int s_first) {
    if (beta == kFastBeta && S <= kFastMaxS) {
        write_digits_fast<8>(x, valid_row, e, S, digits, plane, off, s_first);
        return;
    }
    uint32_t lo[8], hi[8], sg[8];
    int t[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) digit_source(x[i], valid_row, e, &lo[i], &hi[i], &t[i], &sg[i]);
    const uint32_t mask = (1u << beta) - 1u;
    for (int s = s_first + 1; s <= S; ++s) {
        uint32_t u[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) u[i] = digit_bits(lo[i], hi[i], t[i] - beta * s, mask);
        uint4 v;
        v.x = digits_to_half2(u[0], u[1], sg[0], sg[1]);
        v.y = digits_to_half2(u[2], u[3], sg[2], sg[3]);
        v.z = digits_to_half2(u[4], u[5], sg[4], sg[5]);
        v.w = digits_to_half2(u[6], u[7], sg[6], sg[7]);
        *reinterpret_cast<uint4*>(digits + (s - 1) * plane + off) = v;
    }
}

// Residues of the integer operand A^ = trunc(|x| 2^(bits - e)) sign(x) modulo each p_l, in the
// symmetric range [lo, hi] = [-floor(p/2), floor((p-1)/2)] (|r| <= 127: exact in fp16, products
// < 2^14 as for the digits).  A^ is the top `bits` bits of the 128-bit fraction (the first bits/7
// digits), cut into four 14-bit pieces a_j, signed, held as FP32 integers; per modulus, in exact
// FP32 arithmetic (the FP32 pipes issue twice the integer multiply-adds' rate):
//   t = a_0 + a_1 (2^14 mod p) + a_2 (2^28 mod p) + a_3 (2^42 mod p)   (|t| < 2^24: exact),
//   q = the integer nearest t (1/p)_FP32   (within 1/193 of t / p: one rounding of 1.5 2^23 + t/p),
//   r = t - q p   (exact; |r| < p/2 + 2, r = A^ mod p), one step of p into [lo, hi],
// and the fp16 code of 1536 + r is the low half of the FP32 bits of (1.5 2^23 + 0x6600) + r.
template <int NE>
__device__ __forceinline__ void write_residues(const double (&x)[NE], bool valid_row, int e, const CrtConsts& c,
                                               __half* __restrict__ planes, int64_t plane, int64_t off,
                                               int N, int bits) {
    float a[NE][4];
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        unsigned long long fh, fl;
        uint32_t sg;
        fraction128(x[i], valid_row, e, &fh, &fl, &sg);
        const unsigned long long A = fh >> (64 - bits);  // < 2^56
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            // 2^23 + piece is an FP32 integer with the piece in its low bits; subtracting 2^23 is exact
            const float v = __uint_as_float(0x4B000000u | static_cast<uint32_t>((A >> (14 * j)) & 0x3FFFu)) - 8388608.0f;
            a[i][j] = sg ? -v : v;
        }
    }
    for (int l = 0; l < N; ++l) {
        const float k1 = c.kf[l][0], k2 = c.kf[l][1], k3 = c.kf[l][2];
        const float pf = c.pf[l], inv = c.invf[l], lo = c.lof[l], hi = c.hif[l];
        uint32_t h[NE];
#pragma unroll
        for (int i = 0; i < NE; ++i) {
            const float t = fmaf(a[i][3], k3, fmaf(a[i][2], k2, fmaf(a[i][1], k1, a[i][0])));
            const float q = fmaf(t, inv, 12582912.0f) - 12582912.0f;
            float r = fmaf(-q, pf, t);
            r = r > hi ? r - pf : (r < lo ? r + pf : r);
            // fp16 bits of 1536 + r: in [1024, 2048) the fp16 integers are consecutive codes
            h[i] = __float_as_uint(r + 12609024.0f) & 0xFFFFu;
        }
        uint32_t w[NE / 2];
        const __half2 bias = __half2half2(__ushort_as_half(0x6600));  // 1536
#pragma unroll
        for (int i = 0; i < NE; i += 2) {
            const uint32_t b = h[i] | (h[i + 1] << 16);
            const __half2 v2 = __hsub2(*reinterpret_cast<const __half2*>(&b), bias);  // exact: v
            w[i / 2] = *reinterpret_cast<const uint32_t*>(&v2);
        }
        if constexpr (NE == 8)
            *reinterpret_cast<uint4*>(planes + l * plane + off) = make_uint4(w[0], w[1], w[2], w[3]);
        else
            *reinterpret_cast<uint2*>(planes + l * plane + off) = make_uint2(w[0], w[1]);
    }
}

// Inner dimension contiguous in memory: a thread takes eight consecutive q of one row.
template <bool RES>
__global__ void split_inner_contig(const double* __restrict__ X, int64_t ld, int64_t rows,
                                   int64_t inner, const int32_t* __restrict__ exps,
                                   const uint8_t* __restrict__ flags, int S, int beta,
                                   __half* __restrict__ digits, int64_t rows_pad, int64_t inner_pad,
                                   int s_first, const __grid_constant__ CrtConsts crt, const EmuPlan* plan) {
    int nres = crt.N, rbits = crt.bits;
    if (plan) {  // the device plan decides the encoding, S or (N, width)
        const int pn = plan->N;
        if (RES ? pn == 0 : pn != 0) return;
        if (RES) {
            nres = pn;
            rbits = plan->bits;
        } else {
            S = plan->S;
        }
    }
    const int64_t octs = inner_pad / 8;
    const int64_t total = rows_pad * octs;
    const int64_t plane = rows_pad * inner_pad;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t r = idx / octs;
        const int64_t q = (idx - r * octs) * 8;
        const bool valid = r < rows && !flags[r];
        double x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = (valid && q + t < inner) ? X[q + t + r * ld] : 0.0;
        if constexpr (RES)
            write_residues<8>(x, valid, valid ? exps[r] : 0, crt, digits, plane, r * inner_pad + q, nres, rbits);
        else
            write_digits8(x, valid, valid ? exps[r] : 0, S, beta, digits, plane, r * inner_pad + q, s_first);
    }
}

// Rows contiguous in memory: a 64 x 64 tile is transposed through shared memory so that
// reads are coalesced along r and digit writes along q (four q per thread, 8-byte stores).
// The tile is stored [q][r ^ swz(q)], swz(q) = (q / 4) mod 16: a warp that fills one q row
// (32 consecutive r) and a warp that reads four consecutive q of one r per thread (16
// threads along q) both touch every bank pair evenly, with no padding.
__device__ __forceinline__ int swz(int q) { return (q >> 2) & 15; }
constexpr int TT = 64;
template <bool RES>
__global__ void split_rows_contig(const double* __restrict__ X, int64_t ld, int64_t rows,
                                  int64_t inner, const int32_t* __restrict__ exps,
                                  const uint8_t* __restrict__ flags, int S, int beta,
                                  __half* __restrict__ digits, int64_t rows_pad, int64_t inner_pad,
                                  int s_first, const __grid_constant__ CrtConsts crt, const EmuPlan* plan) {
    __shared__ double tile[TT][TT];  // [q][r ^ swz(q)]
    int nres = crt.N, rbits = crt.bits;
    if (plan) {  // the device plan decides the encoding, S or (N, width)
        const int pn = plan->N;
        if (RES ? pn == 0 : pn != 0) return;
        if (RES) {
            nres = pn;
            rbits = plan->bits;
        } else {
            S = plan->S;
        }
    }
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * TT;
    const int64_t q0 = static_cast<int64_t>(blockIdx.y) * TT;
    const int tid = threadIdx.x;  // 256 threads
    for (int i = tid; i < TT * TT; i += 256) {
        const int rr = i % TT, qq = i / TT;
        const int64_t r = r0 + rr, q = q0 + qq;
        tile[qq][rr ^ swz(qq)] = (r < rows && q < inner) ? X[r + q * ld] : 0.0;
    }
    __syncthreads();
    const int64_t plane = rows_pad * inner_pad;
    const int qg = (tid & 15) * 4;  // four consecutive q
    for (int rr = tid >> 4; rr < TT; rr += 16) {
        const int64_t r = r0 + rr, q = q0 + qg;
        if (r >= rows_pad || q >= inner_pad) continue;
        const bool valid = r < rows && !flags[r];
        double x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = tile[qg + t][rr ^ swz(qg + t)];
        if constexpr (RES)
            write_residues<4>(x, valid, valid ? exps[r] : 0, crt, digits, plane, r * inner_pad + q, nres, rbits);
        else
            write_digits4(x, valid, valid ? exps[r] : 0, S, beta, digits, plane, r * inner_pad + q, s_first);
    }
}

// Logical matrix Y (rows x inner): Y(r, q) = X[r*sr + q*sq]; true when rows are the
// contiguous dimension (sr == 1).
inline bool rows_contiguous(int which, int op) {
    // which 0: rows of op(A) -- op N: A[r + q*ld] (rows contiguous); op T: A[q + r*ld]
    // which 1: columns of op(B) -- op N: B[q + r*ld] (inner contiguous); op T: B[r + q*ld]
    return (which == 0) ? (op == 0) : (op != 0);
}

// ---------------------------------------------------------------- batched passes
// Per-row statistics (exponent, flag, L1 norm) and the row's spread, folded into *spread.
__device__ __forceinline__ void finish_vector(int emax, int nf, float l1, int64_t inner, int32_t* e, uint8_t* ef,
                                              int32_t* spread, bool valid) {
    int v = 0;
    if (valid) {
        *e = (nf || emax == kNoExp) ? 0 : emax;
        *ef = static_cast<uint8_t>(nf != 0);
        if (!nf && emax != kNoExp && l1 > 0.f) {
            const float sp = static_cast<float>(emax) - (log2f(l1) - log2f(static_cast<float>(inner)));
            v = sp > 0.f ? static_cast<int>(ceilf(16.f * sp)) : 0;
        }
    }
    v = __reduce_max_sync(0xFFFFFFFFu, v);
    if (spread && (threadIdx.x & 31) == 0 && v > 0) atomicMax(spread, v);
}

// A (rows contiguous): a thread per row over all of k.
__global__ void batch_scale_a(const EmuBatchPrep* __restrict__ probs, const int2* __restrict__ items) {
    const int2 it = items[blockIdx.x];
    const EmuBatchPrep& pr = probs[it.x];
    const int64_t r = static_cast<int64_t>(it.y) * 256 + threadIdx.x;
    const bool valid = r < pr.m;
    int emax = kNoExp, nf = 0;
    float sum = 0.f;
    if (valid) {
        const double* x = pr.A + r;
        int64_t q = 0;
        for (; q + 4 <= pr.k; q += 4) {
            double v[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) v[t] = x[(q + t) * pr.lda];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int e = elem_exponent(v[t], &nf);
                emax = e > emax ? e : emax;
                if (e != kNoExp) sum += static_cast<float>(fabs(v[t]));
            }
        }
        for (; q < pr.k; ++q) {
            const double v = x[q * pr.lda];
            const int e = elem_exponent(v, &nf);
            emax = e > emax ? e : emax;
            if (e != kNoExp) sum += static_cast<float>(fabs(v));
        }
    }
    finish_vector(emax, nf, sum, pr.k, valid ? pr.e + r : nullptr, valid ? pr.ef + r : nullptr,
                  pr.spread ? pr.spread : nullptr, valid);
}

// B (columns contiguous): a warp per column.
__global__ void batch_scale_b(const EmuBatchPrep* __restrict__ probs, const int2* __restrict__ items) {
    const int2 it = items[blockIdx.x];
    const EmuBatchPrep& pr = probs[it.x];
    const int64_t j = static_cast<int64_t>(it.y) * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    const bool valid = j < pr.n;
    int emax = kNoExp, nf = 0;
    float sum = 0.f;
    if (valid) {
        const double* x = pr.B + j * pr.ldb;
        for (int64_t q = lane; q < pr.k; q += 32) {
            const int e = elem_exponent(x[q], &nf);
            emax = e > emax ? e : emax;
            if (e != kNoExp) sum += static_cast<float>(fabs(x[q]));
        }
    }
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    nf = __reduce_or_sync(0xFFFFFFFFu, nf);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    // one lane per column writes; the spread is reduced over the warp (one column) by finish_vector
    const bool writer = valid && lane == 0;
    finish_vector(emax, nf, sum, pr.k, writer ? pr.f + j : nullptr, writer ? pr.ff + j : nullptr,
                  pr.spread ? pr.spread + 1 : nullptr, writer);
}

// A: 64 (rows) x 64 (k) tile through shared memory, as split_rows_contig.  RES: residues of the
// problem's S moduli (of c) at its `bits` instead of digits.
template <bool RES>
__global__ void batch_split_a(const EmuBatchPrep* __restrict__ probs, const int2* __restrict__ items,
                              const __grid_constant__ CrtConsts c) {
    __shared__ double tile[TT][TT];  // [q][r ^ swz(q)]
    const int2 it = items[blockIdx.x];
    const EmuBatchPrep& pr = probs[it.x];
    if (pr.enc >= 0 && pr.enc != (RES ? 1 : 0)) return;  // the device plan put it on the other encoding
    const int64_t qtiles = pr.k_pad / TT;
    const int64_t r0 = (it.y / qtiles) * TT;
    const int64_t q0 = (it.y % qtiles) * TT;
    const int tid = threadIdx.x;
    for (int i = tid; i < TT * TT; i += 256) {
        const int rr = i % TT, qq = i / TT;
        const int64_t r = r0 + rr, q = q0 + qq;
        tile[qq][rr ^ swz(qq)] = (r < pr.m && q < pr.k) ? pr.A[r + q * pr.lda] : 0.0;
    }
    __syncthreads();
    const int64_t plane = static_cast<int64_t>(pr.m) * pr.k_pad;
    const int qg = (tid & 15) * 4;
    __half* dg = static_cast<__half*>(pr.Ad);
    for (int rr = tid >> 4; rr < TT; rr += 16) {
        const int64_t r = r0 + rr, q = q0 + qg;
        if (r >= pr.m) continue;
        const bool valid = !pr.ef[r];
        double x[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) x[t] = tile[qg + t][rr ^ swz(qg + t)];
        if constexpr (RES)
            write_residues<4>(x, valid, valid ? pr.e[r] : 0, c, dg, plane, r * pr.k_pad + q, pr.S, pr.bits);
        else
            write_digits4(x, valid, valid ? pr.e[r] : 0, pr.S, pr.beta, dg, plane, r * pr.k_pad + q);
    }
}

// B: a thread per four consecutive k of one column, as split_inner_contig.
template <bool RES>
__global__ void batch_split_b(const EmuBatchPrep* __restrict__ probs, const int2* __restrict__ items,
                              const __grid_constant__ CrtConsts c) {
    const int2 it = items[blockIdx.x];
    const EmuBatchPrep& pr = probs[it.x];
    if (pr.enc >= 0 && pr.enc != (RES ? 1 : 0)) return;  // the device plan put it on the other encoding
    const int64_t quads = pr.k_pad / 4;
    const int64_t idx = static_cast<int64_t>(it.y) * 256 + threadIdx.x;
    if (idx >= static_cast<int64_t>(pr.n) * quads) return;
    const int64_t j = idx / quads;
    const int64_t q = (idx - j * quads) * 4;
    const bool valid = !pr.ff[j];
    double x[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) x[t] = (valid && q + t < pr.k) ? pr.B[q + t + j * pr.ldb] : 0.0;
    const int64_t plane = static_cast<int64_t>(pr.n) * pr.k_pad;
    if constexpr (RES)
        write_residues<4>(x, valid, valid ? pr.f[j] : 0, c, static_cast<__half*>(pr.Bd), plane, j * pr.k_pad + q,
                          pr.S, pr.bits);
    else
        write_digits4(x, valid, valid ? pr.f[j] : 0, pr.S, pr.beta, static_cast<__half*>(pr.Bd), plane,
                      j * pr.k_pad + q);
}

}  // namespace split

cudaError_t launch_emu_batch_scale(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                   int n_b, cudaStream_t stream) {
    if (n_a > 0) split::batch_scale_a<<<static_cast<unsigned>(n_a), 256, 0, stream>>>(probs, items_a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_b > 0) split::batch_scale_b<<<static_cast<unsigned>(n_b), 256, 0, stream>>>(probs, items_b);
    return cudaGetLastError();
}

cudaError_t launch_emu_batch_split(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                   int n_b, cudaStream_t stream) {
    const CrtConsts none{};
    if (n_a > 0) split::batch_split_a<false><<<static_cast<unsigned>(n_a), 256, 0, stream>>>(probs, items_a, none);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_b > 0) split::batch_split_b<false><<<static_cast<unsigned>(n_b), 256, 0, stream>>>(probs, items_b, none);
    return cudaGetLastError();
}

cudaError_t launch_emu_batch_residues(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                      int n_b, const CrtConsts& c, cudaStream_t stream) {
    if (n_a > 0) split::batch_split_a<true><<<static_cast<unsigned>(n_a), 256, 0, stream>>>(probs, items_a, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (n_b > 0) split::batch_split_b<true><<<static_cast<unsigned>(n_b), 256, 0, stream>>>(probs, items_b, c);
    return cudaGetLastError();
}

cudaError_t launch_emu_scale(int which, int op, int64_t rows, int64_t inner, const double* X,
                             int64_t ldx, int32_t* exps, uint8_t* flags, float* l1,
                             cudaStream_t stream) {
    using namespace split;
    if (rows <= 0) return cudaSuccess;
    if (split::rows_contiguous(which, op)) {
        cudaError_t e = cudaMemsetAsync(exps, 0x80, static_cast<size_t>(rows) * sizeof(int32_t), stream);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(flags, 0, static_cast<size_t>(rows), stream);
        if (e != cudaSuccess) return e;
        if (l1) {
            e = cudaMemsetAsync(l1, 0, static_cast<size_t>(rows) * sizeof(float), stream);
            if (e != cudaSuccess) return e;
        }
        if (inner > 0) {
            const int64_t bx = (rows + 255) / 256;
            int64_t by = (2 * device_sm_count() * 4 + bx - 1) / bx;  // enough blocks to fill the GPU
            if (by < 1) by = 1;
            if (by > inner) by = inner;
            if (by > 65535) by = 65535;
            const int64_t qchunk = (inner + by - 1) / by;
            by = (inner + qchunk - 1) / qchunk;
            dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(by));
            scale_rows_contig<<<grid, 256, 0, stream>>>(X, ldx, rows, inner, qchunk, exps, flags, l1);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        scale_finalize<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, stream>>>(rows, exps, flags);
        return cudaGetLastError();
    }
    const int64_t blocks = (rows + 7) / 8;
    scale_inner_contig<<<static_cast<unsigned>(blocks), 256, 0, stream>>>(X, ldx, rows, inner, exps, flags, l1);
    return cudaGetLastError();
}

cudaError_t launch_emu_batch_plan(const EmuBatchPlanArgs& a, cudaStream_t stream) {
    if (a.count <= 0) return cudaSuccess;
    split::batch_plan_kernel<<<1, 1024, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_emu_plan(const int* spreads, const EmuPlanTable& t, EmuPlan* out, cudaStream_t stream) {
    split::plan_kernel<<<1, 32, 0, stream>>>(spreads, t, out);
    return cudaGetLastError();
}

cudaError_t launch_emu_spread(int64_t rows, int64_t inner, const int32_t* exps, const uint8_t* flags,
                              const float* l1, int* out, cudaStream_t stream) {
    if (rows <= 0) return cudaSuccess;
    split::spread_kernel<<<static_cast<unsigned>((rows + 255) / 256), 256, 0, stream>>>(rows, inner, exps, flags, l1, out);
    return cudaGetLastError();
}

cudaError_t launch_emu_split(int which, int op, int64_t rows, int64_t inner, const double* X,
                             int64_t ldx, const int32_t* exps, const uint8_t* flags, int S, int beta,
                             void* digits, int64_t rows_pad, int64_t inner_pad, cudaStream_t stream,
                             int s_first, const EmuPlan* plan) {
    using namespace split;
    if (rows_pad <= 0 || inner_pad <= 0) return cudaSuccess;
    if (S < 1 || beta < 1 || beta > 10 || inner_pad % 8 || s_first < 0) return cudaErrorInvalidValue;
    if (s_first >= S) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(digits) % 16) return cudaErrorInvalidValue;
    __half* dg = static_cast<__half*>(digits);
    if (split::rows_contiguous(which, op)) {
        dim3 grid(static_cast<unsigned>((rows_pad + TT - 1) / TT), static_cast<unsigned>((inner_pad + TT - 1) / TT));
        if (grid.y > 65535) return cudaErrorInvalidValue;
        split_rows_contig<false><<<grid, 256, 0, stream>>>(X, ldx, rows, inner, exps, flags, S, beta, dg,
                                                           rows_pad, inner_pad, s_first, CrtConsts{}, plan);
        return cudaGetLastError();
    }
    const int64_t total = rows_pad * (inner_pad / 8);
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(device_sm_count()) * 32;
    if (blocks > cap) blocks = cap;
    split_inner_contig<false><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        X, ldx, rows, inner, exps, flags, S, beta, dg, rows_pad, inner_pad, s_first, CrtConsts{}, plan);
    return cudaGetLastError();
}

cudaError_t launch_emu_residues(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                                const int32_t* exps, const uint8_t* flags, const CrtConsts& c, void* planes,
                                int64_t rows_pad, int64_t inner_pad, cudaStream_t stream, const EmuPlan* plan) {
    using namespace split;
    if (rows_pad <= 0 || inner_pad <= 0) return cudaSuccess;
    if (c.N < 1 || c.N > kCrtMaxModuli || c.bits < 1 || c.bits > 56 || inner_pad % 8) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(planes) % 16) return cudaErrorInvalidValue;
    __half* dg = static_cast<__half*>(planes);
    if (split::rows_contiguous(which, op)) {
        dim3 grid(static_cast<unsigned>((rows_pad + TT - 1) / TT), static_cast<unsigned>((inner_pad + TT - 1) / TT));
        if (grid.y > 65535) return cudaErrorInvalidValue;
        split_rows_contig<true><<<grid, 256, 0, stream>>>(X, ldx, rows, inner, exps, flags, c.N, 7, dg, rows_pad,
                                                          inner_pad, 0, c, plan);
        return cudaGetLastError();
    }
    const int64_t total = rows_pad * (inner_pad / 8);
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = static_cast<int64_t>(device_sm_count()) * 32;
    if (blocks > cap) blocks = cap;
    split_inner_contig<true><<<static_cast<unsigned>(blocks), 256, 0, stream>>>(
        X, ldx, rows, inner, exps, flags, c.N, 7, dg, rows_pad, inner_pad, 0, c, plan);
    return cudaGetLastError();
}

}  // namespace momms
