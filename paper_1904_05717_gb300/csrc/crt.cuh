// crt.cuh -- the per-element arithmetic of the Chinese remainder reconstruction, shared by the
// reconstruction kernel (emu_crt.cu) and the residue product's fused epilogue
// (emu_slice_gemm.cu), so that both give the same bits.
//
// With the product's residues c_l (in [0, p_l)) and the CRT weights w_l (< P, 32-bit limbs):
//   S = sum_l c_l w_l   (so S = Z mod P, and S / P = q + Z / P with |Z / P| <= 1/4 by the
//                        choice of moduli, P > 4 k (2^b - 1)^2),
//   q = round(sum_l c_l F_l / 2^19), F_l = round(2^19 w_l / P)   (error below 2^-8),
//   Z = S - q P computed modulo 2^(32 L) (exact: |Z| < 2^(32 L - 1)),
// then |Z| 2^E rounded once to FP64 with the scale written into the exponent field.
#pragma once
#include <cstdint>

#include "ptx.cuh"

namespace momms {

using u128 = unsigned __int128;

// v rounded to nearest (ties to even) as a double: the leading 64 bits with the rest folded
// into a sticky bit (bit 0 lies below the rounding position of a 53-bit significand), one
// correctly rounded 64-bit conversion, then an exact power-of-two scaling.
MOMMS_DEV double u128_to_double(u128 v) {
    const unsigned long long hi = static_cast<unsigned long long>(v >> 64);
    if (hi == 0) return static_cast<double>(static_cast<unsigned long long>(v));
    const int lz = __clzll(static_cast<long long>(hi));
    const u128 t = v << lz;
    const unsigned long long top = static_cast<unsigned long long>(t >> 64) |
                                   static_cast<unsigned long long>(static_cast<unsigned long long>(t) != 0);
    return static_cast<double>(top) * pow2_normal(64 - lz);
}

// mag 2^(E) with the sign, mag = hi 2^64 + lo, rounded once to FP64 (to nearest, ties to even):
// the 53-bit significand is rounded in integers and the scale goes into the exponent field;
// an exponent outside the normal range takes the FP64 route.
MOMMS_DEV double scaled_double(unsigned long long hi, unsigned long long lo, bool neg, int E) {
    if ((hi | lo) == 0) return 0.0;
    // the leading 64 bits of mag in `top`, the bits below folded into its bit 0 (a sticky bit,
    // under the rounding position of a 53-bit significand)
    int lz;
    unsigned long long top;
    if (hi) {
        lz = __clzll(static_cast<long long>(hi));
        if (lz == 0) {
            top = hi | static_cast<unsigned long long>(lo != 0);
        } else {
            top = (hi << lz) | (lo >> (64 - lz));
            top |= static_cast<unsigned long long>((lo << lz) != 0);
        }
    } else {
        lz = 64 + __clzll(static_cast<long long>(lo));
        top = lo << (lz - 64);
    }
    unsigned long long mant = top >> 11;
    const unsigned long long rem = top & 0x7FFull;
    mant += (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ? 1ull : 0ull;
    int ex = 127 - lz + E;  // unbiased exponent of |y| = mant 2^(ex - 52)
    if (mant == (1ull << 53)) {
        mant >>= 1;
        ++ex;
    }
    if (ex >= -1022 && ex <= 1023)
        return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(neg) << 63) |
                                                           (static_cast<unsigned long long>(ex + 1023) << 52) |
                                                           (mant & ((1ull << 52) - 1))));
    const double y = scale_pow2(u128_to_double((static_cast<u128>(hi) << 64) | lo), E);
    return neg ? -y : y;
}

// One residue c of one element into its limb sums s (L limbs) and quotient sum qs.
template <int L>
MOMMS_DEV void crt_accumulate(unsigned long long (&s)[L], uint32_t& qs, uint32_t c, const uint32_t* w, uint32_t F) {
#pragma unroll
    for (int q = 0; q < L; ++q) s[q] += static_cast<unsigned long long>(c) * w[q];
    qs += c * F;
}

// The element's value Z 2^E rounded to FP64 from its limb sums (Pw: P in 32-bit limbs).
template <int L>
MOMMS_DEV double crt_value(const unsigned long long (&s)[L], uint32_t qs, const uint32_t* Pw, int E) {
    // S mod 2^(32 L) in 32-bit words z[0..L-1]
    uint32_t z[L];
    unsigned long long carry = 0;
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const unsigned long long v = s[q] + carry;
        z[q] = static_cast<uint32_t>(v);
        carry = v >> 32;
    }
    // Z = S - q P modulo 2^(32 L)
    const uint32_t qv = (qs + (1u << 18)) >> 19;
    unsigned long long mc = 0;
    uint32_t borrow = 0;
#pragma unroll
    for (int q = 0; q < L; ++q) {
        const unsigned long long pq = static_cast<unsigned long long>(qv) * Pw[q] + mc;
        mc = pq >> 32;
        const uint32_t sub = static_cast<uint32_t>(pq);
        const unsigned long long d = static_cast<unsigned long long>(z[q]) - sub - borrow;
        z[q] = static_cast<uint32_t>(d);
        borrow = static_cast<uint32_t>(d >> 63);
    }
    const bool neg = (z[L - 1] >> 31) != 0;
    if (neg) {  // two's complement magnitude
        uint32_t c1 = 1;
#pragma unroll
        for (int q = 0; q < L; ++q) {
            const unsigned long long v = static_cast<unsigned long long>(~z[q]) + c1;
            z[q] = static_cast<uint32_t>(v);
            c1 = static_cast<uint32_t>(v >> 32);
        }
    }
    // |Z| = hi 2^64 + lo, scaled by 2^(32 (4 - L)) when L = 3
    if constexpr (L == 4) {
        return scaled_double((static_cast<unsigned long long>(z[3]) << 32) | z[2],
                             (static_cast<unsigned long long>(z[1]) << 32) | z[0], neg, E);
    } else {
        return scaled_double((static_cast<unsigned long long>(z[2]) << 32) | z[1],
                             static_cast<unsigned long long>(z[0]) << 32, neg, E - 32);
    }
}

}  // namespace momms
