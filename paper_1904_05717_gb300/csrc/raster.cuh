// raster.cuh -- the MOMMS family member as a tile visiting order.
//
// The paper composes a member from two loops per cache level and names it by the
// operand that stays resident at each level (Sec. 3.2, 3.3).  On the GPU the L2
// level is decided by which C tiles the ~one wave of concurrently running CTAs
// covers, i.e. by the order in which the persistent CTAs take tiles:
//   C2: grouped raster -- a wave covers a G-tile-row x (wave/G)-tile-column block
//       of C, so the A panels of G tile rows and the B panels of wave/G tile
//       columns are reused through L2 (Resident C at the L2 level).
//   A2: row-major -- the wave walks along n inside a band of tile rows, so that
//       band of A stays in L2 while B streams (Resident A).
//   B2: column-major -- mirror of A2 (Resident B).
//   A1: blocked -- each CTA owns a contiguous run of tiles along n in one tile
//       row (Goto-like: the L2 level is not designed for, Sec. 4.3).
#pragma once
#include <cstdint>

namespace momms {

enum : int { kMemberAuto = 0, kMemberC2 = 1, kMemberA2 = 2, kMemberB2 = 3, kMemberA1 = 4 };

// Division of 32-bit unsigned integers by a divisor d >= 1 fixed for a launch, as a multiply-high,
// two shifts and two adds instead of a division routine (the method of Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Sec. 4: the multiplier is
// 2^32 + m, one bit too wide for a register, so the quotient is t + (n - t) / 2 shifted, t being
// the high word of m n).  With l = ceil(log2 d): m = floor(2^32 (2^l - d) / d) + 1, and
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0) for every 32-bit n.
struct FastDiv {
    uint32_t d, m, s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d) {
    FastDiv f{};
    if (d == 0) d = 1;  // (never used with d = 0; keeps the quotient defined)
    int l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.d = d;
    f.m = static_cast<uint32_t>(((uint64_t(1) << 32) * ((uint64_t(1) << l) - d)) / d + 1);
    f.s1 = l < 1 ? static_cast<uint32_t>(l) : 1u;
    f.s2 = l > 1 ? static_cast<uint32_t>(l - 1) : 0u;
    return f;
}
__host__ __device__ inline uint32_t fdiv(uint32_t n, const FastDiv& f) {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(f.m, n);
#else
    const uint32_t t = static_cast<uint32_t>((static_cast<uint64_t>(f.m) * n) >> 32);
#endif
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// The launch-invariant divisors of a member's tile order (member_tile_fast).
struct TileDiv {
    FastDiv tn, tm;         // tiles_n, tiles_m
    FastDiv gsize;          // C2: G tiles_n
    FastDiv gm, gm_last;    // C2: G, and the tile rows of the last (partial) row group
    int G;
};
inline TileDiv make_tilediv(int group, int tiles_m, int tiles_n) {
    TileDiv t{};
    t.G = group < 1 ? 1 : group;
    t.tn = make_fastdiv(static_cast<uint32_t>(tiles_n));
    t.tm = make_fastdiv(static_cast<uint32_t>(tiles_m));
    t.gsize = make_fastdiv(static_cast<uint32_t>(t.G) * static_cast<uint32_t>(tiles_n));
    t.gm = make_fastdiv(static_cast<uint32_t>(t.G));
    const int rest = tiles_m % t.G;
    t.gm_last = make_fastdiv(static_cast<uint32_t>(rest == 0 ? t.G : rest));
    return t;
}

// Tile t (< tiles_m tiles_n < 2^31) of the A2, B2 and C2 orders as member_tile places it, with
// the divisions by invariant divisors.
__host__ __device__ inline void member_tile_fast(int member, const TileDiv& dv, uint32_t t, int tiles_m, int* tm,
                                                 int* tn) {
    if (member == kMemberA2) {
        const uint32_t q = fdiv(t, dv.tn);
        *tm = static_cast<int>(q);
        *tn = static_cast<int>(t - q * dv.tn.d);
    } else if (member == kMemberB2) {
        const uint32_t q = fdiv(t, dv.tm);
        *tn = static_cast<int>(q);
        *tm = static_cast<int>(t - q * dv.tm.d);
    } else {
        const uint32_t g = fdiv(t, dv.gsize);
        const uint32_t first_m = g * static_cast<uint32_t>(dv.G);
        const FastDiv& gm = static_cast<uint32_t>(tiles_m) - first_m < static_cast<uint32_t>(dv.G) ? dv.gm_last : dv.gm;
        const uint32_t r = t - g * dv.gsize.d;
        const uint32_t q = fdiv(r, gm);
        *tm = static_cast<int>(first_m + (r - q * gm.d));
        *tn = static_cast<int>(q);
    }
}

// Maps the i-th tile taken by CTA `cta` (of `ctas`) to tile coordinates.
// Returns false when the CTA has no i-th tile.
__host__ __device__ inline bool member_tile(int member, int group, int64_t cta, int64_t ctas,
                                            int64_t i, int tiles_m, int tiles_n, int* tm,
                                            int* tn) {
    const int64_t total = static_cast<int64_t>(tiles_m) * tiles_n;
    int64_t t;
    if (member == kMemberA1) {
        const int64_t per = (total + ctas - 1) / ctas;
        if (i >= per) return false;
        t = cta * per + i;
        if (t >= total) return false;
        *tm = static_cast<int>(t / tiles_n);
        *tn = static_cast<int>(t % tiles_n);
        return true;
    }
    t = cta + i * ctas;
    if (t >= total) return false;
    if (member == kMemberA2) {
        *tm = static_cast<int>(t / tiles_n);
        *tn = static_cast<int>(t % tiles_n);
    } else if (member == kMemberB2) {
        *tn = static_cast<int>(t / tiles_m);
        *tm = static_cast<int>(t % tiles_m);
    } else {  // C2, grouped raster with `group` tile rows per group
        const int G = group < 1 ? 1 : group;
        const int64_t gsize = static_cast<int64_t>(G) * tiles_n;
        const int64_t g = t / gsize;
        const int first_m = static_cast<int>(g * G);
        const int gm = (tiles_m - first_m) < G ? (tiles_m - first_m) : G;
        const int64_t r = t - g * gsize;
        *tm = first_m + static_cast<int>(r % gm);
        *tn = static_cast<int>(r / gm);
    }
    return true;
}

// Triangular products (the symmetric rank-k update): of an m x m C, only the tiles that meet
// the stored triangle are visited, tile row by tile row.  Tile rows are 128 high and tile
// columns bn wide, bn dividing 384, so that three tile rows span pc = 384 / bn tile columns.
// Lower: tile row r holds the columns [0, min(tiles_n, floor((128 r + 127) / bn) + 1)) (its
// last row reaches the column's first one); upper: [floor(128 r / bn), tiles_n) (its first row
// reaches the column's last one).

// sum_{r < R} floor((128 r + b) / bn): with r = 3q + j the term is q pc + floor((128 j + b) / bn).
__host__ __device__ inline int64_t tri_floor_sum(int64_t R, int b, int bn) {
    const int64_t pc = 384 / bn;
    const int64_t Q = R / 3, J = R - 3 * Q;
    const int64_t g0 = b / bn, g1 = (128 + b) / bn, g2 = (256 + b) / bn;
    int64_t s = 3 * pc * (Q * (Q - 1) / 2) + Q * (g0 + g1 + g2) + J * Q * pc;
    if (J > 0) s += g0;
    if (J > 1) s += g1;
    return s;
}

// Tiles of the triangle in tile rows [0, R).
__host__ __device__ inline int64_t tri_prefix(bool lower, int64_t R, int tiles_n, int bn) {
    if (!lower) return R * tiles_n - tri_floor_sum(R, 0, bn);
    // rows from rs on are full: floor((128 r + 127) / bn) >= tiles_n - 1
    const int64_t need = static_cast<int64_t>(tiles_n - 1) * bn - 127;
    const int64_t rs = need <= 0 ? 0 : (need + 127) / 128;
    if (R <= rs) return tri_floor_sum(R, 127, bn) + R;
    return tri_floor_sum(rs, 127, bn) + rs + (R - rs) * tiles_n;
}

// The t-th tile of the triangle (row by row); false when t is past the last one.
__host__ __device__ inline bool tri_tile(bool lower, int64_t t, int tiles_m, int tiles_n, int bn, int* tm,
                                         int* tn) {
    if (t < 0 || tiles_m <= 0 || t >= tri_prefix(lower, tiles_m, tiles_n, bn)) return false;
    int64_t lo = 0, hi = tiles_m;  // tri_prefix(lo) <= t < tri_prefix(hi)
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) / 2;
        if (tri_prefix(lower, mid, tiles_n, bn) <= t) lo = mid;
        else hi = mid;
    }
    const int64_t first = lower ? 0 : 128 * lo / bn;
    const int64_t c = first + (t - tri_prefix(lower, lo, tiles_n, bn));
    if (c < 0 || c >= tiles_n) return false;
    *tm = static_cast<int>(lo);
    *tn = static_cast<int>(c);
    return true;
}

}  // namespace momms
