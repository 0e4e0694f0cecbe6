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

}  // namespace momms
