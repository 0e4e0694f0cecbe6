// Host-side check of the product kernels' unit decoding helpers (raster.cuh): the multiply-high
// division by an invariant divisor against the `/` operator, the member orders' 32-bit form
// against member_tile, and the kept-A strips (floor(b T / C) .. floor((b + 1) T / C)) covering
// every (modulus, tile) once.  Exits non-zero on the first mismatch.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../paper_1904_05717_gb300/csrc/raster.cuh"

using namespace momms;

static uint32_t next_u32(uint64_t& s) {  // SplitMix64, high half
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return static_cast<uint32_t>((z ^ (z >> 31)) >> 32);
}

int main() {
    long bad = 0, checks = 0;
    uint64_t seed = 12345;
    // 1. n / d for every d up to 3000, some large d, and n at the edges and at random
    std::vector<uint32_t> ds;
    for (uint32_t d = 1; d <= 3000; ++d) ds.push_back(d);
    for (uint32_t d : {65535u, 65536u, 65537u, 1000003u, 2147483647u, 2147483648u, 4294967295u}) ds.push_back(d);
    for (uint32_t d : ds) {
        const FastDiv f = make_fastdiv(d);
        const uint32_t edge[] = {0u, 1u, d - 1u, d, d + 1u, 2u * d - 1u, 2u * d, 2147483647u, 2147483648u,
                                 4294967294u, 4294967295u};
        for (uint32_t n : edge) {
            ++checks;
            if (fdiv(n, f) != n / d && bad++ < 5) printf("fdiv %u / %u\n", n, d);
        }
        for (int i = 0; i < 300; ++i) {
            const uint32_t n = next_u32(seed);
            ++checks;
            if (fdiv(n, f) != n / d && bad++ < 5) printf("fdiv %u / %u\n", n, d);
        }
    }
    // 2. the A2, B2 and C2 orders in 32-bit form against member_tile (raster groups 1..9, ragged last group)
    for (int tm_ = 1; tm_ <= 33; tm_ += 2)
        for (int tn_ = 1; tn_ <= 40; tn_ += 3)
            for (int G = 1; G <= 9; ++G)
                for (int mem = kMemberC2; mem <= kMemberB2; ++mem) {
                    const TileDiv dv = make_tilediv(G, tm_, tn_);
                    for (int t = 0; t < tm_ * tn_; ++t) {
                        int a = -1, b = -1, c = -1, e = -1;
                        member_tile(mem, G, t % 152, 152, t / 152, tm_, tn_, &a, &b);
                        member_tile_fast(mem, dv, static_cast<uint32_t>(t), tm_, &c, &e);
                        ++checks;
                        if ((a != c || b != e) && bad++ < 5) printf("member %d G %d %dx%d t %d\n", mem, G, tm_, tn_, t);
                    }
                }
    // 3. kept-A strips: every (modulus, tile) exactly once, strips of floor(T / C) or that + 1 tiles
    for (int tiles_m : {1, 3, 7, 128, 130})
        for (int tiles_n : {1, 3, 86, 87})
            for (int N : {1, 5, 15, 16})
                for (int ctas : {1, 5, 152}) {
                    const uint32_t T = static_cast<uint32_t>(tiles_m * tiles_n);
                    if (T < static_cast<uint32_t>(ctas)) continue;
                    const FastDiv fc = make_fastdiv(ctas), f0 = make_fastdiv(T / ctas), f1 = make_fastdiv(T / ctas + 1);
                    const FastDiv ftn = make_fastdiv(tiles_n);
                    std::vector<int> seen(static_cast<size_t>(T) * N, 0);
                    for (uint32_t blk = 0; blk < static_cast<uint32_t>(ctas); ++blk) {
                        const uint32_t start = fdiv(blk * T, fc), len = fdiv((blk + 1) * T, fc) - start;
                        if (len != f0.d && len != f1.d) {
                            if (bad++ < 5) printf("strip length %u\n", len);
                            continue;
                        }
                        const FastDiv& fl = len == f0.d ? f0 : f1;
                        for (uint32_t it = 0;; ++it) {
                            const uint32_t l = fdiv(it, fl);
                            if (l >= static_cast<uint32_t>(N)) break;
                            const uint32_t t = start + (it - l * fl.d);
                            const uint32_t q = fdiv(t, ftn);
                            ++checks;
                            if ((t >= T || q >= static_cast<uint32_t>(tiles_m)) && bad++ < 5) printf("strip unit %u\n", t);
                            else seen[static_cast<size_t>(l) * T + t]++;
                        }
                    }
                    for (int v : seen)
                        if (v != 1 && bad++ < 5) printf("unit visited %d times\n", v);
                }
    printf("checks %ld mismatches %ld\n", checks, bad);
    return bad != 0;
}
