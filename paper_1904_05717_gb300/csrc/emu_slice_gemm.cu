// emu_slice_gemm.cu -- the slice products of the emulated FP64 product on the
// fifth-generation tensor cores, with the recombination fused into the epilogue.
//
// For a C tile (BM x BN = 128 x 192, or 128 x 96) the kernel computes, for every diagonal
// d = S+1 down to 2 of the triangular pair set,
//     P_d = sum_{s+t=d} A_s B_t          (A_s, B_t: integer digit slices in fp16)
// exactly, and combines the diagonals from the least significant one: consecutive
// diagonals exactly in int64, Q = sum_j P_{hi-j} 2^(beta j), for as many as the host proves
// stay below 2^63 (emu_group_ends); FP64 only where a group ends,
// R = 2^(-beta (hi-lo)) (Q + 2^-beta R_prev); and at d = 2
//     C := alpha * 2^(e_i + f_j - 2 beta) R + beta_c C.
//
// Exactness.  A tcgen05 kind::f16 MMA multiplies fp16 integers exactly and accumulates in
// FP32 in tensor memory (TMEM).  Every partial sum of at most `chunk` products of digits
// |d| <= 2^beta - 1 stays an integer below 2^24, so the FP32 accumulator is exact; after each
// chunk the accumulator is drained (tcgen05.ld -> exact float->int conversion -> int32 add).
// The int32 diagonal sums stay below 2^31 because one launch covers at most
// emu_max_k_per_pass(S, beta) of k.
//
// Memory levels (the paper's Sec. 3.3 vocabulary): the C tile is the resident block of
// TMEM/registers (Resident C at L0, Sec. 3.4); A and B digit tiles stream through a
// multi-stage shared-memory ring filled by TMA; which panels stay in L2 is set by the
// member's tile order (raster.cuh).
//
// Roles (512 threads, one CTA per SM): warp 0 = TMA producer (one thread), warp 1 = TMEM
// owner and MMA issuer (one thread), warps 4..15 = drain / recombination, three per TMEM
// lane quadrant, each thread one row and BN/3 columns.  TMEM holds two FP32 accumulators
// (columns 0 and 256) so that draining one overlaps MMAs into the other; the rest holds
// half of the int32 sums (wide tile) or the int64 group sums (narrow tile).  Every mbarrier
// wait is bounded; on expiry the kernel raises a CTA-wide abort flag, lets in-flight copies
// and MMAs finish, frees TMEM, and reports status 1002 (timeout) through p.status.
// A single-problem launch may be followed by a tail launch (the last, partial round of
// tiles cut along k) and a fix-up launch that adds the parts and recombines.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "crt.cuh"
#include "internal.h"
#include "ptx.cuh"
#include "raster.cuh"

namespace momms {
namespace emu {

constexpr int BM = kEmuBM, BK = kEmuBK;
constexpr int CTRL_WARPS = 4;   // warp 0: TMA producer, warp 1: TMEM owner + MMA issuer, 2-3 idle
constexpr int EPI_WARPS = 12;   // three warps per TMEM lane quadrant
constexpr int THREADS = 32 * (CTRL_WARPS + EPI_WARPS);  // 512: four warps per SM sub-partition
constexpr uint32_t A_TILE = BM * BK * 2;                 // 16 KB
constexpr uint32_t TMEM_COLS = 512;                      // two BN-column FP32 accumulators
constexpr size_t SMEM_BUDGET = 225 * 1024;

// Two tile widths.  BN = 192: a drain thread owns 64 columns, the int32 sums of 32 in registers
// and of 32 in spare TMEM, the int64 group sums Q in a global scratch block.  BN = 96 (small k
// or narrow n): 32 columns, all sums in registers, and Q in TMEM next to the accumulators --
// the recombination of a diagonal then makes no round trip to L2.
template <int BN>
struct Cfg {
    static_assert(BN == 192 || BN == 96, "three drain warps per TMEM lane quadrant");
    static constexpr int CW = BN / 3;                    // columns per drain warp (64 or 32)
    static constexpr int CR = 32;                        // of which summed in registers
    static constexpr int CT = CW - CR;                   // and summed as int32 in spare TMEM columns
    static constexpr bool QT = (BN == 96);               // int64 group sums in TMEM
    static constexpr uint32_t B_TILE = BN * BK * 2;
    static constexpr uint32_t STAGE = A_TILE + B_TILE;
    static constexpr int STAGES = static_cast<int>((SMEM_BUDGET - 2048) / STAGE) > 6
                                      ? 6 : static_cast<int>((SMEM_BUDGET - 2048) / STAGE);
    static constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE + 256 + 5 * BN;
    static constexpr uint32_t IDESC = idesc_f16_f32(BM, BN);
    static_assert(STAGE % 1024 == 0, "stage bases stay 1024-byte aligned for the 128-B swizzle");
};

// The residue product of short k with each CTA's A tile kept in shared memory (AK): units of
// one modulus walk along a tile row, so consecutive units of a CTA share their A tile; it is
// loaded once per (modulus, tile row) into a region of AK_SLABS slabs, and only B streams
// through the ring (24 KB stages instead of 40).
constexpr int AK_SLABS = 4;                               // k <= 256
constexpr uint32_t AK_REGION = AK_SLABS * A_TILE;         // 64 KB
constexpr uint32_t AK_STAGE = kEmuBNMax * BK * 2;         // 24 KB: one B slab
constexpr int AK_STAGES = 6;
constexpr size_t AK_SMEM_BYTES = 1024 + AK_REGION + static_cast<size_t>(AK_STAGES) * AK_STAGE + 256 + 5 * kEmuBNMax;
static_assert(AK_SMEM_BYTES <= SMEM_BUDGET + 1024, "kept-A residue product fits one CTA's shared memory");
static_assert(AK_STAGE % 1024 == 0 && AK_REGION % 1024 == 0, "1024-byte aligned slabs for the 128-B swizzle");

// The per-problem quantities every role needs for one tile.
struct Prob {
    int m, n;
    int S, beta;
    int chunk_slabs;
    int slab0, nslab;
    uint32_t group_end;       // bit d set: diagonal d closes an exact int64 group
    const int32_t* e;
    const uint8_t* ef;
    const int32_t* f;
    const uint8_t* ff;
    double alpha, beta_c;
    double* C;
    int64_t ldc;
};

struct Params {
    Prob one;                 // single problem (unused when table != nullptr)
    int tiles_m, tiles_n;
    int member, group;
    const EmuBatchProblem* table;  // batched: one entry per problem, ordered by tile0
    int count;
    int64_t total_tiles;
    const int64_t* total_dev;      // batched with a device plan: the total, written by the plan kernel
    double* scratch;          // FP64 partial recombination R, one BN x BM block per CTA
    long long* qscratch;      // int64 exact group sums Q, one BN x BM block per CTA
    int32_t* status;
    // Tail split (single problem, round-robin members): the main launch stops after its whole
    // rounds; the tiles of the last, partial round go to a second launch that cuts each along k
    // into tail_parts units, one per CTA, each storing its int32 diagonal sums; a third launch
    // adds the parts and recombines.
    int full_rounds;          // whole-tile rounds of the main launch
    int main_ctas;            // CTAs of the main launch (its round-robin order places the tail tiles)
    int tail_tiles;           // tiles in the tail round
    int tail_parts;           // k parts per tail tile (< 2: no split)
    int32_t* tail_sums;       // [tail tile][part][diagonal d-2][column / 4][row][4] int32 partial sums
    // Modular encoding (single problem): `one.S` moduli, the unit of modulus l multiplies residue
    // plane l of A by plane l of B and its epilogue stores (sum mod modp[l]) as a byte.
    uint8_t* res;             // [l][col][row] residues of the product, m n bytes per modulus
    int group_tiles;          // the unit order: groups of this many tiles, moduli in turn
    // Fused reconstruction: the epilogue of a tile's last modulus rebuilds C itself once done[tile]
    // shows the other moduli's residues stored (crt_fused; else a separate reconstruction launch).
    int crt_fused;
    // Triangular product (modular encoding, m = n): only the tri_tiles tiles that meet the lower
    // (tri = 1) or upper (tri = 2) triangle of C are units, taken row by row (tri_tile).
    int tri;
    int tri_bn;
    int64_t tri_tiles;
    // Triangular operand (modular encoding, single problem): the k slabs where op(A) or op(B) is
    // zero are skipped per unit.  1: op(A) lower (k < (tm + 1) BM), 2: op(A) upper (k >= tm BM),
    // 3: op(B) lower (k >= tn BN), 4: op(B) upper (k < (tn + 1) BN); 0: every slab.
    int kcap;
    // Test hook of the timeout path (momms_debug_withhold_load): CTA 0's producer announces its
    // first stage but issues no copy into it, so the MMA thread's bounded wait on that stage runs
    // out -- the abort, drain and status path runs without any fault.
    int withhold;
    // Device plan (single problem, AUTO slice count): plan_kind 1 = this is the modular launch (N
    // moduli from the plan, nothing to do when it chose slices), 2 = the digit launch (S from the
    // plan and its group ends from group_end_by_s, nothing to do when it chose moduli); 0 = none.
    const EmuPlan* plan;
    int plan_kind;
    uint32_t group_end_by_s[17];
    int crt_L;                // limbs of the reconstruction arithmetic (3: P < 2^96, else 4)
    int crt_bits;             // integer width of the operands
    int* done;                // per tile: moduli whose residues are stored
    uint32_t crt_w[kCrtMaxModuli][4];
    uint32_t crt_F[kCrtMaxModuli];
    uint32_t crt_Pw[4];
    uint32_t modp[kCrtMaxModuli];
    uint32_t modmagic[kCrtMaxModuli];  // floor(2^32 / p) + 1
    uint32_t modoff[kCrtMaxModuli];    // p ceil(2^31 / p): makes any int32 sum a uint32 of equal residue
    uint32_t modmagic_up[kCrtMaxModuli];  // ceil(2^32 / p): exact floor quotients of u < 2^24
    uint32_t modoff22[kCrtMaxModuli];     // p ceil(2^22 / p): makes a sum |x| < 2^22 a u < 2^24
    // 32-bit unit decoding (u32dec: every unit index of a single problem below 2^31): the
    // launch-invariant divisors of tile_of, as multiply-high divisions -- every warp role decodes
    // every unit, and 64-bit division routines cost those warps microseconds per small-k unit.
    int u32dec;
    // Kept-A order (akeep): CTA b takes the tiles [floor(b T / C), floor((b + 1) T / C)) of every
    // modulus in turn, row-major (T tiles, C CTAs); fd_ctas divides by C, fd_len and fd_len1 by the
    // two strip lengths floor(T / C) and floor(T / C) + 1.
    int akeep;
    FastDiv fd_ctas, fd_len, fd_len1;
    FastDiv fd_n[17];         // moduli counts 1..16 (the count may come from the device plan)
    FastDiv fd_gt, fd_gt_last;  // group_tiles, and the tiles of the last (partial) group
    TileDiv tdv;              // the member order's divisors
};

// S of the single problem (moduli for the modular launch): the launch's, or the device plan's (0
// when the plan chose the other encoding).
MOMMS_DEV int one_S(const Params& p) {
    if (p.plan_kind == 0) return p.one.S;
    const int N = p.plan->N;
    return p.plan_kind == 1 ? N : (N != 0 ? 0 : p.plan->S);
}

// The it-th tile of this CTA: its problem (-1 = the single problem of p.one) and tile
// coordinates.  A single problem uses the member's tile order; a batch walks the
// concatenated tile list of all problems cyclically.
template <bool TAIL, bool MOD = false>
MOMMS_DEV bool tile_of(const Params& p, int it, int* prob, int* tm, int* tn, int* part, int* lmod = nullptr,
                       int64_t* tile = nullptr) {
    *part = -1;
    if constexpr (MOD) {
        if (p.table != nullptr) {
            // a batch: the units of each problem (its tiles times its moduli) follow one another,
            // modulus-major inside the problem; tile0 is the problem's first unit
            const int64_t u = static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x;
            if (u >= (p.total_dev ? *p.total_dev : p.total_tiles)) return false;
            int lo = 0, hi = p.count - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (p.table[mid].tile0 <= u) lo = mid;
                else hi = mid - 1;
            }
            const EmuBatchProblem& b = p.table[lo];
            const int64_t tiles = static_cast<int64_t>((b.m + BM - 1) / BM) * b.tiles_n;
            const int64_t v = u - b.tile0;
            if (tiles <= 0 || v >= tiles * b.S) return false;
            const int64_t t = v % tiles;
            *prob = lo;
            *lmod = static_cast<int>(v / tiles);
            *tm = static_cast<int>(t / b.tiles_n);
            *tn = static_cast<int>(t % b.tiles_n);
            if (tile) *tile = 0;
            return true;
        }
        // modular encoding: the unit is one modulus of one tile, units handed out round-robin over
        // groups of group_tiles tiles (the member's order; A1 visits rows as A2 does), each group
        // modulus by modulus.  A wave covers one modulus of a block of tiles (the L2 footprint of a
        // digit pair), only the last round is partial, and with group_tiles = the grid a full
        // group keeps every modulus of a tile on one CTA.
        if (p.akeep) {  // kept-A order: this CTA's strip of tiles, modulus after modulus
            const uint32_t tiles = static_cast<uint32_t>(p.tiles_m) * static_cast<uint32_t>(p.tiles_n);
            const int N = one_S(p);
            const uint32_t start = fdiv(blockIdx.x * tiles, p.fd_ctas);
            const uint32_t len = fdiv((blockIdx.x + 1) * tiles, p.fd_ctas) - start;
            if (N < 1 || N > 16 || len == 0) return false;
            const FastDiv& fl = len == p.fd_len.d ? p.fd_len : p.fd_len1;  // the strip's length
            const uint32_t l = fdiv(static_cast<uint32_t>(it), fl);
            if (l >= static_cast<uint32_t>(N)) return false;
            const uint32_t t = start + (static_cast<uint32_t>(it) - l * fl.d);
            const uint32_t q = fdiv(t, p.tdv.tn);
            *prob = -1;
            *lmod = static_cast<int>(l);
            *tm = static_cast<int>(q);
            *tn = static_cast<int>(t - q * p.tdv.tn.d);
            if (tile) *tile = t;
            return true;
        }
        if (p.u32dec && !p.tri) {  // the same order in 32-bit arithmetic
            const uint32_t tiles = static_cast<uint32_t>(p.tiles_m) * static_cast<uint32_t>(p.tiles_n);
            const int N = one_S(p);
            const uint32_t u = blockIdx.x + static_cast<uint32_t>(it) * gridDim.x;
            if (N < 1 || N > 16 || u >= tiles * static_cast<uint32_t>(N)) return false;
            const uint32_t g = fdiv(fdiv(u, p.fd_gt), p.fd_n[N]);  // floor(u / (GT N))
            const uint32_t first = g * p.fd_gt.d;
            const FastDiv& gt = tiles - first < p.fd_gt.d ? p.fd_gt_last : p.fd_gt;
            const uint32_t r = u - first * static_cast<uint32_t>(N);
            const uint32_t l = fdiv(r, gt);
            const uint32_t t = first + (r - l * gt.d);
            *prob = -1;
            *lmod = static_cast<int>(l);
            if (tile) *tile = t;
            member_tile_fast(p.member == kMemberA1 ? kMemberA2 : p.member, p.tdv, t, p.tiles_m, tm, tn);
            return true;
        }
        const int64_t tiles = p.tri ? p.tri_tiles : static_cast<int64_t>(p.tiles_m) * p.tiles_n;
        const int64_t N = one_S(p);
        const int64_t u = static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x;
        if (u >= tiles * N) return false;
        const int64_t GT = p.group_tiles;
        const int64_t g = u / (GT * N);
        const int64_t first = g * GT;
        const int64_t gt = tiles - first < GT ? tiles - first : GT;  // tiles of this group
        const int64_t r = u - g * GT * N;
        *prob = -1;
        *lmod = static_cast<int>(r / gt);
        const int64_t t = first + r % gt;
        if (tile) *tile = t;
        if (p.tri) return tri_tile(p.tri == 1, t, p.tiles_m, p.tiles_n, p.tri_bn, tm, tn);
        const int member = p.member == kMemberA1 ? kMemberA2 : p.member;
        return member_tile(member, p.group, t % gridDim.x, gridDim.x, t / gridDim.x, p.tiles_m, p.tiles_n, tm, tn);
    }
    if constexpr (TAIL) {
        // the tail launch: CTA b takes k part b % parts of tail tile b / parts, the tail tiles
        // being the last, partial round of the main launch's round-robin order
        if (it > 0) return false;
        *prob = -1;
        *part = static_cast<int>(blockIdx.x) % p.tail_parts;
        const int64_t t = static_cast<int64_t>(p.full_rounds) * p.main_ctas + static_cast<int>(blockIdx.x) / p.tail_parts;
        return member_tile(p.member, p.group, t % p.main_ctas, p.main_ctas, t / p.main_ctas, p.tiles_m, p.tiles_n,
                           tm, tn);
    }
    if (p.table == nullptr) {
        *prob = -1;
        if (p.plan_kind != 0 && one_S(p) == 0) return false;  // the plan chose the modular encoding
        if (p.tail_parts >= 2 && it >= p.full_rounds) return false;  // the rest is the tail launch's
        if (p.u32dec && p.member != kMemberA1) {
            const uint32_t t = blockIdx.x + static_cast<uint32_t>(it) * gridDim.x;
            if (t >= static_cast<uint32_t>(p.tiles_m) * static_cast<uint32_t>(p.tiles_n)) return false;
            member_tile_fast(p.member, p.tdv, t, p.tiles_m, tm, tn);
            return true;
        }
        return member_tile(p.member, p.group, blockIdx.x, gridDim.x, it, p.tiles_m, p.tiles_n, tm, tn);
    }
    const int64_t t = static_cast<int64_t>(blockIdx.x) + static_cast<int64_t>(it) * gridDim.x;
    if (t >= (p.total_dev ? *p.total_dev : p.total_tiles)) return false;
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.table[mid].tile0 <= t) lo = mid;
        else hi = mid - 1;
    }
    const int64_t local = t - p.table[lo].tile0;
    const int tiles_n = p.table[lo].tiles_n;
    *prob = lo;
    *tm = static_cast<int>(local / tiles_n);
    *tn = static_cast<int>(local % tiles_n);
    return true;
}

// Small per-tile integers every role keeps in registers.
struct TileInts {
    int S, beta, chunk_slabs, slab0, nslab;
    uint32_t group_end;
};
MOMMS_DEV TileInts tile_ints(const Params& p, int prob, int part) {
    TileInts t;
    if (prob < 0) {
        t.S = one_S(p); t.beta = p.one.beta; t.chunk_slabs = p.one.chunk_slabs;
        t.slab0 = p.one.slab0; t.nslab = p.one.nslab;
        t.group_end = p.plan_kind != 0 ? p.group_end_by_s[t.S < 17 ? t.S : 16] : p.one.group_end;
        if (part >= 0) {  // this unit's share of the pass's k slabs (every part gets at least one)
            const int lo = part * t.nslab / p.tail_parts, hi = (part + 1) * t.nslab / p.tail_parts;
            t.slab0 += lo;
            t.nslab = hi - lo;
        }
    } else {
        const EmuBatchProblem& b = p.table[prob];
        t.S = b.S; t.beta = b.beta; t.chunk_slabs = b.chunk_slabs;
        t.slab0 = 0; t.nslab = b.nslab; t.group_end = b.group_end;
    }
    return t;
}

// The unit's k slabs narrowed to where its triangular operand is not zero (Params::kcap); the
// skipped slabs would add exact zeros.  Every role applies it, so all agree on the slab count.
template <int BN>
MOMMS_DEV void apply_kcap(const Params& p, int tm, int tn, TileInts& t) {
    if (p.kcap == 0) return;
    int lo = t.slab0, hi = t.slab0 + t.nslab;
    if (p.kcap == 1) hi = min(hi, (tm + 1) * (BM / BK));
    else if (p.kcap == 2) lo = max(lo, tm * (BM / BK));
    else if (p.kcap == 3) lo = max(lo, (tn * BN) / BK);
    else hi = min(hi, (tn * BN + BN + BK - 1) / BK);
    if (hi <= lo) return;  // (not for a square triangle) keep the whole range
    t.slab0 = lo;
    t.nslab = hi - lo;
}


// ---------------------------------------------------------------- recombination
// One drain thread's columns after the last chunk of diagonal d.  Q / R point at the
// thread's row in the per-CTA int64 / FP64 scratch blocks (column stride BM).
struct RecombineCtx {
    long long* Q;
    double* R;
    uint32_t qt;       // TMEM address of the thread's int64 group sums (tile width 96): low words at
                       // qt + c, high words at qt + 32 + c for column c
    uint64_t keep;     // L2 policy of the scratch accesses (evict last)
    uint32_t tsum;     // TMEM address of the int32 sums of the last CT columns
    int sh;            // beta * (position of d in its group)
    int gsh;           // -beta * position: R is 2^gsh times the group's fold
    double rb;         // 2^-beta
    bool gfirst;       // d is the least significant diagonal of its group
    bool rfirst;       // no earlier group has produced R yet
};
struct FinalCtx {
    bool row_ok, eflag;
    int ei;
    const int* colexp;       // f_j - 2 beta of the thread's columns (shared memory)
    const uint8_t* colflag;  // non-finite flags of the thread's columns (shared memory)
    int ncols;               // columns of the thread inside the matrix
    int tri, lim;            // triangle mask: 1 keeps columns c <= lim, 2 keeps c >= lim (c local)
    double* cp;              // &C[row, first column of the thread]
    int64_t ldc;
    double alpha, beta_c, qnan;
    bool unit_alpha, beta_zero;  // alpha == 1, beta_c == 0, decided once per tile
};
enum { kMid = 0, kGroupEnd = 1, kLast = 2 };
constexpr int BM_ = kEmuBM;

// 8 columns [c0, c0 + 8): exact int64 group sum, FP64 fold at the group end, C at the end.  The
// FP64 pipe is this epilogue's bottleneck, so every power-of-two scaling is an exponent-field add
// (mul_pow2) and alpha = 1 multiplies nothing: per element the conversion and the fold at a group
// end, the conversion, the fold and beta_c's multiply-add at the end.
template <int MODE, bool QT = false>
MOMMS_DEV void recombine8(const RecombineCtx& rc, const int32_t (&pv)[8], int c0, const FinalCtx* fc) {
    long long qv[8];
    double rv[8];
    if constexpr (QT) {
        if (!rc.gfirst) {
            uint32_t lo[8], hi[8];
            tmem_ld_32x32b_x8(rc.qt + c0, lo);
            tmem_ld_32x32b_x8(rc.qt + 32 + c0, hi);
            tmem_ld_wait(lo);
            tmem_ld_wait(hi);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                qv[j] = static_cast<long long>((static_cast<unsigned long long>(hi[j]) << 32) | lo[j]);
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) qv[j] = 0ll;
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if constexpr (!QT) qv[j] = rc.gfirst ? 0ll : ld_l2_hint(rc.Q + (c0 + j) * BM_, rc.keep);
        if (MODE != kMid) rv[j] = rc.rfirst ? 0.0 : ld_l2_hint(rc.R + (c0 + j) * BM_, rc.keep);
    }
    uint32_t qlo[8], qhi[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const long long p64 = static_cast<long long>(pv[j]);
        const long long v = rc.gfirst ? p64 : qv[j] + (p64 << rc.sh);
        if (MODE == kMid) {
            if constexpr (QT) {
                qlo[j] = static_cast<uint32_t>(static_cast<unsigned long long>(v));
                qhi[j] = static_cast<uint32_t>(static_cast<unsigned long long>(v) >> 32);
            } else {
                st_l2_hint(rc.Q + (c0 + j) * BM_, v, rc.keep);
            }
        } else {
            const double x = static_cast<double>(v);
            const double f = rc.rfirst ? x : fma(rv[j], rc.rb, x);  // exact but for this rounding
            if (MODE == kGroupEnd) {
                st_l2_hint(rc.R + (c0 + j) * BM_, mul_pow2(f, rc.gsh), rc.keep);
            } else if (fc->row_ok && c0 + j < fc->ncols &&
                       (fc->tri == 0 || (fc->tri == 1 ? c0 + j <= fc->lim : c0 + j >= fc->lim))) {
                // f 2^gsh is exact (no partial sum comes near the subnormal range), so one scaling by
                // 2^(gsh + e_i + f_j - 2 beta) rounds as the two would
                double y = (fc->eflag || fc->colflag[c0 + j]) ? fc->qnan
                                                              : mul_pow2(f, rc.gsh + fc->ei + fc->colexp[c0 + j]);
                if (!fc->unit_alpha) y *= fc->alpha;
                double* cp = fc->cp + static_cast<int64_t>(c0 + j) * fc->ldc;
                *cp = fc->beta_zero ? y : fma(fc->beta_c, *cp, y);
            }
        }
    }
    if constexpr (QT) {
        if (MODE == kMid) {
            tmem_st_32x32b_x8(rc.qt + c0, qlo);
            tmem_st_32x32b_x8(rc.qt + 32 + c0, qhi);
            tmem_st_wait();
        }
    }
    asm volatile("" ::: "memory");  // one batch of loads in flight at a time
}

template <int MODE, int CR, int CT>
MOMMS_DEV void recombine(const RecombineCtx& rc, const int32_t (&acc)[CR], const FinalCtx* fc) {
    constexpr bool QT = (CT == 0);  // the narrow tile keeps every sum in registers and Q in TMEM
#pragma unroll
    for (int b = 0; b < CR / 8; ++b) {
        int32_t pv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) pv[j] = acc[b * 8 + j];
        recombine8<MODE, QT>(rc, pv, b * 8, fc);
    }
#pragma unroll
    for (int q = 0; q < CT / 16; ++q) {
        uint32_t t[16];
        tmem_ld_32x32b_x16(rc.tsum + q * 16, t);
        tmem_ld_wait(t);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int32_t pv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) pv[j] = static_cast<int32_t>(t[h * 8 + j]);
            recombine8<MODE>(rc, pv, CR + q * 16 + h * 8, fc);
        }
    }
}

// Wait used while shutting down after an abort: ignores the abort flag, keeps the time limit.
MOMMS_DEV bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    volatile int never = 0;
    return mbar_wait(bar, parity, &never);
}

// Recombination of diagonal d of tile (tm, tn) once its int32 sums are complete: the first CR
// columns of the thread in `acc`, the other CT in TMEM at `tsum`.  Diagonals arrive from the
// least significant (d = S + 1) to the most significant (d = 2).  Inside a group the diagonal
// sums are combined exactly in int64, Q = sum_j P_{hi-j} 2^(beta j) (the host chose the groups
// so that |Q| < 2^63); at the group's most significant diagonal lo, R = 2^(-beta (hi-lo))
// (Q + 2^-beta R_prev) in FP64.  The last group ends at d = 2 and goes straight to C:
//     C := alpha 2^(e_i + f_j - 2 beta) R + beta_c C.
template <int BN, int CR, int CT>
MOMMS_DEV void recombine_diagonal(const Params& p, int prob, int tm, int tn, int d, const TileInts& pr,
                                  long long* Q, double* R, uint64_t keep, uint32_t tsum, double rb, int third,
                                  int rloc, const int* colexp, const uint8_t* colflag, double qnan,
                                  const int32_t (&acc)[CR], int& gj, bool& rfirst) {
    constexpr int CW = BN / 3;
    const bool gfirst = (gj == 0);
    const bool gend = (pr.group_end >> d) & 1u;
    const RecombineCtx rc{Q, R, tsum, keep, tsum, pr.beta * gj, -pr.beta * gj, rb, gfirst, rfirst};
    if (!gend) {
        recombine<kMid, CR, CT>(rc, acc, nullptr);
    } else if (d != 2) {
        recombine<kGroupEnd, CR, CT>(rc, acc, nullptr);
    } else {
        const int row = tm * BM + rloc;
        FinalCtx fc;
        const Prob& one = p.one;
        const EmuBatchProblem* bp = prob < 0 ? nullptr : &p.table[prob];
        const int m_ = bp ? bp->m : one.m;
        const int n_ = bp ? bp->n : one.n;
        fc.row_ok = row < m_;
        fc.ei = fc.row_ok ? (bp ? bp->e : one.e)[row] : 0;
        fc.eflag = fc.row_ok ? ((bp ? bp->ef : one.ef)[row] != 0) : false;
        fc.colexp = colexp + third * CW;
        fc.colflag = colflag + third * CW;
        fc.ncols = min(CW, n_ - (tn * BN + third * CW));
        fc.tri = bp ? bp->tri : 0;
        fc.lim = bp ? row + bp->diag - (tn * BN + third * CW) : 0;
        fc.ldc = bp ? bp->ldc : one.ldc;
        fc.cp = (bp ? bp->C : one.C) + row + static_cast<int64_t>(tn * BN + third * CW) * fc.ldc;
        fc.alpha = bp ? bp->alpha : one.alpha;
        fc.beta_c = bp ? bp->beta_c : one.beta_c;
        fc.qnan = qnan;
        fc.unit_alpha = fc.alpha == 1.0;
        fc.beta_zero = fc.beta_c == 0.0;
        recombine<kLast, CR, CT>(rc, acc, &fc);
    }
    if (gend) {
        gj = 0;
        rfirst = false;
    } else {
        ++gj;
    }
}

// The int32 partial sums of diagonal d of k part `part` of a tail tile: a 192 x 128 block
// stored as [column / 4][row][4], so that a thread's four consecutive columns are one 16-byte
// word and a warp's 32 rows one contiguous 512-byte segment.  Returns this thread's first
// word (columns c0 .. c0 + 3, row rloc); the next four columns are 128 words on.
MOMMS_DEV int4* tail_slot(const Params& p, int tail, int part, int S, int d, int c0, int rloc) {
    const size_t blk = (static_cast<size_t>(tail) * p.tail_parts + part) * S + (d - 2);
    return reinterpret_cast<int4*>(p.tail_sums) + (blk * kEmuBNMax + c0) / 4 * BM + rloc;
}

template <int CR, int CT>
MOMMS_DEV void store_partial(int4* dst, const int32_t (&acc)[CR], uint32_t tsum) {
#pragma unroll
    for (int c = 0; c < CR; c += 4) __stcg(dst + c / 4 * BM, make_int4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]));
#pragma unroll
    for (int q = 0; q < CT / 16; ++q) {
        uint32_t t[16];
        tmem_ld_32x32b_x16(tsum + q * 16, t);
        tmem_ld_wait(t);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
            __stcg(dst + (CR + q * 16 + j) / 4 * BM, make_int4(static_cast<int>(t[j]), static_cast<int>(t[j + 1]),
                                                               static_cast<int>(t[j + 2]), static_cast<int>(t[j + 3])));
    }
}

// x mod p in [0, p) for an int32 sum |x| <= k 127^2 < 2^31 - 255: u = x + p ceil(2^31 / p) lies
// in [0, 2^32) with the same residue, and one multiply-high quotient (floor or one over) with a
// correction finishes it -- no integer division (whose reciprocal estimate runs on the slow
// conversion pipe).
MOMMS_DEV uint32_t residue_of(int32_t x, uint32_t p, uint32_t magic, uint32_t off) {
    const uint32_t u = static_cast<uint32_t>(x) + off;
    const uint32_t q = __umulhi(u, magic);
    int r = static_cast<int>(u - q * p);
    if (r < 0) r += static_cast<int>(p);
    return static_cast<uint32_t>(r);
}

// x mod p in [0, p) from the FP32 bits of an accumulator sum x, an integer with |x| < 2^22 (the
// residue-product sums of k <= 256).  1.5 2^23 + x lies in [2^23, 2^24), where FP32 holds every
// integer, so its bits are 0x4B400000 + x (an FP32 add instead of a float-to-int conversion,
// whose pipe takes 16 lanes per clock per SM); off = p ceil(2^22 / p) - 0x4B400000 turns them into
// u = x + p ceil(2^22 / p) in [0, 2^24), where the multiply-high by ceil(2^32 / p) is the exact
// floor of u / p (its excess, below u 2^-32 < 2^-8, stays under 1/p for p < 256): no correction.
MOMMS_DEV uint32_t residue_small_bits(uint32_t bits, uint32_t p, uint32_t magic_up, uint32_t off) {
    const uint32_t u = __float_as_uint(__uint_as_float(bits) + 12582912.0f) + off;
    return u - __umulhi(u, magic_up) * p;
}

// Four columns' bytes of one row (column c in byte c) transposed across the four lanes of each
// group (rows 4g .. 4g + 3 of the warp): lane q of the group returns column q's bytes of the
// group's four rows, row 4g + t in byte t.
// The two byte-permute selectors of a lane (one per exchange step), taken once per call site:
// each step is then one shuffle and one permute with a register selector.
struct Transpose4Sel {
    uint32_t s1, s2;
};
MOMMS_DEV Transpose4Sel transpose4_sel(int lane) {
    return Transpose4Sel{(lane & 1) ? 0x3715u : 0x6240u, (lane & 2) ? 0x3276u : 0x5410u};
}
MOMMS_DEV uint32_t transpose4x4_bytes(uint32_t w, const Transpose4Sel& sel) {
    const uint32_t o1 = __shfl_xor_sync(0xffffffffu, w, 1);
    const uint32_t t1 = __byte_perm(w, o1, sel.s1);
    const uint32_t o2 = __shfl_xor_sync(0xffffffffu, t1, 2);
    return __byte_perm(t1, o2, sel.s2);
}

// The modular epilogue of modulus l: the thread's int32 sums (CR in `acc`, CT in TMEM at
// `tsum`) reduced into [0, p) and stored as bytes at res[l][col][row].  With m a multiple of 4
// (and res 4-byte aligned) every four columns of the four rows of a lane group are transposed
// across the group and stored as one 32-bit word per lane: a quarter of the store instructions,
// 4 x 32 contiguous bytes each (one byte store per element and column measured 1.2 of the 5.2 us
// a rank-k unit of 128 x 192 x 256 takes).  Else one byte per element (a warp's 32 rows: one
// 32-byte sector per column).  The TMEM reads and the shuffles are warp-wide, so every lane takes
// them before the bounds checks.
template <int BN, int CR, int CT>
MOMMS_DEV void store_residues(const Params& p, int prob, int tm, int tn, int l, int third, int rloc,
                              const int32_t (&acc)[CR], uint32_t tsum) {
    const int row = tm * BM + rloc;
    const int col0 = tn * BN + third * (BN / 3);
    const uint32_t pl = p.modp[l], mg = p.modmagic[l], off = p.modoff[l];
    auto residue = [&](int32_t v) { return residue_of(v, pl, mg, off); };
    const int m = prob < 0 ? p.one.m : p.table[prob].m;
    const int n = prob < 0 ? p.one.n : p.table[prob].n;
    uint8_t* res = prob < 0 ? p.res : p.table[prob].res;
    const bool row_ok = row < m;
    const size_t cstep = static_cast<size_t>(m);
    const int ncols = min(BN / 3, n - col0);
    const int lane = static_cast<int>(threadIdx.x & 31);
    if ((m & 3) == 0 && (reinterpret_cast<uintptr_t>(res) & 3) == 0) {
        // word store: lane 4g + q writes column 4j + q of rows 4g .. 4g + 3 (all inside m or none)
        uint8_t* base = res + static_cast<size_t>(l) * m * n + static_cast<size_t>(col0) * m + (row & ~3);
        const int cq = lane & 3;
        const Transpose4Sel tsel = transpose4_sel(lane);
#pragma unroll
        for (int c = 0; c < CR; c += 4) {
            const uint32_t w = residue(acc[c]) | (residue(acc[c + 1]) << 8) |
                               (residue(acc[c + 2]) << 16) |
                               (residue(acc[c + 3]) << 24);
            const uint32_t x = transpose4x4_bytes(w, tsel);
            if (row_ok && c + cq < ncols) *reinterpret_cast<uint32_t*>(base + (c + cq) * cstep) = x;
        }
#pragma unroll
        for (int q = 0; q < CT / 16; ++q) {
            uint32_t t[16];
            tmem_ld_32x32b_x16(tsum + q * 16, t);
            tmem_ld_wait(t);
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
                const int c = CR + q * 16 + j;
                const uint32_t w = residue(static_cast<int32_t>(t[j])) |
                                   (residue(static_cast<int32_t>(t[j + 1])) << 8) |
                                   (residue(static_cast<int32_t>(t[j + 2])) << 16) |
                                   (residue(static_cast<int32_t>(t[j + 3])) << 24);
                const uint32_t x = transpose4x4_bytes(w, tsel);
                if (row_ok && c + cq < ncols) *reinterpret_cast<uint32_t*>(base + (c + cq) * cstep) = x;
            }
        }
        return;
    }
    uint8_t* dst = res + static_cast<size_t>(l) * m * n + static_cast<size_t>(col0) * m + row;
#pragma unroll
    for (int c = 0; c < CR; ++c) {
        const uint32_t r = residue(acc[c]);
        if (row_ok && c < ncols) dst[c * cstep] = static_cast<uint8_t>(r);
    }
#pragma unroll
    for (int q = 0; q < CT / 16; ++q) {
        uint32_t t[16];
        tmem_ld_32x32b_x16(tsum + q * 16, t);
        tmem_ld_wait(t);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int c = CR + q * 16 + j;
            const uint32_t r = residue(static_cast<int32_t>(t[j]));
            if (row_ok && c < ncols) dst[c * cstep] = static_cast<uint8_t>(r);
        }
    }
}

// The tile's residues of this modulus are stored: once every drain thread has issued its
// stores, one thread publishes them (fence, then the tile's counter).
MOMMS_DEV void signal_tile(const Params& p, int64_t tile) {
    named_bar_sync(1, 32 * EPI_WARPS);
    if (threadIdx.x == 32 * CTRL_WARPS) {
        __threadfence();
        atomicAdd(p.done + tile, 1);
    }
}

// Waits (bounded) until `need` moduli of the tile are published; false if the wait gave up.
MOMMS_DEV bool wait_tile(const Params& p, int64_t tile, int need, volatile int* abort_flag, volatile int* wait_ok) {
    if (threadIdx.x == 32 * CTRL_WARPS) {
        int ok = 1;
        const volatile int* cnt = p.done + tile;
        if (*cnt < need) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1; *cnt < need; ++it) {
                if ((it & 63u) == 0) {
                    if (*abort_flag || globaltimer_ns() - t0 > kWaitTimeoutNs) {
                        *abort_flag = 1;
                        ok = 0;
                        break;
                    }
                    __nanosleep(256);
                }
            }
        }
        __threadfence();
        *wait_ok = ok;
    }
    named_bar_sync(1, 32 * EPI_WARPS);
    return *wait_ok != 0;
}

// L2 prefetch of the residues a final unit will read (other moduli of the warp's 32 rows and the
// thread's columns), issued before the unit's products so that they arrive under them: one
// prefetch per 32-byte sector, spread over the lanes.
template <int BN>
MOMMS_DEV void prefetch_residues(const Params& p, int tm, int tn, int last, int third, int quad, int lane) {
    constexpr int CW = BN / 3;
    const int row0 = tm * BM + quad * 32;
    const int col0 = tn * BN + third * CW;
    if (row0 >= p.one.m) return;
    const int ncols = min(CW, p.one.n - col0);
    const size_t mn = static_cast<size_t>(p.one.m) * p.one.n;
    for (int idx = lane; idx < last * ncols; idx += 32) {
        const int l = idx / ncols, c = idx - l * ncols;
        const uint8_t* a = p.res + l * mn + static_cast<size_t>(col0 + c) * p.one.m + row0;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
    }
}

// Two elements of the fused reconstruction (columns col and col + 1 of one row, the second only
// when `two`): the other moduli's residues from res (all loads issued first), this modulus's
// `own`, then C := alpha y + beta C as the separate reconstruction kernel computes it (crt.cuh).
template <int L>
MOMMS_DEV void crt_pair(const Params& p, int row, int col, bool two, uint32_t own0, uint32_t own1, int last, int Erow,
                        bool flag_row, const int* colexp, const uint8_t* colflag) {
    const size_t mn = static_cast<size_t>(p.one.m) * p.one.n;
    const uint8_t* src = p.res + static_cast<size_t>(col) * p.one.m + row;
    uint32_t r0[kCrtMaxModuli], r1[kCrtMaxModuli];
#pragma unroll
    for (int l = 0; l < kCrtMaxModuli; ++l) {
        r0[l] = l < last ? __ldcg(src + l * mn) : 0u;
        r1[l] = (two && l < last) ? __ldcg(src + l * mn + p.one.m) : 0u;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        if (e == 1 && !two) break;
        unsigned long long s[L];
#pragma unroll
        for (int q = 0; q < L; ++q) s[q] = 0;
        uint32_t qs = 0;
#pragma unroll
        for (int l = 0; l < kCrtMaxModuli; ++l)
            if (l < last) crt_accumulate<L>(s, qs, e == 0 ? r0[l] : r1[l], p.crt_w[l], p.crt_F[l]);
        crt_accumulate<L>(s, qs, e == 0 ? own0 : own1, p.crt_w[last], p.crt_F[last]);
        double y = (flag_row || colflag[e] != 0) ? __longlong_as_double(0x7ff8000000000000ll)
                                                 : crt_value<L>(s, qs, p.crt_Pw, Erow + colexp[e]);
        if (p.one.alpha != 1.0) y *= p.one.alpha;
        double* cp = p.one.C + row + static_cast<int64_t>(col + e) * p.one.ldc;
        *cp = p.one.beta_c == 0.0 ? y : fma(p.one.beta_c, *cp, y);
    }
}

// The last modulus of a tile with the reconstruction fused: this modulus's residues of the
// thread's columns, then each element of C.
template <int BN, int CR, int CT, int L>
MOMMS_DEV void crt_final(const Params& p, int tm, int tn, int last, int third, int rloc, const int32_t (&acc)[CR],
                         uint32_t tsum, const int* colexp, const uint8_t* colflag) {
    constexpr int CW = BN / 3;
    const int row = tm * BM + rloc;
    const int col0 = tn * BN + third * CW;
    const uint32_t pl = p.modp[last], mg = p.modmagic[last], off = p.modoff[last];
    const bool row_ok = row < p.one.m;
    const int ncols = min(CW, p.one.n - col0);
    const int Erow = row_ok ? p.one.e[row] : 0;
    const bool frow = row_ok ? p.one.ef[row] != 0 : false;
    // this modulus's residues of the thread's columns, packed four to a word (static indexing
    // keeps `acc` in registers for the drain of every unit)
    uint32_t own[CW / 4];
#pragma unroll
    for (int c = 0; c < CR; c += 4)
        own[c / 4] = residue_of(acc[c], pl, mg, off) | (residue_of(acc[c + 1], pl, mg, off) << 8) |
                     (residue_of(acc[c + 2], pl, mg, off) << 16) | (residue_of(acc[c + 3], pl, mg, off) << 24);
#pragma unroll
    for (int q = 0; q < CT / 16; ++q) {
        uint32_t t[16];
        tmem_ld_32x32b_x16(tsum + q * 16, t);
        tmem_ld_wait(t);
#pragma unroll
        for (int j = 0; j < 16; j += 4)
            own[(CR + q * 16 + j) / 4] = residue_of(static_cast<int32_t>(t[j]), pl, mg, off) |
                                         (residue_of(static_cast<int32_t>(t[j + 1]), pl, mg, off) << 8) |
                                         (residue_of(static_cast<int32_t>(t[j + 2]), pl, mg, off) << 16) |
                                         (residue_of(static_cast<int32_t>(t[j + 3]), pl, mg, off) << 24);
    }
    if (!row_ok) return;
    for (int c = 0; c < ncols; c += 2)
        crt_pair<L>(p, row, col0 + c, c + 1 < ncols, (own[c >> 2] >> (8 * (c & 3))) & 0xFFu,
                    (own[(c + 1) >> 2] >> (8 * ((c + 1) & 3))) & 0xFFu, last, Erow, frow, colexp + third * CW + c,
                    colflag + third * CW + c);
}

// Stages the column exponents (minus 2 beta) and non-finite flags of tile column tn in shared
// memory, between two barriers of the drain warps (the previous tile's columns are no longer read).
template <int BN>
MOMMS_DEV void stage_columns(const Params& p, int prob, int tn, int beta, int* colexp, uint8_t* colflag) {
    named_bar_sync(1, 32 * EPI_WARPS);
    for (int c = threadIdx.x - 32 * CTRL_WARPS; c < BN; c += 32 * EPI_WARPS) {
        const int col = tn * BN + c;
        const int n_ = prob < 0 ? p.one.n : p.table[prob].n;
        const int32_t* f_ = prob < 0 ? p.one.f : p.table[prob].f;
        const uint8_t* ff_ = prob < 0 ? p.one.ff : p.table[prob].ff;
        colexp[c] = col < n_ ? f_[col] - 2 * beta : 0;
        colflag[c] = col < n_ ? ff_[col] : 0;
    }
    named_bar_sync(1, 32 * EPI_WARPS);
}

// Drains the accumulator chunks of one diagonal (`units` k slabs, `chunk_slabs` per chunk) into
// int32 sums: the first CR of the thread's columns in `acc`, the other CT in TMEM at `tsum`.
// `tacc` is the thread's first accumulator column in buffer 0 (buffer 1 is 256 columns on).
// `remote_empty` (CTA pairs): the shared::cluster address of the pair leader's acc_empty[0], on
// which the peer's warps arrive instead of their own (0: this CTA's acc_empty).
// Returns false if a bounded wait gave up.
template <int CR, int CT>
MOMMS_DEV bool drain_diagonal(int units, int chunk_slabs, uint64_t* acc_full, uint64_t* acc_empty, uint32_t& abuf,
                              uint32_t (&aphase)[2], volatile int* abort_flag, uint32_t tacc, uint32_t tsum,
                              int lane, int32_t (&acc)[CR], uint32_t remote_empty = 0, bool remote_full = false) {
#pragma unroll
    for (int c = 0; c < CR; ++c) acc[c] = 0;
    bool first = true;
    for (int u = 0; u < units;) {
        const int cnt = min(chunk_slabs, units - u);
        const bool ready = remote_full ? mbar_wait_cluster(&acc_full[abuf], aphase[abuf], abort_flag)
                                       : mbar_wait(&acc_full[abuf], aphase[abuf], abort_flag);
        if (!ready) return false;
        tc_fence_after();
        const uint32_t taddr = tacc + abuf * 256u;
#pragma unroll
        for (int q = 0; q < CR / 16; ++q) {
            uint32_t r[16];
            tmem_ld_32x32b_x16(taddr + q * 16, r);
            tmem_ld_wait(r);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[q * 16 + j] += __float2int_rn(__uint_as_float(r[j]));
        }
#pragma unroll
        for (int q = 0; q < CT / 16; ++q) {
            uint32_t r[16];
            tmem_ld_32x32b_x16(taddr + CR + q * 16, r);
            tmem_ld_wait(r);
            uint32_t t[16];
            if (first) {
#pragma unroll
                for (int j = 0; j < 16; ++j) t[j] = static_cast<uint32_t>(__float2int_rn(__uint_as_float(r[j])));
            } else {
                tmem_ld_32x32b_x16(tsum + q * 16, t);
                tmem_ld_wait(t);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    t[j] = static_cast<uint32_t>(static_cast<int32_t>(t[j]) + __float2int_rn(__uint_as_float(r[j])));
            }
            tmem_st_32x32b_x16(tsum + q * 16, t);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
            if (remote_empty) mbar_arrive_cluster(remote_empty + 8u * abuf);
            else mbar_arrive(&acc_empty[abuf]);
        }
        aphase[abuf] ^= 1u;
        abuf ^= 1u;
        u += cnt;
        first = false;
    }
    return true;
}

// The kept-A kernel's unit (one chunk: every k <= 256 sum is an FP32 integer below 2^22 in
// magnitude) from the accumulator straight to its residues: 16 of the thread's columns per
// tensor-memory load, the next load in flight while the current 16 are reduced
// (residue_small_bits), packed, transposed across each group of four lanes and stored
// four rows to a word.  The accumulator goes back to the MMA thread once its last load has landed
// (no int32 sums staged in tensor memory, one exposed load latency per unit).  Requires m % 4 == 0.
template <int BN>
MOMMS_DEV bool drain_store_small(const Params& p, int tm, int tn, int l, int third, int rloc, int lane,
                                 uint64_t* acc_full, uint64_t* acc_empty, uint32_t& abuf, uint32_t (&aphase)[2],
                                 volatile int* abort_flag, uint32_t tacc) {
    constexpr int CW = BN / 3;
    constexpr int G = CW / 16;
    if (!mbar_wait(&acc_full[abuf], aphase[abuf], abort_flag)) return false;
    tc_fence_after();
    const uint32_t taddr = tacc + abuf * 256u;
    const int row = tm * BM + rloc;
    const int col0 = tn * BN + third * CW;
    const int m = p.one.m, n = p.one.n;
    const uint32_t pl = p.modp[l], mg = p.modmagic_up[l];
    const uint32_t off = p.modoff22[l] - 0x4B400000u;  // residue_small_bits' offset
    const bool row_ok = row < m;
    const size_t cstep = static_cast<size_t>(m);
    const int ncols = min(CW, n - col0);
    uint8_t* base = p.res + static_cast<size_t>(l) * m * n + static_cast<size_t>(col0) * m + (row & ~3);
    const int cq = lane & 3;
    const Transpose4Sel tsel = transpose4_sel(lane);
    uint32_t r[2][16];
    tmem_ld_32x32b_x16(taddr, r[0]);
    tmem_ld_wait(r[0]);
#pragma unroll
    for (int g = 0; g < G; ++g) {
        if (g + 1 < G) tmem_ld_32x32b_x16(taddr + (g + 1) * 16, r[(g + 1) & 1]);
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
            uint32_t w = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) w |= residue_small_bits(r[g & 1][c + j], pl, mg, off) << (8 * j);
            const uint32_t x = transpose4x4_bytes(w, tsel);
            const int cc = g * 16 + c + cq;
            if (row_ok && cc < ncols) *reinterpret_cast<uint32_t*>(base + cc * cstep) = x;
        }
        if (g + 1 < G) {
            tmem_ld_wait(r[(g + 1) & 1]);
            if (g + 2 == G) {  // every load has landed: the accumulator is free
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[abuf]);
            }
        }
    }
    aphase[abuf] ^= 1u;
    abuf ^= 1u;
    return true;
}

// A drain warp's share of a k part of a split tail tile (always the CTA's last unit): drain
// every diagonal and store its int32 sums for the fix-up launch (tail_fixup_kernel), which
// adds the parts and recombines once all of them are done.
template <int BN>
MOMMS_DEV void drain_tail_unit(const Params& p, int tn, int part, uint64_t* acc_full, uint64_t* acc_empty,
                               uint32_t abuf, uint32_t ph0, uint32_t ph1, volatile int* abort_flag, uint32_t tacc,
                               uint32_t tsum, int lane, int third, int rloc) {
    using C_ = Cfg<BN>;
    constexpr int CR = C_::CR, CT = C_::CT, CW = C_::CW;
    const TileInts pr = tile_ints(p, -1, part);
    const int tail = static_cast<int>(blockIdx.x) / p.tail_parts;
    uint32_t aphase[2] = {ph0, ph1};
    (void)tn;
    for (int d = pr.S + 1; d >= 2; --d) {
        int32_t acc[CR];
        if (!drain_diagonal<CR, CT>((d - 1) * pr.nslab, pr.chunk_slabs, acc_full, acc_empty, abuf, aphase,
                                    abort_flag, tacc, tsum, lane, acc))
            return;
        store_partial<CR, CT>(tail_slot(p, tail, part, pr.S, d, third * CW, rloc), acc, tsum);
    }
}

// The fix-up of the split tail tiles, one thread per row and 8 columns of a tile: the int32
// diagonal sums of all k parts are added (integer addition: they equal the unsplit sums) and
// recombined in registers with the arithmetic of recombine8 -- exact int64 group sums, FP64
// only at group ends, the final scaling and alpha / beta_c -- so C is bit-identical to the
// unsplit kernel's.
__global__ void __launch_bounds__(256) tail_fixup_kernel(const __grid_constant__ Params p) {
    constexpr int GROUPS = kEmuBNMax / 8;  // column groups of a tile
    const int64_t gid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t per_tile = static_cast<int64_t>(BM) * GROUPS;
    const int tail = static_cast<int>(gid / per_tile);
    if (tail >= p.tail_tiles) return;
    const int w = static_cast<int>(gid - tail * per_tile);
    const int rloc = w % BM, cg = w / BM;  // consecutive threads: consecutive rows
    const int64_t t = static_cast<int64_t>(p.full_rounds) * p.main_ctas + tail;
    int tm, tn;
    if (!member_tile(p.member, p.group, t % p.main_ctas, p.main_ctas, t / p.main_ctas, p.tiles_m, p.tiles_n, &tm, &tn))
        return;
    const Prob& one = p.one;
    const int S = one.S, beta = one.beta;
    const double rb = pow2_normal(-beta);
    long long q[8];
    double r[8];
    int gj = 0;
    bool rfirst = true;
    for (int d = S + 1; d >= 2; --d) {
        int32_t pv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int part = 0; part < p.tail_parts; ++part) {
            const int4* src = tail_slot(p, tail, part, S, d, cg * 8, rloc);
            const int4 a = __ldcg(src), b = __ldcg(src + BM);
            pv[0] += a.x; pv[1] += a.y; pv[2] += a.z; pv[3] += a.w;
            pv[4] += b.x; pv[5] += b.y; pv[6] += b.z; pv[7] += b.w;
        }
        const bool gfirst = (gj == 0);
        const bool gend = (one.group_end >> d) & 1u;
        const int sh = beta * gj;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const long long p64 = static_cast<long long>(pv[j]);
            const long long v = gfirst ? p64 : q[j] + (p64 << sh);
            if (!gend) {
                q[j] = v;
            } else {
                const double x = static_cast<double>(v);
                r[j] = mul_pow2(rfirst ? x : fma(r[j], rb, x), -beta * gj);
            }
        }
        if (gend) {
            gj = 0;
            rfirst = false;
        } else {
            ++gj;
        }
    }
    const int row = tm * BM + rloc;
    if (row >= one.m) return;
    const int ei = one.e[row];
    const bool eflag = one.ef[row] != 0;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    const bool unit_alpha = one.alpha == 1.0, beta_zero = one.beta_c == 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int col = tn * kEmuBNMax + cg * 8 + j;
        if (col >= one.n) break;
        double y = (eflag || one.ff[col]) ? qnan : mul_pow2(r[j], ei + (one.f[col] - 2 * beta));
        if (!unit_alpha) y *= one.alpha;
        double* cp = one.C + row + static_cast<int64_t>(col) * one.ldc;
        *cp = beta_zero ? y : fma(one.beta_c, *cp, y);
    }
}

// MOD: the modular encoding -- a unit is one modulus l of one tile (p.one.S moduli), one pair
// (residue plane l of A, plane l of B), and its epilogue stores residues instead of recombining.
// AK: the kept-A residue product (MOD, BN = kEmuBNMax, k <= AK_SLABS slabs): the A region holds
// the unit's A slabs, loaded once per (modulus, tile row) of the CTA's strip (a_full / a_empty),
// and the ring stages hold B slabs only.
template <int BN, bool TAIL, bool MOD = false, bool AK = false>
__global__ void __launch_bounds__(THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const __grid_constant__ Params p) {
    using C_ = Cfg<BN>;
    static_assert(!AK || (MOD && !TAIL && BN == kEmuBNMax), "kept A: residue products of wide tiles");
    constexpr int STAGES = AK ? AK_STAGES : C_::STAGES;
    constexpr uint32_t STAGE = AK ? AK_STAGE : C_::STAGE;
    constexpr uint32_t RING = AK ? AK_REGION : 0;   // the ring's offset (the A region before it)
    constexpr uint32_t B_OFF = AK ? 0 : A_TILE;     // B slab inside a stage
    constexpr int CW = C_::CW;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint8_t* ring = smem + RING;
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + STAGES * STAGE);
    uint64_t* full = bars;                        // STAGES
    uint64_t* empty = bars + STAGES;              // STAGES
    uint64_t* acc_full = bars + 2 * STAGES;       // 2
    uint64_t* acc_empty = bars + 2 * STAGES + 2;  // 2
    uint64_t* drain = bars + 2 * STAGES + 4;      // 1
    uint64_t* a_full = bars + 2 * STAGES + 5;     // 1 (AK)
    uint64_t* a_empty = bars + 2 * STAGES + 6;    // 1 (AK)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 7);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* wait_ok = reinterpret_cast<volatile int*>(tmem_slot + 2);  // fused reconstruction
    int* colexp = reinterpret_cast<int*>(ring + STAGES * STAGE + 256);   // BN column exponents
    uint8_t* colflag = reinterpret_cast<uint8_t*>(colexp + BN);          // BN column flags

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], EPI_WARPS);
        }
        mbar_init(drain, 1);
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        *abort_flag = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            if (p.table == nullptr) {
                prefetch_tensormap(&tmA);
                prefetch_tensormap(&tmB);
            }
            uint32_t stage = 0, phase = 0;
            int last_phase[STAGES];
            for (int i = 0; i < STAGES; ++i) last_phase[i] = -1;
            bool ok = true;
            bool withhold = p.withhold != 0 && blockIdx.x == 0;
            int ag = -1, a_lm = -1, a_tm = -1;  // AK: group of units sharing the A region
            int a_armed = -1;                   // AK: the last group whose A loads were issued
            for (int it = 0; ok; ++it) {
                int tm, tn, prob, part, lm = 0;
                if (!tile_of<TAIL, MOD>(p, it, &prob, &tm, &tn, &part, &lm)) break;
                TileInts pr = tile_ints(p, prob, part);
                if constexpr (MOD) apply_kcap<BN>(p, tm, tn, pr);
                const CUtensorMap* mapA = prob < 0 ? &tmA : &p.table[prob].mapA;
                const CUtensorMap* mapB = prob < 0 ? &tmB : &p.table[prob].mapB;
                if constexpr (AK) {
                    if (lm != a_lm || tm != a_tm) {
                        // a new (modulus, tile row): once the MMAs of the last group are done with the
                        // region, load this unit's A slabs into it
                        ++ag;
                        if (!mbar_wait(a_empty, static_cast<uint32_t>(ag & 1) ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        mbar_arrive_expect_tx(a_full, static_cast<uint32_t>(pr.nslab) * A_TILE);
                        for (int j = 0; j < pr.nslab; ++j)
                            tma_load_3d(smem + j * A_TILE, mapA, a_full, (pr.slab0 + j) * BK, tm * BM, lm);
                        a_armed = ag;
                        a_lm = lm;
                        a_tm = tm;
                    }
                }

                for (int d = MOD ? 2 : pr.S + 1; d >= 2 && ok; --d) {
                    const int npairs = MOD ? 1 : d - 1;
                    for (int s = 1; s <= npairs && ok; ++s) {
                        const int plane_a = MOD ? lm : s - 1;
                        const int plane_b = MOD ? plane_a : d - s - 1;
                        for (int j = 0; j < pr.nslab; ++j) {
                            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
                                ok = false;
                                break;
                            }
                            uint8_t* sa = ring + stage * STAGE;
                            mbar_arrive_expect_tx(&full[stage], STAGE);
                            const int x = (pr.slab0 + j) * BK;
                            // A slice s rows [tm*BM, +BM), B slice d-s rows [tn*BN, +BN) (MOD: the
                            // residue planes of one modulus); rows past the end of a plane are
                            // zero-filled by the copy engine (AK: B only, A is in its region)
                            if (!withhold) {
                                if constexpr (!AK) tma_load_3d(sa, mapA, &full[stage], x, tm * BM, plane_a);
                                tma_load_3d(sa + B_OFF, mapB, &full[stage], x, tn * BN, plane_b);
                            }
                            withhold = false;  // (test hook: only the first stage stays empty)
                            last_phase[stage] = static_cast<int>(phase);
                            if (++stage == STAGES) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                    }
                }
            }
            if (!ok) {
                // let every issued copy land before the CTA's shared memory goes away
                for (int i = 0; i < STAGES; ++i)
                    if (last_phase[i] >= 0) mbar_wait_drain(&full[i], static_cast<uint32_t>(last_phase[i]));
                // (AK: and the A loads of the last group that issued any)
                if (AK && a_armed >= 0) mbar_wait_drain(a_full, static_cast<uint32_t>(a_armed & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t stage = 0, phase = 0;
            uint32_t abuf = 0;
            uint32_t aphase[2] = {0u, 0u};
            bool ok = true;
            bool issued = false;
            int ag = -1, a_lm = -1, a_tm = -1;  // AK: as the producer's
            for (int it = 0; ok; ++it) {
                int tm, tn, prob, part, lm = 0;
                if (!tile_of<TAIL, MOD>(p, it, &prob, &tm, &tn, &part, &lm)) break;
                TileInts pr = tile_ints(p, prob, part);
                if constexpr (MOD) apply_kcap<BN>(p, tm, tn, pr);
                if constexpr (AK) {
                    if (lm != a_lm || tm != a_tm) {
                        ++ag;
                        // the A region goes back to the producer once every MMA issued so far is done
                        if (ag > 0) umma_commit(a_empty);
                        if (!mbar_wait(a_full, static_cast<uint32_t>(ag & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        a_lm = lm;
                        a_tm = tm;
                    }
                }
                for (int d = MOD ? 2 : pr.S + 1; d >= 2 && ok; --d) {
                    const int units = (MOD ? 1 : d - 1) * pr.nslab;
                    for (int u = 0; u < units && ok;) {
                        const int cnt = min(pr.chunk_slabs, units - u);
                        if (!mbar_wait(&acc_empty[abuf], aphase[abuf] ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = tmem_base + abuf * 256u;
                        for (int c = 0; c < cnt; ++c) {
                            if (!mbar_wait(&full[stage], phase, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t sa = smem_u32(ring + stage * STAGE);
                            const uint64_t da = smem_desc_k_sw128(AK ? smem_u32(smem + (u + c) * A_TILE) : sa);
                            const uint64_t db = smem_desc_k_sw128(sa + B_OFF);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                umma_f16_ss(dt, da + 2ull * kk, db + 2ull * kk, C_::IDESC,
                                            static_cast<uint32_t>((c | kk) != 0));
                            issued = true;
                            umma_commit(&empty[stage]);
                            if (++stage == STAGES) {
                                stage = 0;
                                phase ^= 1u;
                            }
                        }
                        umma_commit(&acc_full[abuf]);
                        aphase[abuf] ^= 1u;
                        abuf ^= 1u;
                        u += cnt;
                    }
                }
            }
            if (!ok && issued) {
                // wait for every MMA issued so far before TMEM is released
                umma_commit(drain);
                mbar_wait_drain(drain, 0);
            }
        }
    } else if (warp >= CTRL_WARPS) {
        // ------------------------------------------------------------ drain + recombination
        // Each drain thread owns one row and CW = 64 columns of the tile.  The int32
        // diagonal sums of the first CR = 32 columns live in registers; those of the
        // other CT = 32 columns live in TMEM columns the accumulators do not use
        // (192..255 and 448..511), which keeps the thread clear of register spills.
        constexpr int CR = C_::CR, CT = C_::CT;
        const int quad = warp & 3;                         // TMEM lanes this warp may read: 32*quad ..
        const int third = (warp - CTRL_WARPS) >> 2;        // columns [CW*third, CW*third + CW)
        const int rloc = quad * 32 + lane;                 // row within the tile
        const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
        // wide tile: half the int32 sums in TMEM columns 192..255 / 448..511; narrow tile: the int64
        // group sums Q in TMEM columns 96..223 / 352..415 (64 per third: low and high words)
        const uint32_t tsum = C_::QT ? tmem_base + lane_off + (third < 2 ? 96u + 64u * third : 352u)
                                     : tmem_base + lane_off + (third < 2 ? 192u + 32u * third : 448u);
        uint32_t abuf = 0;
        uint32_t aphase[2] = {0u, 0u};
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        long long* Q = p.qscratch + (static_cast<size_t>(blockIdx.x) * BN + third * CW) * BM + rloc;
        double* R = p.scratch + (static_cast<size_t>(blockIdx.x) * BN + third * CW) * BM + rloc;
        const uint64_t keep = l2_policy_evict_last();
        if constexpr (TAIL) {
            int tm, tn, prob, part;
            if (tile_of<true>(p, 0, &prob, &tm, &tn, &part))
                drain_tail_unit<BN>(p, tn, part, acc_full, acc_empty, abuf, aphase[0], aphase[1], abort_flag,
                                    tmem_base + lane_off + third * CW, tsum, lane, third, rloc);
        } else {
            bool ok = true;
            for (int it = 0; ok; ++it) {
                int tm, tn, prob, part, lm = 0;
                int64_t tile = 0;
                if (!tile_of<false, MOD>(p, it, &prob, &tm, &tn, &part, &lm, &tile)) break;
                TileInts pr = tile_ints(p, prob, -1);
                if constexpr (MOD) apply_kcap<BN>(p, tm, tn, pr);
                const double rb = pow2_normal(-pr.beta);
                int gj = 0;           // position of the current diagonal inside its int64 group
                bool rfirst = true;   // no FP64 partial R yet for this tile
                const bool final_unit = MOD && p.crt_fused && lm == pr.S - 1;
                if constexpr (!MOD) stage_columns<BN>(p, prob, tn, pr.beta, colexp, colflag);
                else if (final_unit) {
                    stage_columns<BN>(p, prob, tn, p.crt_bits, colexp, colflag);
                    prefetch_residues<BN>(p, tm, tn, lm, third, quad, lane);
                }
                if constexpr (AK) {
                    if (!drain_store_small<BN>(p, tm, tn, lm, third, rloc, lane, acc_full, acc_empty, abuf, aphase,
                                               abort_flag, tmem_base + lane_off + third * CW)) {
                        ok = false;
                        break;
                    }
                } else {
                    for (int d = MOD ? 2 : pr.S + 1; d >= 2; --d) {
                        int32_t acc[CR];
                        if (!drain_diagonal<CR, CT>((MOD ? 1 : d - 1) * pr.nslab, pr.chunk_slabs, acc_full, acc_empty,
                                                    abuf, aphase, abort_flag, tmem_base + lane_off + third * CW, tsum,
                                                    lane, acc)) {
                            ok = false;
                            break;
                        }
                        if constexpr (MOD) {
                            if (!final_unit) {
                                store_residues<BN, CR, CT>(p, prob, tm, tn, lm, third, rloc, acc, tsum);
                                if (p.crt_fused) signal_tile(p, tile);
                            } else if (wait_tile(p, tile, pr.S - 1, abort_flag, wait_ok)) {
                                if (p.crt_L == 3)
                                    crt_final<BN, CR, CT, 3>(p, tm, tn, lm, third, rloc, acc, tsum, colexp, colflag);
                                else
                                    crt_final<BN, CR, CT, 4>(p, tm, tn, lm, third, rloc, acc, tsum, colexp, colflag);
                            } else {
                                ok = false;
                                break;
                            }
                        } else
                            recombine_diagonal<BN, CR, CT>(p, prob, tm, tn, d, pr, Q, R, keep, tsum, rb, third, rloc,
                                                           colexp, colflag, qnan, acc, gj, rfirst);
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status, kStatusTimeout);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- residue product on CTA pairs
// The modular encoding's residue product with the tensor cores of two SMs per MMA
// (tcgen05.mma.cta_group::2, M = 256): a cluster of two CTAs takes a 256 x 192 tile of one
// modulus; each CTA stages its own 128 rows of A and its own 96 of the tile's 192 B rows, so per
// MMA flop a CTA's shared memory is written by TMA and read by the tensor core 30 % less than with
// one CTA per 128 x 192 tile (28 instead of 40 KB per 64-deep slab), and L2 sends 30 % fewer bytes
// per flop.  The even CTA (leader) issues the MMAs; each CTA receives its 128 rows of the
// accumulator in its own tensor memory and drains, reduces and stores them as in slice_gemm_kernel.
//
// Barriers.  Each CTA's producer fills its own stage and completes its own full barrier; the
// peer's warp 1 forwards each completed stage to the leader's full barrier (count 2: the leader's
// own arrival plus the forward), so the leader's MMA thread waits on one barrier for both halves.
// The leader's commits release the stage (empty) and hand over the accumulator (acc_full) in both
// CTAs; both CTAs' drain warps arrive on the leader's acc_empty.  All waits are bounded; a CTA that
// gives up raises its abort flag, the other one's waits then run out too, and both wait for their
// own copies (and the leader for its MMAs) before the closing cluster barrier frees tensor memory.
namespace pairk {
constexpr int BN = kEmuBNMax;                       // 192 columns per pair tile
constexpr int BNH = BN / 2;                         // B rows staged per CTA
constexpr uint32_t B_HALF = BNH * BK * 2;           // 12 KB
constexpr uint32_t STAGE = A_TILE + B_HALF;         // 28 KB
constexpr int STAGES = 7;
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE + 256 + 5 * BN;
constexpr uint32_t IDESC = idesc_f16_f32(2 * BM, BN);
static_assert(STAGE % 1024 == 0, "stage bases stay 1024-byte aligned for the 128-B swizzle");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");

// Unit `it` of this pair: modulus lm of pair tile (tm2, tn); p.tiles_m counts pair rows.
MOMMS_DEV bool unit_of(const Params& p, int it, int* lm, int* tm2, int* tn) {
    const int64_t ncl = gridDim.x >> 1, cl = blockIdx.x >> 1;
    const int64_t tiles = static_cast<int64_t>(p.tiles_m) * p.tiles_n;
    const int64_t u = cl + static_cast<int64_t>(it) * ncl;
    if (u >= tiles * one_S(p)) return false;
    *lm = static_cast<int>(u / tiles);
    const int64_t t = u - *lm * tiles;
    const int member = p.member == kMemberA1 ? kMemberA2 : p.member;
    return member_tile(member, p.group, t % ncl, ncl, t / ncl, p.tiles_m, p.tiles_n, tm2, tn);
}
}  // namespace pairk

__global__ void __launch_bounds__(THREADS, 1)
    residue_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                        const __grid_constant__ Params p) {
    using namespace pairk;
    using C_ = Cfg<BN>;
    constexpr int CR = C_::CR, CT = C_::CT, CW = C_::CW;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
    uint64_t* full = bars;                        // STAGES
    uint64_t* empty = bars + STAGES;              // STAGES
    uint64_t* acc_full = bars + 2 * STAGES;       // 2
    uint64_t* acc_empty = bars + 2 * STAGES + 2;  // 2 (the leader's count both CTAs' drain warps)
    uint64_t* drain = bars + 2 * STAGES + 4;      // 1
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], leader ? 2 : 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], 2 * EPI_WARPS);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbarrier_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(tmem_slot, TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // both CTAs' barriers are initialised before any remote arrive or commit
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer (both CTAs)
        if (lane == 0) {
            prefetch_tensormap(&tmA);
            prefetch_tensormap(&tmB);
            uint32_t stage = 0, phase = 0;
            int last_phase[STAGES];
            for (int i = 0; i < STAGES; ++i) last_phase[i] = -1;
            bool ok = true;
            bool withhold = p.withhold != 0 && blockIdx.x == 0;
            const int nslab = p.one.nslab, slab0 = p.one.slab0;
            for (int it = 0; ok; ++it) {
                int lm, tm2, tn;
                if (!unit_of(p, it, &lm, &tm2, &tn)) break;
                for (int j = 0; j < nslab; ++j) {
                    // the peer's stages are released by the leader's commits
                    const bool freed = leader ? mbar_wait(&empty[stage], phase ^ 1u, abort_flag)
                                              : mbar_wait_cluster(&empty[stage], phase ^ 1u, abort_flag);
                    if (!freed) {
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + stage * STAGE;
                    mbar_arrive_expect_tx(&full[stage], STAGE);
                    const int x = (slab0 + j) * BK;
                    // this CTA's 128 rows of A and 96 rows of B (rows past a plane's end read as zero)
                    if (!withhold) {
                        tma_load_3d_cta(sa, &tmA, &full[stage], x, (2 * tm2 + static_cast<int>(rank)) * BM, lm);
                        tma_load_3d_cta(sa + A_TILE, &tmB, &full[stage], x, tn * BN + static_cast<int>(rank) * BNH,
                                        lm);
                    }
                    withhold = false;  // (test hook: only the first stage stays empty)
                    last_phase[stage] = static_cast<int>(phase);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                for (int i = 0; i < STAGES; ++i)
                    if (last_phase[i] >= 0) mbar_wait_drain(&full[i], static_cast<uint32_t>(last_phase[i]));
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            // -------------------------------------------------------- MMA issuer (leader)
            const uint32_t peer_empty = cluster_addr(empty, 1);
            const uint32_t peer_acc_full = cluster_addr(acc_full, 1);
            uint32_t stage = 0, phase = 0, abuf = 0;
            uint32_t aphase[2] = {0u, 0u};
            bool ok = true, issued = false;
            const int nslab = p.one.nslab, chunk = p.one.chunk_slabs;
            for (int it = 0; ok; ++it) {
                int lm, tm2, tn;
                if (!unit_of(p, it, &lm, &tm2, &tn)) break;
                for (int u = 0; u < nslab && ok;) {
                    const int cnt = min(chunk, nslab - u);
                    if (!mbar_wait_cluster(&acc_empty[abuf], aphase[abuf] ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + abuf * 256u;
                    for (int c = 0; c < cnt; ++c) {
                        if (!mbar_wait_cluster(&full[stage], phase, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(smem + stage * STAGE);
                        const uint64_t da = smem_desc_k_sw128(sa);
                        const uint64_t db = smem_desc_k_sw128(sa + A_TILE);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk)
                            umma_f16_ss_pair(dt, da + 2ull * kk, db + 2ull * kk, IDESC,
                                             static_cast<uint32_t>((c | kk) != 0));
                        issued = true;
                        umma_commit_pair(smem_u32(&empty[stage]));
                        umma_commit_pair(peer_empty + 8u * stage);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    umma_commit_pair(smem_u32(&acc_full[abuf]));
                    umma_commit_pair(peer_acc_full + 8u * abuf);
                    aphase[abuf] ^= 1u;
                    abuf ^= 1u;
                    u += cnt;
                }
            }
            if (!ok && issued) {
                umma_commit_pair(smem_u32(drain));
                mbar_wait_drain(drain, 0);
            }
        } else if (lane == 0) {
            // -------------------------------------------------------- stage forwarder (peer)
            // every stage of this CTA that completes is announced on the leader's full barrier
            const uint32_t leader_full = cluster_addr(full, 0);
            uint32_t stage = 0, phase = 0;
            bool ok = true;
            const int nslab = p.one.nslab;
            for (int it = 0; ok; ++it) {
                int lm, tm2, tn;
                if (!unit_of(p, it, &lm, &tm2, &tn)) break;
                for (int j = 0; j < nslab; ++j) {
                    // polled: a suspended wait here was observed to hand each stage over about 0.9 us late
                    if (!mbar_wait_cluster(&full[stage], phase, abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(leader_full + 8u * stage);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
        }
    } else if (warp >= CTRL_WARPS) {
        // ------------------------------------------------------------ drain + residues (both CTAs)
        const int quad = warp & 3;
        const int third = (warp - CTRL_WARPS) >> 2;
        const int rloc = quad * 32 + lane;
        const uint32_t lane_off = static_cast<uint32_t>(quad * 32) << 16;
        const uint32_t tsum = tmem_base + lane_off + (third < 2 ? 192u + 32u * third : 448u);
        const uint32_t remote_empty = leader ? 0u : cluster_addr(acc_empty, 0);
        uint32_t abuf = 0;
        uint32_t aphase[2] = {0u, 0u};
        for (int it = 0;; ++it) {
            int lm, tm2, tn;
            if (!unit_of(p, it, &lm, &tm2, &tn)) break;
            int32_t acc[CR];
            if (!drain_diagonal<CR, CT>(p.one.nslab, p.one.chunk_slabs, acc_full, acc_empty, abuf, aphase,
                                        abort_flag, tmem_base + lane_off + third * CW, tsum, lane, acc, remote_empty,
                                        !leader))
                break;
            store_residues<BN, CR, CT>(p, -1, 2 * tm2 + static_cast<int>(rank), tn, lm, third, rloc, acc, tsum);
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();  // no CTA leaves while its peer may still arrive on its barriers or MMAs write its TMEM
    if (threadIdx.x == 0 && *abort_flag) atomicExch(p.status, kStatusTimeout);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------------------------ host side
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

static EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        fn = reinterpret_cast<EncodeFn>(ptr);
    }
    return fn;
}

}  // namespace emu

// 3-D fp16 digit tensor [S][rows][k_pad] (k contiguous), box 64 x box_rows x 1, 128-B swizzle.
bool emu_make_digit_map(CUtensorMap* map, const void* base, int64_t k_pad, int64_t rows, int S, int box_rows,
                        int64_t plane_rows, int64_t row_pitch) {
    using namespace emu;
    EncodeFn enc = get_encode();
    if (!enc) return false;
    // The map covers k_pad digits of `rows` rows from `base`; in memory a row is row_pitch digits
    // and a slice plane_rows rows (a block of rows or a range of k may start inside the tensor).
    if (plane_rows <= 0) plane_rows = rows;
    if (row_pitch <= 0) row_pitch = k_pad;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(k_pad), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(S)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(row_pitch) * 2,
                             static_cast<cuuint64_t>(row_pitch) * 2 * static_cast<cuuint64_t>(plane_rows)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, const_cast<void*>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

namespace emu {

// Tail split of a single-problem launch.  With a round-robin member the last round holds only
// tiles % ctas tiles; cutting each into `parts` k ranges (parts = ctas / that count, at most the
// slabs of the shortest pass) lets parts x as many CTAs share that round.
// Armed by momms_debug_withhold_load(); the next slice-product launch takes it (Params::withhold).
static std::atomic<int> g_withhold{0};

struct TailPlan {
    int full_rounds = 0, tiles = 0, parts = 0;
    size_t sums_bytes = 0;
};
static size_t align256_(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static TailPlan tail_plan(int64_t tiles, int64_t ctas, int64_t kslabs, int64_t pass_slabs, int S, int member) {
    TailPlan t;
    if (member == kMemberA1 || ctas <= 1 || kslabs <= 0 || pass_slabs <= 0) return t;
    const int64_t r = tiles % ctas;
    if (r == 0 || tiles < ctas) return t;
    const int64_t last_pass = kslabs - (kslabs - 1) / pass_slabs * pass_slabs;  // slabs of the shortest pass
    // One wave of parts only (r * parts <= ctas), and only when the saving clearly beats the
    // fixed cost of the two extra launches (launch gaps, pipeline fill, the fix-up pass: a few
    // tens of microseconds) -- a tile takes ~0.31 us per pair and k slab on the whole chip.
    int64_t best_p = ctas / r;
    if (best_p > last_pass) best_p = last_pass;
    const double tile_us = 0.31 * (S * (S + 1) / 2) * static_cast<double>(last_pass);
    if (best_p < 2 || tile_us * (1.0 - 1.0 / static_cast<double>(best_p)) < 60.0) return t;
    t.full_rounds = static_cast<int>(tiles / ctas);
    t.tiles = static_cast<int>(r);
    t.parts = static_cast<int>(best_p);
    t.sums_bytes = align256_(static_cast<size_t>(r) * best_p * S * kEmuBNMax * BM * sizeof(int32_t));
    return t;
}

template <int BN>
static cudaError_t launch_bn(const EmuGemmArgs& a, int* passes, cudaStream_t stream) {
    using C_ = Cfg<BN>;
    const int sms = device_sm_count();
    const int64_t tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
    // a triangular product visits the tiles that meet the triangle (modular encoding, m = n)
    if (a.tri && (a.crt == nullptr || a.crt_fuse != nullptr || a.m != a.n || 384 % BN != 0))
        return cudaErrorInvalidValue;
    const int64_t tiles = a.tri ? tri_prefix(a.tri == 1, tiles_m, static_cast<int>(tiles_n), BN) : tiles_m * tiles_n;
    const int64_t units = a.crt ? tiles * a.crt->N : tiles;  // modular encoding: one unit per modulus and tile
    int64_t ctas = a.max_ctas > 0 && a.max_ctas < sms ? a.max_ctas : sms;  // one CTA per SM at most
    if (ctas > units) ctas = units;
    const size_t half = static_cast<size_t>(ctas) * BN * BM * sizeof(double);
    if (a.scratch_bytes < 2 * half) return cudaErrorInvalidValue;
    // int64 group sums Q in the first half, FP64 partial sums R (several groups only) in the second

    CUtensorMap mapA, mapB;
    if (!emu_make_digit_map(&mapA, a.Ad, a.k_pad, a.m_pad, a.S, BM)) return cudaErrorInvalidValue;
    if (!emu_make_digit_map(&mapB, a.Bd, a.k_pad, a.n_pad, a.S, BN)) return cudaErrorInvalidValue;

    static PerDeviceFlag attr_set;  // idempotent; per device, atomic for concurrent first calls
    if (!attr_set.done()) {
        cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel<BN, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C_::SMEM_BYTES));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(slice_gemm_kernel<BN, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(C_::SMEM_BYTES));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(slice_gemm_kernel<BN, false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(C_::SMEM_BYTES));
        if (e != cudaSuccess) return e;
        attr_set.mark();
    }
    const bool mod = a.crt != nullptr;
    const int64_t kslabs = (a.k + BK - 1) / BK;
    // modular encoding: one pass (every k the moduli were planned for keeps the int32 sums exact)
    const int64_t pass_slabs = mod ? kslabs : emu_max_k_per_pass(a.S, a.beta) / BK;
    if (kslabs <= 0 || pass_slabs <= 0) return cudaErrorInvalidValue;
    if (mod && (a.res == nullptr || a.crt->N != a.S || kslabs * BK > crt_max_k())) return cudaErrorInvalidValue;
    const int member = a.member == kMemberAuto ? kMemberC2 : a.member;
    // (with a device plan the digit launch keeps whole tiles: the tail split is planned for one S)
    TailPlan tp = BN == kEmuBNMax && !mod && !a.plan ? tail_plan(tiles, ctas, kslabs, pass_slabs, a.S, member)
                                                     : TailPlan{};
    if (tp.parts && a.scratch_bytes < 2 * half + tp.sums_bytes) tp = TailPlan{};  // whole tiles
    char* tail_base = static_cast<char*>(a.scratch) + 2 * half;
    int npass = 0, nlaunch = 0;
    for (int64_t s0 = 0; s0 < kslabs; s0 += pass_slabs) {
        Params p{};
        p.one.m = static_cast<int>(a.m);
        p.one.n = static_cast<int>(a.n);
        p.one.S = a.S;
        p.one.beta = a.beta;
        p.one.chunk_slabs = emu_chunk_slabs(a.beta);
        p.one.slab0 = static_cast<int>(s0);
        p.one.nslab = static_cast<int>(kslabs - s0 < pass_slabs ? kslabs - s0 : pass_slabs);
        p.one.group_end = emu_group_ends(a.S, a.beta, p.one.nslab * static_cast<int64_t>(BK));
        p.one.e = a.e;
        p.one.ef = a.ef;
        p.one.f = a.f;
        p.one.ff = a.ff;
        p.one.alpha = a.alpha;
        p.one.beta_c = npass == 0 ? a.beta_c : 1.0;
        p.one.C = a.C;
        p.one.ldc = a.ldc;
        p.tiles_m = static_cast<int>(tiles_m);
        p.tiles_n = static_cast<int>(tiles_n);
        p.member = member;
        p.group = a.group > 0 ? a.group : emu_default_group(ctas, static_cast<int>(tiles_m), static_cast<int>(tiles_n));
        if (tp.parts) {
            p.full_rounds = tp.full_rounds;
            p.main_ctas = static_cast<int>(ctas);
            p.tail_tiles = tp.tiles;
            p.tail_parts = tp.parts;
            p.tail_sums = reinterpret_cast<int32_t*>(tail_base);
        }
        if (a.used_ctas) *a.used_ctas = static_cast<int>(ctas);
        if (a.used_group) *a.used_group = p.group;
        p.table = nullptr;
        // unit indices below 2^31 (blockIdx + it ctas stays below tiles N + ctas): 32-bit decoding
        if (tiles_m * tiles_n * kCrtMaxModuli + ctas < (int64_t(1) << 31)) {
            p.u32dec = 1;
            for (int q = 1; q <= 16; ++q) p.fd_n[q] = make_fastdiv(static_cast<uint32_t>(q));
            p.tdv = make_tilediv(p.group, static_cast<int>(tiles_m), static_cast<int>(tiles_n));
        }
        p.withhold = a.withhold > 0 ? 1 : g_withhold.exchange(0);
        if (a.plan) {
            // S or N from the device plan; the pass above was sized for the largest the plan may pick
            p.plan = a.plan;
            p.plan_kind = mod ? 1 : 2;
            for (int q = 1; q <= 16; ++q)
                p.group_end_by_s[q] = emu_group_ends(q, a.beta, p.one.nslab * static_cast<int64_t>(BK));
        }
        p.qscratch = static_cast<long long*>(a.scratch);
        p.scratch = reinterpret_cast<double*>(static_cast<char*>(a.scratch) + half);
        p.status = a.status;
        if (mod) {
            p.res = a.res;
            // Separate reconstruction: one group, modulus-major over all tiles (consecutive waves of
            // the same modulus reuse operand panels in L2).  Fused: groups of four waves' tiles keep a
            // tile's moduli on one CTA and spread the last-modulus epilogues over the launch, while
            // four consecutive waves still share a modulus (groups of one wave's tiles lost that reuse:
            // 8.3 -> 10.9 ms at 8192^3)
            p.group_tiles = a.crt_fuse ? static_cast<int>(std::min<int64_t>(tiles, 4 * ctas)) : static_cast<int>(tiles);
            p.fd_gt = make_fastdiv(static_cast<uint32_t>(p.group_tiles));
            p.fd_gt_last = make_fastdiv(static_cast<uint32_t>(tiles % p.group_tiles == 0 ? p.group_tiles
                                                                                        : tiles % p.group_tiles));
            if (a.crt_fuse) {
                if (a.done == nullptr || a.crt_fuse->N != a.crt->N) return cudaErrorInvalidValue;
                p.crt_fused = 1;
                p.done = a.done;
                p.crt_bits = a.crt_fuse->bits;
                p.crt_L = a.crt_fuse->Pw[3] == 0 ? 3 : 4;
                for (int l = 0; l < a.crt->N; ++l) {
                    for (int q = 0; q < 4; ++q) p.crt_w[l][q] = a.crt_fuse->w[l][q];
                    p.crt_F[l] = a.crt_fuse->frac[l];
                }
                for (int q = 0; q < 4; ++q) p.crt_Pw[q] = a.crt_fuse->Pw[q];
            }
            for (int l = 0; l < a.crt->N; ++l) {
                const uint32_t pl = a.crt->p[l];
                p.modp[l] = pl;
                p.modmagic[l] = a.crt->magic[l];
                p.modoff[l] = static_cast<uint32_t>(pl * (((1ull << 31) + pl - 1) / pl));
                p.modmagic_up[l] = static_cast<uint32_t>(((1ull << 32) + pl - 1) / pl);
                p.modoff22[l] = static_cast<uint32_t>(pl * (((1ull << 22) + pl - 1) / pl));
            }
            if (a.tri) {
                p.tri = a.tri;
                p.tri_bn = BN;
                p.tri_tiles = tiles;
            }
            if (a.kcap < 0 || a.kcap > 4) return cudaErrorInvalidValue;
            p.kcap = a.kcap;
            cudaError_t e;
            const int64_t pair_rows = (tiles_m + 1) / 2;
            if (BN == kEmuBNMax && a.cta_pairs && !a.crt_fuse && !a.tri && !a.kcap && tiles_m >= 2 && ctas >= 4) {
                // CTA pairs over 256 x 192 tiles: B staged as two 96-row halves, one per CTA
                CUtensorMap mapBh;
                if (!emu_make_digit_map(&mapBh, a.Bd, a.k_pad, a.n_pad, a.S, pairk::BNH)) return cudaErrorInvalidValue;
                static PerDeviceFlag pair_attr;
                if (!pair_attr.done()) {
                    e = cudaFuncSetAttribute(residue_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(pairk::SMEM_BYTES));
                    if (e != cudaSuccess) return e;
                    pair_attr.mark();
                }
                // as many pairs as can be resident at once (a GPC with an odd SM count leaves one SM out)
                static std::atomic<int> resident[kMaxDevices] = {};
                const int dev = current_device();
                int max_cl = dev >= 0 && dev < kMaxDevices ? resident[dev].load() : 0;
                if (max_cl <= 0) {
                    cudaLaunchConfig_t q{};
                    q.gridDim = dim3(static_cast<unsigned>(2 * (sms / 2)));
                    q.blockDim = dim3(THREADS);
                    q.dynamicSmemBytes = pairk::SMEM_BYTES;
                    cudaLaunchAttribute qa[1];
                    qa[0].id = cudaLaunchAttributeClusterDimension;
                    qa[0].val.clusterDim.x = 2;
                    qa[0].val.clusterDim.y = 1;
                    qa[0].val.clusterDim.z = 1;
                    q.attrs = qa;
                    q.numAttrs = 1;
                    if (cudaOccupancyMaxActiveClusters(&max_cl, residue_pair_kernel, &q) != cudaSuccess || max_cl <= 0) {
                        cudaGetLastError();
                        max_cl = sms / 2;
                    }
                    if (dev >= 0 && dev < kMaxDevices) resident[dev].store(max_cl);
                }
                const int64_t ncl = std::min<int64_t>({ctas / 2, static_cast<int64_t>(max_cl),
                                                       pair_rows * tiles_n * a.crt->N});
                p.tiles_m = static_cast<int>(pair_rows);
                p.group = a.group > 0 ? a.group : emu_default_group(ncl, static_cast<int>(pair_rows),
                                                                     static_cast<int>(tiles_n));
                p.group_tiles = static_cast<int>(pair_rows * tiles_n);
                if (a.used_ctas) *a.used_ctas = static_cast<int>(2 * ncl);
                if (a.used_group) *a.used_group = p.group;
                if (a.used_pairs) *a.used_pairs = 1;
                cudaLaunchConfig_t cfg{};
                cfg.gridDim = dim3(static_cast<unsigned>(2 * ncl));
                cfg.blockDim = dim3(THREADS);
                cfg.dynamicSmemBytes = pairk::SMEM_BYTES;
                cfg.stream = stream;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = 2;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelEx(&cfg, residue_pair_kernel, mapA, mapBh, p);
            } else {
                bool kept = false;
                if constexpr (BN == kEmuBNMax) {
                    // (the fused drain stores four rows to a word: m a multiple of 4)
                    if (!a.crt_fuse && !a.tri && !a.kcap && p.u32dec && p.one.nslab <= AK_SLABS && tiles >= ctas &&
                        a.m % 4 == 0 && (reinterpret_cast<uintptr_t>(a.res) & 3) == 0 &&
                        ctas * tiles < (int64_t(1) << 32)) {
                        // short k: the kept-A order and kernel (each CTA loads its A tile once per tile
                        // row of its strip and modulus)
                        static PerDeviceFlag ak_attr;
                        if (!ak_attr.done()) {
                            e = cudaFuncSetAttribute(slice_gemm_kernel<BN, false, true, true>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     static_cast<int>(AK_SMEM_BYTES));
                            if (e != cudaSuccess) return e;
                            ak_attr.mark();
                        }
                        p.akeep = 1;
                        p.fd_ctas = make_fastdiv(static_cast<uint32_t>(ctas));
                        p.fd_len = make_fastdiv(static_cast<uint32_t>(tiles / ctas));
                        p.fd_len1 = make_fastdiv(static_cast<uint32_t>(tiles / ctas + 1));
                        slice_gemm_kernel<BN, false, true, true>
                            <<<static_cast<unsigned>(ctas), THREADS, AK_SMEM_BYTES, stream>>>(mapA, mapB, p);
                        e = cudaGetLastError();
                        kept = true;
                    }
                }
                if (!kept) {
                    slice_gemm_kernel<BN, false, true><<<static_cast<unsigned>(ctas), THREADS, C_::SMEM_BYTES, stream>>>(
                        mapA, mapB, p);
                    e = cudaGetLastError();
                }
            }
            if (e != cudaSuccess) return e;
            ++nlaunch;
            ++npass;
            continue;
        }
        // main launch: the whole rounds (all tiles without a tail split)
        slice_gemm_kernel<BN, false><<<static_cast<unsigned>(ctas), THREADS, C_::SMEM_BYTES, stream>>>(mapA, mapB, p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++nlaunch;
        p.withhold = 0;  // the test hook acts on the first launch only
        if (tp.parts) {
            // tail launch: one CTA per k part of every tile of the last, partial round ...
            slice_gemm_kernel<BN, true><<<static_cast<unsigned>(tp.tiles * tp.parts), THREADS, C_::SMEM_BYTES,
                                          stream>>>(mapA, mapB, p);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            // ... and the fix-up: sum of the parts and recombination, one thread per row x 8 columns
            const int64_t threads = static_cast<int64_t>(tp.tiles) * BM * (kEmuBNMax / 8);
            tail_fixup_kernel<<<static_cast<unsigned>((threads + 255) / 256), 256, 0, stream>>>(p);
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            nlaunch += 2;
        }
        ++npass;
    }
    if (passes) *passes = npass;
    if (a.used_launches) *a.used_launches = nlaunch;
    return cudaSuccess;
}

template <int BN>
static cudaError_t launch_bn_batched(const EmuBatchProblem* table, int count, int64_t total_tiles, void* scratch,
                                     size_t scratch_bytes, int32_t* status, cudaStream_t stream,
                                     const int64_t* total_dev) {
    using C_ = Cfg<BN>;
    int64_t ctas = device_sm_count();
    if (ctas > total_tiles) ctas = total_tiles;  // (with total_dev: an upper bound of the total)
    const size_t half = static_cast<size_t>(ctas) * BN * BM * sizeof(double);
    if (scratch_bytes < 2 * half) return cudaErrorInvalidValue;
    static PerDeviceFlag attr_set;  // idempotent; per device, atomic for concurrent first calls
    if (!attr_set.done()) {
        cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel<BN, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C_::SMEM_BYTES));
        if (e != cudaSuccess) return e;
        attr_set.mark();
    }
    Params p{};
    p.table = table;
    p.count = count;
    p.total_tiles = total_tiles;
    p.total_dev = total_dev;
    p.withhold = g_withhold.exchange(0);
    p.qscratch = static_cast<long long*>(scratch);
    p.scratch = reinterpret_cast<double*>(static_cast<char*>(scratch) + half);
    p.status = status;
    CUtensorMap unused{};  // the batch reads each problem's maps from the table
    slice_gemm_kernel<BN, false><<<static_cast<unsigned>(ctas), THREADS, C_::SMEM_BYTES, stream>>>(unused, unused, p);
    return cudaGetLastError();
}

// The residue products of a batch: one persistent launch over every problem's (modulus, tile)
// units; the epilogue stores each problem's residues in its own planes.
template <int BN>
static cudaError_t launch_bn_batched_mod(const EmuBatchProblem* table, int count, int64_t total_units,
                                         const CrtConsts& c, void* scratch, size_t scratch_bytes, int32_t* status,
                                         cudaStream_t stream, const int64_t* total_dev) {
    using C_ = Cfg<BN>;
    int64_t ctas = device_sm_count();
    if (ctas > total_units) ctas = total_units;
    const size_t half = static_cast<size_t>(ctas) * BN * BM * sizeof(double);
    if (scratch_bytes < 2 * half) return cudaErrorInvalidValue;
    static PerDeviceFlag attr_set;  // idempotent; per device, atomic for concurrent first calls
    if (!attr_set.done()) {
        cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel<BN, false, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C_::SMEM_BYTES));
        if (e != cudaSuccess) return e;
        attr_set.mark();
    }
    Params p{};
    p.table = table;
    p.count = count;
    p.total_tiles = total_units;
    p.total_dev = total_dev;
    p.withhold = g_withhold.exchange(0);
    p.qscratch = static_cast<long long*>(scratch);
    p.scratch = reinterpret_cast<double*>(static_cast<char*>(scratch) + half);
    p.status = status;
    for (int l = 0; l < c.N; ++l) {
        const uint32_t pl = c.p[l];
        p.modp[l] = pl;
        p.modmagic[l] = c.magic[l];
        p.modoff[l] = static_cast<uint32_t>(pl * (((1ull << 31) + pl - 1) / pl));
    }
    CUtensorMap unused{};
    slice_gemm_kernel<BN, false, true><<<static_cast<unsigned>(ctas), THREADS, C_::SMEM_BYTES, stream>>>(unused, unused,
                                                                                                      p);
    return cudaGetLastError();
}

}  // namespace emu

cudaError_t launch_emu_residue_gemm_batched(const EmuBatchProblem* dev_table, int count, int64_t total_units,
                                            const CrtConsts& c, void* scratch, size_t scratch_bytes,
                                            int32_t* status, cudaStream_t stream, const int64_t* total_dev) {
    if (count <= 0 || total_units <= 0) return cudaSuccess;
    if (c.N < 1 || c.N > kCrtMaxModuli) return cudaErrorInvalidValue;
    return emu::launch_bn_batched_mod<192>(dev_table, count, total_units, c, scratch, scratch_bytes, status, stream,
                                           total_dev);
}

cudaError_t launch_emu_slice_gemm_batched(const EmuBatchProblem* dev_table, int count, int64_t total_tiles,
                                          void* scratch, size_t scratch_bytes, int32_t* status,
                                          cudaStream_t stream, const int64_t* total_dev) {
    if (count <= 0 || total_tiles <= 0) return cudaSuccess;
    return emu::launch_bn_batched<192>(dev_table, count, total_tiles, scratch, scratch_bytes, status, stream,
                                       total_dev);
}

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return dev;
}

int device_sm_count() {
    // looked up once per device ordinal, thread-safely (a racing first call stores the same value)
    static std::atomic<int> sms[kMaxDevices] = {};
    const int dev = current_device();
    if (dev >= 0 && dev < kMaxDevices) {
        const int v = sms[dev].load(std::memory_order_relaxed);
        if (v > 0) return v;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) cudaGetLastError();
    n = n > 0 ? n : 1;
    if (dev >= 0 && dev < kMaxDevices) sms[dev].store(n, std::memory_order_relaxed);
    return n;
}

size_t emu_scratch_bytes(int num_sms) { return emu_scratch_bytes_for_ctas(num_sms); }

size_t emu_scratch_bytes_tail(int64_t m, int64_t n, int64_t k, int S, int max_ctas, int beta) {
    const int sms = device_sm_count();
    const int64_t tiles = ((m + emu::BM - 1) / emu::BM) * ((n + kEmuBNMax - 1) / kEmuBNMax);
    int64_t ctas = max_ctas > 0 && max_ctas < sms ? max_ctas : sms;
    if (ctas > tiles) ctas = tiles;
    if (ctas < 1) ctas = 1;
    // the recombination blocks for every SM (what momms_emu_slice_gemm requires), whatever the grid
    const size_t base = emu_scratch_bytes_for_ctas(sms);
    const int64_t kslabs = (k + emu::BK - 1) / emu::BK;
    const int64_t pass_slabs = emu_max_k_per_pass(S, beta) / emu::BK;
    const emu::TailPlan tp = emu::tail_plan(tiles, ctas, kslabs, pass_slabs, S, kMemberC2);
    return base + tp.sums_bytes;
}

size_t emu_scratch_bytes_for_ctas(int ctas) {
    // FP64 partial sums R and int64 group sums Q, one 128 x 192 block each per CTA
    return 2 * static_cast<size_t>(ctas) * kEmuBNMax * emu::BM * sizeof(double);
}

int64_t emu_max_k_per_pass(int S, int beta) {
    const int64_t dmax = (1ll << beta) - 1;
    int64_t kmax = ((1ll << 31) - 1) / (dmax * dmax * S);
    kmax -= kmax % emu::BK;
    return kmax;
}

int emu_chunk_slabs(int beta) {
    const int64_t dmax = (1ll << beta) - 1;
    int64_t prods = (1ll << 24) / (dmax * dmax);
    int slabs = static_cast<int>(prods / emu::BK);
    return slabs < 1 ? 1 : slabs;
}

// Tile width: an explicit request of 96 or 192, else the narrow tile only when the wide tiles
// (times the units per tile: the moduli of the modular encoding) are fewer than the SMs (the
// narrow ones then put more of the chip to work; measured: 1024^3 +28 %).  With enough wide tiles the narrow one loses -- twice the tiles' fixed costs and 40 %
// more operand traffic per flop (rank-k 16384 x 16384 x 256: -10 %, panel: -16 %).
int emu_pick_bn(int64_t m, int64_t n, int64_t, int requested, int units_per_tile) {
    if (requested == 96 || requested == 192) return requested;
    const int64_t wide_units = ((m + emu::BM - 1) / emu::BM) * ((n + kEmuBNMax - 1) / kEmuBNMax) * units_per_tile;
    return wide_units < device_sm_count() ? 96 : 192;
}

// The C2 group (tile rows of the block of C one wave covers) with the fewest operand rows
// read over all waves: a wave of `ctas` consecutive tiles of the raster reads the A rows of
// its distinct tile rows and the B rows of its distinct tile columns once per unit of k
// (Resident C at the L2 level, Sec. 2.2.1).  The continuous optimum r = sqrt(ctas*BN/BM)
// ignores waves that straddle two groups, so the candidates around it are counted exactly.
int emu_default_group(int64_t ctas, int tiles_m, int tiles_n) {
    if (tiles_m <= 1 || tiles_n <= 0 || ctas <= 1) return 1;
    static std::mutex mu;
    static std::map<std::tuple<int64_t, int, int>, int> cache;
    const auto key = std::make_tuple(ctas, tiles_m, tiles_n);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const int64_t total = static_cast<int64_t>(tiles_m) * tiles_n;
    const int r0 = static_cast<int>(std::sqrt(static_cast<double>(ctas) * kEmuBNMax / kEmuBM));
    const int lo = std::max(1, r0 / 2), hi = std::min(tiles_m, std::max(1, 2 * r0 + 1));
    std::vector<int64_t> row_seen(tiles_m), col_seen(tiles_n);
    int best = std::min(std::max(1, r0), tiles_m);
    int64_t best_cost = -1;
    for (int r = lo; r <= hi; ++r) {
        std::fill(row_seen.begin(), row_seen.end(), -1);
        std::fill(col_seen.begin(), col_seen.end(), -1);
        int64_t cost = 0;
        for (int64_t t = 0; t < total; ++t) {
            const int64_t wave = t / ctas;
            int tm, tn;
            member_tile(kMemberC2, r, t % ctas, ctas, wave, tiles_m, tiles_n, &tm, &tn);
            if (row_seen[tm] != wave) { row_seen[tm] = wave; cost += kEmuBM; }
            if (col_seen[tn] != wave) { col_seen[tn] = wave; cost += kEmuBNMax; }
        }
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = r; }
    }
    std::lock_guard<std::mutex> g(mu);
    cache[key] = best;
    return best;
}

void emu_debug_withhold_load() { emu::g_withhold.store(1); }
int emu_debug_take_withhold() { return emu::g_withhold.exchange(0); }

cudaError_t launch_emu_slice_gemm(const EmuGemmArgs& a, int* passes, cudaStream_t stream) {
    using namespace emu;
    if (passes) *passes = 0;
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    if (a.S < 1 || a.S > 16 || a.beta < 1 || a.beta > 8) return cudaErrorInvalidValue;
    if (a.crt && (a.beta != 7 || a.crt->N < 1 || a.crt->N > kCrtMaxModuli)) return cudaErrorInvalidValue;
    if (a.m_pad < a.m || a.n_pad < a.n || a.k_pad < a.k || a.k_pad % BK) return cudaErrorInvalidValue;
    if (emu_chunk_slabs(a.beta) * BK * ((1ll << a.beta) - 1) * ((1ll << a.beta) - 1) > (1ll << 24))
        return cudaErrorInvalidValue;  // beta too wide for one 64-wide slab per chunk
    if (a.m > (1ll << 30) || a.n > (1ll << 30)) return cudaErrorInvalidValue;
    if (emu_pick_bn(a.m, a.n, a.k, a.tile_n, a.crt ? a.crt->N : 1) == 96) return launch_bn<96>(a, passes, stream);
    return launch_bn<192>(a, passes, stream);
}

}  // namespace momms
