// internal.h -- launchers shared between the C-ABI layer and the kernel files.
#pragma once
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace momms {

// ---------------------------------------------------------------- native FP64
// C := alpha*op(A)*op(B) + beta*C on the FP64 DMMA tensor instructions.
// tri: 0 = all of C, 1 = lower triangle only (j <= i), 2 = upper only (j >= i); tiles wholly
// outside the triangle do no work.
cudaError_t launch_native_gemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               double beta, double* C, int64_t ldc, int member, int max_ctas,
                               int group, cudaStream_t stream, int* used_ctas = nullptr,
                               int* used_group = nullptr, int tri = 0);
constexpr int kNativeBM = 64, kNativeBN = 64;

// One problem of a batched call (device-resident table entry).
struct BatchProblem {
    const double* A;
    const double* B;
    double* C;
    int64_t lda, ldb, ldc;
    int32_t m, n, k;
    int32_t tiles_n;   // tiles along n of this problem
    int64_t tile0;     // first global tile index of this problem
    double alpha, beta;
};
// One persistent launch over all problems' tiles (problems sorted by tile0).
cudaError_t launch_native_batched(const BatchProblem* dev_problems, int count, int64_t total_tiles,
                                  cudaStream_t stream);

// ------------------------------------------------------------- emulated FP64
// Scaling exponents of the rows of op(X) (which = 0, op(X) rows x inner) or the
// columns of op(X) (which = 1, op(X) inner x rows).
// l1 (optional, may be null): per-vector sum of |x| in FP32, for the slice-count rule.
cudaError_t launch_emu_scale(int which, int op, int64_t rows, int64_t inner, const double* X,
                             int64_t ldx, int32_t* exps, uint8_t* flags, float* l1,
                             cudaStream_t stream);
// Kernels one launch_emu_scale call enqueues (the row-contiguous case adds a finalize kernel).
inline int emu_scale_kernel_count(int which, int op) { return ((which == 0) == (op == 0)) ? 2 : 1; }
// atomicMax into *out of ceil(16 * max_r log2(2^e_r * inner / l1_r)).
cudaError_t launch_emu_spread(int64_t rows, int64_t inner, const int32_t* exps, const uint8_t* flags,
                              const float* l1, int* out, cudaStream_t stream);
// The plan of one emulated product when the data decide it (AUTO slice count), chosen on the
// device so that no call waits for a readback: written by launch_emu_plan after the spreads,
// read at launch time by the split, product and reconstruction kernels of that product.
struct EmuPlan {
    int S;        // digit slices of the width rule (the digit encoding's S)
    int bits;     // operand width: the modular encoding's, or 7 S for digit slices
    int N;        // moduli; 0 = the digit encoding serves the product
    int pad;
    double est;   // estimated max error / bound (the rule's margin)
};
// Largest operand width whose moduli count the plan kernel looks up.
constexpr int kPlanMaxBits = 16 * 7;
// One thread: spreads[0..1] (ceil(16 x spread) of op(A) rows, op(B) columns; `tri`: op(B) is
// op(A)^T and spreads[1] is not read) -> rule bits = c0 + 1.25 (s_A + s_B) with c0 the k-dependent
// part of the rule, S = ceil(bits / 7) in [3, smax], the modular width min(7 S, max(ceil(bits),
// 7 S - 6)), its moduli count ntab[width] (0: none) and the encoding: moduli when ntab gives N,
// N <= n_alloc and (scheme_moduli or N + 2 <= S (S + 1) / 2).
struct EmuPlanTable {
    double c0;
    int smax, n_alloc, scheme_moduli, tri;
    uint8_t ntab[kPlanMaxBits + 1];
};
cudaError_t launch_emu_plan(const int* spreads, const EmuPlanTable& t, EmuPlan* out, cudaStream_t stream);
// Truncation digits (fp16, integer valued), layout [S][rows_pad][inner_pad].  Only the
// slices s_first .. S-1 (0-based) are written; a slice's digits do not depend on S.
// plan (optional): S comes from the device plan, and nothing is written when it chose moduli.
cudaError_t launch_emu_split(int which, int op, int64_t rows, int64_t inner, const double* X,
                             int64_t ldx, const int32_t* exps, const uint8_t* flags, int S,
                             int beta, void* digits, int64_t rows_pad, int64_t inner_pad,
                             cudaStream_t stream, int s_first = 0, const EmuPlan* plan = nullptr);

// ----------------------------------------------- emulated FP64, modular (CRT) encoding
// The operands are truncated to integers of `bits` bits (the first bits/7 digits of the slice
// encoding, A^ = trunc(A 2^(bits - e))), the exact integer product A^ B^ is computed modulo N
// pairwise coprime moduli p_l <= 255 -- one fp16 tensor product of residues |r| <= 127 per
// modulus -- and rebuilt by the Chinese remainder theorem; C := alpha 2^(e + f - 2 bits) A^B^
// + beta C.  N products instead of the S(S+1)/2 of the slice encoding.
constexpr int kCrtMaxModuli = 16;
// Largest k one modular product keeps exact in int32: k 127^2 < 2^31, rounded down to a multiple of 64.
constexpr int64_t kCrtMaxK = (((int64_t(1) << 31) - 1) / (127 * 127)) / 64 * 64;
struct CrtConsts {                 // residue split and slice-product epilogue
    int N;                         // moduli in use
    int bits;                      // integer width of the operands (7 x slices)
    uint32_t p[kCrtMaxModuli];
    uint32_t magic[kCrtMaxModuli]; // floor(2^32 / p) + 1: exact quotients of a < 2^26
    uint32_t c16[kCrtMaxModuli];   // 2^16 mod p
    uint32_t c32[kCrtMaxModuli];   // 2^32 mod p
    // the residue split's FP32 arithmetic: 2^14, 2^28, 2^42 mod p; p; 1 / p rounded to FP32; the
    // centred range [lo, hi] = [-floor(p / 2), floor((p - 1) / 2)]
    float kf[kCrtMaxModuli][3];
    float pf[kCrtMaxModuli], invf[kCrtMaxModuli], lof[kCrtMaxModuli], hif[kCrtMaxModuli];
};
struct CrtRecon {                  // reconstruction
    int N, bits;
    uint32_t w[kCrtMaxModuli][4];  // CRT weights w_l < P in 32-bit limbs, least significant first
    uint32_t frac[kCrtMaxModuli];  // w_l / P as 19-bit fixed point (quotient estimates)
    uint32_t Pw[4];                // P = prod p_l in 32-bit limbs
};
// The moduli for `bits`-bit operands and contraction length k (P > 4 k (2^bits - 1)^2, so
// |A^ B^| <= P/4); false when more than kCrtMaxModuli would be needed.
bool crt_plan(int bits, int64_t k, CrtConsts* c, CrtRecon* r);
// The constants of the first N moduli for `bits`-bit operands (no check of the range).
void crt_consts(int N, int bits, CrtConsts* c, CrtRecon* r);
// Largest k one modular product keeps exact in int32 (k * 127^2 < 2^31), a multiple of 64.
int64_t crt_max_k();
// Residues of the integer operand, layout [N][rows_pad][inner_pad] fp16 (as the digit slices).
// plan (optional): N and the width come from the device plan (c then holds all kCrtMaxModuli
// moduli), and nothing is written when it chose digit slices.
cudaError_t launch_emu_residues(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                                const int32_t* exps, const uint8_t* flags, const CrtConsts& c, void* planes,
                                int64_t rows_pad, int64_t inner_pad, cudaStream_t stream,
                                const EmuPlan* plan = nullptr);
// C from the residue planes of the product ([N][n][m] bytes, residue in [0, p_l)); tri = 1 / 2
// (m = n): only the lower / upper triangle of C is read from the residues and written.
cudaError_t launch_crt_reconstruct(int64_t m, int64_t n, const uint8_t* res, const CrtRecon& r, const int32_t* e,
                                   const uint8_t* ef, const int32_t* f, const uint8_t* ff, double alpha,
                                   double beta, double* C, int64_t ldc, cudaStream_t stream, int tri = 0);
struct CrtReconSet;
// The same with the moduli count and width from the device plan (constants of every count in
// `set`); nothing is written when the plan chose digit slices.
cudaError_t launch_crt_reconstruct_plan(int64_t m, int64_t n, const uint8_t* res, const CrtReconSet& set,
                                        const EmuPlan* plan, const int32_t* e, const uint8_t* ef, const int32_t* f,
                                        const uint8_t* ff, double alpha, double beta, double* C, int64_t ldc,
                                        cudaStream_t stream);

// ----------------------------------------------- triangular solve (leaf step)
constexpr int kTrsmNb = 64;       // order of the blocks inverted by substitution
constexpr int kTrsmLeaf = 512;    // order of the diagonal blocks applied through their inverses
constexpr int kTrsmLower = 0;     // MOMMS_LOWER
// Bytes of the inverses of the ceil(t / kTrsmLeaf) leaf blocks (dense kTrsmLeaf^2 each).
size_t tri_inverse_bytes(int64_t t);
// The inverses of the kTrsmNb-blocks of the t x t triangle of A (uplo 0 lower / 1 upper; unit: the
// diagonal is taken as ones and not read), each in the stored orientation, into the diagonal
// sub-blocks of W's leaf blocks (the rest of W is left as it is).
cudaError_t launch_tri_inverse(int64_t t, const double* A, int64_t lda, int uplo, int unit, double* W,
                               cudaStream_t stream);

struct EmuGemmArgs {
    int64_t m, n, k;
    int S, beta;
    const void* Ad;
    const void* Bd;
    int64_t m_pad, n_pad, k_pad;
    const int32_t* e;
    const uint8_t* ef;
    const int32_t* f;
    const uint8_t* ff;
    double alpha, beta_c;
    double* C;
    int64_t ldc;
    int member, group;
    void* scratch;
    size_t scratch_bytes;
    int32_t* status;
    int max_ctas;  // 0 = number of SMs
    int tile_n;    // CTA tile width request (96 or 192; 0 = automatic)
    int* used_ctas;   // optional out: persistent CTAs launched
    int* used_group;  // optional out: C2 raster group used
    int* used_launches;  // optional out: kernels launched (a tail launch per pass when split)
    const CrtConsts* crt;  // modular encoding: S = N moduli, the epilogue writes residues to `res`
    uint8_t* res;          // [N][n][m] residues of the product (modular encoding only)
    const CrtRecon* crt_fuse;  // non-null: the last modulus of each tile rebuilds C itself
    int* done;             // fused: one zeroed counter per tile (device)
    int tri;               // modular, m = n, separate reconstruction: 1 / 2 = only the tiles meeting the
                           // lower / upper triangle of C
    int kcap;              // modular: a triangular operand, its zero k range skipped per tile (1 op(A)
                           // lower, 2 op(A) upper, 3 op(B) lower, 4 op(B) upper; 0 none)
    int cta_pairs;         // modular, 192-wide tiles: the residue product on CTA pairs (one MMA over two
                           // SMs, 256 x 192 pair tiles) where the problem allows it
    // Device plan (AUTO slice count): S (digit slices) or N (moduli, with `crt` holding all moduli)
    // is read at launch time; the launch does nothing when the plan chose the other encoding.  The
    // pass structure is that of S (or N) as given here, the largest the plan can pick.
    const EmuPlan* plan;
    int* used_pairs;       // optional out: 1 when the residue product ran on CTA pairs
    int withhold;          // 1: the timeout test hook for this launch (else the armed process flag)
};
constexpr int kEmuBM = 128, kEmuBK = 64, kEmuBNMax = 192;

// One problem of a batched emulated call (device table entry; the tensor maps describe
// the problem's digit slices and keep the alignment CUtensorMap demands).
struct EmuBatchProblem {
    CUtensorMap mapA;
    CUtensorMap mapB;
    const int32_t* e;
    const uint8_t* ef;
    const int32_t* f;
    const uint8_t* ff;
    double* C;
    int64_t ldc;
    double alpha, beta_c;
    int64_t tile0;     // first tile of this problem in the concatenated tile list (modular batch: first
                       // unit, a unit being one modulus of one tile)
    int32_t m, n, S, beta, nslab, chunk_slabs, tiles_n;
    uint32_t group_end;
    // triangle of C written (symmetric rank-k updates): 0 = all, 1 = lower (column <= row +
    // diag), 2 = upper (column >= row + diag), rows and columns local to the problem
    int32_t tri, diag;
    uint8_t* res;      // modular batch (S = N moduli): the product's residues, [N][n][m] bytes
};
// Per-problem inputs and outputs of the batched scale and split passes (op = N, N).
struct EmuBatchPrep {
    const double* A;
    const double* B;
    int64_t lda, ldb;
    int32_t m, n, k, k_pad, S, beta;
    int32_t* e;
    uint8_t* ef;
    int32_t* f;
    uint8_t* ff;
    void* Ad;          // S slices [S][m][k_pad] fp16 (unused by the scale passes)
    void* Bd;          // S slices [S][n][k_pad] fp16
    int32_t* spread;   // 2 values (A, B): ceil(16 x spread) by atomicMax, or null
    int32_t bits;      // modular batch: operand width, the S planes being residues of S moduli
    int32_t enc;       // device plan: 0 = digit slices, 1 = moduli (the split of the other encoding
                       // skips the problem); -1 = no plan (every split launch takes it)
    int32_t scheme;    // device plan: the problem's encoding rule (MOMMS_SCHEME_*)
    double c0;         // device plan: the k-dependent constant of the slice-count rule
};
struct CrtBatchProblem;
// The batched device plan: per problem the slice-count rule on its spreads, its encoding and the
// fields of the four tables that depend on them (split passes, both product launches'
// tables with their unit offsets, the reconstruction table), the two launches' unit totals, and
// the largest S / moduli / width of the call as a summary plan.
struct EmuBatchPlanArgs {
    EmuBatchPrep* prep;
    EmuBatchProblem* slices;   // digit-slice launch table (every problem; 0 tiles when on moduli)
    EmuBatchProblem* moduli;   // residue-product launch table (every problem; 0 units when on slices)
    CrtBatchProblem* crt;      // reconstruction table (N = 0 when on slices)
    int count;
    int smax;                  // largest slice count of the rule
    int64_t* totals;           // [0] digit-slice tiles, [1] residue units
    EmuPlan* summary;
    uint64_t P[17][2];         // product of the first N moduli (low, high 64 bits), N = 0..16
};
cudaError_t launch_emu_batch_plan(const EmuBatchPlanArgs& a, cudaStream_t stream);
// Work items are (problem, block) pairs; the block's meaning depends on the pass:
//   scale A: 256 rows   scale B: 8 columns   split A: a 64 x 64 (row, k) tile   split B: 1024 digits.
cudaError_t launch_emu_batch_scale(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                   int n_b, cudaStream_t stream);
cudaError_t launch_emu_batch_split(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                   int n_b, cudaStream_t stream);
// The residue split of a batch: the same work items, the planes of each problem holding its
// operands' residues modulo the first S (= N) moduli of c at that problem's `bits`.
cudaError_t launch_emu_batch_residues(const EmuBatchPrep* probs, const int2* items_a, int n_a, const int2* items_b,
                                      int n_b, const CrtConsts& c, cudaStream_t stream);
// Work-list sizes of one problem.
inline int64_t emu_batch_scale_a_blocks(int64_t m) { return (m + 255) / 256; }
inline int64_t emu_batch_scale_b_blocks(int64_t n) { return (n + 7) / 8; }
inline int64_t emu_batch_split_a_blocks(int64_t m, int64_t k_pad) { return ((m + 63) / 64) * (k_pad / 64); }
inline int64_t emu_batch_split_b_blocks(int64_t n, int64_t k_pad) { return (n * (k_pad / 4) + 255) / 256; }

// Tensor map of S digit slices [S][rows][k_pad] (fp16, k contiguous); box 64 x box_rows.
// TMA map of digit slices [S][plane_rows][row_pitch] (fp16, K-major): k_pad digits of `rows`
// rows from `base`, boxes of 64 digits x box_rows rows (plane_rows, row_pitch 0 = rows, k_pad).
bool emu_make_digit_map(CUtensorMap* map, const void* base, int64_t k_pad, int64_t rows, int S, int box_rows,
                        int64_t plane_rows = 0, int64_t row_pitch = 0);
// One persistent launch of the slice-product kernel over the tiles of all problems.
// Residue products of a batch (modular encoding): units (problem, modulus, tile), problem by
// problem and modulus-major inside a problem; each problem's moduli are the first S of c.
cudaError_t launch_emu_residue_gemm_batched(const EmuBatchProblem* dev_table, int count, int64_t total_units,
                                            const CrtConsts& c, void* scratch, size_t scratch_bytes,
                                            int32_t* status, cudaStream_t stream, const int64_t* total_dev = nullptr);
// Reconstruction of a batch of modular products: work items (problem, block of 8 columns), a warp
// per column.  The reconstruction constants depend only on the number of moduli.
struct CrtBatchProblem {
    const uint8_t* res;  // [N][n][m] residue bytes
    const int32_t* e;
    const uint8_t* ef;
    const int32_t* f;
    const uint8_t* ff;
    double* C;
    int64_t ldc;
    double alpha, beta;
    int32_t m, n, N, bits;
};
struct CrtReconSet {
    CrtRecon by_n[kCrtMaxModuli + 1];  // index: number of moduli
};
inline int64_t crt_batch_blocks(int64_t n) { return (n + 7) / 8; }
cudaError_t launch_crt_reconstruct_batched(const CrtBatchProblem* probs, const int2* items, int n_items,
                                           const CrtReconSet& set, cudaStream_t stream);
cudaError_t launch_emu_slice_gemm_batched(const EmuBatchProblem* dev_table, int count, int64_t total_tiles,
                                          void* scratch, size_t scratch_bytes, int32_t* status,
                                          cudaStream_t stream, const int64_t* total_dev = nullptr);
// The CTA tile width used for n columns (tile_n request 0 = automatic).
int emu_pick_bn(int64_t m, int64_t n, int64_t k, int requested, int units_per_tile = 1);
// Default C2 group of the slice-product kernel for `ctas` persistent CTAs (tile rows of the
// block of C one wave covers; fewest operand rows read per unit of k over all waves).
int emu_default_group(int64_t ctas, int tiles_m, int tiles_n);
// Arms the timeout test hook: the next slice-product launch leaves one stage of CTA 0 empty.
void emu_debug_withhold_load();
// Takes (and clears) the armed test hook: a call that enqueues several product launches of which
// the device plan picks one hands it to each of them.
int emu_debug_take_withhold();
// Launches the slice-product kernel once per k pass; *passes receives the count.
cudaError_t launch_emu_slice_gemm(const EmuGemmArgs& a, int* passes, cudaStream_t stream);
size_t emu_scratch_bytes(int num_sms);
// Scratch for one single-problem launch including the tail split's partial sums (the launch
// falls back to whole tiles when it is given only emu_scratch_bytes).
size_t emu_scratch_bytes_tail(int64_t m, int64_t n, int64_t k, int S, int max_ctas, int beta);
size_t emu_scratch_bytes_for_ctas(int ctas);
// Bit d set: diagonal d is the most significant of an exact int64 group (S, beta, k per pass).
// Diagonal d sums (d - 1) pair products over k_pass, each |digit product| <= (2^beta - 1)^2:
// |P_d| <= (d - 1) (2^beta - 1)^2 k_pass.  Walking from the least significant diagonal, a group
// [lo, hi] holds Q = sum_{d=lo}^{hi} P_d 2^(beta (hi - d)); a group is closed before the bound on
// |Q| would reach 2^63.  (Host and device: the batched device plan evaluates it per problem.)
__host__ __device__ inline uint32_t emu_group_ends(int S, int beta, int64_t k_pass) {
    const unsigned __int128 limit = static_cast<unsigned __int128>(1) << 63;
    const unsigned __int128 dmax = static_cast<unsigned __int128>((1ll << beta) - 1);
    uint32_t mask = 0;
    unsigned __int128 acc = 0;
    int j = 0;
    for (int d = S + 1; d >= 2; --d) {
        const unsigned __int128 pb =
            static_cast<unsigned __int128>(d - 1) * dmax * dmax * static_cast<unsigned __int128>(k_pass);
        bool fits = (j == 0);
        if (j > 0 && beta * j < 64) fits = acc + (pb << (beta * j)) < limit;
        if (!fits) {
            mask |= 1u << (d + 1);  // diagonal d + 1 closed the previous group
            acc = 0;
            j = 0;
        }
        acc += pb << (beta * j);
        ++j;
    }
    mask |= 1u << 2;  // the most significant diagonal always closes the last group
    return mask;
}
// Largest k one pass may cover so that every diagonal sum stays below 2^31.
int64_t emu_max_k_per_pass(int S, int beta);
// Products per FP32 accumulation chunk (every partial sum below 2^24), in 64-wide slabs.
int emu_chunk_slabs(int beta);

// SM count of the current device (looked up once per device ordinal).
int device_sm_count();

// Kernel attributes (the dynamic shared-memory limit) belong to a device's context, so the
// "already set" flags of the launchers are kept per device ordinal.  done() / mark() act on the
// current device; ordinals beyond kMaxDevices are never marked (the attribute is set every call).
constexpr int kMaxDevices = 64;
int current_device();
struct PerDeviceFlag {
    std::atomic<bool> set[kMaxDevices] = {};
    bool done() const {
        const int d = current_device();
        return d >= 0 && d < kMaxDevices && set[d].load(std::memory_order_acquire);
    }
    void mark() {
        const int d = current_device();
        if (d >= 0 && d < kMaxDevices) set[d].store(true, std::memory_order_release);
    }
};

// ------------------------------------------------------------------ probes
cudaError_t probe_peak(int kind, double* tflops, cudaStream_t stream);
// Copies `bytes` (multiple of 16, 16-byte aligned) `repeats` times on `ctas` SMs (0 = all).
cudaError_t stream_copy(void* dst, const void* src, size_t bytes, int ctas, int repeats, cudaStream_t stream);

}  // namespace momms
