/*
 * momms.h -- C ABI of the GB300-native MOMMS library (libmomms.so).
 *
 * The operation is the dense product of the MOMMS paper (Smith & van de Geijn,
 * "The MOMMS Family of Matrix Multiplication Algorithms", SC19), Sec. 2.1
 * footnote (gamma_ij = sum_p alpha_ip beta_pj) and Sec. 2.2.1 (C += AB),
 * extended to BLAS dgemm semantics:
 *
 *     C := alpha * op(A) * op(B) + beta * C,   op(X) = X or X^T,
 *
 * op(A) m x k, op(B) k x n, C m x n, all FP64 and column-major with leading
 * dimensions (element (i, j) of X is X[i + j * ldX]).
 *
 * Conventions shared by every entry point
 *   - Pointers named A, B, C, X, dC, dA, dB, digits, e, f, flags, workspace and
 *     scratch are DEVICE pointers owned by the caller.  The library never frees
 *     them and never uses them after the work enqueued by the call has finished.
 *   - Every call is asynchronous on `stream` (0 = the legacy default stream);
 *     results are ready when the stream reaches the enqueued work.  The
 *     data-driven slice count is chosen on the device (momms_set_plan_on_device),
 *     so the product calls do not wait for the GPU; the exceptions are the
 *     first call that sizes a workspace (it may allocate), momms_syrk with the
 *     data-driven slice count (it reads the spread back), and the calls that say
 *     they synchronise (status, report, probes, tuning).
 *   - Return value: MOMMS_OK (0), a negative number -i when argument i
 *     (1-based, in the order of the prototype) is invalid, or one of the
 *     positive MOMMS_ERR_* codes.  Nothing is enqueued when a call fails.
 *   - BLAS argument rules: m, n, k >= 0; ld >= max(1, rows of the stored
 *     matrix); m == 0 or n == 0 is a no-op; k == 0 or alpha == 0 gives
 *     C := beta * C; beta == 0 makes C write-only (NaNs in C do not
 *     propagate).  C must not overlap A or B.
 *   - No exception crosses the ABI.  A handle may be used by one host thread at
 *     a time; different handles are independent.
 */
#ifndef MOMMS_H
#define MOMMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without including the CUDA headers */
typedef struct CUstream_st* momms_stream_t;

typedef struct momms_handle_s* momms_handle_t;

enum {
    MOMMS_OK = 0,
    MOMMS_ERR_CUDA = 1001,        /* a CUDA launch or runtime call failed          */
    MOMMS_ERR_TIMEOUT = 1002,     /* a bounded device wait expired (the kernel     */
                                  /* returned early; its output is undefined)      */
    MOMMS_ERR_NONFINITE = 1003,   /* emulated mode met Inf/NaN input (a warning:   */
                                  /* affected rows/columns of C were set to NaN)   */
    MOMMS_ERR_WORKSPACE = 1004,   /* the caller's workspace is too small           */
    MOMMS_ERR_UNSUPPORTED = 1005, /* size or option outside what the build handles */
    MOMMS_ERR_ALLOC = 1006,       /* the library could not allocate device memory  */
    MOMMS_ERR_HANDLE = 1007,      /* null or destroyed handle                      */
    MOMMS_ERR_IO = 1008           /* plan cache file could not be read or written  */
};

typedef enum { MOMMS_OP_N = 0, MOMMS_OP_T = 1 } momms_op_t;
typedef enum { MOMMS_LOWER = 0, MOMMS_UPPER = 1 } momms_uplo_t;
typedef enum { MOMMS_LEFT = 0, MOMMS_RIGHT = 1 } momms_side_t;
typedef enum { MOMMS_NON_UNIT = 0, MOMMS_UNIT = 1 } momms_diag_t;

/* How the product is computed.
 *   NATIVE    FP64 DMMA tensor instructions, C micro-tile resident in registers
 *             (Resident C at L0, Sec. 3.4).
 *   EMULATED  FP64 emulated by signed integer digit slices on the fp16 tensor
 *             cores (tcgen05 kind::f16, exact FP32 accumulation in tensor memory,
 *             drained to exact integers, recombined in FP64).
 *   AUTO      the plan (tuned or default) decides per size bucket. */
typedef enum { MOMMS_MODE_AUTO = 0, MOMMS_MODE_NATIVE = 1, MOMMS_MODE_EMULATED = 2 } momms_mode_t;

/* Family member = the order in which C tiles and k blocks are visited, which
 * decides the operand block that stays resident in L2 (Sec. 3.2, Sec. 3.3 naming):
 *   C2  grouped raster: a wave of CTAs covers a block of C, A and B panels are
 *       reused through L2 (Resident C at the L2 level, like C3A2C0 of Sec. 5.4).
 *   A2  a block of rows of A (all of its k) stays in L2 while the wave sweeps
 *       the columns of C (Resident A, like A3B2C0).
 *   B2  mirror of A2: a block of columns of B stays in L2 (like B3A2C0).
 *   A1  plain row-major raster: each CTA keeps its A tile and walks n
 *       (Goto-like A2C0: the L2 level is not designed for, Sec. 4.3).
 * Residue products (modular encoding) with k <= 256, at least one tile per CTA and m a
 * multiple of 4 -- not SYRK's triangle, TRMM's skipped k ranges or the fused
 * reconstruction -- take A1's order whatever the member, with the A tile held in shared
 * memory over each CTA's strip of tiles (the report keeps the member the handle asked for). */
typedef enum {
    MOMMS_MEMBER_AUTO = 0,
    MOMMS_MEMBER_C2 = 1,
    MOMMS_MEMBER_A2 = 2,
    MOMMS_MEMBER_B2 = 3,
    MOMMS_MEMBER_A1 = 4
} momms_member_t;

/* What the last call on a handle did. */
typedef struct {
    int mode;            /* MOMMS_MODE_NATIVE or MOMMS_MODE_EMULATED actually used   */
    int member;          /* member actually used                                     */
    int slices;          /* S (emulated), 0 for native                               */
    int digit_bits;      /* beta (bits per digit), 0 for native                      */
    int k_passes;        /* launches along k (emulated: keeps int32 sums exact)      */
    int tile_m, tile_n;  /* CTA tile                                                 */
    int ctas;            /* CTAs of the (last) product launch                        */
    int group;           /* C2 raster group: tile rows of the C block a wave covers  */
    int64_t launches;    /* kernels enqueued by the call                             */
    double est_err_ratio;/* emulated: estimated truncation error / bound (heuristic) */
    int64_t ooc_block;   /* momms_gemm_host: block size b (0 for the other calls)    */
    int64_t h2d_bytes;   /* momms_gemm_host: bytes copied host -> device             */
    int64_t d2h_bytes;   /* momms_gemm_host: bytes copied device -> host             */
    int moduli;          /* emulated, modular encoding: N moduli (0: digit slices)   */
    int operand_bits;    /* emulated: integer width of the operands (7 S for slices) */
    int crt_fused;       /* moduli: 1 when the residue product rebuilt C itself       */
    int cta_pairs;       /* moduli: 1 when the residue products ran on CTA pairs      */
    int ooc_resident;    /* momms_gemm_host: 0 Resident C, 1 Resident A at HBM level  */
} momms_report_t;

/* ---------------------------------------------------------------- handles */
int momms_create(momms_handle_t* handle);
int momms_destroy(momms_handle_t handle);
int momms_set_mode(momms_handle_t handle, int mode);      /* momms_mode_t            */
int momms_set_member(momms_handle_t handle, int member);  /* momms_member_t          */
/* S = number of digit slices for EMULATED mode: 0 = automatic (from the exponent
 * spread of the inputs), else 1..MOMMS_MAX_SLICES. */
int momms_set_slices(momms_handle_t handle, int slices);
#define MOMMS_MAX_SLICES 16
/* Integer encoding of an EMULATED single product.  Either way the operands become integers of
 * b bits (b = 7S unless noted below): each row of op(A) and column of op(B) is scaled by its
 * power-of-two maximum, A^ = trunc(A 2^(b - e_i)), B^ likewise.
 *   SLICES  each operand as S signed 7-bit digit slices; the S(S+1)/2 most significant digit
 *           pairs are multiplied (fp16 tensor products) and recombined in exact int64 groups
 *           and FP64 (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 2012: the error-free split).
 *   MODULI  the exact integer product A^B^ computed modulo N pairwise coprime moduli <= 255 --
 *           residues |r| <= 127 as fp16, one tensor product per modulus -- and rebuilt by the
 *           Chinese remainder theorem, P = prod p > 4 k (2^b - 1)^2 (Ozaki, Uchino & Imamura,
 *           "Ozaki Scheme II", 2025).  N products instead of S(S+1)/2 (S = 6, k = 8192: 13
 *           instead of 21), and no dropped digit pairs: the only error is the truncation of the
 *           operands.  Needs N <= 16 (any S <= 7; S = 8 for k <= 2048) and k <= 133,120;
 *           otherwise the product falls back to SLICES (report.moduli = 0).
 *   AUTO    MODULI when it takes at least two tensor products fewer than SLICES, else SLICES.
 * With the automatic slice count (momms_set_slices(0)) the modular encoding takes the width
 * the slice-count rule asks for, rounded up to whole bits rather than whole 7-bit digits
 * (report.operand_bits), which can save a modulus.
 * Single products (momms_gemm, its host-memory and triangular forms); batched calls and SYRK
 * use SLICES.  Returns -2 for other values. */
typedef enum { MOMMS_SCHEME_AUTO = 0, MOMMS_SCHEME_SLICES = 1, MOMMS_SCHEME_MODULI = 2 } momms_scheme_t;
int momms_set_scheme(momms_handle_t handle, int scheme);
/* Where the modular encoding rebuilds C: 1 = a separate reconstruction launch after the residue
 * products; 2 = fused: the epilogue of a tile's last modulus (the units run modulus by modulus,
 * so the other moduli of the tile finished long before) reads the other moduli's residues
 * (published per tile through a device counter; a bounded wait) and writes C -- the same
 * arithmetic, the same bits, without the separate pass over C; 0 = automatic = 1 (the fused form
 * measured slower: the drain warps rebuild C at a fraction of the separate kernel's rate and the
 * products wait behind them -- 11.9 against 10.4 ms per 8192^3 step).  Returns -2 for other
 * values. */
int momms_set_crt_fusion(momms_handle_t handle, int mode);
/* Where a product with the data-driven slice count (slices = 0, EMULATED or AUTO mode) makes its
 * choices.  1 (default) = on the device: a one-thread kernel after the scaling pass turns the
 * measured spreads into S, the operand width and the encoding, and every later kernel of the
 * product reads that plan when it starts (the kernels of the encoding not chosen return at once),
 * so the call only enqueues work and can be captured in a CUDA graph once its workspace exists;
 * the report's slices / moduli / operand_bits / est_err_ratio are fetched from the device when
 * momms_get_last_report is called.  0 = on the host: the spreads are read back (the call waits
 * for them) and only the chosen encoding's kernels are launched.  Both give the same plan and the
 * same C.  Triangular updates (momms_syrk) always choose on the host.  Returns -2 for other values. */
int momms_set_plan_on_device(momms_handle_t handle, int on);
/* CTA pairs for the modular encoding's residue products (192-wide tiles, no triangle or k-range
 * skipping): two CTAs of a cluster share each MMA (tcgen05.mma.cta_group::2, M = 256) on a
 * 256 x 192 tile, each staging its own 128 rows of A and 96 rows of B.  Per MMA flop a CTA's shared
 * memory is written and read 30 % less than with one CTA per 128 x 192 tile, and L2 sends 30 %
 * fewer operand bytes.  Both CTAs load only their own tiles (no shared loads).  Results are
 * bit-identical either way.  0 = automatic, 1 = off, 2 = on.  Returns -2 for other values. */
int momms_set_cta_pairs(momms_handle_t handle, int mode);
/* Caps the grid of the single-product launches of this handle at `ctas` CTAs that each
 * loop over their share of the member's tiles (0 = default: one CTA per SM for the
 * emulated slice products, one CTA per tile for the native kernel).  Fewer CTAs lower
 * the engine's compute rate while the memory system stays the same, which moves the
 * compute-to-bandwidth ratio the paper varies between its experiments (Sec. 5.2,
 * Fig. 6) -- the knob of the bandwidth-ratio sweep.  Values above the SM count are
 * clamped to it in emulated mode.  Batched calls ignore it.  Returns -2 for ctas < 0. */
int momms_set_max_ctas(momms_handle_t handle, int ctas);
/* Tile rows of the block of C that one wave of CTAs covers under member C2 (the
 * resident block's m_c in tiles, Sec. 2.2.1; its n_c is the wave size over this).
 * 0 = default: for the emulated kernel the group, near sqrt(wave * 192 / 128), that
 * minimises the operand rows all waves read per unit of k (counted over the actual tile
 * order, so waves straddling two groups are included); 16 for the native kernel.
 * Single-product calls only.  Returns -2 for group < 0. */
int momms_set_raster_group(momms_handle_t handle, int group);
/* Emulated tile width: 192 (wide: half the int32 sums in spare TMEM, the int64 group sums of
 * the recombination in a global scratch block) or 96 (narrow: every sum in registers and the
 * group sums in TMEM, so a diagonal's recombination stays on chip; twice the operand-tile
 * reloads per flop).  0 = automatic: 96 when the 192-wide tiles would be fewer than the SMs
 * (small products: more SMs at work), else 192.  Results are bit-identical either way.
 * Single-product calls only.  Returns -2 for other values. */
int momms_set_tile_n(momms_handle_t handle, int tile_n);
/* What the handle's last call used.  When that call chose its slice count on the device
 * (momms_set_plan_on_device), the plan is copied back from the device here, which waits for the
 * work already enqueued; a replayed CUDA graph of such a call updates it again. */
int momms_get_last_report(momms_handle_t handle, momms_report_t* report);
/* Device status word of the handle (0 = fine, MOMMS_ERR_TIMEOUT after a capped
 * wait expired).  Synchronises `stream` first.  Clears the word. */
int momms_check_device_status(momms_handle_t handle, momms_stream_t stream);
/* Test hook of the timeout path (no counterpart in the paper): the next slice- or
 * residue-product launch of this process (any handle, or the allocation-free entry
 * point) leaves the first shared-memory stage of its first CTA empty -- the producer
 * announces the stage's bytes but issues no copy.  The MMA thread's bounded wait on that
 * stage then runs out (about 2 s), the CTA raises its abort flag, lets its issued copies
 * and MMAs finish, frees its tensor memory and writes MOMMS_ERR_TIMEOUT to the status
 * word the launch was given (momms_check_device_status, momms_noalloc_status).  The C of
 * that call is not valid; later calls are unaffected.  Nothing faults and no wait is
 * unbounded. */
void momms_debug_withhold_load(void);
/* Per-launch timing of the dominant kernel (no counterpart in the paper; measurement only):
 * with max_launches > 0 every later emulated single product of this handle records a CUDA
 * event pair on its stream around its slice- or residue-product launch(es), for up to
 * max_launches products (further ones are not timed); 0 switches it off.  The events are
 * created here, never in the product calls.  Returns -2 for max_launches < 0. */
int momms_set_kernel_timing(momms_handle_t handle, int max_launches);
/* Sum of the recorded launch durations in milliseconds and their number since the last
 * read (waits for the last recorded event), then starts counting again.  Returns -2 / -3
 * for a NULL total_ms / launches. */
int momms_kernel_timing(momms_handle_t handle, double* total_ms, int64_t* launches);
const char* momms_status_string(int status);

/* -------------------------------------------------------------- workspace */
/* Bytes of device workspace a momms_gemm_ex call of this size needs in the
 * handle's current mode/slices (worst case over modes when AUTO).  Without a
 * caller workspace the handle allocates (and keeps) its own. */
int momms_workspace_size(momms_handle_t handle, int op_a, int op_b, int64_t m, int64_t n,
                         int64_t k, size_t* bytes);
/* Caller-owned device workspace (NULL, 0 = return to library-owned memory).
 * Must stay valid until all work enqueued with it has finished. */
int momms_set_workspace(momms_handle_t handle, void* workspace, size_t bytes);

/* --------------------------------------------------------------- products */
/* C := alpha*A*B + beta*C (op = N, N) with a per-thread default handle in AUTO
 * mode.  Sec. 2.2.1; the BLAS dgemm signature. */
int momms_gemm(int64_t m, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb,
               double beta, double* C, int64_t ldc, momms_stream_t stream);

/* C := alpha*op(A)*op(B) + beta*C with the handle's mode, member and slices.
 * op(A) = A (m x k, lda >= m) or A^T (A stored k x m, lda >= k); likewise B. */
int momms_gemm_ex(momms_handle_t handle, int op_a, int op_b, int64_t m, int64_t n,
                  int64_t k, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                  momms_stream_t stream);

/* Gradients of L(C) with C = A*B (A m x k, B k x n): given dC = dL/dC (m x n),
 *   dA = dC * B^T   (m x k; contraction over n)   -- skipped when dA == NULL
 *   dB = A^T * dC   (k x n; contraction over m)   -- skipped when dB == NULL
 * computed through the transposed-operand paths of momms_gemm_ex (dA, dB are
 * overwritten, beta = 0). */
int momms_gemm_backward(momms_handle_t handle, int64_t m, int64_t n, int64_t k,
                        const double* A, int64_t lda, const double* B, int64_t ldb,
                        const double* dC, int64_t lddc, double* dA, int64_t ldda,
                        double* dB, int64_t lddb, momms_stream_t stream);

/* `count` independent products C_i := alpha_i*A_i*B_i + beta_i*C_i (op = N, N),
 * of uneven sizes, in ONE persistent kernel launch over a device tile table
 * (plus, in EMULATED mode, one scale and one split launch over all problems).
 * EMULATED mode chooses the integer encoding per problem (the handle's scheme; in
 * AUTO the modular one where it saves two or more tensor products AND its
 * reconstruction is paid for, N (k + 850) <= 0.9 S (S + 1) / 2 k): the problems on
 * moduli get one residue split, ONE persistent residue-product launch over their
 * (modulus, tile) units and one reconstruction launch, the others the digit split
 * and the slice-product launch (up to 9 launches in all); report.slices and
 * report.moduli give the largest of each.
 * All array arguments are HOST arrays of length `count`; the matrix pointers in
 * them are device pointers.  The tile table lives in the handle, so the
 * enqueued launches can be captured in a CUDA graph and replayed as long as the
 * handle and the problem pointers stay alive and the sizes do not change: a call
 * whose problem table equals the previous call's enqueues only the kernel (make
 * one eager call before capturing). */
int momms_gemm_batched(momms_handle_t handle, int64_t count, const int64_t* m,
                       const int64_t* n, const int64_t* k, const double* alpha,
                       const double* const* A, const int64_t* lda,
                       const double* const* B, const int64_t* ldb, const double* beta,
                       double* const* C, const int64_t* ldc, momms_stream_t stream);

/* --------------------------------------------- steps of the emulated path */
/* These expose each step separately (used by the parity tests).  The digit
 * layout: S slices, slice s (0-based = digit s+1) a rows_pad x inner_pad fp16
 * matrix stored inner-contiguous at digits + s*rows_pad*inner_pad; rows_pad >=
 * rows, inner_pad >= inner and a multiple of 64; padding holds zeros.  The
 * pointer must be 16-byte aligned. */

/* Scaling exponents.  which = 0: the rows of op(X) where op(X) is rows x inner
 * (X = A, op = op_a); which = 1: the columns of op(X) where op(X) is
 * inner x rows (X = B).  exps[r] = floor(log2 max_q |x_rq|) + 1 (0 for an
 * all-zero vector), flags[r] = 1 when the vector holds Inf or NaN. */
int momms_emu_scale(int which, int op, int64_t rows, int64_t inner, const double* X,
                    int64_t ldx, int32_t* exps, uint8_t* flags, momms_stream_t stream);

/* Truncation digits: x * 2^-e = sum_{s=1..S} d_s 2^(-beta s) + remainder,
 * |d_s| <= 2^beta - 1, signs of x; flagged vectors give zero digits.
 * digits: fp16 (integer-valued) as described above; 1 <= beta <= 10. */
int momms_emu_split(int which, int op, int64_t rows, int64_t inner, const double* X,
                    int64_t ldx, const int32_t* exps, const uint8_t* flags, int slices,
                    int digit_bits, void* digits, int64_t rows_pad, int64_t inner_pad,
                    momms_stream_t stream);

/* Moduli of the modular encoding (MOMMS_SCHEME_MODULI) for operands of `bits` bits and
 * contraction length k: the fewest of the library's pairwise coprime moduli <= 255 (walking
 * down from 255, each coprime to all taken before) whose product P exceeds 4 k (2^bits - 1)^2:
 * the centred residue of the exact integer product modulo P is then the product itself, with
 * |product| <= P/4 (the margin the reconstruction's quotient estimate uses).  moduli: host
 * array of 16 entries; *count receives N.  Host only (no device work).  Returns -1 for bits
 * outside 1..56, -2 for k < 1, MOMMS_ERR_UNSUPPORTED when more than 16 moduli or k > 133,120
 * would be needed. */
int momms_crt_moduli(int bits, int64_t k, int* count, uint32_t* moduli);

/* Residues of the integer operand X^ = sign(x) trunc(|x| 2^(bits - e)) (e from
 * momms_emu_scale; X^ is the first bits/7 digits of momms_emu_split when 7 divides bits)
 * modulo each of the N moduli momms_crt_moduli(bits, k) returns, centred in
 * [-floor(p/2), floor((p-1)/2)] and stored as fp16 in plane l of `planes` (layout of the
 * digit slices: [N][rows_pad][inner_pad]; flagged vectors and padding give zeros).
 * Returns the argument errors of momms_emu_split (bits in place of slices: -9 outside 1..56)
 * and MOMMS_ERR_UNSUPPORTED when momms_crt_moduli would. */
int momms_emu_residues(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                       const int32_t* exps, const uint8_t* flags, int bits, int64_t k, void* planes,
                       int64_t rows_pad, int64_t inner_pad, momms_stream_t stream);

/* Slice products and recombination on the tcgen05 tensor cores:
 *   P_d = sum_{s+t=d} A_s B_t  (d = 2..S+1, triangular pair set), exact;
 *   C := alpha * 2^(e_i+f_j) * sum_d 2^(-beta d) P_d + beta*C, the diagonals combined
 *   exactly in int64 groups and in FP64 only between groups (one rounding when a single
 *   group covers all diagonals).
 * Ad: S slices of m_pad x k_pad, Bd: S slices of n_pad x k_pad (layout above,
 * m_pad >= m, n_pad >= n, k_pad a multiple of 64; digit_bits <= 8).
 * scratch: device memory of at least momms_emu_scratch_bytes() bytes (int64 / FP64
 * partial sums of the recombination, one 128 x 192 block per CTA).  Given
 * momms_emu_scratch_bytes_for(m, n, k, slices) bytes, the launch also splits the
 * tiles of its last, partial round of CTAs along k (each part stores its exact int32
 * diagonal sums there; the last part of a tile adds them up and recombines), so that
 * round keeps most SMs busy; the result is bit-identical either way.  status: a
 * device int32 set to MOMMS_ERR_TIMEOUT if a bounded wait expires.
 * member: momms_member_t. */
int momms_emu_slice_gemm(int64_t m, int64_t n, int64_t k, int slices, int digit_bits,
                         const void* Ad, const void* Bd, int64_t m_pad, int64_t n_pad,
                         int64_t k_pad, const int32_t* e, const uint8_t* eflags,
                         const int32_t* f, const uint8_t* fflags, double alpha,
                         double beta, double* C, int64_t ldc, int member, void* scratch,
                         size_t scratch_bytes, int32_t* status, momms_stream_t stream);
size_t momms_emu_scratch_bytes(void);
size_t momms_emu_scratch_bytes_for(int64_t m, int64_t n, int64_t k, int slices);

/* Residue products of the modular encoding on the tcgen05 tensor cores: for each of the N
 * moduli p_l of momms_crt_moduli(bits, k),
 *     res[l][j][i] = (sum_p Ar[l][i][p] Br[l][j][p]) mod p_l   in [0, p_l),
 * the sum exact (FP32 chunks of 1024 products in tensor memory drained to int32).  Ar / Br:
 * residue planes from momms_emu_residues (N planes of m_pad x k_pad / n_pad x k_pad fp16,
 * k_pad a multiple of 64); res: device bytes, N m n of them ([l][column][row], column-major m
 * x n per modulus).  scratch / status as for momms_emu_slice_gemm (its recombination blocks are
 * not used, but the launch keeps the same per-CTA layout).  Errors: -i for argument i, and
 * MOMMS_ERR_UNSUPPORTED when the moduli do not exist for (bits, k). */
int momms_emu_residue_gemm(int64_t m, int64_t n, int64_t k, int bits, const void* Ar, const void* Br,
                           int64_t m_pad, int64_t n_pad, int64_t k_pad, int member, uint8_t* res, void* scratch,
                           size_t scratch_bytes, int32_t* status, momms_stream_t stream);

/* Chinese remainder reconstruction of the modular encoding: from the residues of
 * momms_emu_residue_gemm, the exact product Z = A^B^ (the centred representative modulo
 * P = prod p_l), then
 *     C := alpha * round(Z_ij) 2^(e_i + f_j - 2 bits) + beta * C
 * with round() to nearest FP64 (ties to even) and the power-of-two scaling exact for normal
 * results; beta != 0 uses one fma(beta, C, alpha y); beta == 0 makes C write-only.  Rows i
 * with eflags[i] or columns j with fflags[j] give NaN.  e, eflags, f, fflags from
 * momms_emu_scale.  Errors: -i for argument i, MOMMS_ERR_UNSUPPORTED as above. */
int momms_crt_reconstruct(int64_t m, int64_t n, int64_t k, int bits, const uint8_t* res, const int32_t* e,
                          const uint8_t* eflags, const int32_t* f, const uint8_t* fflags, double alpha,
                          double beta, double* C, int64_t ldc, momms_stream_t stream);

/* --------------------------------------------------- symmetric rank-k update */
/* C := alpha*op(A)*op(A)^T + beta*C on the uplo triangle of the n x n matrix C
 * (BLAS dsyrk: trans = N uses A n x k, trans = T uses A k x n; the other triangle is
 * neither read nor written).  The paper names the other level-3 BLAS as the next use
 * of the family (Sec. 7); this one needs half the products of a GEMM.  Native mode:
 * the DMMA kernel over the triangle's tiles, elements masked on the diagonal tiles.
 * Emulated mode: op(A) is scaled and split ONCE and serves as both operands.  With
 * the modular encoding (chosen as for momms_gemm_ex) the residue products visit only
 * the tiles that meet the triangle (momms_tri_tile gives their order) and the
 * reconstruction writes only the triangle; with digit slices the slice products run
 * over the 128-row blocks of the triangle in one batched launch per k pass.  The
 * error bound is the GEMM one with B = op(A)^T.
 * Device pointers, asynchronous on `stream`.  Errors: BLAS-style negative index
 * (uplo -2, trans -3, n -4, k -5, A -7, lda -8, C -10, ldc -11), MOMMS_ERR_*. */
int momms_syrk(momms_handle_t handle, int uplo, int trans, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, double beta, double* C, int64_t ldc,
               momms_stream_t stream);

/* ------------------------------------------------------ triangular product */
/* B := alpha*op(A)*B (side LEFT, A m x m) or B := alpha*B*op(A) (side RIGHT, A n x n),
 * A triangular (uplo; diag UNIT: ones on the diagonal, which is not read), B m x n
 * overwritten (BLAS dtrmm).  The triangle is first copied into a dense zero-filled
 * operand kept by the handle; the product then runs as a GEMM in the handle's mode --
 * emulated: in place (both operands are split before the products write B), and with
 * the modular encoding each tile's residue products skip the k range where op(A) is
 * zero (half the tensor work; the skipped products are exact zeros, so the result is
 * unchanged); native: from a copy of B.  Device pointers, asynchronous on `stream`.  The
 * bound is the GEMM one with the zero triangle counted as exact zeros.  Errors:
 * BLAS-style negative index (side -2, uplo -3, trans -4, diag -5, m -6, n -7, A -9,
 * lda -10, B -11, ldb -12), MOMMS_ERR_*. */
int momms_trmm(momms_handle_t handle, int side, int uplo, int trans, int diag, int64_t m, int64_t n,
               double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
               momms_stream_t stream);

/* ------------------------------------------------------- triangular solve */
/* B := alpha*op(A)^-1*B (side LEFT: solves op(A) X = alpha B, A m x m) or
 * B := alpha*B*op(A)^-1 (side RIGHT: X op(A) = alpha B, A n x n), A triangular (uplo;
 * diag UNIT: ones on the diagonal, which is not read), B m x n overwritten by X (BLAS
 * dtrsm).  Recursive blocked solve: op(A) is halved (at multiples of 512) until blocks of
 * order <= 512 remain; the off-diagonal half becomes one GEMM update of the right-hand sides
 * (this library's product, in the handle's mode -- the updates carry ~all m^2 n (n^2 m)
 * flops), and each 512 x 512 diagonal block is applied as a GEMM with its explicit inverse:
 * the inverses of its 64 x 64 blocks come from an FP64 substitution kernel (one CTA per
 * block) and are joined pairwise by batched products.  The error is that of the
 * GEMMs plus the inverses' (well-conditioned diagonal blocks: a small multiple of
 * 2^-53 (|op(A)| |X|) componentwise).  Device pointers, asynchronous on `stream` (the
 * emulated GEMMs choose their slice counts on the device).  Errors:
 * BLAS-style negative index (side -2, uplo -3, trans -4, diag -5, m -6, n -7, A -9,
 * lda -10, B -11, ldb -12), MOMMS_ERR_*. */
int momms_trsm(momms_handle_t handle, int side, int uplo, int trans, int diag, int64_t m, int64_t n,
               double alpha, const double* A, int64_t lda, double* B, int64_t ldb,
               momms_stream_t stream);

/* ------------------------------------------------------- out-of-core product */
/* C := alpha*A*B + beta*C with A, B and C in HOST memory (column-major, leading
 * dimensions as for momms_gemm; no transposes), for problems larger than the device
 * memory one wants to give them.  The paper proposes MOMMS for out-of-core use with
 * the slow level reached by explicit transfers overlapped with computation (Sec. 7);
 * here host memory is the slow level and HBM the fast one, with Resident C at the HBM
 * level (Sec. 2.2.1): a b x b block of C stays on the device while b x b blocks of A
 * and B are copied in along k, so A is read ceil(n/b) times, B ceil(m/b) times and C
 * read once (beta != 0) and written once (counts in the report: h2d_bytes, d2h_bytes).
 * Copies run on two streams of the handle, double-buffered against the block products,
 * which run on `stream` in the handle's mode (native / emulated / auto).
 * block: b, a multiple of 256, or 0 to take the largest b whose six b x b FP64 buffers
 * plus one b x b x b product's workspace fit in `device_bytes` (0 = half the free
 * device memory).  Asynchronous on `stream`: C is complete in host memory when the
 * stream is; A, B and C must stay valid until then.  Pinned host memory lets the copies
 * overlap the products; pageable memory works but the copies then block the host.
 * Block buffers are kept by the handle.  Errors: BLAS-style negative index (-14: block
 * not a multiple of 256), MOMMS_ERR_ALLOC, MOMMS_ERR_CUDA. */
int momms_gemm_host(momms_handle_t handle, int64_t m, int64_t n, int64_t k, double alpha,
                    const double* A, int64_t lda, const double* B, int64_t ldb, double beta,
                    double* C, int64_t ldc, size_t device_bytes, int64_t block,
                    momms_stream_t stream);

/* The member of momms_gemm_host at the HBM level, which with the handle's member inside each
 * block product (momms_set_member: the L2 level) and the accumulator tile (registers / TMEM)
 * makes a four-level member in the paper's naming (Sec. 3.2, Fig. 8's C4A2C0): host memory ->
 * HBM -> L2 -> SM.  0 = Resident C (default): a b x b block of C stays in HBM, A and B stream
 * along k (Sec. 2.2.1).  1 = Resident A: a b x b block of A stays in HBM while the blocks of B and
 * C of its block row stream through (Sec. 2.2.2): host<->device words A m k, B k n ceil(m/b),
 * C read m n (ceil(k/b) - 1 + [beta != 0]) and written m n ceil(k/b) -- better than Resident C
 * when k <= b and n is large (a rank-k update: A crosses the link once instead of ceil(n/b)
 * times).  Returns -2 for other values. */
int momms_set_host_resident(momms_handle_t handle, int resident);

/* ------------------------------------------------ allocation-free variant */
/* The emulated product (scale, split and slice-product kernels of EMULATED mode)
 * for callers that cannot allocate device memory: code that runs while a CUDA graph
 * is being captured, runtimes without a device allocator, or libraries whose
 * owners forbid any allocation outside their own memory pool.  The paper has no
 * counterpart; it exists only for such callers.
 *
 * It makes no cudaMalloc / cudaFree and calls no allocating routine.  All of its
 * scratch (exponents, flags, digit slices, FP64 recombination blocks, the status
 * word) lives in one file-scope device array of momms_noalloc_scratch_bytes()
 * bytes (64 MiB) that every GPU which loads the library holds until the process
 * exits.  The caller passes the inputs and the output as for momms_gemm_ex.
 *   - The first call on a device looks up the array's device address (with that
 *     device current); make the first call on each device before any stream
 *     capture.
 *   - Every call shares the array, which keeps the previous call's contents:
 *     calls that overlap on the GPU (other streams, other host threads on the same
 *     device) race on it.  Issue them in order on one stream.
 *   - slices must be given (1..16).  A problem whose scratch does not fit, or with m,
 *     n or k above 2^30, returns MOMMS_ERR_WORKSPACE before anything is enqueued;
 *     m = 0 or n = 0 is a no-op; k = 0 or alpha = 0 returns MOMMS_ERR_UNSUPPORTED
 *     (use momms_gemm_ex).
 *   - The return value covers the enqueueing only.  A bounded device wait that runs
 *     out writes MOMMS_ERR_TIMEOUT into the array's status word (C is then not
 *     valid); momms_noalloc_status() reports and clears it.
 *   - Arguments: op_a 1, op_b 2, m 3, n 4, k 5, slices 6, alpha 7, A 8, lda 9,
 *     B 10, ldb 11, beta 12, C 13, ldc 14, stream 15 (negative return = index). */
int momms_gemm_emulated_noalloc(int op_a, int op_b, int64_t m, int64_t n, int64_t k, int slices,
                                double alpha, const double* A, int64_t lda, const double* B,
                                int64_t ldb, double beta, double* C, int64_t ldc,
                                momms_stream_t stream);
size_t momms_noalloc_scratch_bytes(void);
/* Status of the allocation-free calls on the current device: waits for `stream`
 * (all calls enqueued on it before this one), then stores in *status MOMMS_OK, or
 * MOMMS_ERR_TIMEOUT if a bounded device wait of one of them ran out since the last
 * read, and clears the word.  Allocates nothing.  Returns -2 for status = NULL,
 * MOMMS_ERR_CUDA if the copy or the synchronisation fails. */
int momms_noalloc_status(momms_stream_t stream, int* status);

/* ---------------------------------------------------------------- tuning */
/* A plan: what runs the products of one size bucket (ceil log2 of m, n, k, and the two
 * transpositions).  The paper's point that different members win under different shapes and
 * bandwidths (Sec. 2.3, Sec. 5.4, Fig. 11) made operational: the tuner times the candidates
 * on the device and keeps the fastest.  Zero in tile_n / scheme / cta_pairs means the
 * library's own rule; a handle setting that is not automatic overrides the plan's. */
typedef struct {
    int tuned;      /* 1: from momms_tune / a plan file; 0: the built-in default       */
    int mode;       /* MOMMS_MODE_NATIVE or MOMMS_MODE_EMULATED                         */
    int member;     /* MOMMS_MEMBER_C2 .. A1                                            */
    int slices;     /* 0 = data-driven                                                  */
    int tile_n;     /* emulated tile width: 0 = automatic, 96 or 192                    */
    int scheme;     /* MOMMS_SCHEME_AUTO / SLICES / MODULI                              */
    int cta_pairs;  /* 0 = automatic, 1 = off, 2 = on (momms_set_cta_pairs)             */
} momms_plan_t;
/* Time the candidate plans for the size buckets of the given shapes (count triples
 * m[i], n[i], k[i]; op_a[i] / op_b[i] the transpositions, NULL = all N) on `stream`, on
 * uniform[-1,1] data with the data-driven slice count: the native engine, and for the
 * emulated engine every member (C2, A2, B2, A1) x tile width (192, 96) x encoding (digit
 * slices, moduli), moduli on 192-wide tiles with and without CTA pairs.  Each candidate
 * runs once untimed, then at least three timed calls and at least 20 ms of them (CUDA
 * events on `stream`, mean).  The fastest becomes the bucket's plan; buckets that already
 * have one are skipped.  The plan table is persisted to `path` (a small text file; NULL =
 * do not persist); a readable file is loaded first.  With the environment variable
 * MOMMS_TUNE_LOG set to a path, every candidate's time is appended there as a text line.
 * Single products (momms_gemm, momms_gemm_ex and the calls built on them) use the plan of
 * their bucket; batched calls take each problem's mode and encoding from its bucket's plan.
 * Returns -3 / -4 for a bad count or NULL size arrays, -7 for a bad transposition. */
int momms_tune_ex(momms_handle_t handle, const char* path, int64_t count, const int64_t* m,
                  const int64_t* n, const int64_t* k, const int* op_a, const int* op_b,
                  momms_stream_t stream);
/* momms_tune_ex with every transposition N. */
int momms_tune(momms_handle_t handle, const char* path, int64_t count, const int64_t* m,
               const int64_t* n, const int64_t* k, momms_stream_t stream);
/* Load a plan table written by momms_tune (a missing or mismatching file is
 * ignored and reported as MOMMS_ERR_IO). */
int momms_load_plans(momms_handle_t handle, const char* path);
/* The plan the handle holds for the bucket of (op_a, op_b, m, n, k): tuned, or the built-in
 * default (tuned = 0).  Returns -2 .. -7 for a bad argument (index). */
int momms_get_plan(momms_handle_t handle, int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                   momms_plan_t* plan);

/* ------------------------------------------------------- schedule query */
/* The member's tile order (host side, no GPU needed): the i-th tile taken by CTA `cta`
 * of `ctas` persistent CTAs over a tiles_m x tiles_n tile grid (group = tile rows per
 * group of the C2 raster; <= 0 means the emulated kernel's default for `ctas` CTAs, see
 * momms_set_raster_group).  Returns 1 and writes (tm, tn), 0 when that CTA
 * has no i-th tile, or a negative argument index.  The kernels use the same function. */
int momms_member_tile(int member, int group, int64_t cta, int64_t ctas, int64_t i, int tiles_m,
                      int tiles_n, int* tm, int* tn);

/* The tile order of a triangular product (the modular symmetric rank-k update; host
 * side, no GPU needed): of an n x n C cut into 128-row by tile_n-column tiles
 * (tile_n = 96 or 192), the t-th tile that meets the uplo triangle, tile row by tile
 * row.  Returns 1 and writes (tm, tn), 0 when t is past the last such tile, or a
 * negative argument index (uplo -1, tile_n -2, n -3, t -4, tm -5, tn -6).  *count, when
 * not null, receives the number of such tiles.  The kernel uses the same function. */
int momms_tri_tile(int uplo, int tile_n, int64_t n, int64_t t, int* tm, int* tn, int64_t* count);

/* ------------------------------------------------------- microbenchmarks */
/* Peak probes used as roofline denominators: kind 0 = FP64 DMMA, 1 = FP64 DFMA; the
 * tcgen05 kind::f16 (FP32 accumulate) instruction shapes of the product kernels issued back
 * to back from operands resident in shared memory: 2 = M 128 x N 192 on one CTA per SM,
 * 3 = M 128 x N 256, 4 = M 256 x N 192 on CTA pairs (cta_group::2), 5 = M 256 x N 256 on CTA
 * pairs.  Writes the achieved rate in TFLOP/s (0 if a bounded wait ran out) to *tflops.
 * Synchronous. */
int momms_probe_peak(int kind, double* tflops, momms_stream_t stream);
/* Copies `bytes` of device memory from src to dst, `repeats` times over, on `ctas` SMs
 * (one CTA of 1024 threads per SM; 0 = every SM), asynchronously on `stream`, with
 * streaming cache hints.  Both pointers 16-byte aligned, bytes a multiple of 16, the
 * ranges disjoint; the caller owns both buffers.  An HBM bandwidth probe, and the
 * background traffic of the bandwidth-ratio experiment: launched on a second stream it
 * takes HBM bandwidth away from a product running beside it on the other SMs, the GPU
 * counterpart of the paper's lowered main-memory bandwidth (Sec. 5.2, Fig. 6).  The
 * paper has no such routine.  Returns -1 (dst), -2 (src), -3 (bytes), -4 (ctas) or
 * -5 (repeats) for a bad argument, MOMMS_ERR_CUDA if the launch fails. */
int momms_stream_copy(void* dst, const void* src, size_t bytes, int ctas, int repeats,
                      momms_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* MOMMS_H */
