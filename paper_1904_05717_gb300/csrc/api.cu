// api.cu -- the C ABI (include/momms.h): handles, BLAS argument rules,
// workspace, mode / member / slice-count selection, the emulated pipeline,
// backward, batched, plan cache and peak probes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/momms.h"
#include "internal.h"
#include "raster.cuh"

using momms::BatchProblem;

namespace {

constexpr int kHandleMagic = 0x4D4F4D53;  // "MOMS"
constexpr int kDigitBits = 7;             // beta: 7-bit digits, FP32 chunk of 1024 products
constexpr int kAutoSliceMax = 14;         // workspace sized for this many slices in AUTO
// Whether the residue product runs on CTA pairs (one MMA over two SMs) when the handle says AUTO.
constexpr bool kCtaPairsAuto = false;
bool pairs_on(int mode) { return mode == 2 || (mode == 0 && kCtaPairsAuto); }

// What runs one product of a size bucket: the engine, the member (tile order), the slice count,
// and for the emulated engine the tile width, the integer encoding and the CTA pairs.  Zero in the
// last four means "the library's rule" (the handle's own setting takes precedence when it is not
// automatic).
struct Plan {
    int mode;
    int member;
    int slices;  // 0 = data-driven rule
    int tile_n;  // 0 = automatic, 96, 192
    int scheme;  // MOMMS_SCHEME_AUTO / SLICES / MODULI
    int pairs;   // 0 = automatic, 1 = off, 2 = on
};

// size bucket = (ceil log2 m, ceil log2 n, ceil log2 k) and the two transpositions
inline int lg2c(int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x && b < 62) ++b;
    return b;
}
inline uint32_t bucket_key(int64_t m, int64_t n, int64_t k, int opa = MOMMS_OP_N, int opb = MOMMS_OP_N) {
    return static_cast<uint32_t>(lg2c(m) | (lg2c(n) << 8) | (lg2c(k) << 16) | ((opa & 1) << 24) |
                                 ((opb & 1) << 25));
}

inline size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }
inline int64_t round_up(int64_t x, int64_t q) { return (x + q - 1) / q * q; }

}  // namespace

struct momms_handle_s {
    int magic = kHandleMagic;
    int mode = MOMMS_MODE_AUTO;
    int member = MOMMS_MEMBER_AUTO;
    int slices = 0;
    int digit_bits = kDigitBits;
    int max_ctas = 0;               // grid cap of the single-product launches (0 = default)
    int tile_n = 0;                 // emulated tile width request (96 / 192; 0 = automatic)
    int group = 0;                  // C2 raster group in tile rows (0 = default)
    int scheme = MOMMS_SCHEME_AUTO; // integer encoding of the emulated product
    int crt_fusion = 0;             // 0 auto, 1 separate reconstruction launch, 2 fused
    int cta_pairs = 0;              // 0 auto, 1 off, 2 on: residue products on CTA pairs (cta_group::2)
    int host_resident = 0;          // momms_gemm_host: 0 = Resident C, 1 = Resident A at the HBM level
    void* user_ws = nullptr;
    size_t user_ws_bytes = 0;
    void* own_ws = nullptr;
    size_t own_ws_bytes = 0;
    int32_t* status = nullptr;  // device word
    int* spread_dev = nullptr;  // device pair of spread values (AUTO slice rule)
    bool plan_mode = true;               // data-driven S chosen on the device (else: host readback)
    momms::EmuPlan* plan_dev = nullptr;  // device plan of the last data-driven product
    bool report_pending = false;         // the report's S / moduli / width are still in plan_dev
    int64_t ntab_k = -1;                 // contraction length and scheme the plan table was built for
    int ntab_scheme = -1;
    momms::EmuPlanTable ntab{};
    int* spread_host = nullptr; // pinned
    cudaEvent_t spread_ready = nullptr;
    int last_auto_slices = 6;   // speculative slice count for the next AUTO call
    bool last_auto_mod = false; // ... whether it went to the modular encoding
    int last_auto_bits = 0;     // ... and with which operand width
    momms_report_t report{};
    BatchProblem* dev_probs = nullptr;
    size_t dev_probs_cap = 0;
    std::vector<BatchProblem> host_probs;  // the table last uploaded to dev_probs
    // batched emulated products: per-problem statistics, device tables, spread readback
    void* batch_meta = nullptr;
    size_t batch_meta_cap = 0;
    void* batch_tables = nullptr;
    size_t batch_tables_cap = 0;
    std::vector<char> host_tables;         // the bytes last uploaded to batch_tables
    int* spread_host_big = nullptr;        // pinned, 2 per problem
    size_t spread_host_cap = 0;
    std::unique_ptr<momms::CrtReconSet> crt_set;  // reconstruction constants by moduli count
    std::map<uint32_t, Plan> plans;
    // out-of-core products (momms_gemm_host): block buffers, copy streams, slot events
    void* ooc_buf = nullptr;
    size_t ooc_bytes = 0;
    cudaStream_t ooc_in = nullptr, ooc_out = nullptr;
    cudaEvent_t ooc_ev[11] = {};
    // the B operand's scale and split run on a second stream beside A's (fork / join events)
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // per-launch timing of the dominant product launch (momms_set_kernel_timing): an event pair
    // recorded on the launching stream around each slice- / residue-product launch
    std::vector<cudaEvent_t> kev;  // 2 per launch: before, after
    size_t kev_used = 0;           // pairs recorded since the last read
};

namespace {

bool valid(momms_handle_t h) { return h && h->magic == kHandleMagic; }

void reset_report(momms_handle_t h) {
    h->report = momms_report_t{};
    h->report_pending = false;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return MOMMS_OK;
    return MOMMS_ERR_CUDA;
}

// Workspace carve-up of one emulated product.
struct EmuLayout {
    int64_t m_pad, n_pad, k_pad;
    size_t off_e, off_ef, off_f, off_ff, off_l1a, off_l1b, off_Ad, off_Bd, off_scratch, scratch_bytes, off_res,
        total;
};

// The modular encoding in place of the S(S+1)/2 digit pairs: the moduli for `bits`-bit
// operands, used when allowed and (AUTO) when they save at least two tensor products.
bool use_moduli(int scheme, int bits, int S, int beta, int64_t k, momms::CrtConsts* c, momms::CrtRecon* r) {
    if (scheme == MOMMS_SCHEME_SLICES || beta != kDigitBits || S < 1) return false;
    if (!momms::crt_plan(bits, k, c, r)) return false;
    return scheme == MOMMS_SCHEME_MODULI || c->N + 2 <= S * (S + 1) / 2;
}

// Moduli the workspace holds room for: those of a fixed S, the most any S may take in AUTO.
int moduli_reserved(int scheme, int S, int64_t k) {
    if (scheme == MOMMS_SCHEME_SLICES) return 0;
    if (S <= 0) return momms::kCrtMaxModuli;
    momms::CrtConsts c;
    momms::CrtRecon r;
    return use_moduli(scheme, kDigitBits * S, S, kDigitBits, k, &c, &r) ? c.N : 0;
}

// S digit planes per operand (or N residue planes when more), the recombination scratch and,
// for N moduli, the N residue bytes of every element of C.  shared_b: the second operand is the
// first one transposed (symmetric rank-k update), its planes are the first operand's.
EmuLayout emu_layout(int64_t m, int64_t n, int64_t k, int S, int max_ctas, int N = 0, bool shared_b = false) {
    EmuLayout L{};
    // digit slices hold exactly m (n) rows: ragged tiles are zero-filled by the copy engine
    L.m_pad = std::max<int64_t>(m, 1);
    L.n_pad = std::max<int64_t>(n, 1);
    L.k_pad = round_up(std::max<int64_t>(k, 1), momms::kEmuBK);
    size_t o = 0;
    L.off_e = o;   o += align256(L.m_pad * sizeof(int32_t));
    L.off_ef = o;  o += align256(L.m_pad);
    L.off_f = o;   o += align256(L.n_pad * sizeof(int32_t));
    L.off_ff = o;  o += align256(L.n_pad);
    L.off_l1a = o; o += align256(L.m_pad * sizeof(float));
    L.off_l1b = o; o += align256(L.n_pad * sizeof(float));
    const int planes = std::max(S, N);
    L.off_Ad = o;  o += align256(static_cast<size_t>(planes) * L.m_pad * L.k_pad * 2);
    L.off_Bd = o;
    if (shared_b) L.off_Bd = L.off_Ad;
    else o += align256(static_cast<size_t>(planes) * L.n_pad * L.k_pad * 2);
    L.scratch_bytes = momms::emu_scratch_bytes_tail(m, n, k, S, max_ctas, kDigitBits);
    L.off_scratch = o; o += align256(L.scratch_bytes);
    L.off_res = o; o += align256(static_cast<size_t>(N) * L.m_pad * L.n_pad);
    L.total = o;
    return L;
}

int ensure_workspace(momms_handle_t h, size_t bytes, void** ws) {
    if (h->user_ws) {
        if (h->user_ws_bytes < bytes) return MOMMS_ERR_WORKSPACE;
        *ws = h->user_ws;
        return MOMMS_OK;
    }
    if (h->own_ws_bytes < bytes) {
        if (h->own_ws) {
            cudaDeviceSynchronize();  // the old block may still be in use by enqueued work
            cudaFree(h->own_ws);
            h->own_ws = nullptr;
            h->own_ws_bytes = 0;
        }
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return MOMMS_ERR_ALLOC;
        }
        h->own_ws = p;
        h->own_ws_bytes = bytes;
    }
    *ws = h->own_ws;
    return MOMMS_OK;
}

// Grows a handle-owned device buffer (contents are not kept).
int grow_device(void** buf, size_t* cap, size_t bytes) {
    if (*cap >= bytes && *buf) return MOMMS_OK;
    if (*buf) {
        cudaDeviceSynchronize();  // enqueued work may still use the old block
        cudaFree(*buf);
        *buf = nullptr;
        *cap = 0;
    }
    if (cudaMalloc(buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        *buf = nullptr;
        return MOMMS_ERR_ALLOC;
    }
    *cap = bytes;
    return MOMMS_OK;
}

// C := beta*C on all of C (tri 0), its lower (1) or its upper (2) triangle.
__global__ void scale_c_kernel(int64_t m, int64_t n, double beta, double* C, int64_t ldc, int tri) {
    const int64_t total = m * n;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = idx % m, j = idx / m;
        if ((tri == 1 && j > i) || (tri == 2 && j < i)) continue;
        double* c = C + i + j * ldc;
        *c = (beta == 0.0) ? 0.0 : beta * *c;
    }
}

int scale_c(int64_t m, int64_t n, double beta, double* C, int64_t ldc, cudaStream_t s, int tri = 0) {
    if (beta == 1.0) return MOMMS_OK;
    int64_t blocks = (m * n + 255) / 256;
    blocks = std::min<int64_t>(blocks, int64_t(momms::device_sm_count()) * 16);
    scale_c_kernel<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(m, n, beta, C, ldc, tri);
    return cuda_fail(cudaGetLastError());
}

// Slice count from the exponent spread of the inputs.  spread_a (spread_b) is the
// largest, over rows of op(A) (columns of op(B)), of log2(2^e * k / sum|x|): how many
// bits the vector maximum sits above the mean magnitude.  The truncation error of
// the digits is relative to 2^(e_i + f_j) while the bound is relative to
// (|A||B|)_ij, so wide spreads need more digit bits; with random signs the error
// grows like sqrt(k) while the bound grows like k^2 * mean|a||b|, hence the
// -1.5 log2 k.  Coefficients were fitted to the CPU oracle's measured error over
// uniform, normal and (u - 0.5) exp(phi g) inputs (phi = 1, 2, 4) at k = 64..16384
// and hold every case there at least 10x inside the bound; the result is clamped
// to [3, 14].
// The k-dependent part of the rule: bits = rule_c0(k) + 1.25 (s_A + s_B).  The device plan kernel
// evaluates the same expression with the same IEEE operations in the same order.
double rule_c0(int64_t k) {
    const double L = std::log2(static_cast<double>(std::max<int64_t>(k, 1)));
    return 55.25 - 1.5 * L + 1.5 * std::max(0.0, 12.0 - L);
}

int slices_from_spread(double spread_a, double spread_b, int64_t k, int beta, double* bits_out) {
    const double bits = rule_c0(k) + 1.25 * (spread_a + spread_b);
    if (bits_out) *bits_out = bits;
    int S = static_cast<int>(std::ceil(bits / static_cast<double>(beta)));
    return std::min(std::max(S, 3), kAutoSliceMax);
}

Plan default_plan(int64_t m, int64_t n, int64_t k) {
    Plan p{};
    const double flops = 2.0 * m * n * k;
    // the FP64 tensor pipe is ~1 TFLOP/s; emulation pays off once its fixed costs (five to
    // seven launches, a slice-count readback, 128-row tiles) are amortised: measured 3.5x the
    // native rate at 512^3 (2.7e8 flops).  Thin products qualify too (a 128 x 8192 x 128 block
    // of a triangular solve: the modular encoding's units are tiles x moduli, enough for all SMs)
    const bool big = std::min(m, n) >= 64 && k >= 64 && flops >= 2.0e8;
    p.mode = big ? MOMMS_MODE_EMULATED : MOMMS_MODE_NATIVE;
    p.member = MOMMS_MEMBER_C2;
    p.slices = 0;
    return p;
}

Plan pick_plan(momms_handle_t h, int64_t m, int64_t n, int64_t k, int opa = MOMMS_OP_N, int opb = MOMMS_OP_N) {
    Plan p = default_plan(m, n, k);
    auto it = h->plans.find(bucket_key(m, n, k, opa, opb));
    if (it != h->plans.end()) p = it->second;
    if (h->mode != MOMMS_MODE_AUTO) p.mode = h->mode;
    if (h->member != MOMMS_MEMBER_AUTO) p.member = h->member;
    if (h->slices > 0) p.slices = h->slices;
    return p;
}

int run_native(momms_handle_t h, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
               const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
               int64_t ldc, int member, cudaStream_t s) {
    int ctas = 0, group = 0;
    cudaError_t e = momms::launch_native_gemm(opa, opb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                                              member, h->max_ctas, h->group, s, &ctas, &group);
    if (e == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return MOMMS_ERR_CUDA;
    reset_report(h);
    h->report.ctas = ctas;
    h->report.group = group;
    h->report.mode = MOMMS_MODE_NATIVE;
    h->report.member = member;
    h->report.tile_m = momms::kNativeBM;
    h->report.tile_n = momms::kNativeBN;
    h->report.k_passes = 1;
    h->report.launches = 1;
    return MOMMS_OK;
}

int ensure_aux(momms_handle_t h) {
    if (!h->aux && cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (!h->ev_fork && cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    if (!h->ev_join && cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    return MOMMS_OK;
}

// The work on the second stream joins the caller's stream.
int join_aux(momms_handle_t h, cudaStream_t s) {
    if (cudaEventRecord(h->ev_join, h->aux) != cudaSuccess || cudaStreamWaitEvent(s, h->ev_join, 0) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    return MOMMS_OK;
}

// Event pair around one product launch when kernel timing is on and a pair is left (else no-op).
struct KernelTimer {
    momms_handle_t h;
    cudaStream_t s;
    cudaEvent_t* pair = nullptr;
    KernelTimer(momms_handle_t h_, cudaStream_t s_) : h(h_), s(s_) {
        if (2 * (h->kev_used + 1) <= h->kev.size()) {
            pair = &h->kev[2 * h->kev_used];
            if (cudaEventRecord(pair[0], s) != cudaSuccess) {
                cudaGetLastError();
                pair = nullptr;
            }
        }
    }
    void done() {
        if (pair && cudaEventRecord(pair[1], s) == cudaSuccess) ++h->kev_used;
        pair = nullptr;
    }
};

// tri = 1 / 2: the symmetric rank-k update C := alpha op(A) op(A)^T + beta C on the lower / upper
// triangle (m = n, B = A with opb the other transposition of A): one scale and residue split
// serve both operands, the residue products visit the tiles that meet the triangle and the
// reconstruction writes only the triangle.  When the slice encoding is chosen instead it returns
// kSlicesChosen before the products (only the scale, the spread and a guessed split have run).
// kcap (triangular product): op(A) or op(B) is triangular with zeros stored elsewhere; the
// modular encoding's residue products skip each tile's zero k range (EmuGemmArgs::kcap).
constexpr int kSlicesChosen = 1;

// Reconstruction constants of every moduli count (built once per handle).
const momms::CrtReconSet& crt_set(momms_handle_t h) {
    if (!h->crt_set) {
        h->crt_set.reset(new momms::CrtReconSet{});
        for (int nm = 1; nm <= momms::kCrtMaxModuli; ++nm) {
            momms::CrtConsts cn;
            momms::crt_consts(nm, 0, &cn, &h->crt_set->by_n[nm]);
        }
    }
    return *h->crt_set;
}

// The plan table of the device plan kernel for contraction length k: the rule's constant and the
// moduli count of every operand width (cached per handle for the last k and scheme).
const momms::EmuPlanTable& plan_table(momms_handle_t h, int64_t k, int n_alloc) {
    if (h->ntab_k != k || h->ntab_scheme != h->scheme || h->ntab.n_alloc != n_alloc) {
        momms::EmuPlanTable& t = h->ntab;
        t = momms::EmuPlanTable{};
        t.c0 = rule_c0(k);
        t.smax = kAutoSliceMax;
        t.n_alloc = n_alloc;
        t.scheme_moduli = h->scheme == MOMMS_SCHEME_MODULI;
        t.tri = 0;
        for (int w = 1; w <= momms::kPlanMaxBits && n_alloc > 0; ++w) {
            momms::CrtConsts c;
            momms::CrtRecon r;
            t.ntab[w] = momms::crt_plan(w, k, &c, &r) ? static_cast<uint8_t>(c.N) : 0;
        }
        h->ntab_k = k;
        h->ntab_scheme = h->scheme;
    }
    return h->ntab;
}

// The data-driven product with every choice made on the device: scale and spreads, the plan kernel
// (S, operand width, moduli or slices), then both encodings' splits and products and the
// reconstruction, each reading the plan at launch time and returning at once when the plan chose
// the other encoding.  Nothing is read back, so the call only enqueues work (and can be captured
// in a CUDA graph once the workspace exists).  The report's slice count, moduli and width are
// fetched from the plan when the report is asked for.
int run_emulated_planned(momms_handle_t h, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
                         const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                         int64_t ldc, int member, cudaStream_t s, int kcap) {
    const int bb = h->digit_bits;
    const int S_alloc = kAutoSliceMax;
    const int N_alloc = k <= momms::crt_max_k() ? moduli_reserved(h->scheme, 0, k) : 0;  // one exact pass
    EmuLayout L = emu_layout(m, n, k, S_alloc, h->max_ctas, N_alloc);
    if (std::max(L.m_pad, L.n_pad) > (int64_t(1) << 30)) return MOMMS_ERR_UNSUPPORTED;
    void* ws = nullptr;
    int rc = ensure_workspace(h, L.total, &ws);
    if (rc) return rc;
    rc = ensure_aux(h);
    if (rc) return rc;
    char* w = static_cast<char*>(ws);
    int32_t* e = reinterpret_cast<int32_t*>(w + L.off_e);
    uint8_t* ef = reinterpret_cast<uint8_t*>(w + L.off_ef);
    float* l1a = reinterpret_cast<float*>(w + L.off_l1a);
    int32_t* f = reinterpret_cast<int32_t*>(w + L.off_f);
    uint8_t* ff = reinterpret_cast<uint8_t*>(w + L.off_ff);
    float* l1b = reinterpret_cast<float*>(w + L.off_l1b);
    void* Ad = w + L.off_Ad;
    void* Bd = w + L.off_Bd;
    uint8_t* res = reinterpret_cast<uint8_t*>(w + L.off_res);
    const momms::EmuPlanTable& table = plan_table(h, k, N_alloc);
    const momms::CrtReconSet& set = crt_set(h);
    cudaStream_t sb = h->aux;
    int64_t launches = 0;
    auto fork = [&]() {
        return cudaEventRecord(h->ev_fork, s) == cudaSuccess && cudaStreamWaitEvent(sb, h->ev_fork, 0) == cudaSuccess;
    };
    // statistics of A on the caller's stream, of B on the second stream, then the plan
    if (cudaMemsetAsync(h->spread_dev, 0, 2 * sizeof(int), s) != cudaSuccess || !fork()) return MOMMS_ERR_CUDA;
    if (momms::launch_emu_scale(0, opa, m, k, A, lda, e, ef, l1a, s) != cudaSuccess ||
        momms::launch_emu_scale(1, opb, n, k, B, ldb, f, ff, l1b, sb) != cudaSuccess ||
        momms::launch_emu_spread(m, k, e, ef, l1a, h->spread_dev, s) != cudaSuccess ||
        momms::launch_emu_spread(n, k, f, ff, l1b, h->spread_dev + 1, sb) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += momms::emu_scale_kernel_count(0, opa) + momms::emu_scale_kernel_count(1, opb) + 2;
    rc = join_aux(h, s);
    if (rc) return rc;
    if (momms::launch_emu_plan(h->spread_dev, table, h->plan_dev, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    launches += 1;
    // both encodings' operand passes (the one the plan did not choose returns at once)
    if (!fork()) return MOMMS_ERR_CUDA;
    momms::CrtConsts call;
    momms::CrtRecon rall;
    momms::crt_consts(momms::kCrtMaxModuli, 56, &call, &rall);  // every modulus; N and width from the plan
    if (N_alloc > 0) {
        if (momms::launch_emu_residues(0, opa, m, k, A, lda, e, ef, call, Ad, L.m_pad, L.k_pad, s, h->plan_dev) !=
                cudaSuccess ||
            momms::launch_emu_residues(1, opb, n, k, B, ldb, f, ff, call, Bd, L.n_pad, L.k_pad, sb, h->plan_dev) !=
                cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 2;
    }
    if (momms::launch_emu_split(0, opa, m, k, A, lda, e, ef, S_alloc, bb, Ad, L.m_pad, L.k_pad, s, 0, h->plan_dev) !=
            cudaSuccess ||
        momms::launch_emu_split(1, opb, n, k, B, ldb, f, ff, S_alloc, bb, Bd, L.n_pad, L.k_pad, sb, 0, h->plan_dev) !=
            cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += 2;
    rc = join_aux(h, s);
    if (rc) return rc;
    momms::EmuGemmArgs a{};
    a.m = m; a.n = n; a.k = k; a.beta = bb;
    a.Ad = Ad; a.Bd = Bd; a.m_pad = L.m_pad; a.n_pad = L.n_pad; a.k_pad = L.k_pad;
    a.e = e; a.ef = ef; a.f = f; a.ff = ff;
    a.alpha = alpha; a.beta_c = beta; a.C = C; a.ldc = ldc;
    a.member = member; a.group = h->group;
    a.scratch = w + L.off_scratch; a.scratch_bytes = L.scratch_bytes;
    a.status = h->status; a.max_ctas = h->max_ctas; a.tile_n = h->tile_n;
    a.plan = h->plan_dev;
    int passes = 0, used_ctas = 0, used_group = 0, used_launches = 0, used_pairs = 0;
    a.used_ctas = &used_ctas; a.used_group = &used_group; a.used_launches = &used_launches;
    a.used_pairs = &used_pairs;
    // the digit encoding's products (nothing to do when the plan chose moduli) ...
    a.withhold = momms::emu_debug_take_withhold();  // (test hook: whichever launch the plan runs)
    momms::EmuGemmArgs as = a;
    as.S = S_alloc;
    cudaError_t ce;
    {
        std::unique_ptr<KernelTimer> timer;  // (with moduli possible, the modular launch below is the one timed)
        if (N_alloc == 0) timer.reset(new KernelTimer(h, s));
        ce = momms::launch_emu_slice_gemm(as, &passes, s);
        if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        if (timer) timer->done();
        launches += used_launches;
    }
    // ... and the modular encoding's residue products and reconstruction (nothing when it chose slices)
    if (N_alloc > 0) {
        momms::EmuGemmArgs am = a;
        am.S = momms::kCrtMaxModuli;
        am.crt = &call;
        am.res = res;
        am.kcap = kcap;
        am.cta_pairs = pairs_on(h->cta_pairs) ? 1 : 0;
        int mpasses = 0;
        KernelTimer timer(h, s);
        ce = momms::launch_emu_slice_gemm(am, &mpasses, s);
        if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        timer.done();
        launches += used_launches;
        if (momms::launch_crt_reconstruct_plan(m, n, res, set, h->plan_dev, e, ef, f, ff, alpha, beta, C, ldc, s) !=
            cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 1;
    }
    reset_report(h);
    h->report.ctas = used_ctas;
    h->report.group = used_group;
    h->report.mode = MOMMS_MODE_EMULATED;
    h->report.member = member;
    h->report.digit_bits = bb;
    h->report.k_passes = passes;
    h->report.tile_m = momms::kEmuBM;
    h->report.tile_n = momms::emu_pick_bn(m, n, k, h->tile_n, N_alloc > 0 ? N_alloc : 1);
    h->report.launches = launches;
    h->report.cta_pairs = used_pairs;
    h->report_pending = true;  // slices, moduli, operand_bits and est_err_ratio come from the plan
    return MOMMS_OK;
}

int run_emulated(momms_handle_t h, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
                 const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                 int64_t ldc, int member, int S, cudaStream_t s, int tri = 0, int kcap = 0) {
    const int bb = h->digit_bits;
    h->report_pending = false;
    // (the fused reconstruction needs the moduli count at launch: it keeps the host plan)
    if (S == 0 && !tri && bb == kDigitBits && h->plan_mode && h->crt_fusion != 2)
        return run_emulated_planned(h, opa, opb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, member, s, kcap);
    if (tri && (m != n || A != B || opa == opb)) return MOMMS_ERR_UNSUPPORTED;
    if (S > MOMMS_MAX_SLICES) return MOMMS_ERR_UNSUPPORTED;
    const int S_alloc = S > 0 ? S : kAutoSliceMax;
    const int N_alloc = moduli_reserved(h->scheme, S, k);
    EmuLayout L = emu_layout(m, n, k, S_alloc, h->max_ctas, N_alloc, tri != 0);
    if (std::max(L.m_pad, L.n_pad) > (int64_t(1) << 30)) return MOMMS_ERR_UNSUPPORTED;
    void* ws = nullptr;
    int rc = ensure_workspace(h, L.total, &ws);
    if (rc) return rc;
    char* w = static_cast<char*>(ws);
    int32_t* e = reinterpret_cast<int32_t*>(w + L.off_e);
    uint8_t* ef = reinterpret_cast<uint8_t*>(w + L.off_ef);
    float* l1a = reinterpret_cast<float*>(w + L.off_l1a);
    void* Ad = w + L.off_Ad;
    // a triangle's second operand is the first one transposed: the same exponents, flags and planes
    int32_t* f = tri ? e : reinterpret_cast<int32_t*>(w + L.off_f);
    uint8_t* ff = tri ? ef : reinterpret_cast<uint8_t*>(w + L.off_ff);
    float* l1b = tri ? l1a : reinterpret_cast<float*>(w + L.off_l1b);
    void* Bd = w + L.off_Bd;  // = Ad for a triangle
    void* scratch = w + L.off_scratch;
    uint8_t* res = reinterpret_cast<uint8_t*>(w + L.off_res);
    int64_t launches = 0;
    cudaError_t ce;
    const bool need_stats = (S == 0);
    momms::CrtConsts cc{};
    momms::CrtRecon cr{};
    bool mod = false;        // the modular encoding serves this product
    bool res_ready = false;  // the planes hold residues of the final width
    int mbits = bb * S;      // operand width of the modular encoding
    // A's scale and split run on the caller's stream, B's on a second stream forked from it, so
    // that the two HBM-bound passes overlap; the slice products wait for both.
    rc = ensure_aux(h);
    if (rc) return rc;
    cudaStream_t sb = h->aux;
    if (need_stats && cudaMemsetAsync(h->spread_dev, 0, 2 * sizeof(int), s) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (cudaEventRecord(h->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(sb, h->ev_fork, 0) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    ce = momms::launch_emu_scale(0, opa, m, k, A, lda, e, ef, need_stats ? l1a : nullptr, s);
    if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
    if (!tri) {
        ce = momms::launch_emu_scale(1, opb, n, k, B, ldb, f, ff, need_stats ? l1b : nullptr, sb);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += momms::emu_scale_kernel_count(1, opb);
    }
    launches += momms::emu_scale_kernel_count(0, opa);
    double est = 0.0;
    int split_done = 0;  // slices already written
    if (S == 0) {
        // Data-driven slice count: the spreads are reduced on the device and read back.  While the
        // readback is in flight the digits are already split for a guessed S (the last call's):
        // a slice's digits do not depend on S, so only missing slices are added afterwards.
        if (momms::launch_emu_spread(m, k, e, ef, l1a, h->spread_dev, s) != cudaSuccess) return MOMMS_ERR_CUDA;
        if (!tri && momms::launch_emu_spread(n, k, f, ff, l1b, h->spread_dev + 1, sb) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        rc = join_aux(h, s);  // the readback needs both spreads
        if (rc) return rc;
        if (cudaMemcpyAsync(h->spread_host, h->spread_dev, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        if (!h->spread_ready || cudaEventRecord(h->spread_ready, s) != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += tri ? 1 : 2;
        const int guess = std::min(std::max(h->last_auto_slices, 1), S_alloc);
        momms::CrtConsts gc;
        momms::CrtRecon gr;
        const int guess_bits = h->last_auto_bits;
        const bool guess_mod = h->last_auto_mod && use_moduli(h->scheme, guess_bits, guess, bb, k, &gc, &gr) &&
                               gc.N <= N_alloc;
        if (guess_mod) {
            // residues depend on the operand width: they serve only if the readback confirms S
            ce = momms::launch_emu_residues(0, opa, m, k, A, lda, e, ef, gc, Ad, L.m_pad, L.k_pad, s);
            if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
            if (!tri) ce = momms::launch_emu_residues(1, opb, n, k, B, ldb, f, ff, gc, Bd, L.n_pad, L.k_pad, sb);
        } else if (!tri) {
            ce = momms::launch_emu_split(0, opa, m, k, A, lda, e, ef, guess, bb, Ad, L.m_pad, L.k_pad, s);
            if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
            ce = momms::launch_emu_split(1, opb, n, k, B, ldb, f, ff, guess, bb, Bd, L.n_pad, L.k_pad, sb);
        }
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        if (guess_mod || !tri) launches += tri ? 1 : 2;
        split_done = guess_mod || tri ? 0 : guess;
        if (cudaEventSynchronize(h->spread_ready) != cudaSuccess) return MOMMS_ERR_CUDA;
        const double sa = h->spread_host[0] / 16.0, sbs = tri ? sa : h->spread_host[1] / 16.0;
        double bits = 0.0;
        S = slices_from_spread(sa, sbs, k, bb, &bits);
        est = 0.1 * std::exp2(bits - static_cast<double>(bb) * S);  // the rule keeps a 10x margin
        h->last_auto_slices = S;
        // the modular encoding takes the rule's width itself (not rounded up to whole digits)
        mbits = std::min(bb * S, std::max(static_cast<int>(std::ceil(bits)), bb * S - bb + 1));
        mod = use_moduli(h->scheme, mbits, S, bb, k, &cc, &cr) && cc.N <= N_alloc;
        if (mod) est = 0.1 * std::exp2(bits - static_cast<double>(mbits));
        h->last_auto_mod = mod;
        h->last_auto_bits = mbits;
        res_ready = mod && guess_mod && mbits == guess_bits;
    } else {
        mod = use_moduli(h->scheme, mbits, S, bb, k, &cc, &cr) && cc.N <= N_alloc;
    }
    if (tri && !mod) {
        // the slice encoding's triangle is the batched slice-product path of the caller
        rc = join_aux(h, s);
        return rc ? rc : kSlicesChosen;
    }
    if (mod && !res_ready) {
        ce = momms::launch_emu_residues(0, opa, m, k, A, lda, e, ef, cc, Ad, L.m_pad, L.k_pad, s);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        if (!tri) {
            ce = momms::launch_emu_residues(1, opb, n, k, B, ldb, f, ff, cc, Bd, L.n_pad, L.k_pad, sb);
            if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        }
        launches += tri ? 1 : 2;
    } else if (!mod && S > split_done) {
        ce = momms::launch_emu_split(0, opa, m, k, A, lda, e, ef, S, bb, Ad, L.m_pad, L.k_pad, s, split_done);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        ce = momms::launch_emu_split(1, opb, n, k, B, ldb, f, ff, S, bb, Bd, L.n_pad, L.k_pad, sb, split_done);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += 2;
    }
    rc = join_aux(h, s);  // the slice products need B's exponents and digits
    if (rc) return rc;
    momms::EmuGemmArgs a{};
    a.m = m; a.n = n; a.k = k; a.S = mod ? cc.N : S; a.beta = bb;
    a.Ad = Ad; a.Bd = Bd; a.m_pad = L.m_pad; a.n_pad = L.n_pad; a.k_pad = L.k_pad;
    a.e = e; a.ef = ef; a.f = f; a.ff = ff;
    a.alpha = alpha; a.beta_c = beta; a.C = C; a.ldc = ldc;
    a.member = member; a.group = h->group;
    a.scratch = scratch; a.scratch_bytes = L.scratch_bytes;
    a.status = h->status; a.max_ctas = h->max_ctas; a.tile_n = h->tile_n;
    int passes = 0, used_ctas = 0, used_group = 0, used_launches = 0, used_pairs = 0;
    a.used_ctas = &used_ctas; a.used_group = &used_group; a.used_launches = &used_launches;
    a.used_pairs = &used_pairs;
    // the reconstruction inside the residue product's epilogue (the last modulus of each tile) only
    // on request: measured slower than the separate launch (8192^3: 11.9 against 10.4 ms per step --
    // twelve drain warps per SM rebuild C at a fraction of the separate kernel's rate and stall the
    // products behind them)
    const bool fuse = mod && h->crt_fusion == 2 && !tri;
    a.cta_pairs = pairs_on(h->cta_pairs) ? 1 : 0;
    if (mod) {
        a.crt = &cc;
        a.res = res;
        a.tri = tri;
        a.kcap = kcap;
        if (fuse) {
            // one counter per tile (either tile width), in the recombination scratch the modular
            // product does not use
            const int64_t tiles = ((m + momms::kEmuBM - 1) / momms::kEmuBM) * ((n + 95) / 96);
            if (static_cast<size_t>(tiles) * sizeof(int) > L.scratch_bytes) return MOMMS_ERR_UNSUPPORTED;
            a.crt_fuse = &cr;
            a.done = static_cast<int*>(scratch);
            if (cudaMemsetAsync(a.done, 0, static_cast<size_t>(tiles) * sizeof(int), s) != cudaSuccess)
                return MOMMS_ERR_CUDA;
        }
    }
    KernelTimer timer(h, s);
    ce = momms::launch_emu_slice_gemm(a, &passes, s);
    if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
    timer.done();
    launches += used_launches;
    if (mod && !fuse) {
        // C from the residues of the product (Chinese remainder theorem), scaled, alpha / beta
        ce = momms::launch_crt_reconstruct(m, n, res, cr, e, ef, f, ff, alpha, beta, C, ldc, s, tri);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += 1;
    }
    reset_report(h);
    h->report.ctas = used_ctas;
    h->report.group = used_group;
    h->report.mode = MOMMS_MODE_EMULATED;
    h->report.member = member;
    h->report.slices = S;
    h->report.digit_bits = bb;
    h->report.k_passes = passes;
    h->report.tile_m = momms::kEmuBM;
    h->report.tile_n = momms::emu_pick_bn(m, n, k, h->tile_n, mod ? cc.N : 1);
    h->report.launches = launches;
    h->report.est_err_ratio = est;
    h->report.moduli = mod ? cc.N : 0;
    h->report.operand_bits = mod ? mbits : bb * S;
    h->report.crt_fused = fuse ? 1 : 0;
    h->report.cta_pairs = used_pairs;
    return MOMMS_OK;
}

// Batched emulated products (op = N, N): 2 scale + 2 split launches over work lists and ONE
// persistent slice-product launch over the concatenated tiles of all problems.  With a fixed
// slice count nothing is read back, and a repeated call with the same problems only re-enqueues
// the five kernels (tables are uploaded only when they change), so it can be graph-captured.
// With the data-driven slice count the per-problem spreads are read back once per call.
int run_emulated_batched(momms_handle_t h, const std::vector<int64_t>& idx, const std::vector<int>& scheme_of,
                         const int64_t* m, const int64_t* n,
                         const int64_t* k, const double* alpha, const double* const* A, const int64_t* lda,
                         const double* const* B, const int64_t* ldb, const double* beta, double* const* C,
                         const int64_t* ldc, cudaStream_t s) {
    const int count = static_cast<int>(idx.size());
    const int bb = h->digit_bits;
    // ---- per-problem statistics region (exponents, flags, spreads)
    std::vector<size_t> off_e(count), off_ef(count), off_f(count), off_ff(count);
    size_t meta = align256(sizeof(int32_t) * 2 * static_cast<size_t>(count));  // spreads first
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        off_e[i] = meta;  meta += align256(sizeof(int32_t) * m[p]);
        off_ef[i] = meta; meta += align256(static_cast<size_t>(m[p]));
        off_f[i] = meta;  meta += align256(sizeof(int32_t) * n[p]);
        off_ff[i] = meta; meta += align256(static_cast<size_t>(n[p]));
    }
    int rc = grow_device(&h->batch_meta, &h->batch_meta_cap, meta);
    if (rc) return rc;
    char* mb = static_cast<char*>(h->batch_meta);
    int32_t* spreads = reinterpret_cast<int32_t*>(mb);

    std::vector<momms::EmuBatchPrep> prep(count);
    std::vector<int2> sa_items, sb_items, pa_items, pb_items;
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        momms::EmuBatchPrep& q = prep[i];
        q.A = A[p]; q.B = B[p]; q.lda = lda[p]; q.ldb = ldb[p];
        q.m = static_cast<int32_t>(m[p]); q.n = static_cast<int32_t>(n[p]); q.k = static_cast<int32_t>(k[p]);
        q.k_pad = static_cast<int32_t>(round_up(k[p], momms::kEmuBK));
        q.S = h->slices; q.beta = bb;
        q.enc = -1;  // encodings chosen on the host: every split launch takes the problems given to it
        q.e = reinterpret_cast<int32_t*>(mb + off_e[i]);
        q.ef = reinterpret_cast<uint8_t*>(mb + off_ef[i]);
        q.f = reinterpret_cast<int32_t*>(mb + off_f[i]);
        q.ff = reinterpret_cast<uint8_t*>(mb + off_ff[i]);
        q.spread = spreads + 2 * i;
        for (int64_t b = 0; b < momms::emu_batch_scale_a_blocks(m[p]); ++b) sa_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_scale_b_blocks(n[p]); ++b) sb_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_split_a_blocks(m[p], q.k_pad); ++b) pa_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_split_b_blocks(n[p], q.k_pad); ++b) pb_items.push_back(make_int2(i, (int)b));
    }
    if (sa_items.size() > INT32_MAX || pa_items.size() > INT32_MAX || pb_items.size() > INT32_MAX)
        return MOMMS_ERR_UNSUPPORTED;

    // ---- slice counts
    std::vector<int> S(count, h->slices);
    std::vector<double> rule_bits(count, 0.0);
    const bool auto_s = h->slices <= 0;
    // ---- device tables: [prep][items sa][sb][pa][pb][gemm table][modular: items pa][pb][gemm
    // table][reconstruction table][items]; rebuilt below once S is known
    std::vector<int2> pa_mod, pb_mod, crt_items;
    std::vector<momms::EmuBatchProblem> gemm_mod;
    std::vector<momms::CrtBatchProblem> crt_probs;
    size_t off_mod[5] = {0, 0, 0, 0, 0};
    auto upload = [&](const std::vector<momms::EmuBatchProblem>& gemm, size_t* off_gemm, size_t* off_items) -> int {
        std::vector<char> buf;
        auto put = [&](const void* src, size_t bytes) {
            size_t o = align256(buf.size());
            buf.resize(o + bytes);
            if (bytes) std::memcpy(buf.data() + o, src, bytes);
            return o;
        };
        put(prep.data(), sizeof(momms::EmuBatchPrep) * prep.size());
        off_items[0] = put(sa_items.data(), sizeof(int2) * sa_items.size());
        off_items[1] = put(sb_items.data(), sizeof(int2) * sb_items.size());
        off_items[2] = put(pa_items.data(), sizeof(int2) * pa_items.size());
        off_items[3] = put(pb_items.data(), sizeof(int2) * pb_items.size());
        *off_gemm = put(gemm.data(), sizeof(momms::EmuBatchProblem) * gemm.size());
        off_mod[0] = put(pa_mod.data(), sizeof(int2) * pa_mod.size());
        off_mod[1] = put(pb_mod.data(), sizeof(int2) * pb_mod.size());
        off_mod[2] = put(gemm_mod.data(), sizeof(momms::EmuBatchProblem) * gemm_mod.size());
        off_mod[3] = put(crt_probs.data(), sizeof(momms::CrtBatchProblem) * crt_probs.size());
        off_mod[4] = put(crt_items.data(), sizeof(int2) * crt_items.size());
        const bool same = buf.size() == h->host_tables.size() && h->batch_tables &&
                          std::memcmp(buf.data(), h->host_tables.data(), buf.size()) == 0;
        if (same) return MOMMS_OK;
        int r = grow_device(&h->batch_tables, &h->batch_tables_cap, buf.size());
        if (r) return r;
        if (cudaMemcpyAsync(h->batch_tables, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        h->host_tables.swap(buf);
        return MOMMS_OK;
    };
    size_t off_gemm = 0, off_items[4] = {0, 0, 0, 0};
    char* tb = nullptr;
    auto items = [&](int w) { return reinterpret_cast<const int2*>(tb + off_items[w]); };
    int64_t launches = 0;
    if (auto_s) {
        // statistics first, then one readback of every problem's spreads
        for (auto& q : prep) q.S = 1;
        rc = upload({}, &off_gemm, off_items);
        if (rc) return rc;
        tb = static_cast<char*>(h->batch_tables);
        if (cudaMemsetAsync(spreads, 0, sizeof(int32_t) * 2 * count, s) != cudaSuccess) return MOMMS_ERR_CUDA;
        if (momms::launch_emu_batch_scale(reinterpret_cast<const momms::EmuBatchPrep*>(tb), items(0),
                                          (int)sa_items.size(), items(1), (int)sb_items.size(), s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 2;
        if (h->spread_host_cap < static_cast<size_t>(2 * count)) {
            if (h->spread_host_big) cudaFreeHost(h->spread_host_big);
            h->spread_host_big = nullptr;
            h->spread_host_cap = 0;
            if (cudaMallocHost(&h->spread_host_big, sizeof(int) * 2 * count) != cudaSuccess) return MOMMS_ERR_ALLOC;
            h->spread_host_cap = 2 * count;
        }
        if (cudaMemcpyAsync(h->spread_host_big, spreads, sizeof(int) * 2 * count, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        for (int i = 0; i < count; ++i)
            S[i] = slices_from_spread(h->spread_host_big[2 * i] / 16.0, h->spread_host_big[2 * i + 1] / 16.0,
                                      k[idx[i]], bb, &rule_bits[i]);
    }
    // ---- encoding per problem: the modular one where the single-problem rule takes it (the
    // operand width of the slice rule, moduli when they save two or more products) and, in AUTO,
    // where its per-element costs that do not shrink with k are covered: the reconstruction and
    // residue split of one element cost about what 650 k-steps of one residue product cost, so
    // moduli are taken when N (k + 650) <= 0.9 S (S + 1) / 2 k; digit slices otherwise (850 when
    // the reconstruction took 1.08 ps per element and modulus against 1.27 fs per tensor
    // multiply-add step; on the 2000-problem workload 850 / 650 / 450 then measured 37.8 / 37.1 /
    // 37.1 ms per call with the faster reconstruction and split)
    std::vector<char> mod(count, 0);
    std::vector<int> planes(count), mbits(count, 0);
    for (int i = 0; i < count; ++i) {
        momms::CrtConsts cc;
        momms::CrtRecon cr;
        const int w = auto_s ? std::min(bb * S[i], std::max(static_cast<int>(std::ceil(rule_bits[i])), bb * S[i] - bb + 1))
                             : bb * S[i];
        // the handle's encoding, or where it is AUTO the problem's plan's
        const int sch = h->scheme == MOMMS_SCHEME_AUTO ? scheme_of[i] : h->scheme;
        mod[i] = S[i] <= MOMMS_MAX_SLICES && use_moduli(sch, w, S[i], bb, k[idx[i]], &cc, &cr);
        if (mod[i] && sch == MOMMS_SCHEME_AUTO) {
            const double kk = static_cast<double>(k[idx[i]]);
            mod[i] = cc.N * (kk + 650.0) <= 0.9 * (S[i] * (S[i] + 1) / 2) * kk;
        }
        if (mod[i]) {
            planes[i] = cc.N;
            mbits[i] = w;
        } else {
            if (S[i] > MOMMS_MAX_SLICES || k[idx[i]] > momms::emu_max_k_per_pass(S[i], bb)) return MOMMS_ERR_UNSUPPORTED;
            planes[i] = S[i];
        }
    }
    // ---- digits (residues), product residues and recombination scratch in the workspace
    std::vector<size_t> off_ad(count), off_bd(count), off_res(count, 0);
    size_t ws_bytes = 0;
    for (int i = 0; i < count; ++i) {
        off_ad[i] = ws_bytes; ws_bytes += align256(size_t(2) * planes[i] * prep[i].m * prep[i].k_pad);
        off_bd[i] = ws_bytes; ws_bytes += align256(size_t(2) * planes[i] * prep[i].n * prep[i].k_pad);
        if (mod[i]) {
            off_res[i] = ws_bytes;
            ws_bytes += align256(static_cast<size_t>(planes[i]) * prep[i].m * prep[i].n);
        }
    }
    const size_t off_scratch = ws_bytes;
    const size_t scratch_bytes = momms::emu_scratch_bytes(momms::device_sm_count());
    ws_bytes += align256(scratch_bytes);
    void* ws = nullptr;
    rc = ensure_workspace(h, ws_bytes, &ws);
    if (rc) return rc;
    char* w = static_cast<char*>(ws);
    std::vector<momms::EmuBatchProblem> gemm;
    gemm.reserve(count);
    int64_t tiles = 0, units_mod = 0;
    int nmax = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        momms::EmuBatchPrep& q = prep[i];
        q.S = planes[i];
        q.bits = mbits[i];
        q.Ad = w + off_ad[i];
        q.Bd = w + off_bd[i];
        momms::EmuBatchProblem g;
        std::memset(&g, 0, sizeof(g));
        if (!momms::emu_make_digit_map(&g.mapA, q.Ad, q.k_pad, q.m, planes[i], momms::kEmuBM) ||
            !momms::emu_make_digit_map(&g.mapB, q.Bd, q.k_pad, q.n, planes[i], momms::kEmuBNMax))
            return MOMMS_ERR_UNSUPPORTED;
        g.e = q.e; g.ef = q.ef; g.f = q.f; g.ff = q.ff;
        g.C = C[p]; g.ldc = ldc[p]; g.alpha = alpha[p]; g.beta_c = beta[p];
        g.m = q.m; g.n = q.n; g.S = planes[i]; g.beta = bb;
        g.nslab = q.k_pad / momms::kEmuBK;
        g.chunk_slabs = momms::emu_chunk_slabs(bb);
        g.tiles_n = static_cast<int32_t>((q.n + momms::kEmuBNMax - 1) / momms::kEmuBNMax);
        const int64_t pt = ((q.m + momms::kEmuBM - 1) / momms::kEmuBM) * g.tiles_n;
        if (mod[i]) {
            // units = tiles x moduli; the residues of the product go to the problem's planes, the
            // reconstruction reads them column by column
            g.res = reinterpret_cast<uint8_t*>(w + off_res[i]);
            g.tile0 = units_mod;
            units_mod += pt * planes[i];
            nmax = std::max(nmax, planes[i]);
            gemm_mod.push_back(g);
            const int ci = static_cast<int>(crt_probs.size());
            crt_probs.push_back(momms::CrtBatchProblem{g.res, q.e, q.ef, q.f, q.ff, g.C, g.ldc, g.alpha, g.beta_c,
                                                       q.m, q.n, planes[i], mbits[i]});
            for (int64_t b = 0; b < momms::crt_batch_blocks(q.n); ++b) crt_items.push_back(make_int2(ci, (int)b));
        } else {
            g.group_end = momms::emu_group_ends(S[i], bb, q.k_pad);
            g.tile0 = tiles;
            tiles += pt;
            gemm.push_back(g);
        }
    }
    // the split work lists of each encoding (the items name the problem's prep entry)
    {
        std::vector<int2> pa_s, pb_s;
        for (const int2& it : pa_items) (mod[it.x] ? pa_mod : pa_s).push_back(it);
        for (const int2& it : pb_items) (mod[it.x] ? pb_mod : pb_s).push_back(it);
        pa_items.swap(pa_s);
        pb_items.swap(pb_s);
    }
    if (crt_items.size() > INT32_MAX) return MOMMS_ERR_UNSUPPORTED;
    rc = upload(gemm, &off_gemm, off_items);
    if (rc) return rc;
    tb = static_cast<char*>(h->batch_tables);
    const auto* dprep = reinterpret_cast<const momms::EmuBatchPrep*>(tb);
    if (!auto_s) {
        if (momms::launch_emu_batch_scale(dprep, items(0), (int)sa_items.size(), items(1), (int)sb_items.size(), s) !=
            cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 2;
    }
    const int nslices = static_cast<int>(gemm.size()), nmod = static_cast<int>(gemm_mod.size());
    if (nslices > 0) {
        if (momms::launch_emu_batch_split(dprep, items(2), (int)pa_items.size(), items(3), (int)pb_items.size(), s) !=
            cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 2;
    }
    momms::CrtConsts c16;
    momms::CrtRecon r16;
    momms::crt_consts(momms::kCrtMaxModuli, 0, &c16, &r16);  // the moduli; each problem takes a prefix
    if (nmod > 0) {
        if (momms::launch_emu_batch_residues(dprep, reinterpret_cast<const int2*>(tb + off_mod[0]), (int)pa_mod.size(),
                                             reinterpret_cast<const int2*>(tb + off_mod[1]), (int)pb_mod.size(), c16,
                                             s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 2;
    }
    if (nslices > 0) {
        cudaError_t ce = momms::launch_emu_slice_gemm_batched(
            reinterpret_cast<const momms::EmuBatchProblem*>(tb + off_gemm), nslices, tiles, w + off_scratch,
            scratch_bytes, h->status, s);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += 1;
    }
    if (nmod > 0) {
        cudaError_t ce = momms::launch_emu_residue_gemm_batched(
            reinterpret_cast<const momms::EmuBatchProblem*>(tb + off_mod[2]), nmod, units_mod, c16, w + off_scratch,
            scratch_bytes, h->status, s);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        // C of the modular problems by the Chinese remainder theorem (the constants by moduli count)
        ce = momms::launch_crt_reconstruct_batched(reinterpret_cast<const momms::CrtBatchProblem*>(tb + off_mod[3]),
                                                   reinterpret_cast<const int2*>(tb + off_mod[4]),
                                                   (int)crt_items.size(), crt_set(h), s);
        if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += 2;
    }
    int smax = 0;
    for (int i = 0; i < count; ++i)
        if (!mod[i]) smax = std::max(smax, S[i]);
    reset_report(h);
    h->report.mode = MOMMS_MODE_EMULATED;
    h->report.member = MOMMS_MEMBER_AUTO;
    h->report.slices = smax;
    h->report.moduli = nmax;
    h->report.digit_bits = bb;
    h->report.k_passes = 1;
    h->report.tile_m = momms::kEmuBM;
    h->report.tile_n = momms::kEmuBNMax;
    h->report.launches = launches;
    return MOMMS_OK;
}

// Batched emulated products with the data-driven slice count chosen on the device: one scale pass,
// the batched plan kernel (each problem's S, width and encoding, and the unit layout of both product
// launches, written into the device tables), then both encodings' split passes, both persistent
// product launches (each walking only the problems and units the plan gave it; their totals are
// read on the device) and the reconstruction.  Nothing is read back: the call only enqueues work,
// and a repeated call with the same problems uploads nothing, so it can be captured in a CUDA graph.
int run_emulated_batched_planned(momms_handle_t h, const std::vector<int64_t>& idx, const std::vector<int>& scheme_of,
                                 const int64_t* m, const int64_t* n, const int64_t* k, const double* alpha,
                                 const double* const* A, const int64_t* lda, const double* const* B,
                                 const int64_t* ldb, const double* beta, double* const* C, const int64_t* ldc,
                                 cudaStream_t s) {
    const int count = static_cast<int>(idx.size());
    const int bb = h->digit_bits;
    constexpr int kPlanes = momms::kCrtMaxModuli;  // room for the most moduli and for S <= kAutoSliceMax
    static_assert(kAutoSliceMax <= kPlanes, "digit planes fit the reserved planes");
    // ---- per-problem statistics (exponents, flags; the spreads first)
    std::vector<size_t> off_e(count), off_ef(count), off_f(count), off_ff(count);
    size_t meta = align256(sizeof(int32_t) * 2 * static_cast<size_t>(count));
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        off_e[i] = meta;  meta += align256(sizeof(int32_t) * m[p]);
        off_ef[i] = meta; meta += align256(static_cast<size_t>(m[p]));
        off_f[i] = meta;  meta += align256(sizeof(int32_t) * n[p]);
        off_ff[i] = meta; meta += align256(static_cast<size_t>(n[p]));
    }
    int rc = grow_device(&h->batch_meta, &h->batch_meta_cap, meta);
    if (rc) return rc;
    char* mb = static_cast<char*>(h->batch_meta);
    int32_t* spreads = reinterpret_cast<int32_t*>(mb);
    // ---- workspace: every problem's planes (kPlanes per operand) and product residues, then scratch
    std::vector<size_t> off_ad(count), off_bd(count), off_res(count);
    size_t ws_bytes = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        const int64_t k_pad = round_up(k[p], momms::kEmuBK);
        off_ad[i] = ws_bytes; ws_bytes += align256(size_t(2) * kPlanes * m[p] * k_pad);
        off_bd[i] = ws_bytes; ws_bytes += align256(size_t(2) * kPlanes * n[p] * k_pad);
        off_res[i] = ws_bytes; ws_bytes += align256(static_cast<size_t>(kPlanes) * m[p] * n[p]);
    }
    const size_t off_scratch = ws_bytes;
    const size_t scratch_bytes = momms::emu_scratch_bytes(momms::device_sm_count());
    ws_bytes += align256(scratch_bytes);
    void* ws = nullptr;
    rc = ensure_workspace(h, ws_bytes, &ws);
    if (rc) return rc;
    char* w = static_cast<char*>(ws);
    // ---- the host-side parts of the tables (the plan kernel fills in S, widths, encodings and offsets)
    std::vector<momms::EmuBatchPrep> prep(count);
    std::vector<momms::EmuBatchProblem> gs(count), gm(count);
    std::vector<momms::CrtBatchProblem> cp(count);
    std::vector<int2> sa_items, sb_items, pa_items, pb_items, crt_items;
    int64_t tiles_all = 0;
    for (int i = 0; i < count; ++i) {
        const int64_t p = idx[i];
        momms::EmuBatchPrep& q = prep[i];
        q.A = A[p]; q.B = B[p]; q.lda = lda[p]; q.ldb = ldb[p];
        q.m = static_cast<int32_t>(m[p]); q.n = static_cast<int32_t>(n[p]); q.k = static_cast<int32_t>(k[p]);
        q.k_pad = static_cast<int32_t>(round_up(k[p], momms::kEmuBK));
        q.S = kPlanes; q.beta = bb; q.bits = 0; q.enc = 0;
        q.scheme = h->scheme == MOMMS_SCHEME_AUTO ? scheme_of[i] : h->scheme;
        q.c0 = rule_c0(k[p]);
        q.e = reinterpret_cast<int32_t*>(mb + off_e[i]);
        q.ef = reinterpret_cast<uint8_t*>(mb + off_ef[i]);
        q.f = reinterpret_cast<int32_t*>(mb + off_f[i]);
        q.ff = reinterpret_cast<uint8_t*>(mb + off_ff[i]);
        q.spread = spreads + 2 * i;
        q.Ad = w + off_ad[i];
        q.Bd = w + off_bd[i];
        for (int64_t b = 0; b < momms::emu_batch_scale_a_blocks(m[p]); ++b) sa_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_scale_b_blocks(n[p]); ++b) sb_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_split_a_blocks(m[p], q.k_pad); ++b) pa_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::emu_batch_split_b_blocks(n[p], q.k_pad); ++b) pb_items.push_back(make_int2(i, (int)b));
        for (int64_t b = 0; b < momms::crt_batch_blocks(n[p]); ++b) crt_items.push_back(make_int2(i, (int)b));
        momms::EmuBatchProblem g;
        std::memset(&g, 0, sizeof(g));
        if (!momms::emu_make_digit_map(&g.mapA, q.Ad, q.k_pad, q.m, kPlanes, momms::kEmuBM) ||
            !momms::emu_make_digit_map(&g.mapB, q.Bd, q.k_pad, q.n, kPlanes, momms::kEmuBNMax))
            return MOMMS_ERR_UNSUPPORTED;
        g.e = q.e; g.ef = q.ef; g.f = q.f; g.ff = q.ff;
        g.C = C[p]; g.ldc = ldc[p]; g.alpha = alpha[p]; g.beta_c = beta[p];
        g.m = q.m; g.n = q.n; g.beta = bb;
        g.nslab = q.k_pad / momms::kEmuBK;
        g.chunk_slabs = momms::emu_chunk_slabs(bb);
        g.tiles_n = static_cast<int32_t>((q.n + momms::kEmuBNMax - 1) / momms::kEmuBNMax);
        tiles_all += ((q.m + momms::kEmuBM - 1) / momms::kEmuBM) * g.tiles_n;
        gs[i] = g;
        g.res = reinterpret_cast<uint8_t*>(w + off_res[i]);
        gm[i] = g;
        cp[i] = momms::CrtBatchProblem{g.res, q.e, q.ef, q.f, q.ff, g.C, g.ldc, g.alpha, g.beta_c, q.m, q.n, 0, 0};
    }
    if (sa_items.size() > INT32_MAX || pa_items.size() > INT32_MAX || pb_items.size() > INT32_MAX ||
        crt_items.size() > INT32_MAX)
        return MOMMS_ERR_UNSUPPORTED;
    // ---- one device block: [prep][sa][sb][pa][pb][gs][gm][crt][crt items][totals]
    std::vector<char> buf;
    auto put = [&](const void* src, size_t bytes) {
        size_t o = align256(buf.size());
        buf.resize(o + bytes);
        if (bytes) std::memcpy(buf.data() + o, src, bytes);
        return o;
    };
    const size_t o_prep = put(prep.data(), sizeof(momms::EmuBatchPrep) * count);
    const size_t o_sa = put(sa_items.data(), sizeof(int2) * sa_items.size());
    const size_t o_sb = put(sb_items.data(), sizeof(int2) * sb_items.size());
    const size_t o_pa = put(pa_items.data(), sizeof(int2) * pa_items.size());
    const size_t o_pb = put(pb_items.data(), sizeof(int2) * pb_items.size());
    const size_t o_gs = put(gs.data(), sizeof(momms::EmuBatchProblem) * count);
    const size_t o_gm = put(gm.data(), sizeof(momms::EmuBatchProblem) * count);
    const size_t o_cp = put(cp.data(), sizeof(momms::CrtBatchProblem) * count);
    const size_t o_ci = put(crt_items.data(), sizeof(int2) * crt_items.size());
    const int64_t zeros[2] = {0, 0};
    const size_t o_tot = put(zeros, sizeof(zeros));
    const bool same = buf.size() == h->host_tables.size() && h->batch_tables &&
                      std::memcmp(buf.data(), h->host_tables.data(), buf.size()) == 0;
    if (!same) {
        rc = grow_device(&h->batch_tables, &h->batch_tables_cap, buf.size());
        if (rc) return rc;
        if (cudaMemcpyAsync(h->batch_tables, buf.data(), buf.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        h->host_tables.swap(buf);
    }
    char* tb = static_cast<char*>(h->batch_tables);
    auto* dprep = reinterpret_cast<momms::EmuBatchPrep*>(tb + o_prep);
    auto items = [&](size_t o) { return reinterpret_cast<const int2*>(tb + o); };
    auto* totals = reinterpret_cast<int64_t*>(tb + o_tot);
    // ---- the launches
    int64_t launches = 0;
    if (cudaMemsetAsync(spreads, 0, sizeof(int32_t) * 2 * count, s) != cudaSuccess ||
        momms::launch_emu_batch_scale(dprep, items(o_sa), (int)sa_items.size(), items(o_sb), (int)sb_items.size(), s) !=
            cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += 2;
    momms::EmuBatchPlanArgs pa{};
    pa.prep = dprep;
    pa.slices = reinterpret_cast<momms::EmuBatchProblem*>(tb + o_gs);
    pa.moduli = reinterpret_cast<momms::EmuBatchProblem*>(tb + o_gm);
    pa.crt = reinterpret_cast<momms::CrtBatchProblem*>(tb + o_cp);
    pa.count = count;
    pa.smax = kAutoSliceMax;
    pa.totals = totals;
    pa.summary = h->plan_dev;
    const momms::CrtReconSet& set = crt_set(h);
    for (int c = 1; c <= momms::kCrtMaxModuli; ++c) {
        const uint32_t* Pw = set.by_n[c].Pw;
        pa.P[c][0] = static_cast<uint64_t>(Pw[0]) | (static_cast<uint64_t>(Pw[1]) << 32);
        pa.P[c][1] = static_cast<uint64_t>(Pw[2]) | (static_cast<uint64_t>(Pw[3]) << 32);
    }
    if (momms::launch_emu_batch_plan(pa, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    launches += 1;
    momms::CrtConsts c16;
    momms::CrtRecon r16;
    momms::crt_consts(momms::kCrtMaxModuli, 0, &c16, &r16);  // the moduli; each problem takes a prefix
    if (momms::launch_emu_batch_split(dprep, items(o_pa), (int)pa_items.size(), items(o_pb), (int)pb_items.size(), s) !=
            cudaSuccess ||
        momms::launch_emu_batch_residues(dprep, items(o_pa), (int)pa_items.size(), items(o_pb), (int)pb_items.size(),
                                         c16, s) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += 4;
    const int wh = momms::emu_debug_take_withhold();  // (test hook: one of the two product launches works)
    if (wh) momms::emu_debug_withhold_load();
    cudaError_t ce = momms::launch_emu_slice_gemm_batched(reinterpret_cast<const momms::EmuBatchProblem*>(tb + o_gs),
                                                          count, tiles_all, w + off_scratch, scratch_bytes, h->status,
                                                          s, totals);
    if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
    if (wh) momms::emu_debug_withhold_load();
    ce = momms::launch_emu_residue_gemm_batched(reinterpret_cast<const momms::EmuBatchProblem*>(tb + o_gm), count,
                                                tiles_all * momms::kCrtMaxModuli, c16, w + off_scratch, scratch_bytes,
                                                h->status, s, totals + 1);
    if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
    momms::emu_debug_take_withhold();
    ce = momms::launch_crt_reconstruct_batched(reinterpret_cast<const momms::CrtBatchProblem*>(tb + o_cp),
                                               items(o_ci), (int)crt_items.size(), set, s);
    if (ce != cudaSuccess) return MOMMS_ERR_CUDA;
    launches += 3;
    reset_report(h);
    h->report.mode = MOMMS_MODE_EMULATED;
    h->report.member = MOMMS_MEMBER_AUTO;
    h->report.digit_bits = bb;
    h->report.k_passes = 1;
    h->report.tile_m = momms::kEmuBM;
    h->report.tile_n = momms::kEmuBNMax;
    h->report.launches = launches;
    h->report_pending = true;  // the largest S / moduli / width of the call, from the plan kernel
    return MOMMS_OK;
}

int gemm_dispatch(momms_handle_t h, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha,
                  const double* A, int64_t lda, const double* B, int64_t ldb, double beta, double* C,
                  int64_t ldc, cudaStream_t s) {
    if (m == 0 || n == 0) {
        reset_report(h);
        return MOMMS_OK;
    }
    if (k == 0 || alpha == 0.0) {
        reset_report(h);
        h->report.launches = beta == 1.0 ? 0 : 1;
        return scale_c(m, n, beta, C, ldc, s);
    }
    const Plan p = pick_plan(h, m, n, k, opa, opb);
    const int member = p.member == MOMMS_MEMBER_AUTO ? MOMMS_MEMBER_C2 : p.member;
    if (p.mode == MOMMS_MODE_EMULATED) {
        // the plan's tile width, encoding and CTA pairs where the handle leaves them automatic
        const int tile_n = h->tile_n, scheme = h->scheme, pairs = h->cta_pairs;
        if (tile_n == 0) h->tile_n = p.tile_n;
        if (scheme == MOMMS_SCHEME_AUTO) h->scheme = p.scheme;
        if (pairs == 0) h->cta_pairs = p.pairs;
        const int rc = run_emulated(h, opa, opb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, member, p.slices, s);
        h->tile_n = tile_n;
        h->scheme = scheme;
        h->cta_pairs = pairs;
        return rc;
    }
    return run_native(h, opa, opb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, member, s);
}

// BLAS argument checks; returns 0 or -(1-based index of the first bad argument).
int check_gemm_args(int base, int opa, int opb, int64_t m, int64_t n, int64_t k, const double* A,
                    int64_t lda, const double* B, int64_t ldb, const double* C, int64_t ldc,
                    double alpha, bool has_ops) {
    // argument indices relative to `base` (index of m)
    if (has_ops) {
        if (opa != MOMMS_OP_N && opa != MOMMS_OP_T) return -(base - 2);
        if (opb != MOMMS_OP_N && opb != MOMMS_OP_T) return -(base - 1);
    }
    if (m < 0) return -(base);
    if (n < 0) return -(base + 1);
    if (k < 0) return -(base + 2);
    const int64_t rows_a = opa == MOMMS_OP_N ? m : k;
    const int64_t rows_b = opb == MOMMS_OP_N ? k : n;
    if (lda < std::max<int64_t>(1, rows_a)) return -(base + 5);
    if (ldb < std::max<int64_t>(1, rows_b)) return -(base + 7);
    if (ldc < std::max<int64_t>(1, m)) return -(base + 10);
    const bool work = m > 0 && n > 0;
    const bool product = work && k > 0 && alpha != 0.0;
    if (product && !A) return -(base + 4);
    if (product && !B) return -(base + 6);
    if (work && !C) return -(base + 9);
    if (product) {
        // C must not overlap A or B (byte ranges of the stored matrices)
        auto span = [](const double* p, int64_t ld, int64_t rows, int64_t cols) {
            return std::make_pair(reinterpret_cast<uintptr_t>(p),
                                  reinterpret_cast<uintptr_t>(p + (cols - 1) * ld + rows));
        };
        const auto sc = span(C, ldc, m, n);
        const auto sa = span(A, lda, rows_a, opa == MOMMS_OP_N ? k : m);
        const auto sb = span(B, ldb, rows_b, opb == MOMMS_OP_N ? n : k);
        if (sc.first < sa.second && sa.first < sc.second) return -(base + 9);
        if (sc.first < sb.second && sb.first < sc.second) return -(base + 9);
    }
    return 0;
}

momms_handle_t thread_default_handle() {
    static thread_local momms_handle_t h = nullptr;
    if (!h) momms_create(&h);
    return h;
}

}  // namespace

extern "C" {

int momms_create(momms_handle_t* handle) {
    if (!handle) return -1;
    *handle = nullptr;
    momms_handle_t h = new (std::nothrow) momms_handle_s();
    if (!h) return MOMMS_ERR_ALLOC;
    if (cudaMalloc(&h->status, 128) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MOMMS_ERR_ALLOC;
    }
    h->spread_dev = reinterpret_cast<int*>(reinterpret_cast<char*>(h->status) + 16);
    h->plan_dev = reinterpret_cast<momms::EmuPlan*>(reinterpret_cast<char*>(h->status) + 64);
    if (cudaEventCreateWithFlags(&h->spread_ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        h->spread_ready = nullptr;
    }
    if (cudaMemset(h->status, 0, 128) != cudaSuccess ||
        cudaMallocHost(&h->spread_host, 2 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(h->status);
        delete h;
        return MOMMS_ERR_ALLOC;
    }
    *handle = h;
    return MOMMS_OK;
}

int momms_destroy(momms_handle_t h) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    cudaDeviceSynchronize();
    if (h->own_ws) cudaFree(h->own_ws);
    if (h->dev_probs) cudaFree(h->dev_probs);
    if (h->batch_meta) cudaFree(h->batch_meta);
    if (h->batch_tables) cudaFree(h->batch_tables);
    if (h->spread_host_big) cudaFreeHost(h->spread_host_big);
    if (h->status) cudaFree(h->status);
    if (h->spread_host) cudaFreeHost(h->spread_host);
    if (h->spread_ready) cudaEventDestroy(h->spread_ready);
    if (h->ooc_buf) cudaFree(h->ooc_buf);
    if (h->ooc_in) cudaStreamDestroy(h->ooc_in);
    if (h->ooc_out) cudaStreamDestroy(h->ooc_out);
    for (cudaEvent_t e : h->ooc_ev)
        if (e) cudaEventDestroy(e);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->kev)
        if (e) cudaEventDestroy(e);
    h->magic = 0;
    delete h;
    return MOMMS_OK;
}

int momms_set_mode(momms_handle_t h, int mode) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (mode < MOMMS_MODE_AUTO || mode > MOMMS_MODE_EMULATED) return -2;
    h->mode = mode;
    return MOMMS_OK;
}

int momms_set_member(momms_handle_t h, int member) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (member < MOMMS_MEMBER_AUTO || member > MOMMS_MEMBER_A1) return -2;
    h->member = member;
    return MOMMS_OK;
}

int momms_set_slices(momms_handle_t h, int slices) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (slices < 0 || slices > MOMMS_MAX_SLICES) return -2;
    h->slices = slices;
    return MOMMS_OK;
}

void momms_debug_withhold_load(void) { momms::emu_debug_withhold_load(); }

int momms_set_kernel_timing(momms_handle_t h, int max_launches) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (max_launches < 0) return -2;
    const size_t want = 2 * static_cast<size_t>(max_launches);
    while (h->kev.size() < want) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return MOMMS_ERR_CUDA;
        }
        h->kev.push_back(e);
    }
    while (h->kev.size() > want) {
        cudaEventDestroy(h->kev.back());
        h->kev.pop_back();
    }
    h->kev_used = 0;
    return MOMMS_OK;
}

int momms_kernel_timing(momms_handle_t h, double* total_ms, int64_t* launches) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (!total_ms) return -2;
    if (!launches) return -3;
    double t = 0.0;
    for (size_t i = 0; i < h->kev_used; ++i) {
        float ms = 0.0f;
        if (cudaEventSynchronize(h->kev[2 * i + 1]) != cudaSuccess ||
            cudaEventElapsedTime(&ms, h->kev[2 * i], h->kev[2 * i + 1]) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        t += ms;
    }
    *total_ms = t;
    *launches = static_cast<int64_t>(h->kev_used);
    h->kev_used = 0;
    return MOMMS_OK;
}

int momms_set_host_resident(momms_handle_t h, int resident) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (resident != 0 && resident != 1) return -2;
    h->host_resident = resident;
    return MOMMS_OK;
}

int momms_set_plan_on_device(momms_handle_t h, int on) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (on != 0 && on != 1) return -2;
    h->plan_mode = on != 0;
    return MOMMS_OK;
}

int momms_set_cta_pairs(momms_handle_t h, int mode) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (mode < 0 || mode > 2) return -2;
    h->cta_pairs = mode;
    return MOMMS_OK;
}

int momms_set_crt_fusion(momms_handle_t h, int mode) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (mode < 0 || mode > 2) return -2;
    h->crt_fusion = mode;
    return MOMMS_OK;
}

int momms_set_scheme(momms_handle_t h, int scheme) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (scheme < MOMMS_SCHEME_AUTO || scheme > MOMMS_SCHEME_MODULI) return -2;
    h->scheme = scheme;
    return MOMMS_OK;
}

int momms_set_max_ctas(momms_handle_t h, int ctas) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (ctas < 0) return -2;
    h->max_ctas = ctas;
    return MOMMS_OK;
}

int momms_set_tile_n(momms_handle_t h, int tile_n) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (tile_n != 0 && tile_n != 96 && tile_n != 192) return -2;
    h->tile_n = tile_n;
    return MOMMS_OK;
}

int momms_set_raster_group(momms_handle_t h, int group) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (group < 0) return -2;
    h->group = group;
    return MOMMS_OK;
}

int momms_get_last_report(momms_handle_t h, momms_report_t* r) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (!r) return -2;
    if (h->report_pending) {
        // the last product chose its slice count on the device: its plan holds what it used
        momms::EmuPlan pl{};
        if (cudaMemcpy(&pl, h->plan_dev, sizeof(pl), cudaMemcpyDeviceToHost) != cudaSuccess) return MOMMS_ERR_CUDA;
        h->report.slices = pl.S;
        h->report.moduli = pl.N;
        h->report.operand_bits = pl.bits;
        h->report.est_err_ratio = pl.est;  // (kept pending: a graph replay updates the plan again)
    }
    *r = h->report;
    return MOMMS_OK;
}

int momms_check_device_status(momms_handle_t h, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t v = 0;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (cudaMemcpy(&v, h->status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (v) cudaMemset(h->status, 0, sizeof(int32_t));
    return v ? static_cast<int>(v) : MOMMS_OK;
}

const char* momms_status_string(int status) {
    switch (status) {
        case MOMMS_OK: return "ok";
        case MOMMS_ERR_CUDA: return "CUDA launch or runtime error";
        case MOMMS_ERR_TIMEOUT: return "a bounded device wait expired";
        case MOMMS_ERR_NONFINITE: return "emulated mode met Inf/NaN input";
        case MOMMS_ERR_WORKSPACE: return "workspace too small";
        case MOMMS_ERR_UNSUPPORTED: return "size or option not supported";
        case MOMMS_ERR_ALLOC: return "device allocation failed";
        case MOMMS_ERR_HANDLE: return "invalid handle";
        case MOMMS_ERR_IO: return "plan cache I/O error";
        default: return status < 0 ? "invalid argument" : "unknown status";
    }
}

int momms_workspace_size(momms_handle_t h, int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                         size_t* bytes) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (op_a != MOMMS_OP_N && op_a != MOMMS_OP_T) return -2;
    if (op_b != MOMMS_OP_N && op_b != MOMMS_OP_T) return -3;
    if (m < 0) return -4;
    if (n < 0) return -5;
    if (k < 0) return -6;
    if (!bytes) return -7;
    const Plan p = pick_plan(h, m, n, k, op_a, op_b);
    if (p.mode == MOMMS_MODE_NATIVE || m == 0 || n == 0 || k == 0) {
        *bytes = 0;
        return MOMMS_OK;
    }
    *bytes = emu_layout(m, n, k, p.slices > 0 ? p.slices : kAutoSliceMax, h->max_ctas,
                        moduli_reserved(h->scheme, p.slices, k)).total;
    return MOMMS_OK;
}

int momms_set_workspace(momms_handle_t h, void* workspace, size_t bytes) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255)) return -2;
    h->user_ws = workspace;
    h->user_ws_bytes = workspace ? bytes : 0;
    return MOMMS_OK;
}

int momms_gemm(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
               const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
               momms_stream_t stream) {
    int rc = check_gemm_args(1, MOMMS_OP_N, MOMMS_OP_N, m, n, k, A, lda, B, ldb, C, ldc, alpha, false);
    if (rc) return rc;
    momms_handle_t h = thread_default_handle();
    if (!h) return MOMMS_ERR_ALLOC;
    return gemm_dispatch(h, MOMMS_OP_N, MOMMS_OP_N, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                         reinterpret_cast<cudaStream_t>(stream));
}

int momms_gemm_ex(momms_handle_t h, int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                  double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                  double beta, double* C, int64_t ldc, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    int rc = check_gemm_args(4, op_a, op_b, m, n, k, A, lda, B, ldb, C, ldc, alpha, true);
    if (rc) return rc;
    return gemm_dispatch(h, op_a, op_b, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc,
                         reinterpret_cast<cudaStream_t>(stream));
}

int momms_gemm_backward(momms_handle_t h, int64_t m, int64_t n, int64_t k, const double* A,
                        int64_t lda, const double* B, int64_t ldb, const double* dC, int64_t lddc,
                        double* dA, int64_t ldda, double* dB, int64_t lddb, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (m < 0) return -2;
    if (n < 0) return -3;
    if (k < 0) return -4;
    if (lda < std::max<int64_t>(1, m)) return -6;
    if (ldb < std::max<int64_t>(1, k)) return -8;
    if (lddc < std::max<int64_t>(1, m)) return -10;
    if (dA && ldda < std::max<int64_t>(1, m)) return -12;
    if (dB && lddb < std::max<int64_t>(1, k)) return -14;
    const bool need_dc = (dA && m > 0 && k > 0 && n > 0) || (dB && k > 0 && n > 0 && m > 0);
    if (need_dc && !dC) return -9;
    if (dA && m > 0 && k > 0 && n > 0 && !B) return -7;
    if (dB && k > 0 && n > 0 && m > 0 && !A) return -5;
    int64_t launches = 0;
    if (dA) {
        // dA (m x k) = dC (m x n) * B^T  -- contraction over n
        int rc = gemm_dispatch(h, MOMMS_OP_N, MOMMS_OP_T, m, k, n, 1.0, dC, lddc, B, ldb, 0.0, dA, ldda,
                               reinterpret_cast<cudaStream_t>(stream));
        if (rc) return rc;
        launches += h->report.launches;
    }
    if (dB) {
        // dB (k x n) = A^T (k x m) * dC (m x n)  -- contraction over m
        int rc = gemm_dispatch(h, MOMMS_OP_T, MOMMS_OP_N, k, n, m, 1.0, A, lda, dC, lddc, 0.0, dB, lddb,
                               reinterpret_cast<cudaStream_t>(stream));
        if (rc) return rc;
        launches += h->report.launches;
    }
    h->report.launches = launches;
    return MOMMS_OK;
}

int momms_gemm_batched(momms_handle_t h, int64_t count, const int64_t* m, const int64_t* n,
                       const int64_t* k, const double* alpha, const double* const* A,
                       const int64_t* lda, const double* const* B, const int64_t* ldb,
                       const double* beta, double* const* C, const int64_t* ldc,
                       momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (count < 0) return -2;
    if (count == 0) return MOMMS_OK;
    if (!m) return -3;
    if (!n) return -4;
    if (!k) return -5;
    if (!alpha) return -6;
    if (!A) return -7;
    if (!lda) return -8;
    if (!B) return -9;
    if (!ldb) return -10;
    if (!beta) return -11;
    if (!C) return -12;
    if (!ldc) return -13;
    if (count > (int64_t(1) << 30)) return MOMMS_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double total_flops = 0.0;
    for (int64_t i = 0; i < count; ++i) {
        int rc = check_gemm_args(1, MOMMS_OP_N, MOMMS_OP_N, m[i], n[i], k[i], A[i], lda[i], B[i], ldb[i],
                                 C[i], ldc[i], alpha[i], false);
        if (rc) return -3;  // the size / pointer arrays hold an invalid entry
        if (m[i] > INT32_MAX / 2 || n[i] > INT32_MAX / 2 || k[i] > INT32_MAX / 2) return MOMMS_ERR_UNSUPPORTED;
        total_flops += 2.0 * static_cast<double>(m[i]) * static_cast<double>(n[i]) * static_cast<double>(k[i]);
    }
    // The engine of each problem: the tuned plan of its size bucket where the handle holds one
    // (AUTO mode), else the call's rule -- the emulated pipeline (five launches for the whole batch)
    // once the batch's work amortises them, as for a single product of that many flops.  A plan's
    // encoding also applies per problem when the handle's scheme is AUTO.
    const bool call_emulated =
        h->mode == MOMMS_MODE_EMULATED || (h->mode == MOMMS_MODE_AUTO && total_flops >= 2.0e9);
    std::vector<int64_t> emu_idx, nat_idx;
    std::vector<int> emu_scheme;
    int64_t launches = 0;
    for (int64_t i = 0; i < count; ++i) {
        if (m[i] == 0 || n[i] == 0) continue;
        if (k[i] == 0 || alpha[i] == 0.0) {  // C := beta C only
            int rc = scale_c(m[i], n[i], beta[i], C[i], ldc[i], s);
            if (rc) return rc;
            ++launches;
            continue;
        }
        bool emu = call_emulated;
        int sch = MOMMS_SCHEME_AUTO;
        auto it = h->plans.find(bucket_key(m[i], n[i], k[i]));
        if (it != h->plans.end()) {
            if (h->mode == MOMMS_MODE_AUTO) emu = it->second.mode == MOMMS_MODE_EMULATED;
            sch = it->second.scheme;
        }
        if (emu) {
            emu_idx.push_back(i);
            emu_scheme.push_back(sch);
        } else {
            nat_idx.push_back(i);
        }
    }
    if (emu_idx.size() > (size_t(1) << 24)) return MOMMS_ERR_UNSUPPORTED;
    momms_report_t rep{};
    bool pending = false;  // the emulated part planned on the device: its S / moduli come from the plan
    if (!emu_idx.empty()) {
        // the data-driven slice count is planned on the device unless the handle says otherwise (or a
        // problem's k exceeds what the largest planned slice count keeps exact in one pass)
        bool planned = h->slices <= 0 && h->plan_mode && h->digit_bits == kDigitBits;
        for (int64_t i : emu_idx)
            if (k[i] > momms::emu_max_k_per_pass(kAutoSliceMax, kDigitBits)) planned = false;
        int rc = planned ? run_emulated_batched_planned(h, emu_idx, emu_scheme, m, n, k, alpha, A, lda, B, ldb, beta,
                                                        C, ldc, s)
                         : run_emulated_batched(h, emu_idx, emu_scheme, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
        if (rc) return rc;
        rep = h->report;
        pending = h->report_pending;
        launches += h->report.launches;
    }
    if (!nat_idx.empty()) {
        // native: one persistent launch over a device tile table
        std::vector<BatchProblem> probs;
        probs.reserve(nat_idx.size());
        int64_t tiles = 0;
        for (int64_t i : nat_idx) {
            BatchProblem p{};
            p.A = A[i]; p.B = B[i]; p.C = C[i];
            p.lda = lda[i]; p.ldb = ldb[i]; p.ldc = ldc[i];
            p.m = static_cast<int32_t>(m[i]); p.n = static_cast<int32_t>(n[i]); p.k = static_cast<int32_t>(k[i]);
            const int64_t tm = (m[i] + momms::kNativeBM - 1) / momms::kNativeBM;
            const int64_t tn = (n[i] + momms::kNativeBN - 1) / momms::kNativeBN;
            p.tiles_n = static_cast<int32_t>(tn);
            p.tile0 = tiles;
            p.alpha = alpha[i]; p.beta = beta[i];
            tiles += tm * tn;
            probs.push_back(p);
        }
        const size_t bytes = probs.size() * sizeof(BatchProblem);
        const bool same_table = h->host_probs.size() == probs.size() && h->dev_probs &&
                                std::memcmp(h->host_probs.data(), probs.data(), bytes) == 0;
        if (!same_table) {
            if (h->dev_probs_cap < bytes) {
                if (h->dev_probs) {
                    cudaDeviceSynchronize();
                    cudaFree(h->dev_probs);
                    h->dev_probs = nullptr;
                    h->dev_probs_cap = 0;
                }
                if (cudaMalloc(&h->dev_probs, bytes) != cudaSuccess) {
                    cudaGetLastError();
                    return MOMMS_ERR_ALLOC;
                }
                h->dev_probs_cap = bytes;
            }
            // A pageable-memory copy: it has completed when the call returns.  An identical
            // table is not uploaded again, so a call repeated with the same problems enqueues
            // only the kernel and can be captured in a CUDA graph after one eager call.
            if (cudaMemcpyAsync(h->dev_probs, probs.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return MOMMS_ERR_CUDA;
            h->host_probs = probs;
        }
        cudaError_t e = momms::launch_native_batched(h->dev_probs, static_cast<int>(probs.size()), tiles, s);
        if (e != cudaSuccess) return MOMMS_ERR_CUDA;
        launches += 1;
        if (emu_idx.empty()) {
            rep.mode = MOMMS_MODE_NATIVE;
            rep.member = MOMMS_MEMBER_C2;
            rep.tile_m = momms::kNativeBM;
            rep.tile_n = momms::kNativeBN;
            rep.k_passes = 1;
        }
    }
    reset_report(h);
    h->report = rep;
    h->report.launches = launches;
    h->report_pending = pending;
    return MOMMS_OK;
}

int momms_emu_scale(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                    int32_t* exps, uint8_t* flags, momms_stream_t stream) {
    if (which != 0 && which != 1) return -1;
    if (op != 0 && op != 1) return -2;
    if (rows < 0) return -3;
    if (inner < 0) return -4;
    const bool rows_contig = (which == 0) ? (op == 0) : (op != 0);
    const int64_t stored_rows = rows_contig ? rows : inner;
    if (rows > 0 && inner > 0 && !X) return -5;
    if (ldx < std::max<int64_t>(1, stored_rows)) return -6;
    if (rows > 0 && !exps) return -7;
    if (rows > 0 && !flags) return -8;
    return cuda_fail(momms::launch_emu_scale(which, op, rows, inner, X, ldx, exps, flags, nullptr,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

int momms_emu_split(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                    const int32_t* exps, const uint8_t* flags, int slices, int digit_bits,
                    void* digits, int64_t rows_pad, int64_t inner_pad, momms_stream_t stream) {
    if (which != 0 && which != 1) return -1;
    if (op != 0 && op != 1) return -2;
    if (rows < 0) return -3;
    if (inner < 0) return -4;
    const bool rows_contig = (which == 0) ? (op == 0) : (op != 0);
    const int64_t stored_rows = rows_contig ? rows : inner;
    if (rows > 0 && inner > 0 && !X) return -5;
    if (ldx < std::max<int64_t>(1, stored_rows)) return -6;
    if (rows > 0 && !exps) return -7;
    if (rows > 0 && !flags) return -8;
    if (slices < 1 || slices > MOMMS_MAX_SLICES) return -9;
    if (digit_bits < 1 || digit_bits > 10) return -10;
    if (!digits) return -11;
    if (rows_pad < std::max<int64_t>(rows, 1)) return -12;
    if (inner_pad < inner || inner_pad % momms::kEmuBK) return -13;
    return cuda_fail(momms::launch_emu_split(which, op, rows, inner, X, ldx, exps, flags, slices,
                                             digit_bits, digits, rows_pad, inner_pad,
                                             reinterpret_cast<cudaStream_t>(stream)));
}

int momms_crt_moduli(int bits, int64_t k, int* count, uint32_t* moduli) {
    if (bits < 1 || bits > 56) return -1;
    if (k < 1) return -2;
    if (!count) return -3;
    if (!moduli) return -4;
    momms::CrtConsts c;
    momms::CrtRecon r;
    if (!momms::crt_plan(bits, k, &c, &r)) return MOMMS_ERR_UNSUPPORTED;
    *count = c.N;
    for (int l = 0; l < c.N; ++l) moduli[l] = c.p[l];
    return MOMMS_OK;
}

int momms_emu_residues(int which, int op, int64_t rows, int64_t inner, const double* X, int64_t ldx,
                       const int32_t* exps, const uint8_t* flags, int bits, int64_t k, void* planes,
                       int64_t rows_pad, int64_t inner_pad, momms_stream_t stream) {
    if (which != 0 && which != 1) return -1;
    if (op != 0 && op != 1) return -2;
    if (rows < 0) return -3;
    if (inner < 0) return -4;
    const bool rows_contig = (which == 0) ? (op == 0) : (op != 0);
    const int64_t stored_rows = rows_contig ? rows : inner;
    if (rows > 0 && inner > 0 && !X) return -5;
    if (ldx < std::max<int64_t>(1, stored_rows)) return -6;
    if (rows > 0 && !exps) return -7;
    if (rows > 0 && !flags) return -8;
    if (bits < 1 || bits > 56) return -9;
    if (k < 1) return -10;
    if (!planes) return -11;
    if (rows_pad < std::max<int64_t>(rows, 1)) return -12;
    if (inner_pad < inner || inner_pad % momms::kEmuBK) return -13;
    momms::CrtConsts c;
    momms::CrtRecon r;
    if (!momms::crt_plan(bits, k, &c, &r)) return MOMMS_ERR_UNSUPPORTED;
    return cuda_fail(momms::launch_emu_residues(which, op, rows, inner, X, ldx, exps, flags, c, planes, rows_pad,
                                                inner_pad, reinterpret_cast<cudaStream_t>(stream)));
}

size_t momms_emu_scratch_bytes(void) { return momms::emu_scratch_bytes(momms::device_sm_count()); }

size_t momms_emu_scratch_bytes_for(int64_t m, int64_t n, int64_t k, int slices) {
    if (m <= 0 || n <= 0 || k <= 0 || slices < 1 || slices > MOMMS_MAX_SLICES) return momms_emu_scratch_bytes();
    return momms::emu_scratch_bytes_tail(m, n, k, slices, 0, kDigitBits);
}

int momms_emu_slice_gemm(int64_t m, int64_t n, int64_t k, int slices, int digit_bits, const void* Ad,
                         const void* Bd, int64_t m_pad, int64_t n_pad, int64_t k_pad, const int32_t* e,
                         const uint8_t* eflags, const int32_t* f, const uint8_t* fflags, double alpha,
                         double beta, double* C, int64_t ldc, int member, void* scratch,
                         size_t scratch_bytes, int32_t* status, momms_stream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 0) return -3;
    if (slices < 1 || slices > MOMMS_MAX_SLICES) return -4;
    if (digit_bits < 1 || digit_bits > 8) return -5;
    if (!Ad) return -6;
    if (!Bd) return -7;
    if (m_pad < std::max<int64_t>(m, 1)) return -8;
    if (n_pad < std::max<int64_t>(n, 1)) return -9;
    if (k_pad < k || k_pad % momms::kEmuBK) return -10;
    if (!e) return -11;
    if (!eflags) return -12;
    if (!f) return -13;
    if (!fflags) return -14;
    if (!C && m > 0 && n > 0) return -17;
    if (ldc < std::max<int64_t>(1, m)) return -18;
    if (member < MOMMS_MEMBER_AUTO || member > MOMMS_MEMBER_A1) return -19;
    if (!scratch) return -20;
    if (scratch_bytes < momms::emu_scratch_bytes(momms::device_sm_count())) return MOMMS_ERR_WORKSPACE;
    if (!status) return -22;
    if (m == 0 || n == 0) return MOMMS_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (k == 0 || alpha == 0.0) return scale_c(m, n, beta, C, ldc, s);
    momms::EmuGemmArgs a{};
    a.m = m; a.n = n; a.k = k; a.S = slices; a.beta = digit_bits;
    a.Ad = Ad; a.Bd = Bd; a.m_pad = m_pad; a.n_pad = n_pad; a.k_pad = k_pad;
    a.e = e; a.ef = eflags; a.f = f; a.ff = fflags;
    a.alpha = alpha; a.beta_c = beta; a.C = C; a.ldc = ldc;
    a.member = member; a.group = 0;
    a.scratch = scratch; a.scratch_bytes = scratch_bytes; a.status = status; a.max_ctas = 0; a.tile_n = 0;
    int passes = 0;
    cudaError_t ce = momms::launch_emu_slice_gemm(a, &passes, s);
    if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    return cuda_fail(ce);
}

int momms_emu_residue_gemm(int64_t m, int64_t n, int64_t k, int bits, const void* Ar, const void* Br,
                           int64_t m_pad, int64_t n_pad, int64_t k_pad, int member, uint8_t* res, void* scratch,
                           size_t scratch_bytes, int32_t* status, momms_stream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 1) return -3;
    if (bits < 1 || bits > 56) return -4;
    if (!Ar) return -5;
    if (!Br) return -6;
    if (m_pad < std::max<int64_t>(m, 1)) return -7;
    if (n_pad < std::max<int64_t>(n, 1)) return -8;
    if (k_pad < k || k_pad % momms::kEmuBK) return -9;
    if (member < MOMMS_MEMBER_AUTO || member > MOMMS_MEMBER_A1) return -10;
    if (!res && m > 0 && n > 0) return -11;
    if (!scratch) return -12;
    if (scratch_bytes < momms::emu_scratch_bytes(momms::device_sm_count())) return MOMMS_ERR_WORKSPACE;
    if (!status) return -14;
    momms::CrtConsts c;
    momms::CrtRecon r;
    if (!momms::crt_plan(bits, k, &c, &r)) return MOMMS_ERR_UNSUPPORTED;
    if (m == 0 || n == 0) return MOMMS_OK;
    momms::EmuGemmArgs a{};
    a.m = m; a.n = n; a.k = k; a.S = c.N; a.beta = kDigitBits;
    a.Ad = Ar; a.Bd = Br; a.m_pad = m_pad; a.n_pad = n_pad; a.k_pad = k_pad;
    a.alpha = 1.0; a.beta_c = 0.0;
    a.member = member; a.group = 0;
    a.scratch = scratch; a.scratch_bytes = scratch_bytes; a.status = status; a.max_ctas = 0; a.tile_n = 0;
    a.crt = &c;
    a.res = res;
    a.cta_pairs = pairs_on(0) ? 1 : 0;
    int passes = 0;
    cudaError_t ce = momms::launch_emu_slice_gemm(a, &passes, reinterpret_cast<cudaStream_t>(stream));
    if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    return cuda_fail(ce);
}

int momms_crt_reconstruct(int64_t m, int64_t n, int64_t k, int bits, const uint8_t* res, const int32_t* e,
                          const uint8_t* eflags, const int32_t* f, const uint8_t* fflags, double alpha,
                          double beta, double* C, int64_t ldc, momms_stream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 1) return -3;
    if (bits < 1 || bits > 56) return -4;
    if (!res && m > 0 && n > 0) return -5;
    if (!e && m > 0) return -6;
    if (!eflags && m > 0) return -7;
    if (!f && n > 0) return -8;
    if (!fflags && n > 0) return -9;
    if (!C && m > 0 && n > 0) return -12;
    if (ldc < std::max<int64_t>(1, m)) return -13;
    momms::CrtConsts c;
    momms::CrtRecon r;
    if (!momms::crt_plan(bits, k, &c, &r)) return MOMMS_ERR_UNSUPPORTED;
    return cuda_fail(momms::launch_crt_reconstruct(m, n, res, r, e, eflags, f, fflags, alpha, beta, C, ldc,
                                                   reinterpret_cast<cudaStream_t>(stream)));
}

// ------------------------------------------------------------------ plan cache
static std::string plan_header() {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    char buf[sizeof(prop.name) + 64];  // the device name (up to 255 characters) and the numbers fit
    std::snprintf(buf, sizeof(buf), "momms-plan v2 %s sms=%d l2=%d", prop.name, prop.multiProcessorCount,
                  prop.l2CacheSize);
    for (char* c = buf; *c; ++c)
        if (*c == '\n') *c = ' ';
    return buf;
}

int momms_load_plans(momms_handle_t h, const char* path) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (!path) return -2;
    FILE* fp = std::fopen(path, "r");
    if (!fp) return MOMMS_ERR_IO;
    char line[512];
    if (!std::fgets(line, sizeof(line), fp)) {
        std::fclose(fp);
        return MOMMS_ERR_IO;
    }
    std::string hdr(line);
    while (!hdr.empty() && (hdr.back() == '\n' || hdr.back() == '\r')) hdr.pop_back();
    if (hdr != plan_header()) {
        std::fclose(fp);
        return MOMMS_ERR_IO;  // written on another device or by another version: ignored
    }
    std::map<uint32_t, Plan> plans;
    unsigned key;
    int mode, member, slices, tile_n, scheme, pairs;
    while (std::fscanf(fp, "%u %d %d %d %d %d %d", &key, &mode, &member, &slices, &tile_n, &scheme, &pairs) == 7) {
        if (mode < MOMMS_MODE_NATIVE || mode > MOMMS_MODE_EMULATED) continue;
        if (member < MOMMS_MEMBER_C2 || member > MOMMS_MEMBER_A1) continue;
        if (slices < 0 || slices > MOMMS_MAX_SLICES) continue;
        if (tile_n != 0 && tile_n != 96 && tile_n != 192) continue;
        if (scheme < MOMMS_SCHEME_AUTO || scheme > MOMMS_SCHEME_MODULI) continue;
        if (pairs < 0 || pairs > 2) continue;
        plans[key] = Plan{mode, member, slices, tile_n, scheme, pairs};
    }
    std::fclose(fp);
    for (auto& kv : plans) h->plans[kv.first] = kv.second;
    return MOMMS_OK;
}

static int save_plans(momms_handle_t h, const char* path) {
    std::string tmp = std::string(path) + ".tmp";
    FILE* fp = std::fopen(tmp.c_str(), "w");
    if (!fp) return MOMMS_ERR_IO;
    std::fprintf(fp, "%s\n", plan_header().c_str());
    for (auto& kv : h->plans)
        std::fprintf(fp, "%u %d %d %d %d %d %d\n", kv.first, kv.second.mode, kv.second.member, kv.second.slices,
                     kv.second.tile_n, kv.second.scheme, kv.second.pairs);
    std::fclose(fp);
    if (std::rename(tmp.c_str(), path) != 0) return MOMMS_ERR_IO;
    return MOMMS_OK;
}

__global__ void fill_uniform_kernel(double* x, int64_t n, uint64_t seed) {
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = 2.0 * static_cast<double>(z >> 11) * 0x1.0p-53 - 1.0;
    }
}

// The candidate plans of one bucket: the native engine (its members time the same: the FP64 pipe
// bounds it), and for the emulated engine every member x tile width x encoding, with CTA pairs on
// and off where they apply (moduli, 192-wide tiles).  The slice count stays data-driven.
static std::vector<Plan> tune_candidates(int64_t k) {
    std::vector<Plan> c = {{MOMMS_MODE_NATIVE, MOMMS_MEMBER_C2, 0, 0, MOMMS_SCHEME_AUTO, 0}};
    for (int mem = MOMMS_MEMBER_C2; mem <= MOMMS_MEMBER_A1; ++mem)
        for (int tn : {192, 96})
            for (int sch : {MOMMS_SCHEME_SLICES, MOMMS_SCHEME_MODULI}) {
                if (sch == MOMMS_SCHEME_MODULI && k > momms::crt_max_k()) continue;
                if (sch == MOMMS_SCHEME_MODULI && tn == 192) {
                    c.push_back({MOMMS_MODE_EMULATED, mem, 0, tn, sch, 1});
                    c.push_back({MOMMS_MODE_EMULATED, mem, 0, tn, sch, 2});
                } else {
                    c.push_back({MOMMS_MODE_EMULATED, mem, 0, tn, sch, 1});
                }
            }
    return c;
}

int momms_tune_ex(momms_handle_t h, const char* path, int64_t count, const int64_t* m, const int64_t* n,
                  const int64_t* k, const int* op_a, const int* op_b, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (count < 0) return -3;
    if (count > 0 && (!m || !n || !k)) return -4;
    for (int64_t i = 0; i < count; ++i)
        if ((op_a && op_a[i] != MOMMS_OP_N && op_a[i] != MOMMS_OP_T) ||
            (op_b && op_b[i] != MOMMS_OP_N && op_b[i] != MOMMS_OP_T))
            return -7;
    if (path) momms_load_plans(h, path);  // a missing or stale file is simply re-tuned
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int saved_mode = h->mode, saved_member = h->member, saved_slices = h->slices;
    const int saved_tile = h->tile_n, saved_scheme = h->scheme, saved_pairs = h->cta_pairs;
    FILE* log = nullptr;
    if (const char* lp = std::getenv("MOMMS_TUNE_LOG")) log = std::fopen(lp, "a");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int status = MOMMS_OK;
    for (int64_t i = 0; i < count && status == MOMMS_OK; ++i) {
        if (m[i] <= 0 || n[i] <= 0 || k[i] <= 0) continue;
        const int oa = op_a ? op_a[i] : MOMMS_OP_N, ob = op_b ? op_b[i] : MOMMS_OP_N;
        const uint32_t key = bucket_key(m[i], n[i], k[i], oa, ob);
        if (h->plans.count(key)) continue;
        // op(A) is m x k, op(B) k x n; stored with the leading dimension of their stored rows
        const int64_t ra = oa == MOMMS_OP_N ? m[i] : k[i], ca = oa == MOMMS_OP_N ? k[i] : m[i];
        const int64_t rb = ob == MOMMS_OP_N ? k[i] : n[i], cb = ob == MOMMS_OP_N ? n[i] : k[i];
        double *A = nullptr, *B = nullptr, *C = nullptr;
        if (cudaMalloc(&A, sizeof(double) * ra * ca) != cudaSuccess ||
            cudaMalloc(&B, sizeof(double) * rb * cb) != cudaSuccess ||
            cudaMalloc(&C, sizeof(double) * m[i] * n[i]) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(A); cudaFree(B); cudaFree(C);
            status = MOMMS_ERR_ALLOC;
            break;
        }
        fill_uniform_kernel<<<1024, 256, 0, s>>>(A, ra * ca, 1);
        fill_uniform_kernel<<<1024, 256, 0, s>>>(B, rb * cb, 2);
        Plan best{MOMMS_MODE_NATIVE, MOMMS_MEMBER_C2, 0, 0, MOMMS_SCHEME_AUTO, 0};
        double best_ms = 1e300;
        for (const Plan& c : tune_candidates(k[i])) {
            h->mode = c.mode; h->member = c.member; h->slices = 0;
            h->tile_n = c.tile_n; h->scheme = c.scheme; h->cta_pairs = c.pairs;
            auto call = [&]() {
                return gemm_dispatch(h, oa, ob, m[i], n[i], k[i], 1.0, A, ra, B, rb, 0.0, C, m[i], s);
            };
            int rc = call();  // warm-up (workspace, kernel attributes)
            if (rc) continue;
            // at least three timed calls and at least 20 ms of them (at most 50 calls)
            int reps = 0;
            float total = 0.f;
            while (rc == MOMMS_OK && reps < 50 && (reps < 3 || total < 20.f)) {
                cudaEventRecord(e0, s);
                rc = call();
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                total += ms;
                ++reps;
            }
            if (rc != MOMMS_OK) continue;
            const double per = total / reps;
            if (log)
                std::fprintf(log, "m=%lld n=%lld k=%lld opa=%d opb=%d mode=%d member=%d tile_n=%d scheme=%d pairs=%d "
                                  "ms=%.4f reps=%d\n",
                             static_cast<long long>(m[i]), static_cast<long long>(n[i]), static_cast<long long>(k[i]),
                             oa, ob, c.mode, c.member, c.tile_n, c.scheme, c.pairs, per, reps);
            if (per < best_ms) {
                best_ms = per;
                best = c;
            }
        }
        h->plans[key] = best;
        cudaStreamSynchronize(s);
        cudaFree(A); cudaFree(B); cudaFree(C);
    }
    h->mode = saved_mode; h->member = saved_member; h->slices = saved_slices;
    h->tile_n = saved_tile; h->scheme = saved_scheme; h->cta_pairs = saved_pairs;
    if (log) std::fclose(log);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status == MOMMS_OK && path) status = save_plans(h, path);
    return status;
}

int momms_tune(momms_handle_t h, const char* path, int64_t count, const int64_t* m, const int64_t* n,
               const int64_t* k, momms_stream_t stream) {
    return momms_tune_ex(h, path, count, m, n, k, nullptr, nullptr, stream);
}

int momms_get_plan(momms_handle_t h, int op_a, int op_b, int64_t m, int64_t n, int64_t k, momms_plan_t* plan) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (op_a != MOMMS_OP_N && op_a != MOMMS_OP_T) return -2;
    if (op_b != MOMMS_OP_N && op_b != MOMMS_OP_T) return -3;
    if (m < 1) return -4;
    if (n < 1) return -5;
    if (k < 1) return -6;
    if (!plan) return -7;
    auto it = h->plans.find(bucket_key(m, n, k, op_a, op_b));
    const Plan p = it != h->plans.end() ? it->second : default_plan(m, n, k);
    plan->tuned = it != h->plans.end() ? 1 : 0;
    plan->mode = p.mode;
    plan->member = p.member;
    plan->slices = p.slices;
    plan->tile_n = p.tile_n;
    plan->scheme = p.scheme;
    plan->cta_pairs = p.pairs;
    return MOMMS_OK;
}

// ------------------------------------------------------------------ symmetric rank-k update
namespace {

// Emulated SYRK: op(A) is split into digits once and serves as both operands; the slice
// products run over the tile rows of the referenced triangle only (one problem of the
// batched slice-product launch per 128-row block, the diagonal tiles masked), in k passes
// that keep the int32 diagonal sums exact.
int run_syrk_emulated(momms_handle_t h, int uplo, int trans, int64_t n, int64_t k, double alpha, const double* A,
                      int64_t lda, double beta, double* C, int64_t ldc, int S, cudaStream_t s) {
    const int bb = h->digit_bits;
    const int64_t k_pad = round_up(std::max<int64_t>(k, 1), momms::kEmuBK);
    const int S_alloc = S > 0 ? S : kAutoSliceMax;
    const int64_t tiles_m = (n + momms::kEmuBM - 1) / momms::kEmuBM;
    // workspace: exponents, flags, norms, digits, recombination scratch
    size_t o = 0;
    const size_t off_e = o;  o += align256(sizeof(int32_t) * n);
    const size_t off_ef = o; o += align256(static_cast<size_t>(n));
    const size_t off_l1 = o; o += align256(sizeof(float) * n);
    const size_t off_d = o;  o += align256(size_t(2) * S_alloc * n * k_pad);
    const size_t scratch_bytes = momms::emu_scratch_bytes(momms::device_sm_count());
    const size_t off_scr = o; o += align256(scratch_bytes);
    void* ws = nullptr;
    int rc = ensure_workspace(h, o, &ws);
    if (rc) return rc;
    char* w = static_cast<char*>(ws);
    int32_t* e = reinterpret_cast<int32_t*>(w + off_e);
    uint8_t* ef = reinterpret_cast<uint8_t*>(w + off_ef);
    float* l1 = reinterpret_cast<float*>(w + off_l1);
    char* Ad = w + off_d;
    int64_t launches = 0;
    if (momms::launch_emu_scale(0, trans, n, k, A, lda, e, ef, S > 0 ? nullptr : l1, s) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += momms::emu_scale_kernel_count(0, trans);
    if (S <= 0) {
        // one spread: the second operand is the first one transposed
        if (cudaMemsetAsync(h->spread_dev, 0, sizeof(int), s) != cudaSuccess ||
            momms::launch_emu_spread(n, k, e, ef, l1, h->spread_dev, s) != cudaSuccess ||
            cudaMemcpyAsync(h->spread_host, h->spread_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 1;
        S = slices_from_spread(h->spread_host[0] / 16.0, h->spread_host[0] / 16.0, k, bb, nullptr);
    }
    if (S > S_alloc) return MOMMS_ERR_UNSUPPORTED;
    if (momms::launch_emu_split(0, trans, n, k, A, lda, e, ef, S, bb, Ad, n, k_pad, s) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    launches += 1;
    // one batched slice-product launch per k pass over the triangle's tile rows
    const int64_t pass = momms::emu_max_k_per_pass(S, bb);
    std::vector<momms::EmuBatchProblem> table;
    std::vector<char> all;
    for (int64_t k0 = 0; k0 < k_pad; k0 += pass) {
        const int64_t kp = std::min(pass, k_pad - k0);
        table.assign(static_cast<size_t>(tiles_m), momms::EmuBatchProblem{});
        int64_t tiles = 0;
        for (int64_t tm = 0; tm < tiles_m; ++tm) {
            momms::EmuBatchProblem& g = table[static_cast<size_t>(tm)];
            std::memset(&g, 0, sizeof(g));
            const int64_t r0 = tm * momms::kEmuBM, mb = std::min<int64_t>(momms::kEmuBM, n - r0);
            const int64_t c0 = uplo == MOMMS_LOWER ? 0 : r0;
            const int64_t nb = uplo == MOMMS_LOWER ? std::min<int64_t>(n, r0 + momms::kEmuBM) : n - r0;
            const char* baseA = Ad + (static_cast<size_t>(r0) * k_pad + k0) * 2;
            const char* baseB = Ad + (static_cast<size_t>(c0) * k_pad + k0) * 2;
            if (!momms::emu_make_digit_map(&g.mapA, baseA, kp, mb, S, momms::kEmuBM, n, k_pad) ||
                !momms::emu_make_digit_map(&g.mapB, baseB, kp, nb, S, momms::kEmuBNMax, n, k_pad))
                return MOMMS_ERR_UNSUPPORTED;
            g.e = e + r0; g.ef = ef + r0; g.f = e + c0; g.ff = ef + c0;
            g.C = C + r0 + c0 * ldc; g.ldc = ldc;
            g.alpha = alpha; g.beta_c = k0 == 0 ? beta : 1.0;
            g.m = static_cast<int32_t>(mb); g.n = static_cast<int32_t>(nb); g.S = S; g.beta = bb;
            g.nslab = static_cast<int32_t>(kp / momms::kEmuBK);
            g.chunk_slabs = momms::emu_chunk_slabs(bb);
            g.group_end = momms::emu_group_ends(S, bb, kp);
            g.tiles_n = static_cast<int32_t>((nb + momms::kEmuBNMax - 1) / momms::kEmuBNMax);
            g.tile0 = tiles;
            g.tri = uplo == MOMMS_LOWER ? 1 : 2;
            g.diag = uplo == MOMMS_LOWER ? static_cast<int32_t>(r0) : 0;
            tiles += g.tiles_n;
        }
        const size_t off = align256(all.size());
        all.resize(off + sizeof(momms::EmuBatchProblem) * table.size());
        std::memcpy(all.data() + off, table.data(), sizeof(momms::EmuBatchProblem) * table.size());
    }
    // upload every pass's table at once (kept by the handle until the next upload)
    rc = grow_device(&h->batch_tables, &h->batch_tables_cap, all.size());
    if (rc) return rc;
    if (cudaMemcpyAsync(h->batch_tables, all.data(), all.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    h->host_tables.swap(all);
    size_t off = 0;
    int npass = 0;
    for (int64_t k0 = 0; k0 < k_pad; k0 += pass, ++npass) {
        off = align256(off);
        const auto* dt = reinterpret_cast<const momms::EmuBatchProblem*>(static_cast<char*>(h->batch_tables) + off);
        int64_t tiles = 0;
        const auto* ht = reinterpret_cast<const momms::EmuBatchProblem*>(h->host_tables.data() + off);
        for (int64_t tm = 0; tm < tiles_m; ++tm) tiles += ht[tm].tiles_n;
        if (momms::launch_emu_slice_gemm_batched(dt, static_cast<int>(tiles_m), tiles, w + off_scr, scratch_bytes,
                                                 h->status, s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        launches += 1;
        off += sizeof(momms::EmuBatchProblem) * static_cast<size_t>(tiles_m);
    }
    reset_report(h);
    h->report.mode = MOMMS_MODE_EMULATED;
    h->report.member = MOMMS_MEMBER_AUTO;
    h->report.slices = S;
    h->report.digit_bits = bb;
    h->report.k_passes = npass;
    h->report.tile_m = momms::kEmuBM;
    h->report.tile_n = momms::kEmuBNMax;
    h->report.launches = launches;
    return MOMMS_OK;
}

}  // namespace

int momms_syrk(momms_handle_t h, int uplo, int trans, int64_t n, int64_t k, double alpha, const double* A,
               int64_t lda, double beta, double* C, int64_t ldc, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (uplo != MOMMS_LOWER && uplo != MOMMS_UPPER) return -2;
    if (trans != MOMMS_OP_N && trans != MOMMS_OP_T) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (lda < std::max<int64_t>(1, trans == MOMMS_OP_N ? n : k)) return -8;
    if (ldc < std::max<int64_t>(1, n)) return -11;
    const bool product = n > 0 && k > 0 && alpha != 0.0;
    if (product && !A) return -7;
    if (n > 0 && !C) return -10;
    if (n > (int64_t(1) << 30) || k > (int64_t(1) << 30)) return MOMMS_ERR_UNSUPPORTED;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int tri = uplo == MOMMS_LOWER ? 1 : 2;
    reset_report(h);
    if (n == 0) return MOMMS_OK;
    if (!product) {
        h->report.launches = beta == 1.0 ? 0 : 1;
        return scale_c(n, n, beta, C, ldc, s, tri);
    }
    const Plan p = pick_plan(h, n, n, k);
    if (p.mode == MOMMS_MODE_EMULATED) {
        if (h->scheme != MOMMS_SCHEME_SLICES && h->digit_bits == kDigitBits) {
            // the modular encoding over the triangle's tiles, when it is chosen (op(A) times its
            // transpose: the product's second operand is A with the other transposition)
            const int rc = run_emulated(h, trans, 1 - trans, n, n, k, alpha, A, lda, A, lda, beta, C, ldc,
                                        MOMMS_MEMBER_AUTO, p.slices, s, tri);
            if (rc != kSlicesChosen) return rc;
        }
        return run_syrk_emulated(h, uplo, trans, n, k, alpha, A, lda, beta, C, ldc, p.slices, s);
    }
    const int member = p.member == MOMMS_MEMBER_AUTO ? MOMMS_MEMBER_C2 : p.member;
    int ctas = 0, group = 0;
    cudaError_t e = momms::launch_native_gemm(trans, 1 - trans, n, n, k, alpha, A, lda, A, lda, beta, C, ldc, member,
                                              h->max_ctas, h->group, s, &ctas, &group, tri);
    if (e == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return MOMMS_ERR_CUDA;
    h->report.mode = MOMMS_MODE_NATIVE;
    h->report.member = member;
    h->report.tile_m = momms::kNativeBM;
    h->report.tile_n = momms::kNativeBN;
    h->report.k_passes = 1;
    h->report.ctas = ctas;
    h->report.group = group;
    h->report.launches = 1;
    return MOMMS_OK;
}

// ------------------------------------------------------------------ triangular product
namespace {

// T (t x t, leading dimension t) := the uplo triangle of A with the other triangle zero and,
// for a unit diagonal, ones on the diagonal (A's diagonal is then not read).
__global__ void tri_extract_kernel(int64_t t, const double* __restrict__ A, int64_t lda, int uplo, int unit,
                                   double* __restrict__ T) {
    const int64_t total = t * t;
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t i = idx % t, j = idx / t;
        const bool inside = uplo == MOMMS_LOWER ? (i >= j) : (i <= j);
        double v = 0.0;
        if (i == j && unit) v = 1.0;
        else if (inside) v = A[i + j * lda];
        T[idx] = v;
    }
}

}  // namespace

int momms_trmm(momms_handle_t h, int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
               const double* A, int64_t lda, double* B, int64_t ldb, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (side != MOMMS_LEFT && side != MOMMS_RIGHT) return -2;
    if (uplo != MOMMS_LOWER && uplo != MOMMS_UPPER) return -3;
    if (trans != MOMMS_OP_N && trans != MOMMS_OP_T) return -4;
    if (diag != MOMMS_NON_UNIT && diag != MOMMS_UNIT) return -5;
    if (m < 0) return -6;
    if (n < 0) return -7;
    const int64_t t = side == MOMMS_LEFT ? m : n;  // order of the triangular matrix
    if (lda < std::max<int64_t>(1, t)) return -10;
    if (ldb < std::max<int64_t>(1, m)) return -12;
    if (m > 0 && n > 0 && alpha != 0.0 && !A) return -9;
    if (m > 0 && n > 0 && !B) return -11;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    reset_report(h);
    if (m == 0 || n == 0) return MOMMS_OK;
    if (alpha == 0.0) {
        h->report.launches = 1;
        return scale_c(m, n, 0.0, B, ldb, s);
    }
    // the triangle (zero elsewhere) as a dense t x t operand; B is overwritten with the product
    const Plan p = pick_plan(h, m, n, t);
    const bool emulated = p.mode == MOMMS_MODE_EMULATED;
    const size_t tbytes = align256(static_cast<size_t>(t) * t * sizeof(double));
    const size_t bbytes = emulated ? 0 : align256(static_cast<size_t>(m) * n * sizeof(double));
    int rc = grow_device(&h->ooc_buf, &h->ooc_bytes, tbytes + bbytes);
    if (rc) return rc;
    double* T = static_cast<double*>(h->ooc_buf);
    int64_t blocks = (t * t + 255) / 256;
    blocks = std::min<int64_t>(blocks, int64_t(momms::device_sm_count()) * 16);
    tri_extract_kernel<<<static_cast<unsigned>(std::max<int64_t>(blocks, 1)), 256, 0, s>>>(t, A, lda, uplo, diag,
                                                                                          T);
    if (cudaGetLastError() != cudaSuccess) return MOMMS_ERR_CUDA;
    int64_t launches = 1;
    if (emulated) {
        // in place: the emulated path splits both operands into digits before the slice products
        // write C, and B is not read again (beta = 0).  With the modular encoding each tile's
        // products skip the k range where op(T) is zero: op(T) is lower when the stored triangle is
        // lower and not transposed, or upper and transposed
        const bool op_lower = (uplo == MOMMS_LOWER) != (trans == MOMMS_OP_T);
        const int member = p.member == MOMMS_MEMBER_AUTO ? MOMMS_MEMBER_C2 : p.member;
        rc = side == MOMMS_LEFT
                 ? run_emulated(h, trans, MOMMS_OP_N, m, n, m, alpha, T, t, B, ldb, 0.0, B, ldb, member, p.slices,
                                s, 0, op_lower ? 1 : 2)
                 : run_emulated(h, MOMMS_OP_N, trans, m, n, n, alpha, B, ldb, T, t, 0.0, B, ldb, member, p.slices,
                                s, 0, op_lower ? 3 : 4);
    } else {
        // the native kernel reads B while it writes C: product from a copy of B
        double* Bc = reinterpret_cast<double*>(reinterpret_cast<char*>(h->ooc_buf) + tbytes);
        if (cudaMemcpy2DAsync(Bc, static_cast<size_t>(m) * sizeof(double), B, static_cast<size_t>(ldb) * sizeof(double),
                              static_cast<size_t>(m) * sizeof(double), static_cast<size_t>(n),
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        const int member = p.member == MOMMS_MEMBER_AUTO ? MOMMS_MEMBER_C2 : p.member;
        rc = side == MOMMS_LEFT
                 ? run_native(h, trans, MOMMS_OP_N, m, n, m, alpha, T, t, Bc, m, 0.0, B, ldb, member, s)
                 : run_native(h, MOMMS_OP_N, trans, m, n, n, alpha, Bc, m, T, t, 0.0, B, ldb, member, s);
    }
    if (rc) return rc;
    h->report.launches += launches;
    return MOMMS_OK;
}

// ------------------------------------------------------------------ triangular solve
namespace {

struct TrsmCtx {
    momms_handle_t h;
    int side, uplo, trans;
    bool eff_lower;        // op(A) is lower triangular
    int64_t m, n;
    const double* A;
    int64_t lda;
    double* B;
    int64_t ldb;
    const double* W;       // inverses of the leaf blocks (kTrsmLeaf^2 each, stride kTrsmLeaf)
    double* T;             // leaf product before it is copied into B
    cudaStream_t s;
    int64_t launches;
};

int trsm_gemm(TrsmCtx& c, int opa, int opb, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
              int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc) {
    const int rc = gemm_dispatch(c.h, opa, opb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, c.s);
    c.launches += c.h->report.launches;
    return rc;
}

// Element (r, q) block of op(A): pointer into A and the op that yields it.
const double* op_block(const TrsmCtx& c, int64_t r, int64_t q, int* op) {
    *op = c.trans;
    return c.trans == MOMMS_OP_N ? c.A + r + q * c.lda : c.A + q + r * c.lda;
}

// Rows [r0, r1) of op(A) X = alpha B (side LEFT) or columns [r0, r1) of X op(A) = alpha B
// (side RIGHT), the blocks of op(A) before (LEFT, lower) or after them already solved.
int trsm_rec(TrsmCtx& c, int64_t r0, int64_t r1, double alpha) {
    const int64_t size = r1 - r0;
    const bool left = c.side == MOMMS_LEFT;
    constexpr int64_t leaf = momms::kTrsmLeaf;
    if (size <= leaf) {
        // leaf: X = alpha op(inv(A_bb)) B_b through the scratch T, then copied into B
        const double* Wb = c.W + (r0 / leaf) * leaf * leaf;
        int rc;
        if (left) {
            rc = trsm_gemm(c, c.trans, MOMMS_OP_N, size, c.n, size, alpha, Wb, leaf, c.B + r0, c.ldb, 0.0,
                           c.T, size);
            if (rc) return rc;
            if (cudaMemcpy2DAsync(c.B + r0, c.ldb * sizeof(double), c.T, size * sizeof(double), size * sizeof(double),
                                  c.n, cudaMemcpyDeviceToDevice, c.s) != cudaSuccess)
                return MOMMS_ERR_CUDA;
        } else {
            rc = trsm_gemm(c, MOMMS_OP_N, c.trans, c.m, size, size, alpha, c.B + r0 * c.ldb, c.ldb, Wb,
                           leaf, 0.0, c.T, c.m);
            if (rc) return rc;
            if (cudaMemcpy2DAsync(c.B + r0 * c.ldb, c.ldb * sizeof(double), c.T, c.m * sizeof(double),
                                  c.m * sizeof(double), size, cudaMemcpyDeviceToDevice, c.s) != cudaSuccess)
                return MOMMS_ERR_CUDA;
        }
        return MOMMS_OK;
    }
    // split at a multiple of the leaf order, near the middle
    const int64_t half_blocks = ((size + leaf - 1) / leaf) / 2;
    const int64_t mid = r0 + half_blocks * leaf;
    // LEFT: op(A) lower -> first half first; RIGHT: op(A) upper -> first half first
    const bool first_half_first = left ? c.eff_lower : !c.eff_lower;
    const int64_t a0 = first_half_first ? r0 : mid, a1 = first_half_first ? mid : r1;   // solved first
    const int64_t b0 = first_half_first ? mid : r0, b1 = first_half_first ? r1 : mid;   // updated, then solved
    int rc = trsm_rec(c, a0, a1, alpha);
    if (rc) return rc;
    int op;
    if (left) {
        // B_b := alpha B_b - op(A)[b, a] X_a
        const double* Aba = op_block(c, b0, a0, &op);
        rc = trsm_gemm(c, op, MOMMS_OP_N, b1 - b0, c.n, a1 - a0, -1.0, Aba, c.lda, c.B + a0, c.ldb, alpha, c.B + b0,
                       c.ldb);
    } else {
        // B_b := alpha B_b - X_a op(A)[a, b]
        const double* Aab = op_block(c, a0, b0, &op);
        rc = trsm_gemm(c, MOMMS_OP_N, op, c.m, b1 - b0, a1 - a0, -1.0, c.B + a0 * c.ldb, c.ldb, Aab, c.lda, alpha,
                       c.B + b0 * c.ldb, c.ldb);
    }
    if (rc) return rc;
    return trsm_rec(c, b0, b1, 1.0);
}

// The inverses of the leaf blocks from those of their kTrsmNb-blocks (already on W's diagonal):
// at each level s = kTrsmNb, 2 kTrsmNb, .. < kTrsmLeaf, every pair of s-blocks of a leaf is joined,
//   lower: [L11 0; L21 L22]^-1 = [I11 0; -I22 (L21 I11) I22],
//   upper: [U11 U12; 0 U22]^-1 = [I11 -I11 (U12 I22); 0 I22],
// as two batched products per level (all the inner products, then all the outer ones) -- emulated
// unless the handle asks for native (the batches are small: ~1 GFLOP per 8192 rows, 1 ms on the
// FP64 tensor pipe).  Tmp holds the inner products.
int trsm_join_inverses(momms_handle_t h, int64_t t, const double* A, int64_t lda, int uplo, double* W, double* Tmp,
                       cudaStream_t s, int64_t* launches) {
    constexpr int64_t leaf = momms::kTrsmLeaf;
    const bool lower = uplo == MOMMS_LOWER;
    struct ModeGuard {  // the batched calls below run emulated in AUTO; the caller's mode comes back after
        momms_handle_t h;
        int saved;
        ~ModeGuard() { h->mode = saved; }
    } guard{h, h->mode};
    if (h->mode == MOMMS_MODE_AUTO) h->mode = MOMMS_MODE_EMULATED;
    for (int64_t sz = momms::kTrsmNb; sz < leaf; sz *= 2) {
        std::vector<int64_t> m1, n1, k1, lda1, ldb1, ldc1, m2, n2, k2, lda2, ldb2, ldc2;
        std::vector<const double*> a1, b1, a2, b2;
        std::vector<double*> c1, c2;
        double* tmp = Tmp;
        for (int64_t b0 = 0; b0 < t; b0 += leaf) {
            const int64_t lsz = std::min(leaf, t - b0);
            double* Wl = W + (b0 / leaf) * leaf * leaf;
            for (int64_t o = 0; o + sz < lsz; o += 2 * sz) {
                const int64_t s1 = sz, s2 = std::min(sz, lsz - o - sz);  // sizes of the two diagonal blocks
                const double* I11 = Wl + o + o * leaf;
                const double* I22 = Wl + (o + sz) + (o + sz) * leaf;
                if (lower) {
                    // Tmp = L21 I11 (s2 x s1); W21 = -I22 Tmp
                    m1.push_back(s2); n1.push_back(s1); k1.push_back(s1);
                    a1.push_back(A + (b0 + o + sz) + (b0 + o) * lda); lda1.push_back(lda);
                    b1.push_back(I11); ldb1.push_back(leaf);
                    c1.push_back(tmp); ldc1.push_back(s2);
                    m2.push_back(s2); n2.push_back(s1); k2.push_back(s2);
                    a2.push_back(I22); lda2.push_back(leaf);
                    b2.push_back(tmp); ldb2.push_back(s2);
                    c2.push_back(Wl + (o + sz) + o * leaf); ldc2.push_back(leaf);
                    tmp += s2 * s1;
                } else {
                    // Tmp = U12 I22 (s1 x s2); W12 = -I11 Tmp
                    m1.push_back(s1); n1.push_back(s2); k1.push_back(s2);
                    a1.push_back(A + (b0 + o) + (b0 + o + sz) * lda); lda1.push_back(lda);
                    b1.push_back(I22); ldb1.push_back(leaf);
                    c1.push_back(tmp); ldc1.push_back(s1);
                    m2.push_back(s1); n2.push_back(s2); k2.push_back(s1);
                    a2.push_back(I11); lda2.push_back(leaf);
                    b2.push_back(tmp); ldb2.push_back(s1);
                    c2.push_back(Wl + o + (o + sz) * leaf); ldc2.push_back(leaf);
                    tmp += s1 * s2;
                }
            }
        }
        const int64_t cnt = static_cast<int64_t>(m1.size());
        if (cnt == 0) continue;
        const std::vector<double> one(cnt, 1.0), minus_one(cnt, -1.0), zero(cnt, 0.0);
        int rc = momms_gemm_batched(h, cnt, m1.data(), n1.data(), k1.data(), one.data(), a1.data(), lda1.data(),
                                    b1.data(), ldb1.data(), zero.data(), c1.data(), ldc1.data(),
                                    reinterpret_cast<momms_stream_t>(s));
        if (rc) return rc;
        *launches += h->report.launches;
        rc = momms_gemm_batched(h, cnt, m2.data(), n2.data(), k2.data(), minus_one.data(), a2.data(), lda2.data(),
                                b2.data(), ldb2.data(), zero.data(), c2.data(), ldc2.data(),
                                reinterpret_cast<momms_stream_t>(s));
        if (rc) return rc;
        *launches += h->report.launches;
    }
    return MOMMS_OK;
}

}  // namespace

int momms_trsm(momms_handle_t h, int side, int uplo, int trans, int diag, int64_t m, int64_t n, double alpha,
               const double* A, int64_t lda, double* B, int64_t ldb, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    if (side != MOMMS_LEFT && side != MOMMS_RIGHT) return -2;
    if (uplo != MOMMS_LOWER && uplo != MOMMS_UPPER) return -3;
    if (trans != MOMMS_OP_N && trans != MOMMS_OP_T) return -4;
    if (diag != MOMMS_NON_UNIT && diag != MOMMS_UNIT) return -5;
    if (m < 0) return -6;
    if (n < 0) return -7;
    const int64_t t = side == MOMMS_LEFT ? m : n;  // order of the triangular matrix
    if (lda < std::max<int64_t>(1, t)) return -10;
    if (ldb < std::max<int64_t>(1, m)) return -12;
    if (m > 0 && n > 0 && alpha != 0.0 && !A) return -9;
    if (m > 0 && n > 0 && !B) return -11;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    reset_report(h);
    if (m == 0 || n == 0) return MOMMS_OK;
    if (alpha == 0.0) {
        h->report.launches = 1;
        return scale_c(m, n, 0.0, B, ldb, s);
    }
    // scratch kept by the handle: the leaf blocks' inverses, one leaf's product, and the inner
    // products of the inverses' assembly (at most half a leaf block per leaf)
    const size_t wbytes = align256(momms::tri_inverse_bytes(t));
    const size_t tbytes =
        align256(static_cast<size_t>(momms::kTrsmLeaf) * (side == MOMMS_LEFT ? n : m) * sizeof(double));
    const size_t jbytes = align256(momms::tri_inverse_bytes(t) / 4);
    int rc = grow_device(&h->ooc_buf, &h->ooc_bytes, wbytes + tbytes + jbytes);
    if (rc) return rc;
    double* W = static_cast<double*>(h->ooc_buf);
    double* J = reinterpret_cast<double*>(reinterpret_cast<char*>(h->ooc_buf) + wbytes + tbytes);
    if (cudaMemsetAsync(W, 0, wbytes, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (momms::launch_tri_inverse(t, A, lda, uplo, diag == MOMMS_UNIT, W, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    int64_t join_launches = 0;
    rc = trsm_join_inverses(h, t, A, lda, uplo, W, J, s, &join_launches);
    if (rc) return rc;
    TrsmCtx c{};
    c.h = h;
    c.side = side;
    c.uplo = uplo;
    c.trans = trans;
    c.eff_lower = (uplo == MOMMS_LOWER) != (trans == MOMMS_OP_T);
    c.m = m;
    c.n = n;
    c.A = A;
    c.lda = lda;
    c.B = B;
    c.ldb = ldb;
    c.W = W;
    c.T = reinterpret_cast<double*>(reinterpret_cast<char*>(h->ooc_buf) + wbytes);
    c.s = s;
    c.launches = 1 + join_launches;
    rc = trsm_rec(c, 0, t, alpha);
    if (rc) return rc;
    h->report.launches = c.launches;
    return MOMMS_OK;
}

// ------------------------------------------------------------------ out-of-core products
// Host memory (Grace LPDDR over NVLink-C2C on GB300) is the slow level and HBM the fast one:
// Resident C at the HBM level (Sec. 2.2.1).  A b x b block of C stays in HBM while b x b
// blocks of A and B stream in along k; A is read ceil(n/b) times, B ceil(m/b) times, C read
// once (beta != 0) and written once.  Two buffers per operand let the copies of the next
// blocks run on their own streams while the current block product computes.
namespace {

constexpr int64_t kOocAlign = 256;

// Device bytes of the out-of-core pipeline for block size b (six b x b FP64 buffers) plus the
// workspace of one b x b x b product in the handle's mode.
size_t ooc_device_bytes(momms_handle_t h, int64_t b) {
    size_t ws = 0;
    const Plan p = pick_plan(h, b, b, b);
    if (p.mode == MOMMS_MODE_EMULATED)
        ws = emu_layout(b, b, b, p.slices > 0 ? p.slices : kAutoSliceMax, h->max_ctas,
                        moduli_reserved(h->scheme, p.slices, b)).total;
    return 6 * static_cast<size_t>(b) * b * sizeof(double) + ws;
}

int64_t ooc_block(momms_handle_t h, int64_t m, int64_t n, int64_t k, size_t budget) {
    const int64_t top = round_up(std::max(std::max(m, n), std::max<int64_t>(k, 1)), kOocAlign);
    int64_t best = kOocAlign;
    for (int64_t b = kOocAlign; b <= top; b += kOocAlign)
        if (ooc_device_bytes(h, b) <= budget) best = b;
    return best;
}

int ooc_setup(momms_handle_t h, size_t bytes) {
    if (!h->ooc_in && cudaStreamCreateWithFlags(&h->ooc_in, cudaStreamNonBlocking) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (!h->ooc_out && cudaStreamCreateWithFlags(&h->ooc_out, cudaStreamNonBlocking) != cudaSuccess) return MOMMS_ERR_CUDA;
    for (cudaEvent_t& e : h->ooc_ev)
        if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (h->ooc_bytes < bytes) {
        if (h->ooc_buf) {
            cudaDeviceSynchronize();
            cudaFree(h->ooc_buf);
            h->ooc_buf = nullptr;
            h->ooc_bytes = 0;
        }
        if (cudaMalloc(&h->ooc_buf, bytes) != cudaSuccess) {
            cudaGetLastError();
            return MOMMS_ERR_ALLOC;
        }
        h->ooc_bytes = bytes;
    }
    return MOMMS_OK;
}

// A rows x cols block of a column-major matrix, copied between host and a device buffer with
// leading dimension `dld`.
cudaError_t copy_block(double* dst, int64_t dld, const double* src, int64_t sld, int64_t rows, int64_t cols,
                       cudaMemcpyKind kind, cudaStream_t st) {
    return cudaMemcpy2DAsync(dst, static_cast<size_t>(dld) * sizeof(double), src, static_cast<size_t>(sld) * sizeof(double),
                             static_cast<size_t>(rows) * sizeof(double), static_cast<size_t>(cols), kind, st);
}

}  // namespace

int momms_gemm_host(momms_handle_t h, int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, double* C, int64_t ldc, size_t device_bytes,
                    int64_t block, momms_stream_t stream) {
    if (!valid(h)) return MOMMS_ERR_HANDLE;
    int rc = check_gemm_args(2, MOMMS_OP_N, MOMMS_OP_N, m, n, k, A, lda, B, ldb, C, ldc, alpha, false);
    if (rc) return rc;
    if (block < 0 || block % kOocAlign) return -14;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    momms_report_t total{};
    if (m == 0 || n == 0) {
        h->report = total;
        return MOMMS_OK;
    }
    if (block == 0) {
        size_t budget = device_bytes;
        if (budget == 0) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return MOMMS_ERR_CUDA;
            budget = free_b / 2;
        }
        block = ooc_block(h, m, n, k, budget);
    }
    const int64_t b = block;
    const size_t blk = static_cast<size_t>(b) * b;
    rc = ooc_setup(h, 6 * blk * sizeof(double));
    if (rc) return rc;
    double* buf = static_cast<double*>(h->ooc_buf);
    double* Cb[2] = {buf, buf + blk};
    double* Ab[2] = {buf + 2 * blk, buf + 3 * blk};
    double* Bb[2] = {buf + 4 * blk, buf + 5 * blk};
    cudaEvent_t* ev = h->ooc_ev;
    cudaEvent_t ab_ready[2] = {ev[0], ev[1]}, ab_free[2] = {ev[2], ev[3]};
    cudaEvent_t c_ready[2] = {ev[4], ev[5]}, c_done[2] = {ev[6], ev[7]}, c_free[2] = {ev[8], ev[9]};
    cudaEvent_t start = ev[10];
    // the copy streams start after the work already on the caller's stream
    if (cudaEventRecord(start, s) != cudaSuccess || cudaStreamWaitEvent(h->ooc_in, start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(h->ooc_out, start, 0) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    const bool kzero = (k == 0 || alpha == 0.0);
    int64_t step = 0, cblk = 0, h2d = 0, d2h = 0, launches = 0;
    auto note = [&](const momms_report_t& r) {
        launches += r.launches;
        total.mode = r.mode;
        total.member = r.member;
        total.slices = std::max(total.slices, r.slices);
        total.digit_bits = r.digit_bits;
        total.k_passes = std::max(total.k_passes, r.k_passes);
        total.tile_m = r.tile_m;
        total.tile_n = r.tile_n;
        total.ctas = r.ctas;
        total.group = r.group;
        total.est_err_ratio = std::max(total.est_err_ratio, r.est_err_ratio);
        total.moduli = std::max(total.moduli, r.moduli);
        total.operand_bits = std::max(total.operand_bits, r.operand_bits);
        total.cta_pairs = r.cta_pairs;
    };
    if (h->host_resident == 1 && !kzero) {
        // Resident A at the HBM level (Sec. 2.2.2): a b x b block of A stays on the device while the
        // b x b blocks of B and C of its block row stream through; A is read once, B ceil(m/b) times,
        // C read ceil(k/b) - 1 (+1 when beta != 0) times and written ceil(k/b) times.  B and C share a
        // buffer slot (they change together); A has its own pair of slots.
        const int64_t nbn = (n + b - 1) / b;
        for (int64_t ic = 0; ic < m; ic += b) {
            const int64_t mb = std::min(b, m - ic);
            for (int64_t pc = 0; pc < k; pc += b, ++step) {
                const int64_t kb = std::min(b, k - pc);
                const int as = static_cast<int>(step & 1);
                if (cudaStreamWaitEvent(h->ooc_in, ab_free[as], 0) != cudaSuccess ||
                    copy_block(Ab[as], b, A + ic + pc * lda, lda, mb, kb, cudaMemcpyHostToDevice, h->ooc_in) !=
                        cudaSuccess ||
                    cudaEventRecord(ab_ready[as], h->ooc_in) != cudaSuccess ||
                    cudaStreamWaitEvent(s, ab_ready[as], 0) != cudaSuccess)
                    return MOMMS_ERR_CUDA;
                h2d += mb * kb * 8;
                for (int64_t jc = 0; jc < n; jc += b, ++cblk) {
                    const int64_t nb = std::min(b, n - jc);
                    const int cs = static_cast<int>(cblk & 1);
                    double* hC = C + ic + jc * ldc;
                    const bool read_c = pc > 0 || beta != 0.0;
                    // the slot's last copy-out is done (copy-outs complete in order, so with two or more
                    // block columns that includes this C block's previous k step; with one, wait for it)
                    if (cudaStreamWaitEvent(h->ooc_in, c_free[cs], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                    if (nbn == 1 && cudaStreamWaitEvent(h->ooc_in, c_free[1 - cs], 0) != cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    if (copy_block(Bb[cs], b, B + pc + jc * ldb, ldb, kb, nb, cudaMemcpyHostToDevice, h->ooc_in) !=
                        cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    h2d += kb * nb * 8;
                    if (read_c) {
                        if (copy_block(Cb[cs], b, hC, ldc, mb, nb, cudaMemcpyHostToDevice, h->ooc_in) != cudaSuccess)
                            return MOMMS_ERR_CUDA;
                        h2d += mb * nb * 8;
                    }
                    if (cudaEventRecord(c_ready[cs], h->ooc_in) != cudaSuccess ||
                        cudaStreamWaitEvent(s, c_ready[cs], 0) != cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    rc = gemm_dispatch(h, MOMMS_OP_N, MOMMS_OP_N, mb, nb, kb, alpha, Ab[as], b, Bb[cs], b,
                                       pc == 0 ? beta : 1.0, Cb[cs], b, s);
                    if (rc) return rc;
                    note(h->report);  // (a device-planned product's S and moduli stay pending: no readback here)
                    if (cudaEventRecord(c_done[cs], s) != cudaSuccess ||
                        cudaStreamWaitEvent(h->ooc_out, c_done[cs], 0) != cudaSuccess ||
                        copy_block(hC, ldc, Cb[cs], b, mb, nb, cudaMemcpyDeviceToHost, h->ooc_out) != cudaSuccess ||
                        cudaEventRecord(c_free[cs], h->ooc_out) != cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    d2h += mb * nb * 8;
                }
                if (cudaEventRecord(ab_free[as], s) != cudaSuccess) return MOMMS_ERR_CUDA;
            }
        }
    } else {
        for (int64_t jc = 0; jc < n; jc += b) {
            const int64_t nb = std::min(b, n - jc);
            for (int64_t ic = 0; ic < m; ic += b, ++cblk) {
                const int64_t mb = std::min(b, m - ic);
                const int cs = static_cast<int>(cblk & 1);
                double* hC = C + ic + jc * ldc;
                const bool read_c = beta != 0.0;
                if (cudaStreamWaitEvent(h->ooc_in, c_free[cs], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                if (read_c) {
                    if (copy_block(Cb[cs], b, hC, ldc, mb, nb, cudaMemcpyHostToDevice, h->ooc_in) != cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    h2d += mb * nb * 8;
                }
                if (cudaEventRecord(c_ready[cs], h->ooc_in) != cudaSuccess) return MOMMS_ERR_CUDA;
                if (cudaStreamWaitEvent(s, c_ready[cs], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                if (kzero) {
                    rc = scale_c(mb, nb, beta, Cb[cs], b, s);
                    if (rc) return rc;
                    launches += beta == 1.0 ? 0 : 1;
                }
                for (int64_t pc = 0; !kzero && pc < k; pc += b, ++step) {
                    const int64_t kb = std::min(b, k - pc);
                    const int as = static_cast<int>(step & 1);
                    if (cudaStreamWaitEvent(h->ooc_in, ab_free[as], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                    if (copy_block(Ab[as], b, A + ic + pc * lda, lda, mb, kb, cudaMemcpyHostToDevice, h->ooc_in) !=
                            cudaSuccess ||
                        copy_block(Bb[as], b, B + pc + jc * ldb, ldb, kb, nb, cudaMemcpyHostToDevice, h->ooc_in) !=
                            cudaSuccess)
                        return MOMMS_ERR_CUDA;
                    h2d += (mb * kb + kb * nb) * 8;
                    if (cudaEventRecord(ab_ready[as], h->ooc_in) != cudaSuccess) return MOMMS_ERR_CUDA;
                    if (cudaStreamWaitEvent(s, ab_ready[as], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                    rc = gemm_dispatch(h, MOMMS_OP_N, MOMMS_OP_N, mb, nb, kb, alpha, Ab[as], b, Bb[as], b,
                                       pc == 0 ? beta : 1.0, Cb[cs], b, s);
                    if (rc) return rc;
                    note(h->report);  // (a device-planned product's S and moduli stay pending: no readback here)
                    if (cudaEventRecord(ab_free[as], s) != cudaSuccess) return MOMMS_ERR_CUDA;
                }
                if (cudaEventRecord(c_done[cs], s) != cudaSuccess) return MOMMS_ERR_CUDA;
                if (cudaStreamWaitEvent(h->ooc_out, c_done[cs], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
                if (copy_block(hC, ldc, Cb[cs], b, mb, nb, cudaMemcpyDeviceToHost, h->ooc_out) != cudaSuccess)
                    return MOMMS_ERR_CUDA;
                d2h += mb * nb * 8;
                if (cudaEventRecord(c_free[cs], h->ooc_out) != cudaSuccess) return MOMMS_ERR_CUDA;
            }
        }
    }
    // the caller's stream completes only after the last block is back in host memory
    for (int cs = 0; cs < 2; ++cs)
        if (cudaStreamWaitEvent(s, c_free[cs], 0) != cudaSuccess) return MOMMS_ERR_CUDA;
    total.launches = launches;
    total.ooc_block = b;
    total.ooc_resident = h->host_resident == 1 && !kzero ? 1 : 0;
    total.h2d_bytes = h2d;
    total.d2h_bytes = d2h;
    h->report = total;
    return MOMMS_OK;
}

int momms_member_tile(int member, int group, int64_t cta, int64_t ctas, int64_t i, int tiles_m, int tiles_n,
                      int* tm, int* tn) {
    if (member < MOMMS_MEMBER_AUTO || member > MOMMS_MEMBER_A1) return -1;
    if (ctas < 1 || cta < 0 || cta >= ctas) return -4;
    if (i < 0) return -5;
    if (tiles_m < 0) return -6;
    if (tiles_n < 0) return -7;
    if (!tm) return -8;
    if (!tn) return -9;
    const int mem = member == MOMMS_MEMBER_AUTO ? MOMMS_MEMBER_C2 : member;
    const int g = group > 0 ? group : momms::emu_default_group(ctas, tiles_m, tiles_n);
    return momms::member_tile(mem, g, cta, ctas, i, tiles_m, tiles_n, tm, tn) ? 1 : 0;
}

int momms_tri_tile(int uplo, int tile_n, int64_t n, int64_t t, int* tm, int* tn, int64_t* count) {
    if (uplo != MOMMS_LOWER && uplo != MOMMS_UPPER) return -1;
    if (tile_n != 96 && tile_n != 192) return -2;
    if (n < 0 || n > (int64_t(1) << 30)) return -3;
    if (t < 0) return -4;
    if (!tm) return -5;
    if (!tn) return -6;
    const int tiles_m = static_cast<int>((n + momms::kEmuBM - 1) / momms::kEmuBM);
    const int tiles_n = static_cast<int>((n + tile_n - 1) / tile_n);
    const bool lower = uplo == MOMMS_LOWER;
    if (count) *count = tiles_m > 0 ? momms::tri_prefix(lower, tiles_m, tiles_n, tile_n) : 0;
    return momms::tri_tile(lower, t, tiles_m, tiles_n, tile_n, tm, tn) ? 1 : 0;
}

int momms_probe_peak(int kind, double* tflops, momms_stream_t stream) {
    if (kind < 0 || kind > 5) return -1;
    if (!tflops) return -2;
    cudaError_t e = momms::probe_peak(kind, tflops, reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaErrorNotSupported) return MOMMS_ERR_UNSUPPORTED;
    return cuda_fail(e);
}

int momms_stream_copy(void* dst, const void* src, size_t bytes, int ctas, int repeats, momms_stream_t stream) {
    if (!dst || (reinterpret_cast<uintptr_t>(dst) & 15)) return -1;
    if (!src || (reinterpret_cast<uintptr_t>(src) & 15)) return -2;
    if (bytes % 16) return -3;
    if (ctas < 0) return -4;
    if (repeats < 0) return -5;
    const char* d = static_cast<const char*>(dst);
    const char* s = static_cast<const char*>(src);
    if (bytes && d < s + bytes && s < d + bytes) return -1;  // overlapping ranges
    cudaError_t e = momms::stream_copy(dst, src, bytes, ctas, repeats, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? MOMMS_OK : MOMMS_ERR_CUDA;
}

}  // extern "C"
