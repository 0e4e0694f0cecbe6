// emu_slice_gemm.cu -- the slice products of the emulated FP64 product on the
// fifth-generation tensor cores, with the recombination fused into the epilogue.
//
// For a C tile (BM x BN = 128 x 256) the kernel computes, for every diagonal
// d = S+1 down to 2 of the triangular pair set,
//     P_d = sum_{s+t=d} A_s B_t          (A_s, B_t: integer digit slices in fp16)
// exactly, and folds it into the FP64 Horner sum
//     R_{S+1} = P_{S+1},   R_d = P_d + 2^-beta R_{d+1},
// so that C := alpha * 2^(e_i + f_j - 2 beta) R_2 + beta_c C.
//
// Exactness.  A tcgen05 kind::f16 MMA multiplies fp16 integers exactly and
// accumulates in FP32 in tensor memory (TMEM).  Every partial sum of at most
// `chunk` products of digits |d| <= 2^beta - 1 stays an integer below 2^24, so
// the FP32 accumulator is exact; after each chunk the accumulator is drained
// (tcgen05.ld -> exact float->int conversion -> int32 add in registers).  The
// int32 diagonal sums stay below 2^31 because one launch covers at most
// emu_max_k_per_pass(S, beta) of k.
//
// Memory levels (the paper's Sec. 3.3 vocabulary): the C tile is the resident
// block of registers/TMEM (Resident C at L0, Sec. 3.4); A and B digit tiles are
// streamed through a 4-stage shared-memory ring by TMA; which panels stay in L2
// is set by the member's tile order (raster.cuh).
//
// Roles (320 threads): warp 0 = TMA producer (one thread), warp 1 = TMEM owner
// and MMA issuer (one thread), warps 2..9 = drain / recombination; each drain
// thread holds the 128 int32 diagonal sums of its row in registers.  TMEM holds
// two 256-column FP32 accumulators so that draining one overlaps MMAs into the
// other.  Every mbarrier wait is bounded; on expiry the kernel raises a CTA-wide
// abort flag, lets in-flight copies and MMAs finish, frees TMEM, and reports
// status 1002 (timeout) through p.status.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>

#include "internal.h"
#include "ptx.cuh"
#include "raster.cuh"

namespace momms {
namespace emu {

constexpr int BM = kEmuBM, BN = kEmuBN, BK = kEmuBK;
constexpr int STAGES = 4;
constexpr int EPI_WARPS = 8;
constexpr int EPI_WARP0 = 2;                     // warps 2..9 drain and recombine
constexpr int THREADS = 32 * EPI_WARP0 + 32 * EPI_WARPS;  // 320
constexpr uint32_t A_TILE = BM * BK * 2;   // 16 KB
constexpr uint32_t B_TILE = BN * BK * 2;   // 32 KB
constexpr uint32_t STAGE = A_TILE + B_TILE;
constexpr uint32_t TMEM_COLS = 512;        // two 128 x 256 FP32 accumulators
constexpr uint32_t IDESC = idesc_f16_f32(BM, BN);
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE + 256;

struct Params {
    int m, n;
    int S, beta;
    int chunk_slabs;
    int slab0, nslab;
    int tiles_m, tiles_n;
    int member, group;
    int m_pad, n_pad;
    const int32_t* e;
    const uint8_t* ef;
    const int32_t* f;
    const uint8_t* ff;
    double alpha, beta_c;
    double* C;
    int64_t ldc;
    double* scratch;
    int32_t* status;
};

// r * 2^E with one rounding for every E (two exact power-of-two factors outside
// the normal exponent range; results beyond the double range saturate to 0 / inf).
MOMMS_DEV double scale_pow2(double r, int E) {
    if (E >= -1022 && E <= 1023) return r * pow2_normal(E);
    const int E1 = E > 0 ? 960 : -960;
    int E2 = E - E1;
    E2 = E2 > 1023 ? 1023 : (E2 < -1022 ? -1022 : E2);
    return (r * pow2_normal(E1)) * pow2_normal(E2);
}

// Wait used while shutting down after an abort: ignores the abort flag, keeps the time limit.
MOMMS_DEV bool mbar_wait_drain(uint64_t* bar, uint32_t parity) {
    volatile int never = 0;
    return mbar_wait(bar, parity, &never);
}

__global__ void __launch_bounds__(THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, const Params p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE);
    uint64_t* full = bars;                        // STAGES
    uint64_t* empty = bars + STAGES;              // STAGES
    uint64_t* acc_full = bars + 2 * STAGES;       // 2
    uint64_t* acc_empty = bars + 2 * STAGES + 2;  // 2
    uint64_t* drain = bars + 2 * STAGES + 4;      // 1
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

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
            prefetch_tensormap(&tmA);
            prefetch_tensormap(&tmB);
            uint32_t stage = 0, phase = 0;
            int last_phase[STAGES];
            for (int i = 0; i < STAGES; ++i) last_phase[i] = -1;
            bool ok = true;
            for (int64_t it = 0; ok; ++it) {
                int tm, tn;
                if (!member_tile(p.member, p.group, blockIdx.x, gridDim.x, it, p.tiles_m, p.tiles_n,
                                 &tm, &tn))
                    break;
                for (int d = p.S + 1; d >= 2 && ok; --d) {
                    for (int s = 1; s <= d - 1 && ok; ++s) {
                        const int ya = (s - 1) * p.m_pad + tm * BM;
                        const int yb = (d - s - 1) * p.n_pad + tn * BN;
                        for (int j = 0; j < p.nslab; ++j) {
                            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag)) {
                                ok = false;
                                break;
                            }
                            uint8_t* sa = smem + stage * STAGE;
                            mbar_arrive_expect_tx(&full[stage], STAGE);
                            const int x = (p.slab0 + j) * BK;
                            tma_load_2d(sa, &tmA, &full[stage], x, ya);
                            tma_load_2d(sa + A_TILE, &tmB, &full[stage], x, yb);
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
            for (int64_t it = 0; ok; ++it) {
                int tm, tn;
                if (!member_tile(p.member, p.group, blockIdx.x, gridDim.x, it, p.tiles_m, p.tiles_n,
                                 &tm, &tn))
                    break;
                for (int d = p.S + 1; d >= 2 && ok; --d) {
                    const int units = (d - 1) * p.nslab;
                    for (int u = 0; u < units && ok;) {
                        const int cnt = min(p.chunk_slabs, units - u);
                        if (!mbar_wait(&acc_empty[abuf], aphase[abuf] ^ 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = tmem_base + abuf * BN;
                        for (int c = 0; c < cnt; ++c) {
                            if (!mbar_wait(&full[stage], phase, abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t sa = smem_u32(smem + stage * STAGE);
                            const uint64_t da = smem_desc_k_sw128(sa);
                            const uint64_t db = smem_desc_k_sw128(sa + A_TILE);
#pragma unroll
                            for (int kk = 0; kk < BK / 16; ++kk)
                                umma_f16_ss(dt, da + 2ull * kk, db + 2ull * kk, IDESC,
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
    } else if (warp >= EPI_WARP0) {
        // ------------------------------------------------------------ drain + recombination
        const int quad = warp & 3;                 // TMEM lanes this warp may read: 32*quad ..
        const int half = (warp - EPI_WARP0) >> 2;  // columns [128*half, 128*half + 128)
        const int rloc = quad * 32 + lane;  // row within the tile
        uint32_t abuf = 0;
        uint32_t aphase[2] = {0u, 0u};
        const double rb = pow2_normal(-p.beta);
        const double qnan = __longlong_as_double(0x7ff8000000000000ll);
        double* R = p.scratch + (static_cast<size_t>(blockIdx.x) * BN + half * 128) * BM + rloc;
        bool ok = true;
        for (int64_t it = 0; ok; ++it) {
            int tm, tn;
            if (!member_tile(p.member, p.group, blockIdx.x, gridDim.x, it, p.tiles_m, p.tiles_n, &tm,
                             &tn))
                break;
            const int row = tm * BM + rloc;
            const bool row_ok = row < p.m;
            int ei = 0;
            bool eflag = false;
            if (row_ok) {
                ei = p.e[row];
                eflag = p.ef[row] != 0;
            }
            for (int d = p.S + 1; d >= 2 && ok; --d) {
                int32_t acc[128];
#pragma unroll
                for (int c = 0; c < 128; ++c) acc[c] = 0;
                const int units = (d - 1) * p.nslab;
                for (int u = 0; u < units;) {
                    const int cnt = min(p.chunk_slabs, units - u);
                    if (!mbar_wait(&acc_full[abuf], aphase[abuf], abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t taddr =
                        tmem_base + (static_cast<uint32_t>(quad * 32) << 16) + abuf * BN + half * 128;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        uint32_t r[16];
                        tmem_ld_32x32b_x16(taddr + q * 16, r);
                        tmem_ld_wait(r);
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[q * 16 + j] += __float2int_rn(__uint_as_float(r[j]));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acc_empty[abuf]);
                    aphase[abuf] ^= 1u;
                    abuf ^= 1u;
                    u += cnt;
                }
                if (!ok) break;
                if (d != 2) {
                    // Horner step, least significant diagonal first (kept in FP64 scratch)
                    if (d == p.S + 1) {
#pragma unroll
                        for (int c = 0; c < 128; ++c) {
                            R[c * BM] = static_cast<double>(acc[c]);
                            if ((c & 15) == 15) asm volatile("" ::: "memory");  // bound live registers
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 128; ++c) {
                            R[c * BM] = fma(R[c * BM], rb, static_cast<double>(acc[c]));
                            if ((c & 15) == 15) asm volatile("" ::: "memory");
                        }
                    }
                } else {
                    const int col0 = tn * BN + half * 128;
#pragma unroll
                    for (int c = 0; c < 128; ++c) {
                        const double r2 = (d == p.S + 1) ? static_cast<double>(acc[c])
                                                         : fma(R[c * BM], rb, static_cast<double>(acc[c]));
                        const int col = col0 + c;
                        if (row_ok && col < p.n) {
                            double x;
                            if (eflag || p.ff[col]) {
                                x = qnan;
                            } else {
                                const int E = ei + p.f[col] - 2 * p.beta;
                                x = scale_pow2(r2, E);
                            }
                            double* cp = p.C + row + static_cast<int64_t>(col) * p.ldc;
                            *cp = (p.beta_c == 0.0) ? p.alpha * x : fma(p.beta_c, *cp, p.alpha * x);
                        }
                        if ((c & 15) == 15) asm volatile("" ::: "memory");
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

// 2-D fp16 digit tensor [rows_total][k_pad] (k contiguous), box 64 x box_rows, 128-B swizzle.
static bool make_map(CUtensorMap* map, const void* base, int64_t k_pad, int64_t rows_total,
                     int box_rows) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(k_pad), static_cast<cuuint64_t>(rows_total)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(k_pad) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace emu

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

size_t emu_scratch_bytes(int num_sms) {
    return static_cast<size_t>(num_sms) * emu::BN * emu::BM * sizeof(double);
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

cudaError_t launch_emu_slice_gemm(const EmuGemmArgs& a, int* passes, cudaStream_t stream) {
    using namespace emu;
    if (passes) *passes = 0;
    if (a.m <= 0 || a.n <= 0) return cudaSuccess;
    if (a.S < 1 || a.S > 16 || a.beta < 1 || a.beta > 10) return cudaErrorInvalidValue;
    if (a.m_pad % BM || a.n_pad % BN || a.k_pad % BK || a.m_pad < a.m || a.n_pad < a.n ||
        a.k_pad < a.k)
        return cudaErrorInvalidValue;
    if (emu_chunk_slabs(a.beta) * BK * ((1ll << a.beta) - 1) * ((1ll << a.beta) - 1) > (1ll << 24))
        return cudaErrorInvalidValue;  // beta too wide for one 64-wide slab per chunk
    if (static_cast<int64_t>(a.S) * (a.m_pad > a.n_pad ? a.m_pad : a.n_pad) >= (1ll << 31))
        return cudaErrorInvalidValue;
    const int sms = device_sm_count();
    const int64_t tiles_m = a.m_pad / BM, tiles_n = a.n_pad / BN;
    const int64_t tiles = tiles_m * tiles_n;
    int64_t ctas = a.max_ctas > 0 ? a.max_ctas : sms;
    if (ctas > tiles) ctas = tiles;
    if (a.scratch_bytes < static_cast<size_t>(ctas) * BN * BM * sizeof(double))
        return cudaErrorInvalidValue;

    CUtensorMap mapA, mapB;
    if (!make_map(&mapA, a.Ad, a.k_pad, a.S * a.m_pad, BM)) return cudaErrorInvalidValue;
    if (!make_map(&mapB, a.Bd, a.k_pad, a.S * a.n_pad, BN)) return cudaErrorInvalidValue;

    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(slice_gemm_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(SMEM_BYTES));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }

    const int64_t kslabs = (a.k + BK - 1) / BK;
    const int64_t pass_slabs = emu_max_k_per_pass(a.S, a.beta) / BK;
    int npass = 0;
    if (kslabs <= 0 || pass_slabs <= 0) return cudaErrorInvalidValue;
    for (int64_t s0 = 0; s0 < kslabs; s0 += pass_slabs) {
        Params p;
        p.m = static_cast<int>(a.m);
        p.n = static_cast<int>(a.n);
        p.S = a.S;
        p.beta = a.beta;
        p.chunk_slabs = emu_chunk_slabs(a.beta);
        p.slab0 = static_cast<int>(s0);
        p.nslab = static_cast<int>(kslabs - s0 < pass_slabs ? kslabs - s0 : pass_slabs);
        p.tiles_m = static_cast<int>(tiles_m);
        p.tiles_n = static_cast<int>(tiles_n);
        p.member = a.member == kMemberAuto ? kMemberC2 : a.member;
        p.group = a.group > 0 ? a.group : 8;
        p.m_pad = static_cast<int>(a.m_pad);
        p.n_pad = static_cast<int>(a.n_pad);
        p.e = a.e;
        p.ef = a.ef;
        p.f = a.f;
        p.ff = a.ff;
        p.alpha = a.alpha;
        p.beta_c = npass == 0 ? a.beta_c : 1.0;
        p.C = a.C;
        p.ldc = a.ldc;
        p.scratch = static_cast<double*>(a.scratch);
        p.status = a.status;
        slice_gemm_kernel<<<static_cast<unsigned>(ctas), THREADS, SMEM_BYTES, stream>>>(mapA, mapB, p);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ++npass;
    }
    if (passes) *passes = npass;
    return cudaSuccess;
}

}  // namespace momms
