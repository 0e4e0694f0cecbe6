// noalloc.cu -- the emulated FP64 product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA graph that
// is being captured, allocator-less embedded runtimes, or libraries that must not
// touch the device heap (for example a caller that owns every byte through its own
// pool and forbids other allocations).  momms_gemm_emulated_noalloc serves them: it
// runs the same scale, split and slice-product kernels as the emulated path of
// momms_gemm_ex, but takes all of its scratch (exponents, flags, digit slices, the
// FP64 recombination blocks and the status word) from one file-scope device array of
// kNoAllocBytes (64 MiB).  Every GPU that loads the library holds that array until
// the process exits.
//
// Rules of use:
//   * The first call on a device looks up the device address of the array (with that
//     device current) and caches it; make that first call before any stream capture.
//   * All calls share the array and it keeps the last call's contents: calls that
//     overlap on the GPU (different streams, or different host threads on one
//     device) race on it and give wrong results.  Serialise them on one stream.
//   * Problems whose scratch does not fit are rejected with MOMMS_ERR_WORKSPACE
//     before anything is enqueued; the slice count must be given (1..16) because the
//     data-driven choice needs a host readback.
//   * A call only enqueues work.  Whether its bounded device waits all finished in time is
//     recorded in a status word inside the array; momms_noalloc_status() waits for the
//     stream, returns that word and clears it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "../../include/momms.h"
#include "internal.h"

namespace {

constexpr size_t kNoAllocBytes = size_t(64) << 20;
constexpr int kNoAllocMaxCtas = 64;  // FP64 recombination blocks kept in the array
constexpr size_t kStatusOffset = 0;  // the device status word: zero-initialised at load, 0 = no timeout

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_dev_ptr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Largest m, n or k the carve-up below accepts: the int32 tile and slab arithmetic of the kernels,
// and every region's byte count stays far inside 64-bit arithmetic.
constexpr int64_t kNoAllocMaxDim = int64_t(1) << 30;

// a * b * c * d bytes, or SIZE_MAX when the product exceeds the array (no 64-bit wrap-around).
size_t region_bytes(uint64_t a, uint64_t b, uint64_t c, uint64_t d = 1) {
    const unsigned __int128 v = static_cast<unsigned __int128>(a) * b * c * d;
    return v > kNoAllocBytes ? SIZE_MAX : static_cast<size_t>(v);
}

// Device address of the array on the current device (looked up once per device).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MOMMS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MOMMS_ERR_CUDA;
        }
        g_dev_ptr[dev] = p;
    }
    *out = g_dev_ptr[dev];
    return MOMMS_OK;
}

}  // namespace

extern "C" size_t momms_noalloc_scratch_bytes(void) { return kNoAllocBytes; }

extern "C" int momms_gemm_emulated_noalloc(int op_a, int op_b, int64_t m, int64_t n, int64_t k,
                                           int slices, double alpha, const double* A, int64_t lda,
                                           const double* B, int64_t ldb, double beta, double* C,
                                           int64_t ldc, momms_stream_t stream) {
    if (op_a != MOMMS_OP_N && op_a != MOMMS_OP_T) return -1;
    if (op_b != MOMMS_OP_N && op_b != MOMMS_OP_T) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 0) return -5;
    if (slices < 1 || slices > MOMMS_MAX_SLICES) return -6;
    const int64_t rows_a = op_a == MOMMS_OP_N ? m : k;
    const int64_t rows_b = op_b == MOMMS_OP_N ? k : n;
    const bool work = m > 0 && n > 0 && k > 0 && alpha != 0.0;
    if (work && !A) return -8;
    if (lda < std::max<int64_t>(1, rows_a)) return -9;
    if (work && !B) return -10;
    if (ldb < std::max<int64_t>(1, rows_b)) return -11;
    if (m > 0 && n > 0 && !C) return -13;
    if (ldc < std::max<int64_t>(1, m)) return -14;
    if (m == 0 || n == 0) return MOMMS_OK;
    if (!work) return MOMMS_ERR_UNSUPPORTED;  // C := beta*C needs no product: use momms_gemm_ex
    if (m > kNoAllocMaxDim || n > kNoAllocMaxDim || k > kNoAllocMaxDim) return MOMMS_ERR_WORKSPACE;

    constexpr int beta_bits = 7;
    const int64_t k_pad = (k + momms::kEmuBK - 1) / momms::kEmuBK * momms::kEmuBK;
    const int64_t tiles = ((m + momms::kEmuBM - 1) / momms::kEmuBM) *
                          ((n + momms::kEmuBNMax - 1) / momms::kEmuBNMax);
    const int ctas = static_cast<int>(std::min<int64_t>(
        {static_cast<int64_t>(momms::device_sm_count()), tiles, static_cast<int64_t>(kNoAllocMaxCtas)}));
    // carve the array: status word, exponents, flags, digit slices, recombination blocks (each
    // region's size checked against the array before it is added: no sum can wrap)
    const size_t digits_a = region_bytes(2, static_cast<uint64_t>(slices), static_cast<uint64_t>(m),
                                         static_cast<uint64_t>(k_pad));
    const size_t digits_b = region_bytes(2, static_cast<uint64_t>(slices), static_cast<uint64_t>(n),
                                         static_cast<uint64_t>(k_pad));
    if (digits_a == SIZE_MAX || digits_b == SIZE_MAX) return MOMMS_ERR_WORKSPACE;
    size_t o = kStatusOffset + 256;  // the status word leads the array
    const size_t off_e = o;       o += up256(sizeof(int32_t) * m);
    const size_t off_ef = o;      o += up256(static_cast<size_t>(m));
    const size_t off_f = o;       o += up256(sizeof(int32_t) * n);
    const size_t off_ff = o;      o += up256(static_cast<size_t>(n));
    if (o > kNoAllocBytes) return MOMMS_ERR_WORKSPACE;
    const size_t off_Ad = o;      o += up256(digits_a);
    if (o > kNoAllocBytes) return MOMMS_ERR_WORKSPACE;
    const size_t off_Bd = o;      o += up256(digits_b);
    if (o > kNoAllocBytes) return MOMMS_ERR_WORKSPACE;
    const size_t off_R = o;
    const size_t r_bytes = momms::emu_scratch_bytes_for_ctas(ctas);
    o += up256(r_bytes);
    if (o > kNoAllocBytes) return MOMMS_ERR_WORKSPACE;

    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    char* w = static_cast<char*>(base);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t* status = reinterpret_cast<int32_t*>(w + kStatusOffset);
    int32_t* e = reinterpret_cast<int32_t*>(w + off_e);
    uint8_t* ef = reinterpret_cast<uint8_t*>(w + off_ef);
    int32_t* f = reinterpret_cast<int32_t*>(w + off_f);
    uint8_t* ff = reinterpret_cast<uint8_t*>(w + off_ff);
    // The status word is not cleared here: a timeout of an earlier call stays visible until
    // momms_noalloc_status() reads and clears it.  Every other region is fully written before it
    // is read.
    if (momms::launch_emu_scale(0, op_a, m, k, A, lda, e, ef, nullptr, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (momms::launch_emu_scale(1, op_b, n, k, B, ldb, f, ff, nullptr, s) != cudaSuccess) return MOMMS_ERR_CUDA;
    if (momms::launch_emu_split(0, op_a, m, k, A, lda, e, ef, slices, beta_bits, w + off_Ad, m, k_pad, s) !=
        cudaSuccess)
        return MOMMS_ERR_CUDA;
    if (momms::launch_emu_split(1, op_b, n, k, B, ldb, f, ff, slices, beta_bits, w + off_Bd, n, k_pad, s) !=
        cudaSuccess)
        return MOMMS_ERR_CUDA;
    momms::EmuGemmArgs a{};
    a.m = m; a.n = n; a.k = k; a.S = slices; a.beta = beta_bits;
    a.Ad = w + off_Ad; a.Bd = w + off_Bd; a.m_pad = m; a.n_pad = n; a.k_pad = k_pad;
    a.e = e; a.ef = ef; a.f = f; a.ff = ff;
    a.alpha = alpha; a.beta_c = beta; a.C = C; a.ldc = ldc;
    a.member = 0; a.group = 0;
    a.scratch = w + off_R; a.scratch_bytes = r_bytes; a.status = status;
    a.max_ctas = ctas; a.tile_n = 0;
    int passes = 0;
    cudaError_t ce = momms::launch_emu_slice_gemm(a, &passes, s);
    if (ce == cudaErrorInvalidValue) return MOMMS_ERR_UNSUPPORTED;
    return ce == cudaSuccess ? MOMMS_OK : MOMMS_ERR_CUDA;
}

extern "C" int momms_noalloc_status(momms_stream_t stream, int* status) {
    if (!status) return -2;
    *status = MOMMS_OK;
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t* word = reinterpret_cast<int32_t*>(static_cast<char*>(base) + kStatusOffset);
    int32_t v = 0;
    // the copy waits for every call enqueued on `stream` before it; the clear follows it in order
    if (cudaMemcpyAsync(&v, word, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MOMMS_ERR_CUDA;
    if (v != 0) {
        if (cudaMemsetAsync(word, 0, sizeof(int32_t), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
            return MOMMS_ERR_CUDA;
        *status = v == MOMMS_ERR_TIMEOUT ? MOMMS_ERR_TIMEOUT : MOMMS_ERR_CUDA;
    }
    return MOMMS_OK;
}
