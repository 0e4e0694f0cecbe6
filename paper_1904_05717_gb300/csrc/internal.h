// internal.h -- launchers shared between the C-ABI layer and the kernel files.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace momms {

// ---------------------------------------------------------------- native FP64
// C := alpha*op(A)*op(B) + beta*C on the FP64 DMMA tensor instructions.
cudaError_t launch_native_gemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               double beta, double* C, int64_t ldc, int member,
                               cudaStream_t stream);
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
// atomicMax into *out of ceil(16 * max_r log2(2^e_r * inner / l1_r)).
cudaError_t launch_emu_spread(int64_t rows, int64_t inner, const int32_t* exps, const uint8_t* flags,
                              const float* l1, int* out, cudaStream_t stream);
// Truncation digits (fp16, integer valued), layout [S][rows_pad][inner_pad].
cudaError_t launch_emu_split(int which, int op, int64_t rows, int64_t inner, const double* X,
                             int64_t ldx, const int32_t* exps, const uint8_t* flags, int S,
                             int beta, void* digits, int64_t rows_pad, int64_t inner_pad,
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
    int tile_n;    // CTA tile width request (only 192 is built; 0 = automatic)
};
constexpr int kEmuBM = 128, kEmuBK = 64, kEmuBNMax = 192;
// The CTA tile width used for n columns (tile_n request 0 = automatic).
int emu_pick_bn(int64_t n, int requested);
// Launches the slice-product kernel once per k pass; *passes receives the count.
cudaError_t launch_emu_slice_gemm(const EmuGemmArgs& a, int* passes, cudaStream_t stream);
size_t emu_scratch_bytes(int num_sms);
size_t emu_scratch_bytes_for_ctas(int ctas);
// Bit d set: diagonal d is the most significant of an exact int64 group (S, beta, k per pass).
uint32_t emu_group_ends(int S, int beta, int64_t k_pass);
// Largest k one pass may cover so that every diagonal sum stays below 2^31.
int64_t emu_max_k_per_pass(int S, int beta);
// Products per FP32 accumulation chunk (every partial sum below 2^24), in 64-wide slabs.
int emu_chunk_slabs(int beta);

int device_sm_count();

// ------------------------------------------------------------------ probes
cudaError_t probe_peak(int kind, double* tflops, cudaStream_t stream);

}  // namespace momms
