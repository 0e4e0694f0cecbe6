// probe.cu -- peak-rate microbenchmarks used as roofline denominators:
// kind 0 = FP64 DMMA (mma.sync m16n8k4), kind 1 = FP64 DFMA.  Each thread runs
// independent dependency chains long enough to fill the pipe; the rate is the
// counted flops over the CUDA-event time of the launch.
// kinds 2-5 = the tcgen05 kind::f16 instruction shapes of the product kernels issued back to back
// from shared-memory operands that stay in place (no loads, no drains): 2 = M 128 x N 192 on one
// CTA (the residue product's), 3 = M 128 x N 256, 4 = M 256 x N 192 on a CTA pair
// (cta_group::2, the pair kernel's), 5 = M 256 x N 256 on a CTA pair.  They bound what the
// instruction alone reaches on each SM.
#include "internal.h"
#include "ptx.cuh"

namespace momms {
namespace probe {

__global__ void dmma_kernel(double* out, int iters) {
    double a0 = 1e-3 * threadIdx.x, a1 = 2e-3 * threadIdx.x, b = 1e-3;
    double c[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) c[j][i] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            asm volatile(
                "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
                "{%0,%1,%2,%3};"
                : "+d"(c[j][0]), "+d"(c[j][1]), "+d"(c[j][2]), "+d"(c[j][3])
                : "d"(a0), "d"(a1), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) s += c[j][i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dfma_kernel(double* out, int iters) {
    double x[8];
    const double y = 1.0000001, z = 1e-9;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], y, z);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Streaming copy of 16-byte words, grid-strided, four loads in flight per thread before the
// stores; the streaming cache hints keep the copy from occupying L2.
__global__ void __launch_bounds__(1024, 1)
    copy_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, int64_t words, int repeats) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int r = 0; r < repeats; ++r) {
        int64_t i = first;
        for (; i + 3 * stride < words; i += 4 * stride) {
            const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride);
            const uint4 c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
            __stcs(dst + i, a);
            __stcs(dst + i + stride, b);
            __stcs(dst + i + 2 * stride, c);
            __stcs(dst + i + 3 * stride, d);
        }
        for (; i < words; i += stride) __stcs(dst + i, __ldcs(src + i));
    }
}

// One CTA per SM (or one pair of CTAs per two SMs): thread 0 of the (leading) CTA issues `iters` x 4
// MMAs of K = 16 from zero operands in shared memory into two alternating TMEM accumulators, commits
// them, and waits (bounded) until they are done.
constexpr int kProbeSmem = 120 * 1024;  // one CTA per SM
template <int M, int N, bool PAIR>
__global__ void __launch_bounds__(128, 1) mma_probe_kernel(int iters, int32_t* status) {
    extern __shared__ uint8_t raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~uintptr_t(1023));
    constexpr int RA = PAIR ? M / 2 : M;       // A rows this CTA holds
    constexpr int RB = PAIR ? N / 2 : N;       // B rows this CTA holds
    constexpr uint32_t A_BYTES = RA * 64 * 2, B_BYTES = RB * 64 * 2;
    uint64_t* done = reinterpret_cast<uint64_t*>(smem + A_BYTES + B_BYTES);
    uint32_t* slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(slot + 1);
    for (uint32_t i = threadIdx.x * 16; i < A_BYTES + B_BYTES; i += blockDim.x * 16)
        *reinterpret_cast<uint4*>(smem + i) = make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
    const uint32_t rank = PAIR ? cluster_ctarank() : 0;
    if (threadIdx.x == 0) {
        mbar_init(done, 1);
        *abort_flag = 0;
        fence_mbarrier_init();
    }
    if (threadIdx.x < 32) {
        if constexpr (PAIR) {
            tmem_alloc_pair(slot, 512);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(slot, 512);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    tc_fence_after();
    const uint32_t base = *slot;
    if (threadIdx.x == 0 && rank == 0) {
        const uint64_t da = smem_desc_k_sw128(smem_u32(smem));
        const uint64_t db = smem_desc_k_sw128(smem_u32(smem + A_BYTES));
        constexpr uint32_t idesc = idesc_f16_f32(M, N);
        for (int it = 0; it < iters; ++it) {
            const uint32_t d = base + (it & 1) * 256u;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                if constexpr (PAIR) umma_f16_ss_pair(d, da + 2ull * kk, db + 2ull * kk, idesc, 1u);
                else umma_f16_ss(d, da + 2ull * kk, db + 2ull * kk, idesc, 1u);
            }
        }
        if constexpr (PAIR) umma_commit_pair(smem_u32(done));
        else umma_commit(done);
        if (!mbar_wait(done, 0, abort_flag)) atomicExch(status, kStatusTimeout);
    }
    tc_fence_before();
    __syncthreads();
    if constexpr (PAIR) cluster_sync();
    if (threadIdx.x < 32) {
        tc_fence_after();
        if constexpr (PAIR) tmem_dealloc_pair(base, 512);
        else tmem_dealloc(base, 512);
    }
}

}  // namespace probe

template <int M, int N, bool PAIR>
static cudaError_t mma_probe(double* tflops, cudaStream_t stream) {
    static PerDeviceFlag attr;
    if (!attr.done()) {
        cudaError_t e = cudaFuncSetAttribute(probe::mma_probe_kernel<M, N, PAIR>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, probe::kProbeSmem);
        if (e != cudaSuccess) return e;
        attr.mark();
    }
    const int sms = device_sm_count();
    const int ctas = PAIR ? 2 * (sms / 2) : sms;
    const int iters = 20000;
    int32_t* status = nullptr;
    cudaError_t e = cudaMalloc(&status, sizeof(int32_t));
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(status, 0, sizeof(int32_t), stream);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms = 0.f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, stream);
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(static_cast<unsigned>(ctas));
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = probe::kProbeSmem;
        cfg.stream = stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = PAIR ? 2 : 1;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, probe::mma_probe_kernel<M, N, PAIR>, iters, status);
        cudaEventRecord(e1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
    int32_t st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof(st), cudaMemcpyDeviceToHost);
    const double issuers = PAIR ? sms / 2 : sms;
    const double flops = issuers * static_cast<double>(iters) * 4.0 * 2.0 * M * N * 16.0;
    *tflops = (e == cudaSuccess && st == 0 && ms > 0.f) ? flops / (ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(status);
    return e;
}

// The dynamic shared memory asked for makes the copy CTAs one per SM, so `ctas` counts SMs.
constexpr int kCopyThreads = 1024, kCopySmem = 120 * 1024;

cudaError_t stream_copy(void* dst, const void* src, size_t bytes, int ctas, int repeats,
                        cudaStream_t stream) {
    if (bytes == 0 || repeats == 0) return cudaSuccess;
    static PerDeviceFlag attr_set;  // idempotent; per device, atomic for concurrent first calls
    if (!attr_set.done()) {
        cudaError_t e = cudaFuncSetAttribute(probe::copy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kCopySmem);
        if (e != cudaSuccess) return e;
        attr_set.mark();
    }
    const int sms = device_sm_count();
    const int grid = (ctas <= 0 || ctas > sms) ? sms : ctas;
    probe::copy_kernel<<<grid, kCopyThreads, kCopySmem, stream>>>(
        static_cast<const uint4*>(src), static_cast<uint4*>(dst), static_cast<int64_t>(bytes / 16), repeats);
    return cudaGetLastError();
}

cudaError_t probe_peak(int kind, double* tflops, cudaStream_t stream) {
    if (kind == 2) return mma_probe<128, 192, false>(tflops, stream);
    if (kind == 3) return mma_probe<128, 256, false>(tflops, stream);
    if (kind == 4) return mma_probe<256, 192, true>(tflops, stream);
    if (kind == 5) return mma_probe<256, 256, true>(tflops, stream);
    const int sms = device_sm_count();
    const int threads = 256, blocks = sms * 4;
    double* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(double) * threads * blocks);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int iters = kind == 0 ? 1000 : 4000;
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {
        cudaEventRecord(e0, stream);
        if (kind == 0) probe::dmma_kernel<<<blocks, threads, 0, stream>>>(out, iters);
        else probe::dfma_kernel<<<blocks, threads, 0, stream>>>(out, iters);
        cudaEventRecord(e1, stream);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) break;
        cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    const double flops = kind == 0 ? 1024.0 * 4 * iters * blocks * (threads / 32)
                                   : 2.0 * 8 * iters * static_cast<double>(blocks) * threads;
    *tflops = (e == cudaSuccess && ms > 0.f) ? flops / (ms * 1e-3) / 1e12 : 0.0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return e;
}

}  // namespace momms
