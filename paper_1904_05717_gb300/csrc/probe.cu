// probe.cu -- peak-rate microbenchmarks used as roofline denominators:
// kind 0 = FP64 DMMA (mma.sync m16n8k4), kind 1 = FP64 DFMA.  Each thread runs
// independent dependency chains long enough to fill the pipe; the rate is the
// counted flops over the CUDA-event time of the launch.
#include "internal.h"

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

}  // namespace probe

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
    if (kind == 2) return cudaErrorNotSupported;
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
