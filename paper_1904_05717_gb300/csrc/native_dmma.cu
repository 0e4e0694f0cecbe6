// native_dmma.cu -- native FP64 product on the DMMA tensor instructions.
//
// C := alpha * op(A) * op(B) + beta * C.  A CTA owns a 64 x 64 block of C held
// in registers for the whole k loop (the Resident C block of registers, L0 in
// the paper's Sec. 3.4: on a GPU the MMA latency x throughput product fixes a
// minimum accumulator block exactly as the paper argues for CPUs).  k is
// streamed in 16-wide panels of op(A) and op(B) through a double-buffered
// shared-memory ring (the guest panels of the SMEM level, Sec. 3.3), loaded
// with coalesced 8-byte reads for any leading dimension and either operand
// orientation, so the transposed paths of the backward pass need no copy.
//
// The FP64 tensor pipe of this GPU is narrow (about 1 TFLOP/s for the whole
// chip), so the kernel is compute-bound by a wide margin; the member only
// decides the order in which CTAs take tiles (raster.cuh), and with it the L2
// reuse of the A and B panels.
//
// Warp tiling: 4 warps in a 2 x 2 grid, warp tile 32 x 32 = 2 x 4 fragments of
// mma.sync.m16n8k4.f64 (row.col).  Fragment ownership (g = lane / 4, t = lane % 4):
//   A 16x4: a0 = (g, t), a1 = (g + 8, t);   B 4x8: b0 = (t, g);
//   C 16x8: c0 = (g, 2t), c1 = (g, 2t+1), c2 = (g+8, 2t), c3 = (g+8, 2t+1).
#include "internal.h"
#include "raster.cuh"

namespace momms {
namespace native {

constexpr int BM = kNativeBM, BN = kNativeBN, BK = 16;
constexpr int THREADS = 128;
constexpr int PAD = 8;  // row pad (doubles) of the shared tiles: 2-way bank spread
constexpr int LDS_A = BM + PAD, LDS_B = BN + PAD;

__device__ __forceinline__ void dmma_16x8x4(double (&c)[4], double a0, double a1, double b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k4.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
        "{%0,%1,%2,%3};"
        : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
        : "d"(a0), "d"(a1), "d"(b0));
}

struct Smem {
    double a[2][BK][LDS_A];  // [buf][p][i]  = op(A)(i, p)
    double b[2][BK][LDS_B];  // [buf][p][j]  = op(B)(p, j)
};

// Each thread moves 8 elements of the A panel and 8 of the B panel per k step.
template <bool TA, bool TB>
__device__ __forceinline__ void load_panels(const double* __restrict__ A, int64_t lda,
                                            const double* __restrict__ B, int64_t ldb, int m,
                                            int n, int k, int i0, int j0, int p0, double (&ra)[8],
                                            double (&rb)[8]) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int i, p;
        if (!TA) {  // A[i + p*lda]: i fastest
            i = tid & 63;
            p = (tid >> 6) + 2 * r;
        } else {  // A[p + i*lda]: p fastest
            p = tid & 15;
            i = (tid >> 4) + 8 * r;
        }
        const int gi = i0 + i, gp = p0 + p;
        double v = 0.0;
        if (gi < m && gp < k) v = TA ? A[gp + static_cast<int64_t>(gi) * lda] : A[gi + static_cast<int64_t>(gp) * lda];
        ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int j, p;
        if (!TB) {  // B[p + j*ldb]: p fastest
            p = tid & 15;
            j = (tid >> 4) + 8 * r;
        } else {  // B[j + p*ldb]: j fastest
            j = tid & 63;
            p = (tid >> 6) + 2 * r;
        }
        const int gj = j0 + j, gp = p0 + p;
        double v = 0.0;
        if (gj < n && gp < k) v = TB ? B[gj + static_cast<int64_t>(gp) * ldb] : B[gp + static_cast<int64_t>(gj) * ldb];
        rb[r] = v;
    }
}

template <bool TA, bool TB>
__device__ __forceinline__ void store_panels(Smem& sm, int buf, const double (&ra)[8], const double (&rb)[8]) {
    const int tid = threadIdx.x;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int i, p;
        if (!TA) { i = tid & 63; p = (tid >> 6) + 2 * r; }
        else { p = tid & 15; i = (tid >> 4) + 8 * r; }
        sm.a[buf][p][i] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        int j, p;
        if (!TB) { p = tid & 15; j = (tid >> 4) + 8 * r; }
        else { j = tid & 63; p = (tid >> 6) + 2 * r; }
        sm.b[buf][p][j] = rb[r];
    }
}

// One 64 x 64 tile of C.
template <bool TA, bool TB>
__device__ void gemm_tile(Smem& sm, int m, int n, int k, double alpha, const double* __restrict__ A,
                          int64_t lda, const double* __restrict__ B, int64_t ldb, double beta,
                          double* __restrict__ C, int64_t ldc, int tm, int tn, int tri = 0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
    const int i0 = tm * BM, j0 = tn * BN;

    double acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0;

    double ra[8], rb[8];
    const int ksteps = (k + BK - 1) / BK;
    if (ksteps > 0) {
        load_panels<TA, TB>(A, lda, B, ldb, m, n, k, i0, j0, 0, ra, rb);
        store_panels<TA, TB>(sm, 0, ra, rb);
    }
    __syncthreads();
    for (int ks = 0; ks < ksteps; ++ks) {
        const int buf = ks & 1;
        const bool more = ks + 1 < ksteps;
        if (more) load_panels<TA, TB>(A, lda, B, ldb, m, n, k, i0, j0, (ks + 1) * BK, ra, rb);
#pragma unroll
        for (int kk = 0; kk < BK; kk += 4) {
            double af[2][2], bf[4];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                af[mi][0] = sm.a[buf][kk + t][wm + mi * 16 + g];
                af[mi][1] = sm.a[buf][kk + t][wm + mi * 16 + g + 8];
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) bf[ni] = sm.b[buf][kk + t][wn + ni * 8 + g];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) dmma_16x8x4(acc[mi][ni], af[mi][0], af[mi][1], bf[ni]);
        }
        if (more) store_panels<TA, TB>(sm, buf ^ 1, ra, rb);
        __syncthreads();
    }

    // epilogue: C = alpha * acc + beta * C (beta == 0: C is not read)
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int i = i0 + wm + mi * 16 + g + ((c & 2) ? 8 : 0);
                const int j = j0 + wn + ni * 8 + 2 * t + (c & 1);
                if (i < m && j < n && (tri == 0 || (tri == 1 ? j <= i : j >= i))) {
                    double* cp = C + i + static_cast<int64_t>(j) * ldc;
                    const double v = alpha * acc[mi][ni][c];
                    *cp = (beta == 0.0) ? v : fma(beta, *cp, v);
                }
            }
        }
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(THREADS)
    gemm_kernel(int m, int n, int k, double alpha, const double* __restrict__ A, int64_t lda,
                const double* __restrict__ B, int64_t ldb, double beta, double* __restrict__ C,
                int64_t ldc, int member, int group, int tiles_m, int tiles_n, int tri) {
    __shared__ Smem sm;
    int tm, tn;
    // one tile per CTA by default; a capped grid loops over the CTA's share in member order
    bool synced = true;
    for (int64_t i = 0; member_tile(member, group, blockIdx.x, gridDim.x, i, tiles_m, tiles_n, &tm, &tn); ++i) {
        // a triangle-only product skips the tiles that lie wholly outside its triangle
        if (tri == 1 && tn * BN > tm * BM + BM - 1) continue;
        if (tri == 2 && tn * BN + BN - 1 < tm * BM) continue;
        if (!synced) __syncthreads();  // the shared panels are reused by the next tile
        gemm_tile<TA, TB>(sm, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tm, tn, tri);
        synced = false;
    }
}

// Persistent launch over the tiles of many problems (op = N, N).
__global__ void __launch_bounds__(THREADS)
    batched_kernel(const BatchProblem* __restrict__ probs, int count, int64_t total_tiles) {
    __shared__ Smem sm;
    for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
        // binary search: last problem with tile0 <= t
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (probs[mid].tile0 <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchProblem& pr = probs[lo];
        const int64_t local = t - pr.tile0;
        const int tm = static_cast<int>(local / pr.tiles_n);
        const int tn = static_cast<int>(local % pr.tiles_n);
        gemm_tile<false, false>(sm, pr.m, pr.n, pr.k, pr.alpha, pr.A, pr.lda, pr.B, pr.ldb, pr.beta,
                                pr.C, pr.ldc, tm, tn);
        __syncthreads();  // the shared panels are reused by the next tile
    }
}

}  // namespace native

cudaError_t launch_native_gemm(int op_a, int op_b, int64_t m, int64_t n, int64_t k, double alpha,
                               const double* A, int64_t lda, const double* B, int64_t ldb,
                               double beta, double* C, int64_t ldc, int member, int max_ctas,
                               int group_req, cudaStream_t stream, int* used_ctas, int* used_group, int tri) {
    using namespace native;
    if (m <= 0 || n <= 0) return cudaSuccess;
    if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > INT32_MAX / 2) return cudaErrorInvalidValue;
    const int tiles_m = static_cast<int>((m + BM - 1) / BM);
    const int tiles_n = static_cast<int>((n + BN - 1) / BN);
    const int64_t tiles = static_cast<int64_t>(tiles_m) * tiles_n;
    if (tiles > INT32_MAX) return cudaErrorInvalidValue;
    const int mem = member == kMemberAuto ? kMemberC2 : member;
    const int group = group_req > 0 ? group_req : 16;
    const dim3 grid(static_cast<unsigned>(max_ctas > 0 && max_ctas < tiles ? max_ctas : tiles));
    if (used_ctas) *used_ctas = static_cast<int>(grid.x);
    if (used_group) *used_group = group;
    const int mi = static_cast<int>(m), ni = static_cast<int>(n), ki = static_cast<int>(k);
    if (!op_a && !op_b)
        gemm_kernel<false, false><<<grid, THREADS, 0, stream>>>(mi, ni, ki, alpha, A, lda, B, ldb, beta, C, ldc, mem, group, tiles_m, tiles_n, tri);
    else if (op_a && !op_b)
        gemm_kernel<true, false><<<grid, THREADS, 0, stream>>>(mi, ni, ki, alpha, A, lda, B, ldb, beta, C, ldc, mem, group, tiles_m, tiles_n, tri);
    else if (!op_a && op_b)
        gemm_kernel<false, true><<<grid, THREADS, 0, stream>>>(mi, ni, ki, alpha, A, lda, B, ldb, beta, C, ldc, mem, group, tiles_m, tiles_n, tri);
    else
        gemm_kernel<true, true><<<grid, THREADS, 0, stream>>>(mi, ni, ki, alpha, A, lda, B, ldb, beta, C, ldc, mem, group, tiles_m, tiles_n, tri);
    return cudaGetLastError();
}

cudaError_t launch_native_batched(const BatchProblem* dev_problems, int count, int64_t total_tiles,
                                  cudaStream_t stream) {
    using namespace native;
    if (count <= 0 || total_tiles <= 0) return cudaSuccess;
    int64_t grid = static_cast<int64_t>(device_sm_count()) * 8;  // 8 resident CTAs per SM
    if (grid > total_tiles) grid = total_tiles;
    batched_kernel<<<static_cast<unsigned>(grid), THREADS, 0, stream>>>(dev_problems, count, total_tiles);
    return cudaGetLastError();
}

}  // namespace momms
