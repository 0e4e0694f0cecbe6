// trsm.cu -- inverses of the diagonal blocks of a triangular matrix, the leaf step of the
// blocked triangular solve (momms_trsm in api.cu).
//
// The solve op(A) X = alpha B (or X op(A) = alpha B) is done recursively: the off-diagonal
// blocks become GEMM updates of the right-hand sides (the product of this library), and each
// kTrsmLeaf x kTrsmLeaf diagonal block is applied as a GEMM with its explicit inverse.  The
// inverses of the nb x nb blocks inside a leaf are computed here in FP64, one CTA per block, by
// forward substitution on the block's columns (api.cu then joins them into the leaf's inverse
// with batched GEMMs, [L11 0; L21 L22]^-1 = [I11 0; -I22 L21 I11 I22]):
// for a lower triangle L, column t of L^-1 is x with x_t = 1 / L_tt and
//     x_i = -(sum_{k=t}^{i-1} L_ik x_k) / L_ii,   i > t.
// An upper triangle U is handled as L = U^T (inv(U) = inv(U^T)^T).
#include "internal.h"

namespace momms {

namespace {

// Packed lower triangle by rows: element (i, k), k <= i, at i (i + 1) / 2 + k.
__device__ __forceinline__ int tri_row(int i, int k) { return i * (i + 1) / 2 + k; }

// One CTA (kTrsmNb threads) per diagonal block g of the t x t triangle.  The block's inverse goes
// to the diagonal sub-block g % (kTrsmLeaf / nb) of leaf block g / (kTrsmLeaf / nb) of W (dense
// kTrsmLeaf x kTrsmLeaf column-major blocks), zero outside the triangle and outside the block's
// size for the last, partial block.
__global__ void __launch_bounds__(kTrsmNb) tri_inverse_kernel(int64_t t, const double* __restrict__ A, int64_t lda,
                                                              int uplo, int unit, double* __restrict__ W) {
    extern __shared__ double sm[];
    constexpr int nb = kTrsmNb;
    constexpr int packed = nb * (nb + 1) / 2;
    double* L = sm;            // the block as a lower triangle, packed by rows
    double* X = sm + packed;   // its inverse, packed by rows as well
    const int64_t b0 = static_cast<int64_t>(blockIdx.x) * nb;
    const int sz = static_cast<int>(t - b0 < nb ? t - b0 : nb);
    const double* Ab = A + b0 + b0 * lda;
    // L(i, k), k <= i: the stored lower triangle, or the transpose of the stored upper one; the
    // global reads run down the stored columns (coalesced)
    if (uplo == kTrsmLower) {
        for (int k = 0; k < nb; ++k)
            for (int i = k + threadIdx.x; i < nb; i += blockDim.x)
                L[tri_row(i, k)] = (i < sz && k < sz) ? ((i == k && unit) ? 1.0 : Ab[i + static_cast<int64_t>(k) * lda])
                                                      : 0.0;
    } else {
        for (int i = 0; i < nb; ++i)
            for (int k = threadIdx.x; k <= i; k += blockDim.x)
                L[tri_row(i, k)] = (i < sz && k < sz) ? ((i == k && unit) ? 1.0 : Ab[k + static_cast<int64_t>(i) * lda])
                                                      : 0.0;
    }
    __syncthreads();
    const int tc = threadIdx.x;  // column of the inverse this thread computes
    if (tc < sz) {
        X[tri_row(tc, tc)] = 1.0 / L[tri_row(tc, tc)];
        for (int i = tc + 1; i < sz; ++i) {
            double acc = 0.0;
            const double* Li = L + tri_row(i, 0);
            for (int k = tc; k < i; ++k) acc = fma(Li[k], X[tri_row(k, tc)], acc);
            X[tri_row(i, tc)] = -acc / Li[i];
        }
    }
    __syncthreads();
    constexpr int per_leaf = kTrsmLeaf / nb;
    constexpr int64_t ldw = kTrsmLeaf;
    double* Wb = W + static_cast<int64_t>(blockIdx.x / per_leaf) * ldw * ldw +
                 static_cast<int64_t>(blockIdx.x % per_leaf) * nb * (ldw + 1);
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int r = idx % nb, c = idx / nb;  // element (r, c) of the stored-orientation inverse
        double v = 0.0;
        if (r < sz && c < sz) {
            if (uplo == kTrsmLower) v = r >= c ? X[tri_row(r, c)] : 0.0;
            else v = r <= c ? X[tri_row(c, r)] : 0.0;  // inv(U) = inv(U^T)^T
        }
        Wb[r + c * ldw] = v;
    }
}

}  // namespace

size_t tri_inverse_bytes(int64_t t) {
    const int64_t leaves = (t + kTrsmLeaf - 1) / kTrsmLeaf;
    return static_cast<size_t>(leaves) * kTrsmLeaf * kTrsmLeaf * sizeof(double);
}

cudaError_t launch_tri_inverse(int64_t t, const double* A, int64_t lda, int uplo, int unit, double* W,
                               cudaStream_t stream) {
    if (t <= 0) return cudaSuccess;
    const int64_t blocks = (t + kTrsmNb - 1) / kTrsmNb;
    if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
    constexpr size_t smem = 2 * sizeof(double) * kTrsmNb * (kTrsmNb + 1) / 2;
    static PerDeviceFlag attr_set;  // idempotent; per device, atomic for concurrent first calls
    if (!attr_set.done()) {
        const cudaError_t e =
            cudaFuncSetAttribute(tri_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess) return e;
        attr_set.mark();
    }
    tri_inverse_kernel<<<static_cast<unsigned>(blocks), kTrsmNb, smem, stream>>>(t, A, lda, uplo, unit, W);
    return cudaGetLastError();
}

}  // namespace momms
