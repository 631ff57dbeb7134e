// Dense operations on sets of vectors, for the subspace iteration that finds
// the lowest eigenpairs of the LB operator (Sec. 4.3): Gram matrices G = X^T Y
// and block combinations Y = X C.  FP64 throughout.
//
// A set of p vectors of length n is stored in blocks of w interleaved columns,
// so each block is a right-hand-side array [n][w] of the solver:
//   element (r, c) at (c / w) * n * w + r * w + (c % w),  p a multiple of w.
//
// The Gram matrix is reduced in a fixed order (kGramBlocks row ranges, each
// summed by one block in row order, then the ranges in order), so its value
// depends on neither the GPU nor the launch.
#include "common.cuh"

namespace mvgd {
namespace {

constexpr int kGramBlocks = 256;  // row ranges of the first reduction stage
constexpr int kGramRows = 16;     // rows staged in shared memory at a time
constexpr int kMaxCols = 128;     // p, q <= kMaxCols

__device__ __forceinline__ int64_t at(int64_t r, int c, int64_t n, int w) {
    return (int64_t)(c / w) * n * w + r * w + (c % w);
}

// partial[b][i][j] = sum over the rows of range b of X(r, i) Y(r, j)
__global__ void __launch_bounds__(256) k_gram_partial(const double* __restrict__ X, int p, const double* __restrict__ Y,
                                                      int q, int64_t n, int w, double* __restrict__ partial) {
    __shared__ double xs[kGramRows][kMaxCols];
    __shared__ double ys[kGramRows][kMaxCols];
    const int64_t per = (n + kGramBlocks - 1) / kGramBlocks;
    const int64_t r0 = blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
    const int outs = p * q;
    double acc[(kMaxCols * kMaxCols + 255) / 256];
#pragma unroll
    for (int t = 0; t < (kMaxCols * kMaxCols + 255) / 256; t++) acc[t] = 0.0;
    for (int64_t base = r0; base < r1; base += kGramRows) {
        const int rows = (int)(r1 - base < kGramRows ? r1 - base : kGramRows);
        __syncthreads();
        for (int e = threadIdx.x; e < rows * p; e += blockDim.x) xs[e / p][e % p] = X[at(base + e / p, e % p, n, w)];
        for (int e = threadIdx.x; e < rows * q; e += blockDim.x) ys[e / q][e % q] = Y[at(base + e / q, e % q, n, w)];
        __syncthreads();
#pragma unroll
        for (int t = 0; t < (kMaxCols * kMaxCols + 255) / 256; t++) {
            const int o = threadIdx.x + t * 256;
            if (o < outs) {
                const int i = o / q, j = o % q;
                double a = acc[t];
                for (int rr = 0; rr < rows; rr++) a = fma(xs[rr][i], ys[rr][j], a);
                acc[t] = a;
            }
        }
    }
#pragma unroll
    for (int t = 0; t < (kMaxCols * kMaxCols + 255) / 256; t++) {
        const int o = threadIdx.x + t * 256;
        if (o < outs) partial[(int64_t)blockIdx.x * outs + o] = acc[t];
    }
}

// G[o] = sum over the ranges b (in order) of partial[b][o]
__global__ void k_gram_final(const double* __restrict__ partial, int outs, double* __restrict__ G) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < outs; o += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < kGramBlocks; b++) s += partial[(int64_t)b * outs + o];
        G[o] = s;
    }
}

// Y(r, j) = sum_i X(r, i) C[i][j]   (C row-major p x q, at most 128 KB: read
// through the read-only cache, where the threads of a block share it)
__global__ void __launch_bounds__(256) k_block_combine(const double* __restrict__ X, int p,
                                                       const double* __restrict__ Cm, int q, int64_t n, int w,
                                                       double* __restrict__ Y) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * q; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / q;
        const int j = (int)(e % q);
        double s = 0.0;
        for (int i = 0; i < p; i++) s = fma(X[at(r, i, n, w)], __ldg(Cm + i * q + j), s);
        Y[at(r, j, n, w)] = s;
    }
}

// X(r, c) = 0 for every column c of the rows r flagged in mask
__global__ void k_block_zero_rows(double* __restrict__ X, int p, int64_t n, int w, const uint8_t* __restrict__ mask) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * p; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / p;
        if (mask[r]) X[at(r, (int)(e % p), n, w)] = 0.0;
    }
}

bool bad_shape(int64_t n, int p, int q, int w) {
    return n < 1 || w < 1 || w > 8 || p < 1 || q < 1 || p > kMaxCols || q > kMaxCols || p % w != 0 || q % w != 0;
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_block_gram_workspace_bytes(int32_t p, int32_t q) {
    if (p < 1 || q < 1 || p > kMaxCols || q > kMaxCols) return 0;
    return (size_t)kGramBlocks * p * q * sizeof(double);
}

MVGD_API mvgd_status mvgd_block_gram(const double* X, int32_t p, const double* Y, int32_t q, int64_t n, int32_t w,
                                     double* G, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!X || !Y || !G || !ws || bad_shape(n, p, q, w)) return MVGD_EINVAL;
    if (!aligned(X) || !aligned(Y) || !aligned(ws) || (reinterpret_cast<uintptr_t>(G) & 7) != 0) return MVGD_EINVAL;
    if (ws_bytes < mvgd_block_gram_workspace_bytes(p, q)) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    double* partial = static_cast<double*>(ws);
    k_gram_partial<<<kGramBlocks, 256, 0, s>>>(X, p, Y, q, n, w, partial);
    k_gram_final<<<(p * q + 255) / 256, 256, 0, s>>>(partial, p * q, G);
    return launch_status();
}

MVGD_API mvgd_status mvgd_block_combine(const double* X, int32_t p, const double* C, int32_t q, int64_t n, int32_t w,
                                        double* Y, mvgd_stream_t stream) {
    if (!X || !C || !Y || X == Y || bad_shape(n, p, q, w)) return MVGD_EINVAL;
    if (!aligned(X) || !aligned(Y) || (reinterpret_cast<uintptr_t>(C) & 7) != 0) return MVGD_EINVAL;
    const int64_t blocks = (n * q + 255) / 256;
    k_block_combine<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, (cudaStream_t)stream>>>(X, p, C, q, n, w,
                                                                                                  Y);
    return launch_status();
}

MVGD_API mvgd_status mvgd_block_zero_rows(double* X, int32_t p, int64_t n, int32_t w, const uint8_t* mask,
                                          mvgd_stream_t stream) {
    if (!X || !mask || bad_shape(n, p, p, w) || !aligned(X)) return MVGD_EINVAL;
    const int64_t blocks = (n * p + 255) / 256;
    k_block_zero_rows<<<(unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, (cudaStream_t)stream>>>(X, p, n, w, mask);
    return launch_status();
}
