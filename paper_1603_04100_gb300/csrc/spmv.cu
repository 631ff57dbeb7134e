// y = alpha (sigma x - L x) + beta y on the sliced ELL operator (the product a
// Krylov solve of (sigma I - L) u = f repeats; Sec. 3.1, Sec. 4.2).
//
// One thread per row: within a warp the 32 rows of one slice read every slot
// of col / val as one coalesced 128-byte (FP32) or 256-byte (FP64) line; x is
// gathered through L1/L2.  Three arithmetic forms:
//   F64       standard form  w_0 x_i + sum_s w_s x_{c_s}, FP64 weights;
//   F32       difference form sum_s w_s (x_{c_s} - x_i) with FP32 hi weights:
//             rows of L sum to zero, so the self weight is implied and the
//             products act on small differences of a smooth vector;
//   F64_HILO  standard form with w = hi + lo evaluated in FP64.
#include "common.cuh"

namespace mvgd {
namespace {

// The operator's columns and weights are streamed once per product: loaded
// past L1 (read-only path, no L1 allocation), so that L1 keeps the lines of x
// the neighbour gathers reuse.  At 1M rows, K = 20 this took the FP32 product
// from 45 us to 35 us.  (Plain asm: the arrays do not change while a kernel runs.)
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
    double v;
    asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}

// KK > 0: K fixed at compile time (every slot's loads can be issued at once);
// KK == 0: K at run time.
template <int Q, int KK>
__global__ void __launch_bounds__(256) k_spmv_f64(int64_t n, int kr, const int32_t* __restrict__ col,
                                                   const double* __restrict__ val, double sigma, double alpha,
                                                   const double* __restrict__ x, double beta,
                                                   double* __restrict__ y) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = KK > 0 ? KK : kr;
    const int m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    const double w0 = ld_stream(val + vb);
    double xi[Q], acc[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        xi[q] = x[r * Q + q];
        acc[q] = w0 * xi[q];
    }
#pragma unroll (KK > 0 ? KK : 4)
    for (int s = 0; s < k; s++) {
        const int64_t j = ld_stream(col + cb + (int64_t)s * kSlice);
        const double w = ld_stream(val + vb + (int64_t)(s + 1) * kSlice);
#pragma unroll
        for (int q = 0; q < Q; q++) acc[q] = fma(w, x[j * Q + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        double out = alpha * (sigma * xi[q] - acc[q]);
        if (beta != 0.0) out = fma(beta, y[r * Q + q], out);
        y[r * Q + q] = out;
    }
}

template <int Q, int KK>
__global__ void __launch_bounds__(256) k_spmv_f32(int64_t n, int kr, const int32_t* __restrict__ col,
                                                   const float* __restrict__ val, float sigma, float alpha,
                                                   const float* __restrict__ x, float beta,
                                                   float* __restrict__ y) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int k = KK > 0 ? KK : kr;
    const int m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    float xi[Q], acc[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        xi[q] = x[r * Q + q];
        acc[q] = 0.0f;
    }
#pragma unroll (KK > 0 ? KK : 4)
    for (int s = 0; s < k; s++) {
        const int64_t j = ld_stream(col + cb + (int64_t)s * kSlice);
        const float w = ld_stream(val + vb + (int64_t)(s + 1) * kSlice);
#pragma unroll
        for (int q = 0; q < Q; q++) acc[q] = fmaf(w, x[j * Q + q] - xi[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        float out = alpha * (sigma * xi[q] - acc[q]);
        if (beta != 0.0f) out = fmaf(beta, y[r * Q + q], out);
        y[r * Q + q] = out;
    }
}

template <int Q, int KK>
void launch_spmv_k(const mvgd_ell* L, int mode, double sigma, double alpha, const void* x, double beta, void* y,
                   cudaStream_t s) {
    const int64_t n = L->n;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (mode == MVGD_SPMV_F32)
        k_spmv_f32<Q, KK><<<blocks, 256, 0, s>>>(n, L->k, L->col, static_cast<const float*>(L->val), (float)sigma,
                                                 (float)alpha, static_cast<const float*>(x), (float)beta,
                                                 static_cast<float*>(y));
    else
        k_spmv_f64<Q, KK><<<blocks, 256, 0, s>>>(n, L->k, L->col, static_cast<const double*>(L->val), sigma, alpha,
                                                 static_cast<const double*>(x), beta, static_cast<double*>(y));
}

template <int Q>
mvgd_status launch_spmv(const mvgd_ell* L, int mode, double sigma, double alpha, const void* x, double beta,
                        void* y, cudaStream_t s) {
    if (mode == MVGD_SPMV_F32 || mode == MVGD_SPMV_F64) {
        // the common K at compile time, any other at run time
        switch (L->k) {
            case 12: launch_spmv_k<Q, 12>(L, mode, sigma, alpha, x, beta, y, s); break;
            case 16: launch_spmv_k<Q, 16>(L, mode, sigma, alpha, x, beta, y, s); break;
            case 20: launch_spmv_k<Q, 20>(L, mode, sigma, alpha, x, beta, y, s); break;
            case 24: launch_spmv_k<Q, 24>(L, mode, sigma, alpha, x, beta, y, s); break;
            default: launch_spmv_k<Q, 0>(L, mode, sigma, alpha, x, beta, y, s); break;
        }
    } else {
        // hi + lo: hi is stored as float in val; read it through a float view
        return MVGD_EINVAL;
    }
    return launch_status();
}

template <int Q>
__global__ void __launch_bounds__(256) k_spmv_hilo(int64_t n, int k, const int32_t* __restrict__ col,
                                                    const float* __restrict__ hi, const float* __restrict__ lo,
                                                    double sigma, double alpha, const double* __restrict__ x,
                                                    double beta, double* __restrict__ y) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    const double w0 = (double)ld_stream(hi + vb) + (double)ld_stream(lo + vb);
    double xi[Q], acc[Q];
#pragma unroll
    for (int q = 0; q < Q; q++) {
        xi[q] = x[r * Q + q];
        acc[q] = w0 * xi[q];
    }
#pragma unroll 4
    for (int s = 0; s < k; s++) {
        const int64_t j = ld_stream(col + cb + (int64_t)s * kSlice);
        const int64_t e = vb + (int64_t)(s + 1) * kSlice;
        const double w = (double)ld_stream(hi + e) + (double)ld_stream(lo + e);
#pragma unroll
        for (int q = 0; q < Q; q++) acc[q] = fma(w, x[j * Q + q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < Q; q++) {
        double out = alpha * (sigma * xi[q] - acc[q]);
        if (beta != 0.0) out = fma(beta, y[r * Q + q], out);
        y[r * Q + q] = out;
    }
}

template <int Q>
mvgd_status launch_hilo(const mvgd_ell* L, double sigma, double alpha, const void* x, double beta, void* y,
                        cudaStream_t s) {
    unsigned blocks = (unsigned)((L->n + 255) / 256);
    k_spmv_hilo<Q><<<blocks, 256, 0, s>>>(L->n, L->k, L->col, static_cast<const float*>(L->val), L->val_lo,
                                          sigma, alpha, static_cast<const double*>(x), beta,
                                          static_cast<double*>(y));
    return launch_status();
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API mvgd_status mvgd_spmv(const mvgd_ell* L, int32_t mode, int32_t nrhs, double sigma, double alpha,
                               const void* x, double beta, void* y, mvgd_stream_t stream) {
    if (!L || !x || !y || !L->col || !L->val || L->n < 1 || L->k < 1 || L->k > kMaxK) return MVGD_EINVAL;
    if (nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (!aligned(x) || !aligned(y) || !aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo))
        return MVGD_EINVAL;
    if (mode == MVGD_SPMV_F64 && L->prec != MVGD_FP64) return MVGD_EINVAL;
    if ((mode == MVGD_SPMV_F32 || mode == MVGD_SPMV_F64_HILO) && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (mode == MVGD_SPMV_F64_HILO && !L->val_lo) return MVGD_EINVAL;
    if (mode < 0 || mode > 2) return MVGD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == MVGD_SPMV_F64_HILO) {
        switch (nrhs) {
            case 1: return launch_hilo<1>(L, sigma, alpha, x, beta, y, s);
            case 2: return launch_hilo<2>(L, sigma, alpha, x, beta, y, s);
            case 3: return launch_hilo<3>(L, sigma, alpha, x, beta, y, s);
            case 4: return launch_hilo<4>(L, sigma, alpha, x, beta, y, s);
            case 5: return launch_hilo<5>(L, sigma, alpha, x, beta, y, s);
            case 6: return launch_hilo<6>(L, sigma, alpha, x, beta, y, s);
            case 7: return launch_hilo<7>(L, sigma, alpha, x, beta, y, s);
            default: return launch_hilo<8>(L, sigma, alpha, x, beta, y, s);
        }
    }
    switch (nrhs) {
        case 1: return launch_spmv<1>(L, mode, sigma, alpha, x, beta, y, s);
        case 2: return launch_spmv<2>(L, mode, sigma, alpha, x, beta, y, s);
        case 3: return launch_spmv<3>(L, mode, sigma, alpha, x, beta, y, s);
        case 4: return launch_spmv<4>(L, mode, sigma, alpha, x, beta, y, s);
        case 5: return launch_spmv<5>(L, mode, sigma, alpha, x, beta, y, s);
        case 6: return launch_spmv<6>(L, mode, sigma, alpha, x, beta, y, s);
        case 7: return launch_spmv<7>(L, mode, sigma, alpha, x, beta, y, s);
        default: return launch_spmv<8>(L, mode, sigma, alpha, x, beta, y, s);
    }
}
