// Conditioning of the stored system (Sec. 4.1): power iteration on the
// Gauss-Seidel iteration matrix T = M^-1 N of A = sigma I - L, where M is the
// lower triangle of A with its diagonal and N the strictly upper triangle, in
// stored row order.  The paper compares the eigenvalues of T for the MVGD and
// the least-squares rows: inside the unit circle for MVGD, so a plain
// Gauss-Seidel sweep converges; largely outside for least squares.
//
// One cooperative launch runs every step.  A product y = T x is
//   z = N x                  the upper neighbours, read from the previous iterate;
//   M y = z                  forward substitution: y_r = (z_r - sum_{j<r} a_rj y_j) / a_rr.
// The substitution is sync-free: warps take rows in increasing order from a
// per-step ticket counter, and each lane whose neighbour j precedes the row
// waits on flag[j] (= step + 1 once y_j is stored; a release store after the
// value, an acquire load before it is read).  A warp only waits on rows whose
// tickets were taken earlier by warps that are running, so the lowest
// unfinished row always has its inputs and the substitution cannot deadlock;
// every wait is bounded all the same.  Norms are summed over fixed row ranges
// and then over the ranges in order, so the results repeat bit for bit.
#include "common.cuh"

namespace mvgd {
namespace {

constexpr int kGsThreads = 256;
constexpr long long kGsPollLimit = 1ll << 24;  // polls of one flag before MVGD_ETIMEOUT
constexpr long long kGsBarrierLimit = 1ll << 26;
constexpr int kGsMaxIters = 1 << 20;

struct GsArgs {
    mvgd_ell L;
    double sigma;
    const double* x0;
    int iters;
    double* nu;
    double* xout;
    int32_t* status;
    double* buf0;
    double* buf1;
    unsigned* flag;   // [n]
    unsigned* tick;   // [iters]
    double* part;     // [grid]
    unsigned* bar;    // barrier counter
    int* err;
    long long poll_limit;     // polls of one row flag before MVGD_ETIMEOUT
    long long barrier_limit;  // polls of the grid barrier
    int withhold;             // test control: row 0's first flag is never published
};

__device__ __forceinline__ void st_release_gpu(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Weight e of the operator: FP64, or hi + lo (lo == nullptr for FP64 weights)
__device__ __forceinline__ double weight(const void* val, const float* lo, int64_t e) {
    return lo == nullptr ? __ldg(static_cast<const double*>(val) + e)
                         : (double)__ldg(static_cast<const float*>(val) + e) + (double)__ldg(lo + e);
}

// Sum of (c v_r)^2 over this block's fixed row range: each thread over a fixed
// stride, then the warps' butterflies, then the warps in order.
__device__ double range_sumsq(const double* v, double c, int64_t r0, int64_t r1, double* red) {
    double s = 0.0;
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const double y = c * __ldcg(v + r);
        s = fma(y, y, s);
    }
    s = warp_sum(s);
    if (lane_id() == 0) red[threadIdx.x / kWarp] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x / kWarp); w++) t += red[w];
    __syncthreads();
    return t;
}

// All blocks: the sum of part[0 .. gridDim.x) in order, broadcast through shared memory.
__device__ double grid_total(const double* part, double* slot) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) t += __ldcg(part + b);
        *slot = t;
    }
    __syncthreads();
    const double t = *slot;
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kGsThreads) k_gs_power(GsArgs a) {
    __shared__ double red[kGsThreads / kWarp];
    __shared__ double total;
    const int64_t n = a.L.n;
    const int k = a.L.k, m = k + 1;
    const int32_t* __restrict__ col = a.L.col;
    const void* val = a.L.val;
    const float* lo_w = a.L.prec == MVGD_FP64 ? nullptr : a.L.val_lo;
    const int lane = (int)lane_id();
    GridBarrier bar{a.bar, nullptr};
    unsigned epoch = 0;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = blockIdx.x * per < n ? blockIdx.x * per : n;
    const int64_t r1 = r0 + per < n ? r0 + per : n;

    // x_0 = x0 / ||x0||: the copy is stored raw, its scale kept in c
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) __stcg(a.buf0 + r, a.x0[r]);
    __syncthreads();
    double s0 = range_sumsq(a.buf0, 1.0, r0, r1, red);
    if (threadIdx.x == 0) a.part[blockIdx.x] = s0;
    if (!grid_sync(bar, epoch, a.err, a.barrier_limit)) goto done;
    {
        double tot = grid_total(a.part, &total);
        if (!(tot > 0.0) || !isfinite(tot)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.err, 0, (int)MVGD_ENONFINITE);
            goto done;
        }
        double c = 1.0 / sqrt(tot);
        for (int it = 0; it < a.iters; it++) {
            const double* src = (it & 1) ? a.buf1 : a.buf0;
            double* dst = (it & 1) ? a.buf0 : a.buf1;
            const unsigned done_mark = (unsigned)it + 1u;
            for (;;) {
                unsigned t = 0;
                if (lane == 0) t = atomicAdd(a.tick + it, 1u);
                t = __shfl_sync(0xffffffffu, t, 0);
                if ((int64_t)t >= n) break;
                const int64_t r = t;
                double up = 0.0, lo = 0.0, dself = 0.0;
                if (lane < k) {
                    const int64_t j = __ldg(col + sell_index(r, lane, k));
                    const double arj = -weight(val, lo_w, sell_index(r, lane + 1, m));
                    if (j > r) {
                        up = arj * (c * __ldcg(src + j));
                    } else if (j == r) {
                        dself = arj;
                    } else {
                        long long polls = 0;
                        while (ld_acquire_gpu(a.flag + j) != done_mark) {
                            if ((++polls & 255) == 0 && (polls > a.poll_limit || *(volatile int*)a.err != 0)) {
                                atomicCAS(a.err, 0, (int)MVGD_ETIMEOUT);
                                break;
                            }
                        }
                        lo = arj * __ldcg(dst + j);
                    }
                }
                up = warp_sum(up);
                lo = warp_sum(lo);
                dself = warp_sum(dself);
                if (lane == 0) {
                    const double d = a.sigma - weight(val, lo_w, sell_index(r, 0, m)) + dself;
                    __stcg(dst + r, (up - lo) / d);
                    if (!(a.withhold && it == 0 && r == 0)) st_release_gpu(a.flag + r, done_mark);
                }
                if (*(volatile int*)a.err != 0) break;
            }
            if (!grid_sync(bar, epoch, a.err, a.barrier_limit)) goto done;
            const double sb = range_sumsq(dst, 1.0, r0, r1, red);
            if (threadIdx.x == 0) a.part[blockIdx.x] = sb;
            if (!grid_sync(bar, epoch, a.err, a.barrier_limit)) goto done;
            tot = grid_total(a.part, &total);
            const double nrm = sqrt(tot);
            if (blockIdx.x == 0 && threadIdx.x == 0) a.nu[it] = nrm;
            if (!(tot > 0.0) || !isfinite(tot)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.err, 0, (int)MVGD_ENONFINITE);
                goto done;
            }
            c = 1.0 / nrm;
        }
        // x = the last product, normalised
        const double* last = (a.iters & 1) ? a.buf1 : a.buf0;
        for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) a.xout[r] = c * __ldcg(last + r);
    }
done:
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        __threadfence();
        *a.status = *(volatile int*)a.err;
    }
}

struct GsLayout {
    size_t buf0, buf1, flag, tick, part, ctl, total;
};

GsLayout gs_layout(int64_t n, int iters, int grid) {
    GsLayout l{};
    size_t o = 0;
    l.buf0 = o; o += align_up(sizeof(double) * n);
    l.buf1 = o; o += align_up(sizeof(double) * n);
    l.flag = o; o += align_up(sizeof(unsigned) * n);
    l.tick = o; o += align_up(sizeof(unsigned) * iters);
    l.part = o; o += align_up(sizeof(double) * grid);
    l.ctl = o; o += align_up(2 * sizeof(int));
    l.total = o;
    return l;
}

// Blocks of the cooperative launch (the grid is also the number of norm ranges).
constexpr int kGsMaxGrid = 152 * 8;

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_gs_power_workspace_bytes(int64_t n, int32_t iters) {
    if (n < 1 || n >= (1ll << 31) || iters < 1 || iters > kGsMaxIters) return 0;
    return gs_layout(n, iters, kGsMaxGrid).total;
}

MVGD_API mvgd_status mvgd_gs_power(const mvgd_ell* L, double sigma, const double* x0, int32_t iters, double* nu,
                                   double* x, int32_t* status, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!L || !x0 || !nu || !x || !status || !ws || !L->col || !L->val) return MVGD_EINVAL;
    if (L->n < 1 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK || iters < 1 || iters > kGsMaxIters)
        return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!(sigma == sigma) || sigma - sigma != 0.0) return MVGD_EINVAL;
    if (!aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo) || !aligned(ws)) return MVGD_EINVAL;
    if (!aligned(x0) || !aligned(x) || !aligned(nu) || !aligned(status)) return MVGD_EINVAL;
    if (ws_bytes < mvgd_gs_power_workspace_bytes(L->n, iters)) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    MVGD_CUDA_TRY(cudaGetDevice(&dev));
    MVGD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MVGD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs_power, kGsThreads, 0));
    if (per_sm < 1) return MVGD_ECUDA;
    int grid = sms * per_sm;
    if (grid > kGsMaxGrid) grid = kGsMaxGrid;
    const int64_t blocks_needed = (L->n + kGsThreads / kWarp - 1) / (kGsThreads / kWarp);  // a row per warp
    if (grid > blocks_needed) grid = (int)blocks_needed;
    const GsLayout lay = gs_layout(L->n, iters, kGsMaxGrid);
    char* base = static_cast<char*>(ws);
    GsArgs a;
    a.L = *L;
    a.sigma = sigma;
    a.x0 = x0;
    a.iters = iters;
    a.nu = nu;
    a.xout = x;
    a.status = status;
    a.buf0 = reinterpret_cast<double*>(base + lay.buf0);
    a.buf1 = reinterpret_cast<double*>(base + lay.buf1);
    a.flag = reinterpret_cast<unsigned*>(base + lay.flag);
    a.tick = reinterpret_cast<unsigned*>(base + lay.tick);
    a.part = reinterpret_cast<double*>(base + lay.part);
    a.bar = reinterpret_cast<unsigned*>(base + lay.ctl);
    a.err = reinterpret_cast<int*>(base + lay.ctl) + 1;
    a.poll_limit = wait_limit_or(kGsPollLimit);
    a.barrier_limit = wait_limit_or(kGsBarrierLimit);
    a.withhold = take_withhold() ? 1 : 0;
    // flags, tickets and the control words start at zero; the flag and ticket
    // regions are contiguous
    MVGD_CUDA_TRY(cudaMemsetAsync(base + lay.flag, 0, lay.part - lay.flag, s));
    MVGD_CUDA_TRY(cudaMemsetAsync(base + lay.ctl, 0, 2 * sizeof(int), s));
    void* args[] = {(void*)&a};
    MVGD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_gs_power, dim3(grid), dim3(kGsThreads), args, 0, s));
    return MVGD_OK;
}
