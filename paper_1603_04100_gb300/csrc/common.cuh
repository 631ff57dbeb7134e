// Internal helpers shared by the CUDA translation units of libmvgd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mvgd.h"

#define MVGD_API extern "C" __attribute__((visibility("default")))

namespace mvgd {

constexpr int kWarp = 32;
constexpr int kSlice = 32;          // SELL slice height
constexpr int kMaxK = 31;
constexpr int kMinK = 5;
constexpr size_t kAlign = 256;

__host__ __device__ inline size_t align_up(size_t x, size_t a = kAlign) { return (x + a - 1) / a * a; }
__host__ __device__ inline int64_t n_padded(int64_t n) { return (n + kSlice - 1) / kSlice * kSlice; }

// Element (r, s) of a sliced-ELL array of width w.
__host__ __device__ inline int64_t sell_index(int64_t r, int s, int w) {
    return (r / kSlice) * (int64_t)(kSlice * w) + (int64_t)s * kSlice + (r % kSlice);
}

inline bool aligned(const void* p) { return p == nullptr || ((uintptr_t)p % kAlign) == 0; }

// Carves 256-byte aligned sub-buffers out of a caller workspace.
struct Carver {
    char* base;
    size_t used = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count) {
        T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
        used += align_up(sizeof(T) * count);
        return p;
    }
};

#define MVGD_CUDA_TRY(expr)                              \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return MVGD_ECUDA;        \
    } while (0)

inline mvgd_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? MVGD_OK : MVGD_ECUDA;
}

// Host side of mvgd_set_wait_limit / mvgd_test_withhold_arrival (capi.cu):
// the poll limit a launch made now should use (dflt unless the caller set
// one), and the one-shot withhold control (true once after it was armed).
long long wait_limit_or(long long dflt);
bool take_withhold();
// Launch shapes set by mvgd_set_launch_tuning (speed only, never results).
int tuned_solver_blocks_per_sm();  // 0: as many as fit
int tuned_stage_buffers();         // 1 or 2
int tuned_assemble_warps();        // 1, 2, 4 or 8

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & (kWarp - 1); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Compensated FP32 accumulation (the "Dot2" scheme of Ogita, Rump & Oishi,
// SIAM J. Sci. Comput. 26(6), 2005): each product is split exactly into
// p + e with one FMA (TwoProduct) and each addition into s + e (TwoSum), so
// a dot product of FP32 vectors comes out as accurate as if accumulated in
// twice the working precision, using FP32 instructions only.  The _rn
// intrinsics keep the compiler from contracting the error terms away.
// ---------------------------------------------------------------------------
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void f2_add_prod(F2& acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float ep = __fmaf_rn(a, b, -p);  // exact: a*b = p + ep
    float s, es;
    two_sum(acc.hi, p, s, es);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(es, ep));
}

__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
    float s, e;
    two_sum(x.hi, y.hi, s, e);
    F2 r;
    r.hi = s;
    r.lo = __fadd_rn(__fadd_rn(x.lo, y.lo), e);
    return r;
}

__device__ __forceinline__ F2 warp_sum_f2(F2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F2 w;
        w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v = f2_add(v, w);
    }
    return v;
}

__device__ __forceinline__ double f2_to_double(F2 v) { return (double)v.hi + (double)v.lo; }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int m) {
    return __shfl_xor_sync(0xffffffffu, v, m);
}

// ---------------------------------------------------------------------------
// Grid-wide barrier for persistent cooperative kernels, on one monotonic
// arrival counter.  Bounded: after `limit` polls it sets *err and returns
// false, so a kernel whose blocks were not all resident ends with an error
// status instead of spinning forever.
// ---------------------------------------------------------------------------
struct GridBarrier {
    unsigned int* count;   // zeroed before the launch
    volatile unsigned int* gen;  // unused (kept for the control-word layout)
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const volatile unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0 of each block adds its arrival with a release reduction (its
// block's writes, ordered before it by __syncthreads, are released with it)
// and does not wait for the add to return; it then polls the counter with
// acquire loads until every block of this barrier has arrived: the e-th
// barrier of a launch completes at count = e * gridDim.x (compared modulo
// 2^32, so the counter may wrap).  One round trip less than a returning
// atomic followed by a released generation word: about 1 us less per barrier
// for 456 blocks on GB300.  `epoch` is the caller's count of barriers passed,
// the same in every block.
// `arrive` false (only the withhold test control passes it) leaves this block's
// arrival out, so the barrier cannot complete and every block's wait runs out.
__device__ __forceinline__ bool grid_sync(GridBarrier b, unsigned& epoch, int* err, long long limit,
                                          bool arrive = true) {
    __syncthreads();
    bool ok = true;
    epoch += 1u;
    if (threadIdx.x == 0) {
        const unsigned target = epoch * gridDim.x;
        if (arrive) red_release_add_gpu(b.count, 1u);
        long long polls = 0;
        while ((int)(ld_acquire_gpu(b.count) - target) < 0) {
            if ((++polls & 255) == 0 && (polls > limit || *(volatile int*)err != 0)) {
                atomicCAS(err, 0, (int)MVGD_ETIMEOUT);
                ok = false;
                break;
            }
        }
    }
    __syncthreads();
    return ok && (*(volatile int*)err == 0);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies global -> shared (the TMA engine's untiled form)
// completing on an mbarrier.  Addresses and sizes must be multiples of 16
// bytes; every caller copies whole sliced-ELL slices of a 256-byte aligned
// array, which are.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes barrier initialisation, and generic-proxy accesses of shared memory
// that precede an async copy into it, ordered before that copy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// L2 policy that marks streamed data as first to evict.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete: false after
// `limit` polls (the copy did not land), so no caller can spin forever.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    for (long long i = 0; i < limit; i++) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    return false;
}

}  // namespace mvgd
