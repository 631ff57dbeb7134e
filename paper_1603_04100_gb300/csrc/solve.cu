// Device-resident Krylov solves of (sigma I - L) u = f (Sec. 4.2; the paper
// solves with AMG -- here BiCGSTAB, van der Vorst 1992, optionally left-scaled
// by the diagonal).
//
// Every system being solved is a "request" whose whole solver state (Krylov
// vectors, per-RHS scalars, reduction partials) lives in its own caller-owned
// workspace.  One persistent cooperative kernel advances any set of requests
// together; an iteration is a fixed sequence of phases separated by a bounded
// grid barrier:
//   PRE_A  FP64: p = r + beta (p - omega v)       | FP32: fold u += s x on restart
//   A      v = A p  (FP32: p formed on the fly at the neighbours)      -> (rh, v)
//   PRE_B  FP64: s = r - alpha v                   | FP32: skipped
//   B      t = A s  (FP32: s formed on the fly)                     -> (t, s), (t, t)
//   C      x += alpha p + omega s, r = s - omega t                  -> (rh, r), (r, r)
// FP64 materialises p and s because forming them at every neighbour would
// multiply the FP64 work by K on a part whose FP64 pipe is 1/56 of FP32; the
// FP32 path forms them on the fly and saves two barriers.  Rows are cut into
// fixed chunks of kCh rows; a chunk's partials are reduced in a fixed order
// and the block that finishes a request's last chunk of a phase sums that
// request's partials in chunk order and advances its per-RHS state.  Results
// therefore depend neither on the grid size nor on the other requests.
//
// Per right-hand side:
//   RESTART  FP64 true residual r64 = f - A u (FP32 path: on hi + lo weights,
//            after folding the last inner correction into u); stop at rtol,
//            else restart the Krylov vectors from D^-1 r64 (FP32 path: scaled
//            by 1 / ||r64|| and rounded to FP32)
//   INNER    BiCGSTAB until the recursive residual meets the restart target;
//            a diverging FP32 inner solve is abandoned and its correction dropped
//   DONE
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "vcycle.cuh"

namespace mvgd {
namespace {

constexpr int kCh = 256;   // rows per tile: one per thread, 8 slices of 32
constexpr int kThreads = 256;
constexpr int kChan = 2;     // reduced channels a step of the row-scaled flows
constexpr int kChanAmg = 5;  // ... of the multigrid flow (B takes five dot products)
__host__ __device__ constexpr int chan_count(bool amg) { return amg ? kChanAmg : kChan; }
constexpr int kRedSlots = 3;
constexpr int kMaxReq = 1024;
constexpr long long kStageWaitLimit = 1ll << 24;  // polls of an mbarrier: far beyond any copy's landing time

enum Phase : int { P_PRE_A = 0, P_A = 1, P_PRE_B = 2, P_B = 3, P_C = 4, P_COUNT = 5 };
enum Mode : int { M_RESTART = 0, M_INNER = 1, M_SKIP = 2, M_DONE = 3 };

__host__ __device__ constexpr int red_slot(int ph) { return ph == P_A ? 0 : (ph == P_B ? 1 : 2); }

struct RhsState {
    double rho, alpha, omega, beta;
    double fnorm, relres, scale, target;
    double rnorm, rmin;
    int mode, pp, iters, inner_iters, outer, status, discard, stall;
    int best_flag;   // the last iteration reached a new smallest inner residual: copy x to x_best
    int fold_best;   // on restart, fold x_best (not x) into u
    int since_best;  // inner iterations since the smallest residual last dropped by 1%
    int pending;     // multigrid flow: the last step's x += alpha ph + omega sh is still to apply
};

// One request: an operator, its right-hand sides and all solver state.
struct Prob {
    int64_t n;
    int k, Q, prec, precond;
    double sigma;
    const int32_t* col;
    const void* val;
    const float* val_lo;
    const int32_t* order;
    double* f;         // stored order [n][Q]
    double* u;         // stored order [n][Q]
    void* x;
    void* xb;          // FP32 path: the inner iterate with the smallest residual so far
    void* r;
    void* rh;
    void* p[2];
    void* v[2];
    void* s;
    void* t;
    double* r64;
    void* invd;        // [n] VT: 1 / (sigma + sum_s |w_s|), the left scaling (precond == 1)
    RhsState* st;      // [Q]
    void* part;        // [kRedSlots][channels][nchunk][Q] tile partials (Part<MIXED>: F2 or double)
    unsigned* arrive;  // [kRedSlots]
    int nchunk, pad;
    // multigrid right preconditioning (precond == 2); amg == nullptr otherwise
    const AmgHeader* amg;
    int amg_levels, pad3;
    void* ph;                    // [n][Q] VT: M^-1 p
    void* sh;                    // [n][Q] VT: M^-1 s
    float* vy[kAmgMaxLevels];    // per level [n_l][Q]: pre-smoothed y_l = d_l b_l
    float* vr[kAmgMaxLevels];    //                     residual r_l
    float* vb[kAmgMaxLevels];    //                     right-hand side b_l (l >= 1)
    float* vx[kAmgMaxLevels];    //                     correction x_l (l >= 1)
    double rtol, inner_rtol;
    int maxit, inner_maxit, max_outer, pad2;
};

struct Ctl {
    GridBarrier bar;
    int* err;
    int* active;     // right-hand sides not DONE
    int* nrestart;   // right-hand sides in RESTART
    int* stop;
    const int* cancel;
    long long limit;
    int trace;       // record each step's end time (mvgd_trace_enable)
    int withhold;    // test control: block 0 leaves its first barrier arrival out
};

// ------------------------------------------------------------------------------
// Step trace: block 0 of the solver stamps the device clock after every grid
// barrier, with the step it closed, into a static device ring that the host
// reads with mvgd_trace_read.  Off unless mvgd_trace_enable(1).
// ------------------------------------------------------------------------------
constexpr int kTraceMax = 1 << 16;
static __device__ unsigned long long g_trace[kTraceMax];
static __device__ unsigned int g_trace_n;
int g_trace_on = 0;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// step code: Krylov phase ph (0..4), or 0x1000 | side << 8 | kind << 4 | level for a V-cycle step
__device__ __forceinline__ void trace_step(const Ctl& ctl, unsigned code) {
    if (!ctl.trace || blockIdx.x != 0 || threadIdx.x != 0) return;
    const unsigned i = g_trace_n;
    g_trace_n = i + 1;
    g_trace[i % kTraceMax] = ((unsigned long long)code << 48) | (global_ns() & 0xffffffffffffull);
}

__device__ __forceinline__ void load_state(RhsState& dst, const RhsState* src) {
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
#pragma unroll
    for (int w = 0; w < (int)(sizeof(RhsState) / 8); w++) d[w] = __ldcg(s + w);
}

// ------------------------------------------------------------------------------
// Row work
// ------------------------------------------------------------------------------

// PRE_A / PRE_B / C and the RESTART steps: elementwise on row r.
template <bool MIXED, int QT>
__device__ __forceinline__ void elementwise_row(const Prob& P, int64_t r, int ph, const RhsState* S,
                                                const bool (&inner)[QT], const bool (&restart)[QT],
                                                F2 (&af)[kChan][QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q;
#pragma unroll
    for (int q = 0; q < QT; q++) {
        const int64_t e = r * Q + q;
        if (ph == P_PRE_A) {
            if (MIXED && restart[q] && S[q].outer > 0 && !S[q].discard)
                P.u[e] += S[q].scale * (double)static_cast<const VT*>(S[q].fold_best ? P.xb : P.x)[e];
            if (!MIXED && inner[q]) {
                VT* pv = static_cast<VT*>(P.p[0]);
                const VT* vv = static_cast<const VT*>(P.v[0]);
                const VT* rv = static_cast<const VT*>(P.r);
                pv[e] = rv[e] + (VT)S[q].beta * (pv[e] - (VT)S[q].omega * vv[e]);
            }
        } else if (ph == P_PRE_B) {
            if (!MIXED && inner[q]) {
                const VT* vv = static_cast<const VT*>(P.v[0]);
                const VT* rv = static_cast<const VT*>(P.r);
                static_cast<VT*>(P.s)[e] = rv[e] - (VT)S[q].alpha * vv[e];
            }
        } else if (ph == P_C) {
            if (inner[q]) {
                const VT* pv = static_cast<const VT*>(P.p[S[q].pp]);
                VT* X = static_cast<VT*>(P.x);
                const VT sv = static_cast<const VT*>(P.s)[e], tv = static_cast<const VT*>(P.t)[e];
                const VT al = (VT)S[q].alpha, om = (VT)S[q].omega;
                X[e] = X[e] + al * pv[e] + om * sv;
                const VT rn = sv - om * tv;
                static_cast<VT*>(P.r)[e] = rn;
                const VT rhv = static_cast<const VT*>(P.rh)[e];
                f2_add_prod(af[0][q], (float)rhv, (float)rn);
                f2_add_prod(af[1][q], (float)rn, (float)rn);
            }
        }
    }
}

// FP64 partials of the FP64 steps (C of the plain path) go through a double
// accumulator so that nothing is rounded to FP32.
template <int QT>
__device__ __forceinline__ void c_row_f64(const Prob& P, int64_t r, const RhsState* S, const bool (&inner)[QT],
                                          double (&ad)[kChan][QT]) {
    const int Q = P.Q;
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!inner[q]) continue;
        const int64_t e = r * Q + q;
        const double* pv = static_cast<const double*>(P.p[0]);
        double* X = static_cast<double*>(P.x);
        const double sv = static_cast<const double*>(P.s)[e], tv = static_cast<const double*>(P.t)[e];
        X[e] = X[e] + S[q].alpha * pv[e] + S[q].omega * sv;
        const double rn = sv - S[q].omega * tv;
        static_cast<double*>(P.r)[e] = rn;
        ad[0][q] += static_cast<const double*>(P.rh)[e] * rn;
        ad[1][q] += rn * rn;
    }
}

// Warp totals of E F2 values a lane (E a power of two, at most 32) with a
// fraction of the shuffles of E separate butterflies.  At each of the first
// log2 E offsets (16, 8, ...) a lane keeps half of its values -- the upper
// half if its bit at that offset is set -- and adds the partner's copy of
// them; the remaining offsets add the one value left.  Every value is summed
// in exactly the pairs and order of a plain xor butterfly over offsets 16, 8,
// 4, 2, 1 (f2_add is commutative), so the totals are those of E separate
// butterflies, bit for bit.  Returns the total of channel `chan` (set here)
// that this lane ends with; lanes L with L % (32 / E) == 0 hold channels
// 0 .. E-1 once each.
template <int E>
__device__ __forceinline__ F2 warp_sum_f2_multi(F2 (&v)[E], int lane, int& chan) {
    static_assert(E >= 1 && E <= 32 && (E & (E - 1)) == 0, "a power of two, at most 32 values");
    chan = 0;
#pragma unroll
    for (int t = 0; t < 5; t++) {
        const int o = 16 >> t;
        const int h = E >> (t + 1);  // values kept after this offset (0: one value left)
        if (h >= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int j = 0; j < (h >= 1 ? h : 1); j++) {
                const F2 send = up ? v[j] : v[j + h];
                const F2 keep = up ? v[j + h] : v[j];
                F2 recv;
                recv.hi = __shfl_xor_sync(0xffffffffu, send.hi, o);
                recv.lo = __shfl_xor_sync(0xffffffffu, send.lo, o);
                v[j] = f2_add(keep, recv);
            }
            if (up) chan += h;
        } else {
            F2 w;
            w.hi = __shfl_xor_sync(0xffffffffu, v[0].hi, o);
            w.lo = __shfl_xor_sync(0xffffffffu, v[0].lo, o);
            v[0] = f2_add(v[0], w);
        }
    }
    return v[0];
}

__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 1 ? 1 : 2 * pow2_at_least((x + 1) / 2); }

// Tile partials and their sums: F2 (double-float on the FP32 pipe) in the
// FP32 flow, double in the FP64 one.  One SM sums a request's thousands of
// partials in each reducing step.  GB300's FP64 rate (1.25 TFLOP/s nominal)
// is about two FP64 lanes a clock an SM, a warp instruction every 16 clocks,
// with 63 clocks of latency (measured), so in FP64 that sum alone took about
// 1 us a channel at 1M rows; F2 additions (eight FP32 operations) take a
// fraction of it with about 48 bits.  The F2
// range is FP32's: the FP32 flow's squared residual norms stay below 3.4e38
// (||f|| below about 1.8e19) or the step reports a non-finite residual.
template <bool MIXED>
using Part = typename std::conditional<MIXED, F2, double>::type;
__device__ __forceinline__ F2 part_add(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ double part_add(double a, double b) { return a + b; }
__device__ __forceinline__ double part_value(F2 a) { return f2_to_double(a); }
__device__ __forceinline__ double part_value(double a) { return a; }
template <typename PT>
__device__ __forceinline__ PT part_zero() {
    if constexpr (std::is_same<PT, F2>::value) {
        F2 z;
        z.hi = 0.0f;
        z.lo = 0.0f;
        return z;
    } else {
        return 0.0;
    }
}
template <typename PT>
__device__ __forceinline__ PT part_from(double x) {
    if constexpr (std::is_same<PT, F2>::value) {
        F2 z;
        z.hi = __double2float_rn(x);
        z.lo = __double2float_rn(x - (double)z.hi);
        return z;
    } else {
        return x;
    }
}
__device__ __forceinline__ F2 part_warp_sum(F2 v) { return warp_sum_f2(v); }
__device__ __forceinline__ double part_warp_sum(double v) { return warp_sum(v); }
__device__ __forceinline__ F2 part_load(const F2* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    F2 z;
    z.hi = v.x;
    z.lo = v.y;
    return z;
}
__device__ __forceinline__ double part_load(const double* p) { return __ldcg(p); }

// A warp's partials of its slice of a tile, channels 0 .. NCH-1 of every
// right-hand side, into out[ch * QT + q]: the FP32 (F2) products summed over
// the warp, plus the FP64 ones where there are any (`with64`).
template <bool MIXED, int QT, int NC, int NCH>
__device__ __forceinline__ void tile_partials(const F2 (&af)[NC][QT], const double (&ad)[NC][QT], bool with64,
                                              int lane, Part<MIXED>* out) {
    using PT = Part<MIXED>;
    constexpr int E = pow2_at_least(NCH * QT);
    double w64[NCH * QT];
#pragma unroll
    for (int e = 0; e < NCH * QT; e++) w64[e] = with64 ? warp_sum(ad[e / QT][e % QT]) : 0.0;
    if constexpr (MIXED && E > 32) {  // more values than lanes: one butterfly each
#pragma unroll
        for (int e = 0; e < NCH * QT; e++) {
            F2 x = warp_sum_f2(af[e / QT][e % QT]);
            if (with64) x = f2_add(x, part_from<F2>(w64[e]));
            if (lane == 0) out[e] = x;
        }
    } else if constexpr (MIXED) {
        constexpr int E32 = E > 32 ? 32 : E;
        F2 v[E32];
#pragma unroll
        for (int e = 0; e < E32; e++) {
            v[e].hi = 0.0f;
            v[e].lo = 0.0f;
            if (e < NCH * QT) v[e] = af[e / QT][e % QT];
        }
        int chan;
        const F2 tot = warp_sum_f2_multi<E32>(v, lane, chan);
        if ((lane & (32 / E32 - 1)) == 0 && chan < NCH * QT) {
            F2 x = tot;
            if (with64) {
                double w = 0.0;
#pragma unroll
                for (int e = 0; e < NCH * QT; e++)
                    if (e == chan) w = w64[e];
                x = f2_add(x, part_from<F2>(w));
            }
            out[chan] = x;
        }
    } else if (lane == 0) {
#pragma unroll
        for (int e = 0; e < NCH * QT; e++) out[e] = part_from<PT>(w64[e]);
    }
}

// Per-warp staging of operator slices.  A slice -- 32 rows' k column slots
// and k+1 weight slots, each 32 consecutive words in the sliced layout, so two
// contiguous runs -- arrives in the warp's shared memory by two bulk
// asynchronous copies issued by lane 0 and completing on one of the warp's
// mbarriers.  With two buffers the slice of the warp's next tile is requested
// before the current one is used, so the operator keeps streaming while the
// warp gathers and reduces.  The evict-first hint keeps the small, reused
// Krylov vectors in L2 while the operator streams past.
struct Stager {
    unsigned char* base;  // this warp's buffers
    uint32_t bytes;       // one buffer
    uint32_t val_off;     // where the weights start inside a buffer
    uint64_t* bar;        // [2] this warp's mbarriers
    uint64_t pol;
    uint32_t parity;      // bit b: parity of buffer b's next completion
    uint32_t busy;        // bit b: a copy into buffer b has not been waited for
    int nbuf;
    int next_c;           // tile whose slice was requested ahead (-1: none), in buffer next_b
    int next_b;
    bool ok;              // false once a copy missed its wait: nothing more is issued

    __device__ int* col(int b) const { return reinterpret_cast<int*>(base + b * bytes); }
    __device__ const void* val(int b) const { return base + b * bytes + val_off; }

    __device__ void issue(int b, const int32_t* colsrc, const void* valsrc, int esize, int k, int64_t slice) {
        __syncwarp();  // every lane has consumed what buffer b held
        if (!ok) return;  // after a missed wait the warp issues nothing more
        busy |= 1u << b;
        if (lane_id() == 0) {
            const uint32_t cb = (uint32_t)(kSlice * k * 4), vb = (uint32_t)(kSlice * (k + 1) * esize);
            mbar_expect_tx(&bar[b], cb + vb);
            bulk_g2s(col(b), colsrc + slice * (int64_t)(kSlice * k), cb, &bar[b], pol);
            bulk_g2s(base + b * bytes + val_off,
                     static_cast<const char*>(valsrc) + slice * (int64_t)(kSlice * (k + 1)) * esize, vb, &bar[b],
                     pol);
        }
    }

    // The buffer holding tile c's slice: requested now unless it was requested
    // ahead; then, with two buffers, requests tile c2's slice ahead (c2 < 0: none).
    __device__ int acquire(int c, int64_t slice, int c2, int64_t slice2, const int32_t* colsrc, const void* valsrc,
                           int esize, int k, int* err) {
        if (next_c >= 0 && next_c != c) {  // a slice requested ahead for a tile not taken: let it land first
            wait(next_b, err);
            next_c = -1;
        }
        int b;
        if (next_c == c) {
            b = next_b;
        } else {
            b = (busy & 1u) ? 1 : 0;
            issue(b, colsrc, valsrc, esize, k, slice);
        }
        next_c = -1;
        if (nbuf == 2 && c2 >= 0) {
            next_b = b ^ 1;
            next_c = c2;
            issue(next_b, colsrc, valsrc, esize, k, slice2);
        }
        return b;
    }

    // Warp-collective bounded wait for buffer b.  A copy that missed its wait
    // stays marked busy with its parity unchanged, so drain() waits for it
    // again before the block's shared memory is released.
    __device__ bool wait(int b, int* err) {
        if (!ok) return false;  // nothing was issued since the first miss
        const bool landed = __all_sync(0xffffffffu, mbar_wait(&bar[b], (parity >> b) & 1u, kStageWaitLimit));
        if (landed) {
            parity ^= 1u << b;
            busy &= ~(1u << b);
        } else {
            ok = false;
            if (lane_id() == 0) atomicCAS(err, 0, (int)MVGD_ETIMEOUT);
        }
        return ok;
    }

    // Before the block's shared memory goes away: bounded waits for every copy
    // still in flight (landed or not, each buffer's wait ends within its limit).
    __device__ void drain() {
        for (int b = 0; b < 2; b++)
            if (busy & (1u << b)) mbar_wait(&bar[b], (parity >> b) & 1u, kStageWaitLimit);
    }
};

// A / B for INNER right-hand sides: one operator application each, reading
// the row's columns and weights from the warp's staged slice.  Called by every
// lane of a staged warp (`valid`: the lane's row exists); the row's own loads
// are issued before `landed()` waits for the slice, so they overlap the copy.
template <bool MIXED, int QT, typename Landed>
__device__ __forceinline__ void spmv_row(const Prob& P, int64_t r, bool valid, int ph, const RhsState* S,
                                         const bool (&on)[QT], const float (&c1)[QT], const float (&c2)[QT],
                                         F2 (&af)[kChan][QT], double (&ad)[kChan][QT], const int* colS,
                                         const typename std::conditional<MIXED, float, double>::type* valS,
                                         Landed&& landed) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q, k = P.k;
    const int lane = (int)(r % kSlice);
    const VT sig = (VT)P.sigma;
    const VT invd = (valid && P.precond) ? static_cast<const VT*>(P.invd)[r] : (VT)1;
    // vectors written by other blocks during this kernel: plain (coherent) loads
    const VT* R = static_cast<const VT*>(P.r);
    const VT* RH = static_cast<const VT*>(P.rh);
    const VT* src[QT];
    const VT* vold[QT];
    VT si[QT], acc[QT];
#pragma unroll
    for (int q = 0; q < QT; q++) {
        acc[q] = (VT)0;
        si[q] = (VT)0;
        src[q] = nullptr;
        vold[q] = nullptr;
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        if (MIXED) {
            vold[q] = static_cast<const VT*>(P.v[S[q].pp]);
            src[q] = static_cast<const VT*>(P.p[S[q].pp]);
            if (valid)
                si[q] = (ph == P_A) ? R[e] + (VT)c1[q] * (src[q][e] - (VT)c2[q] * vold[q][e])
                                    : R[e] - (VT)c1[q] * vold[q][e];
        } else {
            src[q] = static_cast<const VT*>(ph == P_A ? P.p[0] : P.s);
            if (valid) si[q] = src[q][e];
        }
    }
    if (!landed() || !valid) return;  // landed() is warp-collective: every lane calls it
    const VT w0 = valS[lane];
#pragma unroll 8
    for (int sl = 0; sl < k; sl++) {
        const int64_t j = colS[sl * kSlice + lane];
        const VT w = valS[(sl + 1) * kSlice + lane];
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q]) continue;
            const int64_t e = j * Q + q;
            if (MIXED) {
                const VT sj = (ph == P_A) ? R[e] + (VT)c1[q] * (src[q][e] - (VT)c2[q] * vold[q][e])
                                          : R[e] - (VT)c1[q] * vold[q][e];
                acc[q] = fmaf(w, sj - si[q], acc[q]);
            } else {
                acc[q] = fma(w, src[q][e], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        const VT lx = MIXED ? acc[q] : acc[q] + w0 * si[q];
        const VT res = invd * (sig * si[q] - lx);
        if (ph == P_A) {
            const int np = MIXED ? (S[q].pp ^ 1) : 0;
            if (MIXED) static_cast<VT*>(P.p[np])[e] = si[q];
            // the previous iteration reached a new best residual: keep its iterate
            if (MIXED && S[q].best_flag) static_cast<VT*>(P.xb)[e] = static_cast<const VT*>(P.x)[e];
            static_cast<VT*>(P.v[np])[e] = res;
            if (MIXED) f2_add_prod(af[0][q], (float)RH[e], (float)res);
            else ad[0][q] += (double)(RH[e] * res);
        } else {
            if (MIXED) static_cast<VT*>(P.s)[e] = si[q];
            static_cast<VT*>(P.t)[e] = res;
            if (MIXED) {
                f2_add_prod(af[0][q], (float)res, (float)si[q]);
                f2_add_prod(af[1][q], (float)res, (float)res);
            } else {
                ad[0][q] += (double)(res * si[q]);
                ad[1][q] += (double)(res * res);
            }
        }
    }
}

// RESTART steps: in A the FP64 true residual, in the step that ends the
// iteration (C of the row-scaled flows, B of the multigrid flow) the restart of
// the Krylov vectors.
template <bool MIXED, int QT, int NC>
__device__ __forceinline__ void restart_row(const Prob& P, int64_t r, int ph, const RhsState* S, const bool (&on)[QT],
                                            double (&ad)[NC][QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q, k = P.k, m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    if (ph == P_A) {
        double w0;
        if (MIXED) w0 = (double)static_cast<const float*>(P.val)[vb] + (double)P.val_lo[vb];
        else w0 = static_cast<const double*>(P.val)[vb];
        double acc[QT], ui[QT];
#pragma unroll
        for (int q = 0; q < QT; q++) {
            ui[q] = on[q] ? P.u[r * Q + q] : 0.0;
            acc[q] = w0 * ui[q];
        }
#pragma unroll 4
        for (int sl = 0; sl < k; sl++) {
            const int64_t j = P.col[cb + (int64_t)sl * kSlice];
            const int64_t e = vb + (int64_t)(sl + 1) * kSlice;
            double w;
            if (MIXED) w = (double)static_cast<const float*>(P.val)[e] + (double)P.val_lo[e];
            else w = static_cast<const double*>(P.val)[e];
#pragma unroll
            for (int q = 0; q < QT; q++)
                if (on[q]) acc[q] = fma(w, P.u[j * Q + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q]) continue;
            const int64_t e = r * Q + q;
            const double fv = P.f[e];
            const double res = fv - (P.sigma * ui[q] - acc[q]);
            P.r64[e] = res;
            ad[0][q] += res * res;
            ad[1][q] += fv * fv;
        }
        return;
    }
    // the iteration's last step: restart the Krylov vectors
    const double invd = P.precond ? (double)static_cast<const VT*>(P.invd)[r] : 1.0;
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        double rv = invd * P.r64[e];
        if (MIXED) rv /= S[q].scale;
        const VT rr = (VT)rv;
        static_cast<VT*>(P.r)[e] = rr;
        // shadow residual: r itself; after a refinement step that did not lower the
        // residual, a deterministic relative perturbation of up to +-50% sends the
        // retry down a different Krylov path ((rh, r) stays positive)
        VT rhv = rr;
        if (S[q].stall > 0) {
            uint32_t hsh = (uint32_t)e * 2654435761u ^ (uint32_t)S[q].outer * 40503u;
            hsh ^= hsh >> 16; hsh *= 0x7feb352du; hsh ^= hsh >> 15; hsh *= 0x846ca68bu; hsh ^= hsh >> 16;
            const double u01 = (double)hsh * (1.0 / 4294967296.0);
            rhv = (VT)(rv * (1.0 + (u01 - 0.5)));
        }
        static_cast<VT*>(P.rh)[e] = rhv;
        static_cast<VT*>(P.p[0])[e] = (VT)0;
        static_cast<VT*>(P.v[0])[e] = (VT)0;
        if (MIXED) {
            static_cast<VT*>(P.p[1])[e] = (VT)0;
            static_cast<VT*>(P.v[1])[e] = (VT)0;
            static_cast<VT*>(P.x)[e] = (VT)0;
            static_cast<VT*>(P.xb)[e] = (VT)0;
        }
        ad[0][q] += (double)rr * (double)rr;
    }
}

// ------------------------------------------------------------------------------
// Multigrid-preconditioned flow (precond == 2).  Right preconditioning:
//   p = r + beta (p - omega v);  ph = M^-1 p;  v = A ph;  alpha = rho / (rh, v)
//   s = r - alpha v;             sh = M^-1 s;  t = A sh;  omega = (t, s) / (t, t)
//   x += alpha ph + omega sh;    r = s - omega t
// with M^-1 one V-cycle.  p and s are materialised (the cycle reads them at
// other rows), with their pre-smoothed FP32 copies y_0 = d_0 p for level 0.
// An iteration has six grid steps, PRE_A, (cycle), A, PRE_B, (cycle), B: the
// new residual's two dot products follow from those of s and t,
//   (rh, r) = (rh, s) - omega (rh, t),
//   (r, r)  = (s, s) - 2 omega (t, s) + omega^2 (t, t),
// so B takes all five and r = s - omega t is formed by the next PRE_A, row by
// row, with no step (and no grid barrier) of its own.
// ------------------------------------------------------------------------------
template <bool MIXED, int QT>
__device__ __forceinline__ void amg_pre_row(const Prob& P, int64_t r, int ph, const RhsState* S,
                                            const bool (&inner)[QT], const bool (&restart)[QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q;
    const float d0 = P.amg->lv[0].dinv[r];
    VT* pv = static_cast<VT*>(P.p[0]);
    const VT* vv = static_cast<const VT*>(P.v[0]);
    VT* rv = static_cast<VT*>(P.r);
#pragma unroll
    for (int q = 0; q < QT; q++) {
        const int64_t e = r * Q + q;
        if (q >= Q) break;
        if (ph == P_PRE_A) {
            VT rn = (VT)0;
            if (S[q].pending) {
                // the last iteration's step (alpha, omega still hold its values): its
                // residual r = s - omega t and its iterate x += alpha ph + omega sh
                const VT om = (VT)S[q].omega;
                rn = static_cast<const VT*>(P.s)[e] - om * static_cast<const VT*>(P.t)[e];
                rv[e] = rn;
                VT* X = static_cast<VT*>(P.x);
                X[e] = X[e] + (VT)S[q].alpha * static_cast<const VT*>(P.ph)[e] + om * static_cast<const VT*>(P.sh)[e];
            }
            if (MIXED && restart[q] && S[q].outer > 0 && !S[q].discard)
                P.u[e] += S[q].scale * (double)static_cast<const VT*>(S[q].fold_best ? P.xb : P.x)[e];
            if (inner[q]) {
                if (!S[q].pending) rn = rv[e];
                const VT nv = rn + (VT)S[q].beta * (pv[e] - (VT)S[q].omega * vv[e]);
                pv[e] = nv;
                P.vy[0][e] = d0 * (float)nv;
            }
        } else if (inner[q]) {
            const VT nv = rv[e] - (VT)S[q].alpha * vv[e];
            static_cast<VT*>(P.s)[e] = nv;
            P.vy[0][e] = d0 * (float)nv;
        }
    }
}

// PRE_A / PRE_B of NT rows at once (rows r[k], k < n, of up to NT tiles of one
// request; `ok[k]`: the row exists), for right-hand sides that are INNER or
// have a pending step (no RESTART in the request: its fold goes row by row).
// Every operand of every row is loaded before any is used, so a block's tiles
// cost one memory round trip a group instead of one a tile; each row's
// arithmetic is that of amg_pre_row.
template <bool MIXED, int QT, int NT>
__device__ __forceinline__ void amg_pre_rows(const Prob& P, const int64_t (&r)[NT], const bool (&ok)[NT], int ph,
                                             const RhsState* S, const bool (&inner)[QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q;
    const float* dinv = P.amg->lv[0].dinv;
    VT* pv = static_cast<VT*>(P.p[0]);
    const VT* vv = static_cast<const VT*>(P.v[0]);
    VT* rv = static_cast<VT*>(P.r);
    // PRE_A: a = s, b = t, x, h1 = ph, h2 = sh (a pending step) or a = r; c = p, w = v.
    // PRE_B: a = r, w = v.
    float d0[NT];
    VT a[NT][QT], b[NT][QT], c[NT][QT], w[NT][QT], x[NT][QT], h1[NT][QT], h2[NT][QT];
#pragma unroll
    for (int k = 0; k < NT; k++) {
        d0[k] = ok[k] ? dinv[r[k]] : 0.0f;
#pragma unroll
        for (int q = 0; q < QT; q++) {
            a[k][q] = b[k][q] = c[k][q] = w[k][q] = x[k][q] = h1[k][q] = h2[k][q] = (VT)0;
            if (!ok[k] || q >= Q) continue;
            const int64_t e = r[k] * Q + q;
            if (ph == P_PRE_A && S[q].pending) {
                a[k][q] = static_cast<const VT*>(P.s)[e];
                b[k][q] = static_cast<const VT*>(P.t)[e];
                x[k][q] = static_cast<const VT*>(P.x)[e];
                h1[k][q] = static_cast<const VT*>(P.ph)[e];
                h2[k][q] = static_cast<const VT*>(P.sh)[e];
            } else if (inner[q]) {
                a[k][q] = rv[e];
            }
            if (inner[q]) {
                w[k][q] = vv[e];
                if (ph == P_PRE_A) c[k][q] = pv[e];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NT; k++) {
        if (!ok[k]) continue;
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (q >= Q) break;
            const int64_t e = r[k] * Q + q;
            if (ph == P_PRE_A) {
                VT rn = a[k][q];
                if (S[q].pending) {
                    const VT om = (VT)S[q].omega;
                    rn = a[k][q] - om * b[k][q];
                    rv[e] = rn;
                    static_cast<VT*>(P.x)[e] = x[k][q] + (VT)S[q].alpha * h1[k][q] + om * h2[k][q];
                }
                if (inner[q]) {
                    const VT nv = rn + (VT)S[q].beta * (c[k][q] - (VT)S[q].omega * w[k][q]);
                    pv[e] = nv;
                    P.vy[0][e] = d0[k] * (float)nv;
                }
            } else if (inner[q]) {
                const VT nv = a[k][q] - (VT)S[q].alpha * w[k][q];
                static_cast<VT*>(P.s)[e] = nv;
                P.vy[0][e] = d0[k] * (float)nv;
            }
        }
    }
}

// A: v = A ph and (rh, v); B: t = A sh and (t, s), (t, t), (rh, s), (rh, t),
// (s, s); from the staged slice (every lane of the warp calls).
template <bool MIXED, int QT, typename Landed>
__device__ __forceinline__ void amg_spmv_row(const Prob& P, int64_t r, bool valid, int ph, const RhsState* S,
                                             const bool (&on)[QT], F2 (&af)[kChanAmg][QT],
                                             double (&ad)[kChanAmg][QT], const int* colS,
                                             const typename std::conditional<MIXED, float, double>::type* valS,
                                             Landed&& landed) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q, k = P.k;
    const int lane = (int)(r % kSlice);
    const VT sig = (VT)P.sigma;
    const VT* src = static_cast<const VT*>(ph == P_A ? P.ph : P.sh);
    VT si[QT], acc[QT];
#pragma unroll
    for (int q = 0; q < QT; q++) {
        acc[q] = (VT)0;
        si[q] = (on[q] && valid) ? src[r * Q + q] : (VT)0;
    }
    if (!landed() || !valid) return;  // warp-collective
    const VT w0 = valS[lane];
#pragma unroll 8
    for (int sl = 0; sl < k; sl++) {
        const int64_t j = colS[sl * kSlice + lane];
        const VT w = valS[(sl + 1) * kSlice + lane];
        VT xj[QT];
        load_row<QT>(src, j, Q, xj);  // every right-hand side of neighbour j at once
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q]) continue;
            // FP32: difference form (rows of L sum to zero), as in the plain flow
            if (MIXED) acc[q] = fmaf(w, xj[q] - si[q], acc[q]);
            else acc[q] = fma(w, xj[q], acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        const VT lx = MIXED ? acc[q] : acc[q] + w0 * si[q];
        const VT res = sig * si[q] - lx;
        const VT rhv = static_cast<const VT*>(P.rh)[e];
        if (ph == P_A) {
            static_cast<VT*>(P.v[0])[e] = res;
            if (MIXED && S[q].best_flag) static_cast<VT*>(P.xb)[e] = static_cast<const VT*>(P.x)[e];
            if (MIXED) f2_add_prod(af[0][q], (float)rhv, (float)res);
            else ad[0][q] += (double)(rhv * res);
        } else {
            static_cast<VT*>(P.t)[e] = res;
            const VT sv = static_cast<const VT*>(P.s)[e];
            if (MIXED) {
                f2_add_prod(af[0][q], (float)res, (float)sv);
                f2_add_prod(af[1][q], (float)res, (float)res);
                f2_add_prod(af[2][q], (float)rhv, (float)sv);
                f2_add_prod(af[3][q], (float)rhv, (float)res);
                f2_add_prod(af[4][q], (float)sv, (float)sv);
            } else {
                ad[0][q] += (double)(res * sv);
                ad[1][q] += (double)(res * res);
                ad[2][q] += (double)(rhv * sv);
                ad[3][q] += (double)(rhv * res);
                ad[4][q] += (double)(sv * sv);
            }
        }
    }
}

// ------------------------------------------------------------------------------
// State transitions (run by the block that finishes a request's phase)
// ------------------------------------------------------------------------------
// c[] holds the step's reduced channels for this right-hand side.  The step
// that ends an iteration is C in the row-scaled flows and B in the multigrid
// flow, whose B also yields the new residual's (rh, r) and (r, r).
template <bool MIXED, bool AMG>
__device__ void advance(const Prob& P, int ph, RhsState& T, const double* c, const Ctl& ctl) {
    const int ph_end = AMG ? P_B : P_C;
    if (ph == P_A) T.pending = 0;  // applied by PRE_A of this iteration
    switch (T.mode) {
        case M_INNER:
            if (ph == P_A) {
                const double a = c[0];
                if (MIXED) T.pp ^= 1;
                if (!(fabs(a) > 0.0) || !isfinite(a)) T.mode = M_SKIP;
                else T.alpha = T.rho / a;
            } else if (ph == P_B || ph == P_C) {
                double a = c[0], b = c[1];  // C: (rh, r) and (r, r)
                if (ph == P_B) {
                    T.omega = (b > 0.0 && isfinite(a) && isfinite(b)) ? a / b : 0.0;
                    if (!AMG) break;
                    const double om = T.omega, ts = a, tt = b;
                    a = c[2] - om * c[3];
                    b = c[4] - 2.0 * om * ts + om * om * tt;
                    if (b < 0.0) b = 0.0;  // rounding of a near-cancellation
                }
                T.iters++;
                T.inner_iters++;
                const double rn = sqrt(b);
                T.rnorm = rn;
                const bool finite = isfinite(rn) && isfinite(a);
                // multigrid flow: x moves by this step only if it stayed finite
                T.pending = finite ? 1 : 0;
                // FP32 path: remember the iterate with the smallest residual; an
                // inner solve that stagnates or starts to diverge ends there and
                // hands back that best iterate instead of its last one
                const bool improved = finite && rn < T.rmin;
                if (improved) {
                    T.since_best = (rn < 0.99 * T.rmin) ? 0 : T.since_best + 1;
                    T.rmin = rn;
                } else {
                    T.since_best++;
                }
                T.best_flag = improved ? 1 : 0;
                const bool diverging = MIXED && finite && rn > 1e4 * T.rmin;
                const bool stagnating = MIXED && T.since_best > 200 && 2 * T.since_best > T.inner_iters;
                bool restart = !finite || diverging || stagnating || rn <= T.target || T.iters >= P.maxit ||
                               T.omega == 0.0 || a == 0.0 || (MIXED && T.inner_iters >= P.inner_maxit);
                if (restart) {
                    // x_best only ever holds finite iterates with smaller residuals (or
                    // the zero start), so folding it is always safe
                    T.discard = 0;
                    T.fold_best = improved ? 0 : 1;  // the current iterate is the best one iff it just improved
                    T.best_flag = 0;
                    T.mode = M_RESTART;
                    atomicAdd(ctl.nrestart, 1);
                } else {
                    T.beta = (a / T.rho) * (T.alpha / T.omega);
                    T.rho = a;
                }
            }
            break;
        case M_SKIP:
            if (ph == ph_end) {
                T.mode = M_RESTART;
                T.discard = 0;
                atomicAdd(ctl.nrestart, 1);
            }
            break;
        case M_RESTART:
            if (ph == P_A) {
                const double a = c[0], b = c[1];
                if (T.fnorm < 0) {
                    const double fn = sqrt(b);
                    T.fnorm = fn > 0 ? fn : 1.0;
                }
                const double rn = sqrt(a);
                const double rel = rn / T.fnorm;
                if (T.outer > 0 && !(rel < T.relres)) T.stall++;
                else T.stall = 0;
                T.relres = rel;
                if (!isfinite(rn)) {
                    T.mode = M_DONE;
                    T.status = MVGD_ENONFINITE;
                } else if (rel <= P.rtol) {
                    T.mode = M_DONE;
                    T.status = MVGD_OK;
                } else if (T.iters >= P.maxit) {
                    T.mode = M_DONE;
                    T.status = MVGD_ENOCONV;
                } else if (T.outer >= P.max_outer || T.stall >= 4) {
                    T.mode = M_DONE;
                    T.status = MVGD_EBREAKDOWN;
                } else {
                    T.scale = rn;
                }
                if (T.mode == M_DONE) {
                    atomicSub(ctl.active, 1);
                    atomicSub(ctl.nrestart, 1);
                }
            } else if (ph == ph_end) {
                const double a = c[0];
                const double rn = sqrt(a);
                T.rho = a;
                T.alpha = 1.0;
                T.omega = 1.0;
                T.beta = 0.0;
                T.pp = 0;
                T.rmin = rn;
                T.rnorm = rn;
                double red = 0.5 * P.rtol / T.relres;
                if (MIXED) red = fmax(P.inner_rtol, red);
                T.target = red * rn;
                T.outer++;
                T.inner_iters = 0;
                T.discard = 0;
                T.best_flag = 0;
                T.fold_best = 0;
                T.since_best = 0;
                T.mode = M_INNER;
                atomicSub(ctl.nrestart, 1);
            }
            break;
        default:
            break;
    }
}

// Work units of one kind of step: unit c belongs to request chunk_req[c] and
// is its unit c - chunk_base[request].
struct ChunkTable {
    const int* chunk_req;   // [nchunks]
    const int* chunk_base;  // [count]
    int nchunks, pad;
};

struct ReqTable {
    const Prob* const* prob;       // [count]
    ChunkTable fine;               // kCh-row tiles of level 0 (every Krylov phase; V-cycle level 0)
    ChunkTable lvl[kAmgMaxLevels]; // [l], 1 <= l < mlev: kThreads / amg_group(n_l)-row units of level l
    ChunkTable coarse;             // 8-row groups (a warp each) of every coarsest level
    int mlev;                      // largest (levels - 1) among the requests
    int nreq;                      // requests in the launch (1: every unit is request 0's, no lookups)
    int G[kAmgMaxLevels];          // [l], l >= 1: amg_group of the launch's rows at level l (see amg_lanes)
};

// Request of unit c of table T, and the unit's place in that request.
__device__ __forceinline__ int unit_req(const ReqTable& tab, const ChunkTable& T, int c) {
    return tab.nreq == 1 ? 0 : T.chunk_req[c];
}
__device__ __forceinline__ int unit_base(const ReqTable& tab, const ChunkTable& T, int ri) {
    return tab.nreq == 1 ? 0 : T.chunk_base[ri];
}

template <typename VT>
__host__ __device__ constexpr size_t stage_bytes_per_warp(int kmax) {
    return (size_t)kSlice * kmax * sizeof(int) + (size_t)kSlice * (kmax + 1) * sizeof(VT);
}

// This block has finished `cnt` tiles of request P in a reducing phase: publish
// them (one fence and one atomic per block and request), and if they were the
// request's last tiles, sum all its tile partials and advance the per-RHS state.
// The sum's order depends on the tile count alone: thread t takes tiles t,
// t + 256, ... in batches of kFinBatch whose loads are all issued before any
// is added, each batch summed as a balanced pairwise tree, the batches in
// order; then a butterfly over the warp and a pairwise tree over the 8 warps.
// The dependent chain is log-depth and costs one L2 round trip a batch; the
// additions are F2 in the FP32 flow (see Part).
template <bool MIXED, int QT, bool AMG>
__device__ __forceinline__ void arrive_and_finalize(const Prob& P, int ph, int slot, int cnt, const RhsState* S,
                                                    Part<MIXED> (&fin)[kThreads / 32][chan_count(AMG) * QT],
                                                    double (&tot)[chan_count(AMG) * QT], int* last, const Ctl& ctl) {
    constexpr int NC = chan_count(AMG);
    using PT = Part<MIXED>;
    const int nch = (AMG && ph == P_B) ? kChanAmg : kChan;  // the channels this step reduces
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // the block's partial stores precede the barrier; thread 0's fence releases
    // them (cumulatively) with the arrival, and on the last arrival its second
    // fence orders every block's partials before the loads below
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const bool lst = atomicAdd(&P.arrive[slot], (unsigned)cnt) + (unsigned)cnt == (unsigned)P.nchunk;
        if (lst) __threadfence();
        *last = lst;
    }
    __syncthreads();
    if (*last) {
        constexpr int kFinBatch = (QT == 1 && !MIXED) ? 16 : 8;
        const int nchunk = P.nchunk, Q = P.Q;
        // two channels (or right-hand sides) at a time: 2 x kFinBatch loads in flight
#pragma unroll
        for (int e0 = 0; e0 < NC * QT; e0 += 2) {
            const int e1 = e0 + 1;
            const bool on0 = e0 / QT < nch && e0 % QT < Q;                   // step-uniform
            const bool on1 = e1 < NC * QT && e1 / QT < nch && e1 % QT < Q;  // step-uniform
            PT acc0 = part_zero<PT>(), acc1 = part_zero<PT>();
            if (on0 || on1) {
                const PT* part = static_cast<const PT*>(P.part);
                const PT* b0 = &part[((int64_t)slot * NC + e0 / QT) * nchunk * Q + e0 % QT];
                const PT* b1 = &part[((int64_t)slot * NC + e1 / QT) * nchunk * Q + e1 % QT];
                for (int l0 = tid; l0 < nchunk; l0 += kThreads * kFinBatch) {
                    PT v0[kFinBatch], v1[kFinBatch];
#pragma unroll
                    for (int u = 0; u < kFinBatch; u++) {
                        const int l = l0 + u * kThreads;
                        v0[u] = on0 && l < nchunk ? part_load(b0 + (int64_t)l * Q) : part_zero<PT>();
                        v1[u] = on1 && l < nchunk ? part_load(b1 + (int64_t)l * Q) : part_zero<PT>();
                    }
#pragma unroll
                    for (int w = 1; w < kFinBatch; w <<= 1)
#pragma unroll
                        for (int u = 0; u < kFinBatch; u += 2 * w) {
                            v0[u] = part_add(v0[u], v0[u + w]);
                            v1[u] = part_add(v1[u], v1[u + w]);
                        }
                    acc0 = part_add(acc0, v0[0]);
                    acc1 = part_add(acc1, v1[0]);
                }
            }
            if (on0) acc0 = part_warp_sum(acc0);
            if (on1) acc1 = part_warp_sum(acc1);
            if (lane == 0) {
                fin[wid][e0] = acc0;
                if (e1 < NC * QT) fin[wid][e1] = acc1;
            }
        }
        __syncthreads();
        static_assert(kThreads / 32 == 8, "the warp tree below sums 8 warps");
        if (tid < NC * QT) {
            const PT* f = &fin[0][tid];
            constexpr int W = NC * QT;
            tot[tid] = part_value(part_add(part_add(part_add(f[0], f[W]), part_add(f[2 * W], f[3 * W])),
                                           part_add(part_add(f[4 * W], f[5 * W]), part_add(f[6 * W], f[7 * W]))));
        }
        __syncthreads();
        if (tid < P.Q) {
            RhsState T = S[tid];
            double cv[NC];
#pragma unroll
            for (int ch = 0; ch < NC; ch++) cv[ch] = tot[ch * QT + tid];
            advance<MIXED, AMG>(P, ph, T, cv, ctl);
            P.st[tid] = T;
        }
        // the grid barrier that ends this phase releases the new states and the
        // reset counter before any block reads them
        if (tid == 0) P.arrive[slot] = 0;
    }
    __syncthreads();
}

enum VStep : int { V_DOWN = 0, V_COARSE = 1, V_UP = 2 };

// The tile this block takes after tile c in a step over table T, if it is
// request ri's and this warp's slice of it holds rows (its slice in *slice2);
// else -1.  Such a tile is staged exactly like tile c, so its slice can be
// requested ahead.
__device__ __forceinline__ int next_tile(const ReqTable& tab, const ChunkTable& T, int c, int ri, int64_t nrows,
                                         int wid, int64_t& slice2) {
    const int c2 = c + (int)gridDim.x;
    if (c2 >= T.nchunks || unit_req(tab, T, c2) != ri) return -1;
    slice2 = (int64_t)(c2 - unit_base(tab, T, ri)) * (kCh / kSlice) + wid;
    return slice2 * kSlice < nrows ? c2 : -1;
}

template <bool MIXED, int QT, bool AMG>
__global__ void __launch_bounds__(kThreads, QT <= 2 ? 3 : 2)
    k_solve(ReqTable tab, Ctl ctl, int iter_budget, int kmax, int nbuf) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char stage_smem[];
    __shared__ RhsState S[QT];
    __shared__ __align__(16) Prob sP;
    __shared__ __align__(16) AmgHeader sH;
    static_assert(sizeof(Prob) % 8 == 0 && sizeof(AmgHeader) % 8 == 0, "descriptors are copied in 8-byte words");
    // per-warp partials of the block's pending tiles, summed into tile partials
    // (in warp order) only when kRedTiles are pending or the request changes:
    // the warps of a block do not wait for each other tile by tile
    constexpr int NC = chan_count(AMG);
    // about 5 KB of pending partials at most
    constexpr int kRedTiles = 80 / (NC * QT) > 16 ? 16 : (80 / (NC * QT) < 2 ? 2 : 80 / (NC * QT));
    __shared__ Part<MIXED> red[kRedTiles][kThreads / 32][NC * QT];
    __shared__ int red_lc[kRedTiles];
    __shared__ Part<MIXED> fin[kThreads / 32][NC * QT];
    __shared__ double tot[NC * QT];
    __shared__ int last;
    __shared__ float vagg[kThreads / kAmgAgg];  // a block's row residuals on a small level (agg_sum)
    __shared__ __align__(8) uint64_t stage_bar[kThreads / 32][2];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // this warp's nbuf slice buffers: kmax column slots, then kmax + 1 weight slots each
    Stager st;
    st.bytes = (uint32_t)stage_bytes_per_warp<VT>(kmax);
    st.val_off = (uint32_t)(kSlice * kmax * sizeof(int));
    st.base = stage_smem + (size_t)wid * nbuf * st.bytes;
    st.bar = stage_bar[wid];
    st.pol = 0;
    st.parity = 0;
    st.busy = 0;
    st.nbuf = nbuf;
    st.next_c = -1;
    st.next_b = 0;
    st.ok = true;
    if (lane == 0) {
        mbar_init(&st.bar[0], 1);
        mbar_init(&st.bar[1], 1);
        fence_mbar_init();
        st.pol = l2_evict_first_policy();
    }
    __syncthreads();

    bool inner[QT], restart[QT];
    bool any_inner = false, any_restart = false, all_done = true;
    float c1[QT], c2[QT];
    // the request whose state S holds, while no phase has advanced it since
    int held = -1;
    unsigned bar_epoch = 0;  // grid barriers passed (the same count in every block)
    // The descriptor (and multigrid header) of the request the block works on,
    // copied into shared memory when the request changes.  Each grid barrier's
    // acquire leaves none of them in L1, so read from global memory every step
    // would start with a chain of dependent L2 round trips (table -> descriptor
    // -> header -> level arrays) before the first row is touched.  Neither is
    // written while the solver runs.
    int desc = -1;
    auto load_desc = [&](int ri) {
        if (ri == desc) return;
        __syncthreads();  // every thread is done with the previous one
        const unsigned long long* gp = reinterpret_cast<const unsigned long long*>(tab.prob[ri]);
        for (int w = tid; w < (int)(sizeof(Prob) / 8); w += kThreads)
            reinterpret_cast<unsigned long long*>(&sP)[w] = __ldcg(gp + w);
        __syncthreads();
        if (AMG && sP.amg != nullptr) {
            const unsigned long long* gh = reinterpret_cast<const unsigned long long*>(sP.amg);
            for (int w = tid; w < (int)(sizeof(AmgHeader) / 8); w += kThreads)
                reinterpret_cast<unsigned long long*>(&sH)[w] = __ldcg(gh + w);
            __syncthreads();
            if (tid == 0) sP.amg = &sH;
            __syncthreads();
        }
        desc = ri;
    };
    // Loads request ri's per-RHS state into S (block-wide) and its masks.
    auto enter = [&](int ri, int ph) {
        held = ri;
        load_desc(ri);
        __syncthreads();
        const Prob& P = sP;
        // a K above the one the staging buffers were sized for (a wrong K in the
        // request list) would overrun shared memory, and a hierarchy of another
        // operator would be read out of bounds: do no work and end the launch
        bool fits = P.k <= kmax && ((P.amg != nullptr) == AMG);
        if (AMG && fits) fits = P.amg->n == P.n && P.amg->k == P.k;
        if (!fits && tid == 0) atomicCAS(ctl.err, 0, (int)MVGD_EINVAL);
        if (tid < QT) {
            if (tid < P.Q && fits) {
                load_state(S[tid], P.st + tid);
            } else {  // a slot past the request's RHS count: no work of any kind
                S[tid].mode = M_DONE;
                S[tid].pending = 0;
            }
        }
        __syncthreads();
        any_inner = any_restart = false;
        all_done = true;
#pragma unroll
        for (int q = 0; q < QT; q++) {
            const int md = S[q].mode;
            inner[q] = md == M_INNER;
            restart[q] = md == M_RESTART;
            any_inner |= inner[q];
            any_restart |= restart[q];
            all_done &= (md == M_DONE);
            c1[q] = (float)(ph == P_A ? S[q].beta : S[q].alpha);
            c2[q] = (float)S[q].omega;
        }
    };

    // One Krylov phase over every request's level-0 tiles, then the grid barrier.
    // the step that ends an iteration: it restarts the Krylov vectors of the
    // right-hand sides in RESTART and its barrier precedes the exit test
    constexpr int ph_end = AMG ? P_B : P_C;
    auto fine_phase = [&](int ph) -> bool {
        const bool reduce = ph == P_A || ph == P_B || ph == P_C;
        const int nch = (AMG && ph == P_B) ? kChanAmg : kChan;  // the channels this step reduces
        const int slot = red_slot(ph);
        int cur = -1, tiles = 0, nred = 0;
        // tile partials of the pending tiles of request P: each the sum of its 8 warp partials (a pairwise tree)
        auto flush = [&](const Prob& P) {
            __syncthreads();
            for (int e = tid; e < nred * NC * QT; e += kThreads) {
                const int t = e / (NC * QT), j = e % (NC * QT);
                if (j / QT >= nch) continue;
                const Part<MIXED>* rw = &red[t][0][j];
                constexpr int W = NC * QT;  // stride between warps
                const Part<MIXED> v = part_add(part_add(part_add(rw[0], rw[W]), part_add(rw[2 * W], rw[3 * W])),
                                               part_add(part_add(rw[4 * W], rw[5 * W]), part_add(rw[6 * W], rw[7 * W])));
                const int ch = j / QT, q = j % QT;
                if (q < P.Q)
                    static_cast<Part<MIXED>*>(P.part)[(((int64_t)slot * NC + ch) * P.nchunk + red_lc[t]) * P.Q + q] = v;
            }
            __syncthreads();
            nred = 0;
        };
        for (int c = blockIdx.x;; c += gridDim.x) {
            const int ri = c < tab.fine.nchunks ? unit_req(tab, tab.fine, c) : -1;
            if (ri != cur) {
                // leaving request `cur`: publish this block's tiles of it
                if (cur >= 0 && reduce && tiles > 0) {
                    flush(sP);  // still request cur's descriptor
                    arrive_and_finalize<MIXED, QT, AMG>(sP, ph, slot, tiles, S, fin, tot, &last, ctl);
                }
                if (ri < 0) break;
                cur = ri;
                tiles = 0;
                enter(ri, ph);
            }
            if (all_done) continue;  // the whole request is finished: no work, no arrival
            const Prob& P = sP;
            const int lc = c - unit_base(tab, tab.fine, ri);
            const int64_t r = (int64_t)lc * kCh + tid;
            const int64_t slice = (int64_t)lc * (kCh / kSlice) + wid;
            F2 af[NC][QT];
            double ad[NC][QT];
#pragma unroll
            for (int ch = 0; ch < NC; ch++)
#pragma unroll
                for (int q = 0; q < QT; q++) { af[ch][q].hi = 0.0f; af[ch][q].lo = 0.0f; ad[ch][q] = 0.0; }
            // warp-uniform: lane 0 stages the whole slice and every lane waits for it
            const bool staged = (ph == P_A || ph == P_B) && any_inner && slice * kSlice < P.n && st.ok;
            if (staged) {
                int64_t slice2 = 0;
                const int cn = next_tile(tab, tab.fine, c, ri, P.n, wid, slice2);
                // FP32 multigrid flow: the hierarchy's level-0 weights (the operator's hi
                // values, copied at set-up), the array the V-cycle's level-0 steps read too
                const void* vsrc = (AMG && MIXED) ? static_cast<const void*>(P.amg->lv[0].val) : P.val;
                const int b = st.acquire(c, slice, cn, slice2, P.col, vsrc, (int)sizeof(VT), P.k, ctl.err);
                const int* colS = st.col(b);
                const VT* valS = static_cast<const VT*>(st.val(b));
                auto landed = [&]() { return st.wait(b, ctl.err); };
                if constexpr (AMG) amg_spmv_row<MIXED, QT>(P, r, r < P.n, ph, S, inner, af, ad, colS, valS, landed);
                else spmv_row<MIXED, QT>(P, r, r < P.n, ph, S, inner, c1, c2, af, ad, colS, valS, landed);
            }
            if (r < P.n) {
                // a restart computes its residual in A and resets the Krylov vectors in
                // the iteration's last step, so that its first inner step starts at the
                // next iteration
                if (ph == P_A) {
                    if (any_restart) restart_row<MIXED, QT, NC>(P, r, ph, S, restart, ad);
                } else if (ph == ph_end) {
                    if constexpr (!AMG) {
                        if (any_inner) {
                            if (MIXED) elementwise_row<MIXED, QT>(P, r, ph, S, inner, restart, af);
                            else c_row_f64<QT>(P, r, S, inner, ad);
                        }
                    }
                    if (any_restart) restart_row<MIXED, QT, NC>(P, r, ph, S, restart, ad);
                } else if (ph != P_B) {
                    if constexpr (AMG) amg_pre_row<MIXED, QT>(P, r, ph, S, inner, restart);
                    else elementwise_row<MIXED, QT>(P, r, ph, S, inner, restart, af);
                }
            }
            if (!reduce) continue;
            // tile partials in a fixed order: FP32 partials within the warp in FP32,
            // then (at the next flush) the 8 warps in order
            {
                const bool with64 = any_restart || !MIXED;
                if constexpr (AMG) {
                    if (ph == P_B) tile_partials<MIXED, QT, NC, kChanAmg>(af, ad, with64, lane, red[nred][wid]);
                    else tile_partials<MIXED, QT, NC, kChan>(af, ad, with64, lane, red[nred][wid]);
                } else {
                    tile_partials<MIXED, QT, NC, kChan>(af, ad, with64, lane, red[nred][wid]);
                }
            }
            if (tid == 0) red_lc[nred] = lc;
            nred++;
            tiles++;
            if (nred == kRedTiles) flush(P);
        }
        // the stop word is written only before the last barrier of an iteration and
        // read only after it, so every block takes the same exit decision
        if (ph == ph_end && blockIdx.x == 0 && tid == 0 && ctl.cancel && *(const volatile int*)ctl.cancel != 0)
            *ctl.stop = 1;
        if (reduce) held = -1;  // the states were advanced at the arrivals
        const bool ok = grid_sync(ctl.bar, bar_epoch, ctl.err, ctl.limit,
                                  !(ctl.withhold && blockIdx.x == 0 && bar_epoch == 0));
        trace_step(ctl, (unsigned)ph);
        return ok;
    };

    // PRE_A / PRE_B of the multigrid flow with one or two right-hand sides:
    // up to NT of the block's tiles of one request at a time (amg_pre_rows), so
    // their loads overlap; a request with a RESTART goes row by row (the fold of
    // x into u).  The rows and their arithmetic are those of fine_phase.
    auto pre_phase = [&](int ph) -> bool {
        constexpr int NT = MIXED ? (QT == 1 ? 4 : 2) : (QT == 1 ? 2 : 1);  // operands in registers
        const int G = (int)gridDim.x;
        for (int c = blockIdx.x; c < tab.fine.nchunks;) {
            const int ri = unit_req(tab, tab.fine, c);
            if (ri != held) enter(ri, ph);
            int n = 1;
            while (n < NT && c + n * G < tab.fine.nchunks && unit_req(tab, tab.fine, c + n * G) == ri) n++;
            if (!all_done) {
                const Prob& P = sP;
                const int base = unit_base(tab, tab.fine, ri);
                if (any_restart) {
                    for (int k = 0; k < n; k++) {
                        const int64_t r = (int64_t)(c + k * G - base) * kCh + tid;
                        if (r < P.n) amg_pre_row<MIXED, QT>(P, r, ph, S, inner, restart);
                    }
                } else {
                    int64_t rows[NT];
                    bool ok[NT];
#pragma unroll
                    for (int k = 0; k < NT; k++) {
                        rows[k] = (int64_t)(c + k * G - base) * kCh + tid;
                        ok[k] = k < n && rows[k] < P.n;
                    }
                    amg_pre_rows<MIXED, QT, NT>(P, rows, ok, ph, S, inner);
                }
            }
            c += n * G;
        }
        const bool ok = grid_sync(ctl.bar, bar_epoch, ctl.err, ctl.limit,
                                  !(ctl.withhold && blockIdx.x == 0 && bar_epoch == 0));
        trace_step(ctl, (unsigned)ph);
        return ok;
    };

    // One step of the V-cycle applied to p (side 0) or s (side 1) of every
    // INNER right-hand side, then the grid barrier.
    auto vstep = [&](int kind, int l, int side) -> bool {
        const ChunkTable& T = kind == V_COARSE ? tab.coarse : (l == 0 ? tab.fine : tab.lvl[l]);
        int cur = -1;
        for (int c = blockIdx.x; c < T.nchunks; c += gridDim.x) {
            const int ri = unit_req(tab, T, c);
            if (ri != cur) {
                cur = ri;
                // V-cycle steps leave the states alone: the one loaded by the
                // preceding PRE phase (or step) stays valid
                if (ri != held) enter(ri, P_PRE_A);
            }
            const Prob& P = sP;
            const int m = P.amg_levels - 1;  // the request's coarsest level
            if (!any_inner || (kind != V_COARSE && l >= m)) continue;
            const AmgHeader& H = *P.amg;
            const int Q = P.Q;
            const int lc = c - unit_base(tab, T, ri);
            const VT* B0 = static_cast<const VT*>(side == 0 ? P.p[0] : P.s);
            VT* X0 = static_cast<VT*>(side == 0 ? P.ph : P.sh);
            if (kind == V_COARSE) {
                const int64_t rho = (int64_t)lc * (kThreads / kWarp) + wid;  // a warp per row
                if (rho >= H.nc) continue;
#pragma unroll
                for (int q = 0; q < QT; q++) {
                    if (!inner[q]) continue;
                    float x;
                    if (m == 0) x = coarse_row(H, rho, [&](int64_t cc) { return (float)B0[cc * Q + q]; });
                    else x = coarse_row(H, rho, [&](int64_t cc) { return P.vb[m][cc * Q + q]; });
                    if (lane == 0) {
                        if (m == 0) X0[rho * Q + q] = (VT)x;
                        else P.vx[m][rho * Q + q] = x;
                    }
                }
                continue;
            }
            const int64_t nl = H.lv[l].n;
            // level 0: a lane per row (staged slices); level >= 1: G lanes per row
            const int G = l == 0 ? 1 : amg_lanes(tab.G[l], nl, QT);
            const int64_t r = (int64_t)lc * (kThreads / G) + tid / G;
            const bool valid = r < nl;
            // whole warps past the level's end have nothing to do, except in a down
            // step whose aggregates span warps (G >= 8: block barriers in agg_sum)
            const bool warp_idle = (int64_t)lc * (kThreads / G) + (wid * kWarp) / G >= nl;
            if (warp_idle && (kind == V_UP || G < 8)) continue;
            // level 0 reads the operator's slice from a staged buffer, like A and B
            const int* colS = nullptr;
            const float* w0S = nullptr;
            int b = 0;
            if (l == 0) {
                if (!st.ok) continue;
                const int64_t slice = (int64_t)lc * (kCh / kSlice) + wid;
                int64_t slice2 = 0;
                const int cn = next_tile(tab, tab.fine, c, ri, nl, wid, slice2);
                b = st.acquire(c, slice, cn, slice2, P.col, H.lv[0].val, 4, P.k, ctl.err);
                colS = st.col(b);
                w0S = static_cast<const float*>(st.val(b));
            }
            const float sig = (float)P.sigma;
            const int k = P.k;
            auto a0 = [&](float xi, auto&& xv) {
                return l == 0 ? a0_row_staged(colS, w0S, lane, k, sig, xi, xv) : a0_row(H, r, xi, xv);
            };
            if (kind == V_DOWN) {
                float* Yn = (l + 1 < m) ? P.vy[l + 1] : nullptr;
                const float* Y = P.vy[l];
                float bi[QT], yi[QT];
#pragma unroll
                for (int q = 0; q < QT; q++) {  // the row's own values, loaded while the slice lands
                    bi[q] = (valid && inner[q]) ? (l == 0 ? (float)B0[r * Q + q] : P.vb[l][r * Q + q]) : 0.0f;
                    yi[q] = (valid && inner[q]) ? Y[r * Q + q] : 0.0f;
                }
                if (l == 0) {
                    // level 0: every right-hand side in one pass over the neighbours
                    if (!st.wait(b, ctl.err)) continue;
                    float ay[QT];
#pragma unroll
                    for (int q = 0; q < QT; q++) ay[q] = 0.0f;
                    if (valid)
                        a0_rows_staged<QT>(colS, w0S, lane, k, sig, yi, ay,
                                           [&](int64_t j, float (&x)[QT]) { load_row<QT>(Y, j, Q, x); });
#pragma unroll
                    for (int q = 0; q < QT; q++)
                        if (inner[q]) vdown_finish(H, 0, 1, r, valid, Q, q, bi[q] - ay[q], P.vr[0], P.vb[1], Yn, vagg);
                    continue;
                }
                // level >= 1: every right-hand side in one pass over the row's entries
                float ay[QT];
                al_rows<QT>(H.lv[l], r, valid, G, yi, [&](int64_t j, float (&x)[QT]) { load_row<QT>(Y, j, Q, x); },
                            ay);
#pragma unroll
                for (int q = 0; q < QT; q++) {
                    if (!inner[q]) continue;  // block-uniform
                    vdown_finish(H, l, G, r, valid, Q, q, bi[q] - ay[q], P.vr[l], P.vb[l + 1], Yn, vagg);
                }
            } else {
                const float* Xc = P.vx[l + 1];
                float yi[QT], rr[QT];
#pragma unroll
                for (int q = 0; q < QT; q++) {
                    yi[q] = (valid && inner[q]) ? P.vy[l][r * Q + q] : 0.0f;
                    rr[q] = (valid && inner[q]) ? P.vr[l][r * Q + q] : 0.0f;
                }
                if (l == 0) {
                    // level 0: x = y + x_c + d (r - A_0 P x_c), every right-hand side in one pass
                    if (!st.wait(b, ctl.err) || !valid) continue;
                    float xc[QT], apx[QT];
                    load_row<QT>(Xc, r / kAmgAgg, Q, xc);
                    a0_rows_staged<QT>(colS, w0S, lane, k, sig, xc, apx,
                                       [&](int64_t j, float (&x)[QT]) { load_row<QT>(Xc, j / kAmgAgg, Q, x); });
                    const float d0 = H.lv[0].dinv[r];
#pragma unroll
                    for (int q = 0; q < QT; q++)
                        if (inner[q]) X0[r * Q + q] = (VT)(yi[q] + xc[q] + d0 * (rr[q] - apx[q]));
                    continue;
                }
                if (!valid && G == 1) continue;
                // level >= 1: x = y + x_c + d (r - A_l P x_c), every right-hand side in one pass
                float xc[QT], apx[QT];
#pragma unroll
                for (int q = 0; q < QT; q++) xc[q] = 0.0f;
                if (valid) load_row<QT>(Xc, r / kAmgAgg, Q, xc);
                al_rows<QT>(H.lv[l], r, valid, G, xc,
                            [&](int64_t j, float (&x)[QT]) { load_row<QT>(Xc, j / kAmgAgg, Q, x); }, apx);
                if (!valid || (lane & (G - 1)) != 0) continue;
                const float dl = H.lv[l].dinv[r];
#pragma unroll
                for (int q = 0; q < QT; q++)
                    if (inner[q]) P.vx[l][r * Q + q] = yi[q] + xc[q] + dl * (rr[q] - apx[q]);
            }
        }
        const bool ok = grid_sync(ctl.bar, bar_epoch, ctl.err, ctl.limit,
                                  !(ctl.withhold && blockIdx.x == 0 && bar_epoch == 0));
        trace_step(ctl, 0x1000u | ((unsigned)side << 8) | ((unsigned)kind << 4) | (unsigned)l);
        return ok;
    };
    auto vcycle = [&](int side) -> bool {
        for (int l = 0; l < tab.mlev; l++)
            if (!vstep(V_DOWN, l, side)) return false;
        if (!vstep(V_COARSE, 0, side)) return false;
        for (int l = tab.mlev - 1; l >= 0; l--)
            if (!vstep(V_UP, l, side)) return false;
        return true;
    };

    for (int it = 0; it < iter_budget; ++it) {
        bool ok = true;
        if (AMG) {
            if constexpr (QT <= 2)
                ok = pre_phase(P_PRE_A) && vcycle(0) && fine_phase(P_A) && pre_phase(P_PRE_B) && vcycle(1) &&
                     fine_phase(P_B);
            else
                ok = fine_phase(P_PRE_A) && vcycle(0) && fine_phase(P_A) && fine_phase(P_PRE_B) && vcycle(1) &&
                     fine_phase(P_B);
        } else {
            // read after the last barrier of the previous iteration: identical in every block
            const bool pre_a = !MIXED || *(volatile int*)ctl.nrestart > 0;
            for (int ph = 0; ph < P_COUNT && ok; ++ph) {
                if (ph == P_PRE_A && !pre_a) continue;
                if (ph == P_PRE_B && MIXED) continue;
                ok = fine_phase(ph);
            }
        }
        if (!ok) break;  // error exit, after the drain below
        if (*(volatile int*)ctl.active == 0 || *(volatile int*)ctl.stop != 0) break;
    }
    // copies still landing (a missed wait): bounded waits before the block's
    // shared memory is released
    st.drain();
}

// ------------------------------------------------------------------------------
// Request workspace layout, set-up and tear-down
// ------------------------------------------------------------------------------
struct ReqLayout {
    Prob* prob;
    RhsState* st;
    double* part;
    unsigned* arrive;
    mvgd_solve_info* info;
    double* fs;
    double* us;
    double* r64;
    void* invd;
    void* vec[12];  // x r rh p0 p1 v0 v1 s t x_best ph sh
    int nlev;       // multigrid levels (precond == 2), else 0
    float* vy[kAmgMaxLevels];
    float* vr[kAmgMaxLevels];
    float* vb[kAmgMaxLevels];
    float* vx[kAmgMaxLevels];
    size_t bytes;
};

ReqLayout req_layout(void* ws, int64_t n, int Q, int prec, int precond) {
    ReqLayout L;
    memset(&L, 0, sizeof(L));
    Carver cv(ws);
    const int64_t nchunk = (n + kCh - 1) / kCh;
    const size_t vt = prec == MVGD_FP64 ? sizeof(double) : sizeof(float);
    L.prob = cv.take<Prob>(1);
    L.st = cv.take<RhsState>(Q);
    L.part = cv.take<double>(kRedSlots * chan_count(precond == 2) * nchunk * Q);
    L.arrive = cv.take<unsigned>(kRedSlots);
    L.info = cv.take<mvgd_solve_info>(Q);
    L.fs = cv.take<double>(n * Q);
    L.us = cv.take<double>(n * Q);
    L.r64 = cv.take<double>(n * Q);
    L.invd = cv.take<char>(vt * n);
    const int nvec = precond == 2 ? 12 : 10;
    for (int v = 0; v < nvec; v++) L.vec[v] = cv.take<char>(vt * n * Q);
    if (precond == 2) {
        int64_t sizes[kAmgMaxLevels];
        L.nlev = amg_levels(n, sizes);
        for (int l = 0; l < L.nlev; l++) {
            const int64_t m = n_padded(sizes[l]) * Q;
            L.vy[l] = cv.take<float>(m);
            L.vr[l] = cv.take<float>(m);
            if (l > 0) {
                L.vb[l] = cv.take<float>(m);
                L.vx[l] = cv.take<float>(m);
            }
        }
    }
    L.bytes = cv.used;
    return L;
}

// Chunk tables of one launch: level 0 (Krylov phases), levels 1 .. kAmgMaxLevels-1
// and the coarsest solves; each with its per-request first-unit array.
struct CtlLayout {
    unsigned* bar;
    int* words;     // err, active, nrestart, stop
    const Prob** prob;
    int* chunk_req[kAmgMaxLevels + 1];   // [0] fine, [l] level l, [kAmgMaxLevels] coarsest
    int* chunk_base[kAmgMaxLevels + 1];
    size_t bytes;
};

constexpr int kCoarseUnits = (kAmgCoarsest + kThreads / kWarp - 1) / (kThreads / kWarp);

CtlLayout ctl_layout(void* ws, int max_req, int64_t max_chunks) {
    CtlLayout C;
    memset(&C, 0, sizeof(C));
    Carver cv(ws);
    C.bar = cv.take<unsigned>(2);
    C.words = cv.take<int>(4);
    C.prob = cv.take<const Prob*>(max_req);
    for (int t = 0; t <= kAmgMaxLevels; t++) {
        // level l >= 1 of a request has n_l <= n / 8^l + 1 rows in ceil(n_l G / kThreads)
        // <= n_l / 8 + 1 units (G <= 32): over all requests at most
        // total_rows / 8^(l+1) + 2 count (one more per request kept as margin), and
        // total_rows <= kCh max_chunks
        const int64_t units = t == kAmgMaxLevels ? (int64_t)max_req * kCoarseUnits
                              : (t == 0 ? max_chunks : ((int64_t)kCh * max_chunks >> (3 * (t + 1))) + 3 * max_req);
        C.chunk_req[t] = cv.take<int>(units);
        C.chunk_base[t] = cv.take<int>(max_req);
    }
    C.bytes = cv.used;
    return C;
}

__global__ void k_request_init(Prob P, Prob* dst, int64_t n) {
    // Prob travels by value (kernel parameter), so set-up is capturable in a graph
    if (blockIdx.x == 0 && threadIdx.x == 0) *dst = P;
    if (blockIdx.x == 0 && threadIdx.x < P.Q) {
        RhsState T;
        T.rho = T.alpha = T.omega = 1.0;
        T.beta = 0.0;
        T.fnorm = -1.0;
        T.relres = 1.0;
        T.scale = 0.0;
        T.target = 0.0;
        T.rnorm = 0.0;
        T.rmin = 0.0;
        T.mode = M_RESTART;
        T.pp = 0;
        T.iters = T.inner_iters = T.outer = 0;
        T.status = MVGD_OK;
        T.discard = 0;
        T.stall = 0;
        T.best_flag = T.fold_best = T.since_best = T.pending = 0;
        P.st[threadIdx.x] = T;
    }
    if (blockIdx.x == 0 && threadIdx.x < kRedSlots) P.arrive[threadIdx.x] = 0;
}

// Left scaling of the Krylov system: d_r = sigma + sum_s |w_rs| over the row's
// FP64 (or hi + lo) weights.  Always positive, unlike sigma - w_self: rows of an
// MVGD operator on irregular samples need not be diagonally dominant, and a
// self weight near sigma would make the Jacobi divisor vanish.
__global__ void k_prep_scaling(Prob P) {
    const int k = P.k, m = k + 1;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < P.n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
        double d = fabs(P.sigma);
        for (int s = 0; s < m; s++) {
            const int64_t e = vb + (int64_t)s * kSlice;
            double w = P.prec == MVGD_FP64 ? static_cast<const double*>(P.val)[e]
                                           : (double)static_cast<const float*>(P.val)[e] + (double)P.val_lo[e];
            d += fabs(w);
        }
        const double inv = d > 0 ? 1.0 / d : 1.0;
        if (P.prec == MVGD_FP64) static_cast<double*>(P.invd)[r] = inv;
        else static_cast<float*>(P.invd)[r] = (float)inv;
    }
}

__global__ void k_gather_rows(const double* __restrict__ src, const int32_t* __restrict__ order, int64_t n, int Q,
                              double* __restrict__ dst, int zero) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * Q; e += (int64_t)gridDim.x * blockDim.x) {
        if (zero || src == nullptr) { dst[e] = 0.0; continue; }
        const int64_t r = e / Q, q = e % Q;
        const int64_t from = order ? (int64_t)order[r] : r;
        dst[e] = src[from * Q + q];
    }
}

__global__ void k_finish(const Prob* P, mvgd_solve_info* out) {
    const int q = threadIdx.x;
    if (q >= P->Q) return;
    RhsState T;
    load_state(T, P->st + q);
    mvgd_solve_info I;
    I.iters = T.iters;
    I.outer = T.outer;
    I.relres = T.relres;
    int s = T.status;
    if (T.mode != M_DONE && s == MVGD_OK) s = MVGD_ENOCONV;
    I.status = s;
    I.reserved = 0;
    out[q] = I;
}

__global__ void k_scatter_solution(const Prob* P, double* __restrict__ dst) {
    const int64_t n = P->n;
    const int Q = P->Q;
    const int32_t* order = P->order;
    const double* src = P->u;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * Q; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Q, q = e % Q;
        const int64_t to = order ? (int64_t)order[r] : r;
        dst[to * Q + q] = src[e];
    }
}

constexpr int kTableMax = 256;
struct TableArgs {
    const Prob* prob[kTableMax];
    int nchunk[kTableMax];
    int count;
    int first_chunk;
};

// Request and chunk tables from by-value parameters (capturable in a graph);
// the first group also resets the barrier and the control words.
__global__ void k_build_table(TableArgs A, int base, const Prob** prob, int* chunk_req, int* chunk_base,
                              unsigned* bar, int* words, int first_group) {
    __shared__ int start[kTableMax + 1];
    if (threadIdx.x == 0) {
        start[0] = A.first_chunk;
        for (int i = 0; i < A.count; i++) start[i + 1] = start[i] + A.nchunk[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < A.count; i += blockDim.x) {
        if (prob) prob[base + i] = A.prob[i];
        chunk_base[base + i] = start[i];
    }
    for (int i = 0; i < A.count; i++)
        for (int c = start[i] + threadIdx.x; c < start[i + 1]; c += blockDim.x) chunk_req[c] = base + i;
    if (first_group && threadIdx.x == 0) {
        bar[0] = 0;
        bar[1] = 0;
        words[0] = 0;  // err
        words[3] = 0;  // stop
    }
}

// Counts running and restarting right-hand sides of the listed requests.
__global__ void k_count_active(const Prob** prob, int count, int* words) {
    __shared__ int act, rst;
    if (threadIdx.x == 0) { act = 0; rst = 0; }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const Prob* P = prob[i];
        for (int q = 0; q < P->Q; q++) {
            const int md = __ldcg(&P->st[q].mode);
            if (md != M_DONE) atomicAdd(&act, 1);
            if (md == M_RESTART) atomicAdd(&rst, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        words[1] = act;
        words[2] = rst;
    }
}

// After a launch that a cancel word or a barrier time-out ended, mark the
// right-hand sides that did not finish.
__global__ void k_mark_exit(const Prob** prob, int count, const int* words) {
    const int err = words[0], stop = words[3];
    if (!err && !stop) return;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const Prob* P = prob[i];
        for (int q = 0; q < P->Q; q++)
            if (P->st[q].mode != M_DONE) P->st[q].status = err ? err : MVGD_ECANCELLED;
    }
}

// done[i] = 1 when every right-hand side of request i has finished.
__global__ void k_poll(TableArgs A, int32_t* done) {
    for (int i = threadIdx.x; i < A.count; i += blockDim.x) {
        const Prob* P = A.prob[i];
        int all = 1;
        for (int q = 0; q < P->Q; q++) all &= (__ldcg(&P->st[q].mode) == M_DONE);
        done[i] = all;
    }
}

// Slice buffers per warp.  One by default: a second buffer (the next tile's
// slice requested ahead) costs a resident block per SM, and on GB300 at 1M
// rows, K = 20, three single-buffered blocks ran the FP32 multigrid solve 8 %
// faster than two double-buffered ones (every step that is not a product
// loses the third block's latency hiding).  mvgd_set_launch_tuning selects two.
template <typename VT>
int stage_buffers(int kmax) {
    if (tuned_stage_buffers() == 2 && 2 * stage_bytes_per_warp<VT>(kmax) * (kThreads / kWarp) <= (112u << 10))
        return 2;
    return 1;
}

template <bool MIXED, int QT, bool AMG>
mvgd_status launch_solve(const ReqTable& tab, Ctl ctl, int budget, int kmax, cudaStream_t s) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    auto fn = k_solve<MIXED, QT, AMG>;
    int nbuf = stage_buffers<VT>(kmax);
    const size_t smem = stage_bytes_per_warp<VT>(kmax) * (kThreads / kWarp) * nbuf;
    int dev = 0, sms = 0, per_sm = 0;
    MVGD_CUDA_TRY(cudaGetDevice(&dev));
    MVGD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MVGD_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    MVGD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) return MVGD_ECUDA;
    const int want = tuned_solver_blocks_per_sm();
    if (want > 0 && want < per_sm) per_sm = want;
    int grid = sms * per_sm;
    if (grid > tab.fine.nchunks) grid = tab.fine.nchunks;
    ReqTable t = tab;
    void* args[] = {(void*)&t, (void*)&ctl, (void*)&budget, (void*)&kmax, (void*)&nbuf};
    MVGD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kThreads), args, smem, s));
    return MVGD_OK;
}

template <bool MIXED, bool AMG>
mvgd_status dispatch_q(int Q, const ReqTable& tab, Ctl ctl, int budget, int kmax, cudaStream_t s) {
    if (Q <= 1) return launch_solve<MIXED, 1, AMG>(tab, ctl, budget, kmax, s);
    if (Q <= 2) return launch_solve<MIXED, 2, AMG>(tab, ctl, budget, kmax, s);
    if (Q <= 4) return launch_solve<MIXED, 4, AMG>(tab, ctl, budget, kmax, s);
    return launch_solve<MIXED, 8, AMG>(tab, ctl, budget, kmax, s);
}

int gather_blocks(int64_t elems) {
    int64_t gb = (elems + 255) / 256;
    return (int)(gb > 8192 ? 8192 : (gb < 1 ? 1 : gb));
}

int64_t max_chunks_for(int count, int64_t total_rows) { return total_rows / kCh + count + 1; }

}  // namespace
}  // namespace mvgd

using namespace mvgd;

// ---------------------------------------------------------------------------------
// Requests
// ---------------------------------------------------------------------------------
MVGD_API size_t mvgd_request_workspace_bytes(int64_t n, int32_t k, int32_t nrhs, int32_t prec, int32_t precond) {
    (void)k;
    if (n <= 0 || nrhs < 1 || nrhs > 8 || precond < 0 || precond > 2) return 0;
    if (precond == 2 && amg_levels(n, nullptr) == 0) return 0;
    return req_layout(nullptr, n, nrhs, prec, precond).bytes;
}

MVGD_API mvgd_status mvgd_request_init(void* req_ws, size_t req_bytes, const mvgd_ell* L, int32_t nrhs, double sigma,
                                       const double* f, const double* u0, const mvgd_solve_opts* opts,
                                       mvgd_stream_t stream) {
    if (!req_ws || !L || !f || !opts || nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (L->n < 2 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK || !L->col || !L->val) return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!aligned(f) || !aligned(u0) || !aligned(req_ws) || !aligned(L->col) || !aligned(L->val) ||
        !aligned(L->val_lo) || !aligned(L->order))
        return MVGD_EINVAL;
    if (!(opts->rtol > 0) || opts->maxit < 1 || !(sigma == sigma)) return MVGD_EINVAL;
    if (opts->precond < 0 || opts->precond > 2) return MVGD_EINVAL;
    if (opts->precond == 2 && (!opts->amg || !aligned(opts->amg))) return MVGD_EINVAL;
    const bool mixed = L->prec == MVGD_FP32_REFINE;
    if (mixed && (opts->inner_maxit < 1 || !(opts->inner_rtol > 0) || opts->max_outer < 1)) return MVGD_EINVAL;
    const int64_t n = L->n;
    ReqLayout W = req_layout(req_ws, n, nrhs, L->prec, opts->precond);
    if (req_bytes < W.bytes) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int gb = gather_blocks(n * nrhs);
    k_gather_rows<<<gb, 256, 0, s>>>(f, L->order, n, nrhs, W.fs, 0);
    k_gather_rows<<<gb, 256, 0, s>>>(u0, L->order, n, nrhs, W.us, u0 == nullptr);
    Prob P;
    P.n = n;
    P.k = L->k;
    P.Q = nrhs;
    P.prec = L->prec;
    P.precond = opts->precond == 1 ? 1 : 0;
    P.sigma = sigma;
    P.col = L->col;
    P.val = L->val;
    P.val_lo = L->val_lo;
    P.order = L->order;
    P.f = W.fs;
    P.u = W.us;
    P.x = mixed ? W.vec[0] : (void*)W.us;
    P.xb = W.vec[9];
    P.r = W.vec[1];
    P.rh = W.vec[2];
    P.p[0] = W.vec[3];
    P.p[1] = W.vec[4];
    P.v[0] = W.vec[5];
    P.v[1] = W.vec[6];
    P.s = W.vec[7];
    P.t = W.vec[8];
    P.r64 = W.r64;
    P.invd = W.invd;
    P.st = W.st;
    P.part = W.part;
    P.arrive = W.arrive;
    P.nchunk = (int)((n + kCh - 1) / kCh);
    P.pad = 0;
    P.rtol = opts->rtol;
    P.inner_rtol = mixed ? opts->inner_rtol : 0.0;
    P.maxit = opts->maxit;
    P.inner_maxit = mixed ? opts->inner_maxit : opts->maxit;
    P.max_outer = mixed ? opts->max_outer : 1000;
    P.pad2 = 0;
    P.amg = opts->precond == 2 ? static_cast<const AmgHeader*>(opts->amg) : nullptr;
    P.amg_levels = W.nlev;
    P.pad3 = 0;
    P.ph = W.vec[10];
    P.sh = W.vec[11];
    for (int l = 0; l < kAmgMaxLevels; l++) {
        P.vy[l] = W.vy[l];
        P.vr[l] = W.vr[l];
        P.vb[l] = W.vb[l];
        P.vx[l] = W.vx[l];
    }
    k_request_init<<<1, 32, 0, s>>>(P, W.prob, n);
    if (P.precond) k_prep_scaling<<<gather_blocks(n), 256, 0, s>>>(P);
    return launch_status();
}

MVGD_API size_t mvgd_iterate_workspace_bytes(int32_t max_requests, int64_t max_total_rows) {
    if (max_requests < 1 || max_total_rows < 1) return 0;
    return ctl_layout(nullptr, max_requests, max_chunks_for(max_requests, max_total_rows)).bytes;
}

MVGD_API mvgd_status mvgd_iterate(const mvgd_request* reqs, int32_t count, int32_t prec, int32_t precond,
                                  int32_t max_iterations, const int32_t* cancel, void* ctl_ws, size_t ctl_bytes,
                                  mvgd_stream_t stream) {
    if (!reqs || count < 1 || count > kMaxReq || max_iterations < 0 || !ctl_ws) return MVGD_EINVAL;
    if (prec != MVGD_FP64 && prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (precond < 0 || precond > 2) return MVGD_EINVAL;
    const bool amg = precond == 2;
    int64_t total_rows = 0;
    int maxQ = 1, kmax = kMinK, mlev = 0;
    for (int i = 0; i < count; i++) {
        const mvgd_request& R = reqs[i];
        if (!R.workspace || !aligned(R.workspace) || R.n < 2 || R.n >= (1ll << 31) || R.nrhs < 1 || R.nrhs > 8 ||
            R.k < kMinK || R.k > kMaxK)
            return MVGD_EINVAL;
        total_rows += R.n;
        if (R.nrhs > maxQ) maxQ = R.nrhs;
        if (R.k > kmax) kmax = R.k;
        if (amg) {
            const int nl = amg_levels(R.n, nullptr);
            if (nl == 0) return MVGD_EINVAL;
            if (nl - 1 > mlev) mlev = nl - 1;
        }
    }
    if (!aligned(ctl_ws) || !aligned(cancel)) return MVGD_EINVAL;
    if (ctl_bytes < mvgd_iterate_workspace_bytes(count, total_rows)) return MVGD_EWORKSPACE;
    if (max_iterations == 0) return MVGD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    CtlLayout C = ctl_layout(ctl_ws, count, max_chunks_for(count, total_rows));
    ReqTable tab;
    memset(&tab, 0, sizeof(tab));
    tab.prob = C.prob;
    tab.mlev = mlev;
    tab.nreq = count;
    const int qt = maxQ <= 1 ? 1 : (maxQ <= 2 ? 2 : (maxQ <= 4 ? 4 : 8));  // the solver's right-hand-side width
    for (int l = 0; l < kAmgMaxLevels; l++) {
        int64_t rows = 0;
        for (int i = 0; amg && l > 0 && i < count; i++) {
            int64_t sizes[kAmgMaxLevels];
            const int nl = amg_levels(reqs[i].n, sizes);
            if (l < nl - 1) rows += sizes[l];
        }
        tab.G[l] = l == 0 || rows == 0 ? 1 : amg_group(rows);
    }
    // table t: 0 = level-0 tiles, 1 .. mlev-1 = level-t tiles, kAmgMaxLevels = coarsest rows by 8
    for (int t = 0; t <= kAmgMaxLevels; t++) {
        const bool coarse = t == kAmgMaxLevels;
        if (t > 0 && (!amg || (!coarse && t >= mlev))) continue;
        int units = 0;
        for (int g = 0; g < count; g += kTableMax) {
            TableArgs A;
            A.count = count - g < kTableMax ? count - g : kTableMax;
            A.first_chunk = units;
            for (int i = 0; i < A.count; i++) {
                const mvgd_request& R = reqs[g + i];
                A.prob[i] = reinterpret_cast<const Prob*>(R.workspace);  // the Prob record opens every workspace
                int64_t sizes[kAmgMaxLevels];
                const int nl = amg ? amg_levels(R.n, sizes) : 1;
                if (t == 0) A.nchunk[i] = (int)((R.n + kCh - 1) / kCh);
                else if (coarse) A.nchunk[i] = (int)((sizes[nl - 1] + kThreads / kWarp - 1) / (kThreads / kWarp));
                else if (t < nl - 1) {
                    const int64_t rows = kThreads / amg_lanes(tab.G[t], sizes[t], qt);  // rows per unit
                    A.nchunk[i] = (int)((sizes[t] + rows - 1) / rows);
                } else {
                    A.nchunk[i] = 0;
                }
                units += A.nchunk[i];
            }
            k_build_table<<<1, 256, 0, s>>>(A, g, t == 0 ? C.prob : nullptr, C.chunk_req[t], C.chunk_base[t], C.bar,
                                            C.words, t == 0 && g == 0);
        }
        ChunkTable& T = coarse ? tab.coarse : (t == 0 ? tab.fine : tab.lvl[t]);
        T.chunk_req = C.chunk_req[t];
        T.chunk_base = C.chunk_base[t];
        T.nchunks = units;
    }
    k_count_active<<<1, 256, 0, s>>>(C.prob, count, C.words);
    Ctl ctl;
    ctl.bar.count = C.bar;
    ctl.bar.gen = C.bar + 1;
    ctl.err = C.words;
    ctl.active = C.words + 1;
    ctl.nrestart = C.words + 2;
    ctl.stop = C.words + 3;
    ctl.cancel = cancel;
    ctl.limit = wait_limit_or(20000000ll);  // polls of >= 32 ns each: seconds, never reached by co-resident blocks
    ctl.trace = g_trace_on;
    ctl.withhold = take_withhold() ? 1 : 0;
    mvgd_status st;
    if (prec == MVGD_FP32_REFINE)
        st = amg ? dispatch_q<true, true>(maxQ, tab, ctl, max_iterations, kmax, s)
                 : dispatch_q<true, false>(maxQ, tab, ctl, max_iterations, kmax, s);
    else
        st = amg ? dispatch_q<false, true>(maxQ, tab, ctl, max_iterations, kmax, s)
                 : dispatch_q<false, false>(maxQ, tab, ctl, max_iterations, kmax, s);
    if (st != MVGD_OK) return st;
    k_mark_exit<<<1, 256, 0, s>>>(C.prob, count, C.words);
    return launch_status();
}

MVGD_API mvgd_status mvgd_request_poll(void* const* reqs, int32_t count, int32_t* done, mvgd_stream_t stream) {
    if (!reqs || count < 1 || !done || !aligned(done)) return MVGD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (int g = 0; g < count; g += kTableMax) {
        TableArgs A;
        A.count = count - g < kTableMax ? count - g : kTableMax;
        A.first_chunk = 0;
        for (int i = 0; i < A.count; i++) {
            if (!reqs[g + i] || !aligned(reqs[g + i])) return MVGD_EINVAL;
            A.prob[i] = reinterpret_cast<const Prob*>(reqs[g + i]);
            A.nchunk[i] = 0;
        }
        k_poll<<<1, 256, 0, s>>>(A, done + g);
    }
    return launch_status();
}

MVGD_API mvgd_status mvgd_request_finish(void* req_ws, int64_t n, int32_t nrhs, double* u, mvgd_solve_info* info,
                                         mvgd_stream_t stream) {
    if (!req_ws || !u || !info || n < 1 || nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (!aligned(req_ws) || !aligned(u)) return MVGD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const Prob* P = reinterpret_cast<const Prob*>(req_ws);
    k_scatter_solution<<<gather_blocks(n * nrhs), 256, 0, s>>>(P, u);
    k_finish<<<1, 32, 0, s>>>(P, info);
    return launch_status();
}

// ---------------------------------------------------------------------------------
// One system: init + iterate to the end + finish
// ---------------------------------------------------------------------------------
MVGD_API size_t mvgd_solve_workspace_bytes(int64_t n, int32_t k, int32_t nrhs, int32_t prec, int32_t precond) {
    if (n <= 0 || nrhs < 1 || nrhs > 8) return 0;
    const size_t req = mvgd_request_workspace_bytes(n, k, nrhs, prec, precond);
    if (req == 0) return 0;
    size_t amg = 0;
    if (precond == 2) {
        amg = mvgd_amg_workspace_bytes(n, k);
        if (amg == 0) return 0;
    }
    return req + mvgd_iterate_workspace_bytes(1, n) + align_up(sizeof(mvgd_solve_info) * 8) + align_up(amg);
}

MVGD_API mvgd_status mvgd_solve(const mvgd_ell* L, int32_t nrhs, double sigma, const double* f, double* u,
                                const mvgd_solve_opts* opts, mvgd_solve_info* info, const int32_t* cancel,
                                void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!L || !f || !u || !opts || !info || !ws || nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (L->n < 2 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK || !L->col || !L->val) return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (!(opts->rtol > 0) || opts->maxit < 1 || !(sigma == sigma)) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE &&
        (!L->val_lo || opts->inner_maxit < 1 || !(opts->inner_rtol > 0) || opts->max_outer < 1))
        return MVGD_EINVAL;
    if (opts->precond < 0 || opts->precond > 2 || (opts->amg && !aligned(opts->amg))) return MVGD_EINVAL;
    size_t need = mvgd_solve_workspace_bytes(L->n, L->k, nrhs, L->prec, opts->precond);
    if (need == 0) return MVGD_EINVAL;
    if (opts->precond == 2 && opts->amg) need -= align_up(mvgd_amg_workspace_bytes(L->n, L->k));  // not built here
    if (!aligned(ws) || !aligned(u) || !aligned(f)) return MVGD_EINVAL;
    if (ws_bytes < need) return MVGD_EWORKSPACE;
    cudaPointerAttributes pa;
    MVGD_CUDA_TRY(cudaPointerGetAttributes(&pa, info));
    const bool host_info = pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged;
    char* base = static_cast<char*>(ws);
    const size_t req_bytes = mvgd_request_workspace_bytes(L->n, L->k, nrhs, L->prec, opts->precond);
    const size_t ctl_bytes = mvgd_iterate_workspace_bytes(1, L->n);
    void* req = base;
    void* ctl = base + req_bytes;
    mvgd_solve_info* staged = reinterpret_cast<mvgd_solve_info*>(base + req_bytes + ctl_bytes);
    mvgd_solve_opts o = *opts;
    mvgd_status st;
    if (o.precond == 2 && !o.amg) {
        // no hierarchy given: build one after the info staging area
        void* amg = base + req_bytes + ctl_bytes + align_up(sizeof(mvgd_solve_info) * 8);
        st = mvgd_amg_setup(L, sigma, amg, mvgd_amg_workspace_bytes(L->n, L->k), stream);
        if (st != MVGD_OK) return st;
        o.amg = amg;
    }
    st = mvgd_request_init(req, req_bytes, L, nrhs, sigma, f, u, &o, stream);
    if (st != MVGD_OK) return st;
    // every inner iteration and every restart is one pass of the phases
    const bool mixed = L->prec == MVGD_FP32_REFINE;
    long long budget = (long long)opts->maxit + 2ll * ((mixed ? opts->max_outer : 1000) + 2) + 4;
    if (budget > (1ll << 30)) budget = 1ll << 30;
    mvgd_request one;
    one.workspace = req;
    one.n = L->n;
    one.nrhs = nrhs;
    one.k = L->k;
    st = mvgd_iterate(&one, 1, L->prec, o.precond, (int32_t)budget, cancel, ctl, ctl_bytes, stream);
    if (st != MVGD_OK) return st;
    st = mvgd_request_finish(req, L->n, nrhs, u, host_info ? staged : info, stream);
    if (st != MVGD_OK) return st;
    if (!host_info) return MVGD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    MVGD_CUDA_TRY(cudaMemcpyAsync(info, staged, sizeof(mvgd_solve_info) * nrhs, cudaMemcpyDeviceToHost, s));
    MVGD_CUDA_TRY(cudaStreamSynchronize(s));
    int worst = MVGD_OK;
    for (int i = 0; i < nrhs; i++)
        if (info[i].status != MVGD_OK && worst == MVGD_OK) worst = info[i].status;
    return (mvgd_status)worst;
}

// ---------------------------------------------------------------------------------
// Step trace
// ---------------------------------------------------------------------------------
MVGD_API mvgd_status mvgd_trace_enable(int32_t on) {
    g_trace_on = on ? 1 : 0;
    if (on) {
        const unsigned zero = 0;
        MVGD_CUDA_TRY(cudaMemcpyToSymbol(g_trace_n, &zero, sizeof(zero)));
    }
    return MVGD_OK;
}

MVGD_API int32_t mvgd_trace_read(uint64_t* out, int32_t max) {
    if (!out || max < 1) return -1;
    unsigned n = 0;
    if (cudaMemcpyFromSymbol(&n, g_trace_n, sizeof(n)) != cudaSuccess) return -1;
    const int32_t count = (int32_t)(n < (unsigned)kTraceMax ? n : (unsigned)kTraceMax);
    const int32_t take = count < max ? count : max;
    if (take > 0 && cudaMemcpyFromSymbol(out, g_trace, sizeof(uint64_t) * take) != cudaSuccess) return -1;
    return take;
}
