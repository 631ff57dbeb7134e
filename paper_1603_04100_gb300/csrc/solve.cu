// Device-resident Krylov solve of (sigma I - L) u = f (Sec. 4.2; the paper
// solves with AMG -- here BiCGSTAB, van der Vorst 1992, left-preconditioned by
// the diagonal when asked).
//
// One persistent cooperative kernel runs every iteration of every right-hand
// side of every problem in the batch.  An iteration is three phases separated
// by a grid barrier:
//   A  p = r + beta (p - omega v) formed on the fly at the neighbours, v = A p
//   B  s = r - alpha v formed on the fly,                              t = A s
//   C  x += alpha p + omega s, r = s - omega t
// Each phase ends in dot products.  Rows are cut into fixed chunks of kCh
// rows; a chunk's partial sums are reduced in a fixed order and the block that
// finishes a problem's last chunk of the phase sums that problem's chunks in
// chunk order and advances its per-RHS state.  Results therefore do not depend
// on the grid size or on which other problems share the launch.
//
// Per right-hand side a small state machine runs:
//   RESTART  FP64 true residual r64 = f - A u  (mixed: on hi + lo weights,
//            after folding the last inner correction into u); stop if
//            ||r64|| <= rtol ||f||; else restart the Krylov vectors from
//            D^-1 r64 (mixed: scaled by 1 / ||r64||, in FP32)
//   INNER    BiCGSTAB iterations (mixed: FP32 on hi weights in difference
//            form) until the recursive residual meets the restart target
//   DONE
#include <type_traits>

#include "common.cuh"

namespace mvgd {
namespace {

constexpr int kCh = 2048;
constexpr int kThreads = 256;
constexpr int kRowsPerThread = kCh / kThreads;
constexpr int kChan = 2;

enum Mode : int { M_RESTART = 0, M_INNER = 1, M_SKIP = 2, M_DONE = 3 };

struct RhsState {
    double rho, alpha, omega, beta;
    double fnorm, relres, scale, target;
    double rnorm, pad0;
    int mode, pp, iters, inner_iters, outer, status;
};

struct Prob {
    int64_t n;
    int k, Q;
    double sigma;
    const int32_t* col;
    const void* val;
    const float* val_lo;
    const double* f;
    double* u;
    void* x;
    void* r;
    void* rh;
    void* p[2];
    void* v[2];
    void* s;
    void* t;
    double* r64;
    RhsState* st;
    double* part;      // [3][kChan][nchunk][Q]
    unsigned* arrive;  // [3]
    int chunk0, nchunk;
    double rtol, inner_rtol;
    int maxit, inner_maxit, max_outer, precond;
};

struct Ctl {
    GridBarrier bar;
    int* err;
    int* active;
    const int* cancel;
    int* stop;
    long long limit;
};

template <typename T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

// Row loops --------------------------------------------------------------------

template <bool MIXED, int QT>
__device__ __forceinline__ void inner_row(const Prob& P, int64_t r, int ph, const RhsState* S, const bool (&on)[QT],
                                          float (&af)[kChan][QT], double (&ad)[kChan][QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q, k = P.k, m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    const VT* __restrict__ val = static_cast<const VT*>(P.val);
    // vectors written by other blocks during this kernel: plain (coherent) loads
    const VT* R = static_cast<const VT*>(P.r);
    const VT* RH = static_cast<const VT*>(P.rh);
    const VT sig = (VT)P.sigma;
    const VT w0 = val[vb];
    const VT invd = P.precond ? (VT)1 / (sig - w0) : (VT)1;

    if (ph == 2) {
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q]) continue;
            const int64_t e = r * Q + q;
            const VT* pv = static_cast<const VT*>(P.p[S[q].pp]);
            VT* X = static_cast<VT*>(P.x);
            const VT sv = static_cast<const VT*>(P.s)[e], tv = static_cast<const VT*>(P.t)[e];
            const VT al = (VT)S[q].alpha, om = (VT)S[q].omega;
            X[e] = X[e] + al * pv[e] + om * sv;
            const VT rn = sv - om * tv;
            static_cast<VT*>(P.r)[e] = rn;
            if (MIXED) {
                af[0][q] += (float)(RH[e] * rn);
                af[1][q] += (float)(rn * rn);
            } else {
                ad[0][q] += (double)(RH[e] * rn);
                ad[1][q] += (double)(rn * rn);
            }
        }
        return;
    }
    // phases A and B: one operator application per active right-hand side
    VT si[QT], acc[QT];
    const VT* pold[QT];
    const VT* vold[QT];
    VT c1[QT], c2[QT];
#pragma unroll
    for (int q = 0; q < QT; q++) {
        acc[q] = (VT)0;
        si[q] = (VT)0;
        if (!on[q]) continue;
        const int pp = S[q].pp;
        vold[q] = static_cast<const VT*>(P.v[pp]);
        pold[q] = static_cast<const VT*>(P.p[pp]);
        if (ph == 0) {
            c1[q] = (VT)S[q].beta;
            c2[q] = (VT)S[q].omega;
            const int64_t e = r * Q + q;
            si[q] = R[e] + c1[q] * (pold[q][e] - c2[q] * vold[q][e]);
        } else {
            c1[q] = (VT)S[q].alpha;
            const int64_t e = r * Q + q;
            si[q] = R[e] - c1[q] * vold[q][e];
        }
    }
#pragma unroll 4
    for (int sl = 0; sl < k; sl++) {
        const int64_t j = P.col[cb + (int64_t)sl * kSlice];
        const VT w = val[vb + (int64_t)(sl + 1) * kSlice];
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q]) continue;
            const int64_t e = j * Q + q;
            VT sj;
            if (ph == 0) sj = R[e] + c1[q] * (pold[q][e] - c2[q] * vold[q][e]);
            else sj = R[e] - c1[q] * vold[q][e];
            if (MIXED) acc[q] += w * (sj - si[q]);
            else acc[q] += w * sj;
        }
    }
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        const VT lx = MIXED ? acc[q] : acc[q] + w0 * si[q];
        const VT res = invd * (sig * si[q] - lx);
        if (ph == 0) {
            // new p and v go to the other ping-pong buffers
            const int np = S[q].pp ^ 1;
            static_cast<VT*>(P.p[np])[e] = si[q];
            static_cast<VT*>(P.v[np])[e] = res;
            if (MIXED) af[0][q] += (float)(RH[e] * res);
            else ad[0][q] += (double)(RH[e] * res);
        } else {
            static_cast<VT*>(P.s)[e] = si[q];
            static_cast<VT*>(P.t)[e] = res;
            if (MIXED) {
                af[0][q] += (float)(res * si[q]);
                af[1][q] += (float)(res * res);
            } else {
                ad[0][q] += (double)(res * si[q]);
                ad[1][q] += (double)(res * res);
            }
        }
    }
}

template <bool MIXED, int QT>
__device__ __forceinline__ void restart_row(const Prob& P, int64_t r, int ph, const RhsState* S, const bool (&on)[QT],
                                            double (&ad)[kChan][QT]) {
    using VT = typename std::conditional<MIXED, float, double>::type;
    const int Q = P.Q, k = P.k, m = k + 1;
    const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int64_t cb = (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    if (ph == 0) {
        if (!MIXED) return;
#pragma unroll
        for (int q = 0; q < QT; q++) {
            if (!on[q] || S[q].outer == 0) continue;
            const int64_t e = r * Q + q;
            P.u[e] += S[q].scale * (double)static_cast<const VT*>(P.x)[e];
        }
        return;
    }
    if (ph == 1) {
        // true residual in FP64
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
    // ph == 2: restart the Krylov vectors from D^-1 r64 (scaled in the mixed path)
    double invd = 1.0;
    if (P.precond) {
        double w0 = MIXED ? (double)static_cast<const float*>(P.val)[vb] : static_cast<const double*>(P.val)[vb];
        invd = 1.0 / (P.sigma - w0);
    }
#pragma unroll
    for (int q = 0; q < QT; q++) {
        if (!on[q]) continue;
        const int64_t e = r * Q + q;
        double rv = invd * P.r64[e];
        if (MIXED) rv /= S[q].scale;
        const VT rr = (VT)rv;
        static_cast<VT*>(P.r)[e] = rr;
        static_cast<VT*>(P.rh)[e] = rr;
        static_cast<VT*>(P.p[0])[e] = (VT)0;
        static_cast<VT*>(P.p[1])[e] = (VT)0;
        static_cast<VT*>(P.v[0])[e] = (VT)0;
        static_cast<VT*>(P.v[1])[e] = (VT)0;
        if (MIXED) static_cast<VT*>(P.x)[e] = (VT)0;
        ad[0][q] += (double)rr * (double)rr;
    }
}

// State transitions -------------------------------------------------------------

template <bool MIXED>
__device__ void advance(const Prob& P, int ph, RhsState& T, double a, double b, int* active) {
    switch (T.mode) {
        case M_INNER:
            if (ph == 0) {
                T.pp ^= 1;
                if (!(fabs(a) > 0.0) || !isfinite(a)) T.mode = M_SKIP;
                else T.alpha = T.rho / a;
            } else if (ph == 1) {
                T.omega = (b > 0.0 && isfinite(a) && isfinite(b)) ? a / b : 0.0;
            } else {
                T.iters++;
                T.inner_iters++;
                const double rn = sqrt(b);
                T.rnorm = rn;
                bool restart = !isfinite(rn) || !isfinite(a) || rn <= T.target || T.iters >= P.maxit ||
                               T.omega == 0.0 || a == 0.0 || (MIXED && T.inner_iters >= P.inner_maxit);
                if (restart) {
                    T.mode = M_RESTART;
                } else {
                    T.beta = (a / T.rho) * (T.alpha / T.omega);
                    T.rho = a;
                }
            }
            break;
        case M_SKIP:
            if (ph == 2) T.mode = M_RESTART;
            break;
        case M_RESTART:
            if (ph == 1) {
                if (T.fnorm < 0) {
                    const double fn = sqrt(b);
                    T.fnorm = fn > 0 ? fn : 1.0;
                }
                const double rn = sqrt(a);
                T.relres = rn / T.fnorm;
                if (!isfinite(rn)) {
                    T.mode = M_DONE;
                    T.status = MVGD_ENONFINITE;
                } else if (T.relres <= P.rtol) {
                    T.mode = M_DONE;
                    T.status = MVGD_OK;
                } else if (T.iters >= P.maxit) {
                    T.mode = M_DONE;
                    T.status = MVGD_ENOCONV;
                } else if (T.outer >= P.max_outer) {
                    T.mode = M_DONE;
                    T.status = MVGD_EBREAKDOWN;
                } else {
                    T.scale = rn;
                }
                if (T.mode == M_DONE) atomicSub(active, 1);
            } else if (ph == 2) {
                const double rn = sqrt(a);
                T.rho = a;
                T.alpha = 1.0;
                T.omega = 1.0;
                T.beta = 0.0;
                T.pp = 0;
                double red = 0.5 * P.rtol / T.relres;
                if (MIXED) red = fmax(P.inner_rtol, red);
                T.target = red * rn;
                T.outer++;
                T.inner_iters = 0;
                T.mode = M_INNER;
            }
            break;
        default:
            break;
    }
}

template <bool MIXED, int QT>
__global__ void __launch_bounds__(kThreads) k_solve(const Prob* __restrict__ probs,
                                                     const int* __restrict__ chunk_prob, int nchunks, Ctl ctl,
                                                     int iter_budget) {
    __shared__ RhsState S[QT];
    __shared__ double red[kThreads / 32][kChan * QT];
    __shared__ double tot[kChan * QT];
    __shared__ int last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;

    for (int it = 0; it < iter_budget; ++it) {
        for (int ph = 0; ph < 3; ++ph) {
            for (int c = blockIdx.x; c < nchunks; c += gridDim.x) {
                const Prob& P = probs[chunk_prob[c]];
                const int lc = c - P.chunk0;
                if (tid < QT) {
                    if (tid < P.Q) S[tid] = P.st[tid];
                    else S[tid].mode = M_DONE;
                }
                __syncthreads();
                bool on_inner[QT], on_restart[QT];
                bool any_inner = false, any_restart = false;
#pragma unroll
                for (int q = 0; q < QT; q++) {
                    on_inner[q] = S[q].mode == M_INNER;
                    on_restart[q] = S[q].mode == M_RESTART;
                    any_inner |= on_inner[q];
                    any_restart |= on_restart[q];
                }
                float af[kChan][QT];
                double ad[kChan][QT];
#pragma unroll
                for (int ch = 0; ch < kChan; ch++)
#pragma unroll
                    for (int q = 0; q < QT; q++) { af[ch][q] = 0.0f; ad[ch][q] = 0.0; }
                const int64_t row0 = (int64_t)lc * kCh;
                for (int j = 0; j < kRowsPerThread; ++j) {
                    const int64_t r = row0 + (int64_t)j * kThreads + tid;
                    if (r >= P.n) break;
                    if (any_inner) inner_row<MIXED, QT>(P, r, ph, S, on_inner, af, ad);
                    if (any_restart) restart_row<MIXED, QT>(P, r, ph, S, on_restart, ad);
                }
                // block reduction in a fixed order
#pragma unroll
                for (int ch = 0; ch < kChan; ch++)
#pragma unroll
                    for (int q = 0; q < QT; q++) {
                        double v = ad[ch][q] + (double)af[ch][q];
                        v = warp_sum(v);
                        if (lane == 0) red[wid][ch * QT + q] = v;
                    }
                __syncthreads();
                if (tid < kChan * QT) {
                    double v = 0.0;
                    for (int w = 0; w < kThreads / 32; w++) v += red[w][tid];
                    const int ch = tid / QT, q = tid % QT;
                    if (q < P.Q) P.part[(((int64_t)ph * kChan + ch) * P.nchunk + lc) * P.Q + q] = v;
                }
                __threadfence();
                __syncthreads();
                if (tid == 0) last = (atomicAdd(&P.arrive[ph], 1u) == (unsigned)(P.nchunk - 1));
                __syncthreads();
                if (last) {
                    __threadfence();
                    // sum this problem's chunk partials in chunk order
                    double acc[kChan * QT];
#pragma unroll
                    for (int e = 0; e < kChan * QT; e++) acc[e] = 0.0;
                    for (int l = tid; l < P.nchunk; l += kThreads)
#pragma unroll
                        for (int e = 0; e < kChan * QT; e++) {
                            const int ch = e / QT, q = e % QT;
                            if (q < P.Q) acc[e] += ldcg(&P.part[(((int64_t)ph * kChan + ch) * P.nchunk + l) * P.Q + q]);
                        }
#pragma unroll
                    for (int e = 0; e < kChan * QT; e++) {
                        double v = warp_sum(acc[e]);
                        if (lane == 0) red[wid][e] = v;
                    }
                    __syncthreads();
                    if (tid < kChan * QT) {
                        double v = 0.0;
                        for (int w = 0; w < kThreads / 32; w++) v += red[w][tid];
                        tot[tid] = v;
                    }
                    __syncthreads();
                    if (tid < P.Q) {
                        RhsState T = S[tid];
                        advance<MIXED>(P, ph, T, tot[0 * QT + tid], tot[1 * QT + tid], ctl.active);
                        P.st[tid] = T;
                    }
                    if (tid == 0) P.arrive[ph] = 0;
                    __threadfence();
                }
                __syncthreads();
            }
            // the stop word is written only before the last barrier of an iteration and read
            // only after it, so every block takes the same exit decision
            if (ph == 2 && blockIdx.x == 0 && tid == 0 && ctl.cancel && *(const volatile int*)ctl.cancel != 0)
                *ctl.stop = 1;
            if (!grid_sync(ctl.bar, ctl.err, ctl.limit)) return;
        }
        if (*(volatile int*)ctl.active == 0 || *(volatile int*)ctl.stop != 0) break;
    }
}

// Setup / teardown kernels --------------------------------------------------------

__global__ void k_init_states(RhsState* st, int Q, unsigned* arrive, unsigned* bar, int* ctl_words, int active) {
    int t = threadIdx.x;
    if (t < Q) {
        RhsState T;
        T.rho = T.alpha = T.omega = 1.0;
        T.beta = 0.0;
        T.fnorm = -1.0;
        T.relres = 1.0;
        T.scale = 0.0;
        T.target = 0.0;
        T.rnorm = 0.0;
        T.pad0 = 0.0;
        T.mode = M_RESTART;
        T.pp = 0;
        T.iters = T.inner_iters = T.outer = 0;
        T.status = MVGD_OK;
        st[t] = T;
    }
    if (t < 3) arrive[t] = 0;
    if (t < 2) bar[t] = 0;
    if (t == 0) {
        ctl_words[0] = 0;       // err
        ctl_words[1] = active;  // active
        ctl_words[2] = 0;       // stop
    }
}

__global__ void k_finish(const RhsState* st, int Q, const int* ctl_words, mvgd_solve_info* out) {
    int q = threadIdx.x;
    if (q >= Q) return;
    RhsState T = st[q];
    mvgd_solve_info I;
    I.iters = T.iters;
    I.outer = T.outer;
    I.relres = T.relres;
    int s = T.status;
    if (T.mode != M_DONE) s = ctl_words[0] ? ctl_words[0] : (ctl_words[2] ? MVGD_ECANCELLED : MVGD_ENOCONV);
    I.status = s;
    I.reserved = 0;
    out[q] = I;
}

__global__ void k_gather_rows(const double* __restrict__ src, const int32_t* __restrict__ order, int64_t n, int Q,
                              double* __restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * Q; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / Q, q = e % Q;
        dst[e] = src[(int64_t)order[r] * Q + q];
    }
}

__global__ void k_scatter_rows(const double* __restrict__ src, const int32_t* __restrict__ order, int64_t n, int Q,
                               double* __restrict__ dst) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * Q; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = e / Q, q = e % Q;
        dst[(int64_t)order[r] * Q + q] = src[e];
    }
}

struct SolveLayout {
    Prob* prob;
    int* chunk_prob;
    RhsState* st;
    double* part;
    unsigned* arrive;
    unsigned* bar;
    int* ctl_words;
    mvgd_solve_info* info;
    double* fs;
    double* us;
    double* r64;
    void* vec[9];  // x r rh p0 p1 v0 v1 s t
    size_t bytes;
};

SolveLayout solve_layout(void* ws, int64_t n, int Q, int prec) {
    SolveLayout L;
    Carver cv(ws);
    const int64_t nchunk = (n + kCh - 1) / kCh;
    const size_t vt = prec == MVGD_FP64 ? sizeof(double) : sizeof(float);
    L.prob = cv.take<Prob>(1);
    L.chunk_prob = cv.take<int>(nchunk);
    L.st = cv.take<RhsState>(Q);
    L.part = cv.take<double>(3 * kChan * nchunk * Q);
    L.arrive = cv.take<unsigned>(3);
    L.bar = cv.take<unsigned>(2);
    L.ctl_words = cv.take<int>(4);
    L.info = cv.take<mvgd_solve_info>(Q);
    L.fs = cv.take<double>(n * Q);
    L.us = cv.take<double>(n * Q);
    L.r64 = cv.take<double>(n * Q);
    for (int v = 0; v < 9; v++) L.vec[v] = cv.take<char>(vt * n * Q);
    L.bytes = cv.used;
    return L;
}

template <bool MIXED, int QT>
mvgd_status launch_solve(const Prob* dprob, const int* chunk_prob, int nchunks, Ctl ctl, int budget,
                         cudaStream_t s) {
    auto fn = k_solve<MIXED, QT>;
    int dev = 0, sms = 0, per_sm = 0;
    MVGD_CUDA_TRY(cudaGetDevice(&dev));
    MVGD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    MVGD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0));
    if (per_sm < 1) return MVGD_ECUDA;
    int grid = sms * per_sm;
    if (grid > nchunks) grid = nchunks;
    void* args[] = {(void*)&dprob, (void*)&chunk_prob, (void*)&nchunks, (void*)&ctl, (void*)&budget};
    MVGD_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kThreads), args, 0, s));
    return MVGD_OK;
}

template <bool MIXED>
mvgd_status dispatch_q(int Q, const Prob* dprob, const int* chunk_prob, int nchunks, Ctl ctl, int budget,
                       cudaStream_t s) {
    if (Q <= 1) return launch_solve<MIXED, 1>(dprob, chunk_prob, nchunks, ctl, budget, s);
    if (Q <= 2) return launch_solve<MIXED, 2>(dprob, chunk_prob, nchunks, ctl, budget, s);
    if (Q <= 4) return launch_solve<MIXED, 4>(dprob, chunk_prob, nchunks, ctl, budget, s);
    return launch_solve<MIXED, 8>(dprob, chunk_prob, nchunks, ctl, budget, s);
}

__global__ void k_fill_chunks(int* chunk_prob, int nchunk, int value) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nchunk; c += gridDim.x * blockDim.x) chunk_prob[c] = value;
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_solve_workspace_bytes(int64_t n, int32_t k, int32_t nrhs, int32_t prec) {
    (void)k;
    if (n <= 0 || nrhs < 1 || nrhs > 8) return 0;
    return solve_layout(nullptr, n, nrhs, prec).bytes;
}

MVGD_API mvgd_status mvgd_solve(const mvgd_ell* L, int32_t nrhs, double sigma, const double* f, double* u,
                                const mvgd_solve_opts* opts, mvgd_solve_info* info, const int32_t* cancel,
                                void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!L || !f || !u || !opts || !info || !ws || nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (L->n < 2 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK || !L->col || !L->val) return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!aligned(f) || !aligned(u) || !aligned(ws) || !aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo) ||
        !aligned(L->order))
        return MVGD_EINVAL;
    if (!(opts->rtol > 0) || opts->maxit < 1 || !(sigma == sigma)) return MVGD_EINVAL;
    const bool mixed = L->prec == MVGD_FP32_REFINE;
    if (mixed && (opts->inner_maxit < 1 || !(opts->inner_rtol > 0) || opts->max_outer < 1)) return MVGD_EINVAL;
    const int64_t n = L->n;
    const int Q = nrhs;
    SolveLayout W = solve_layout(ws, n, Q, L->prec);
    if (ws_bytes < W.bytes) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;

    cudaPointerAttributes pa;
    MVGD_CUDA_TRY(cudaPointerGetAttributes(&pa, info));
    const bool host_info = pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged;

    const double* fs = f;
    double* us = u;
    if (L->order) {
        int gb = (int)((n * Q + 255) / 256);
        if (gb > 8192) gb = 8192;
        k_gather_rows<<<gb, 256, 0, s>>>(f, L->order, n, Q, W.fs);
        k_gather_rows<<<gb, 256, 0, s>>>(u, L->order, n, Q, W.us);
        fs = W.fs;
        us = W.us;
    }
    const int nchunk = (int)((n + kCh - 1) / kCh);
    Prob P;
    P.n = n;
    P.k = L->k;
    P.Q = Q;
    P.sigma = sigma;
    P.col = L->col;
    P.val = L->val;
    P.val_lo = L->val_lo;
    P.f = fs;
    P.u = us;
    P.x = mixed ? W.vec[0] : (void*)us;
    P.r = W.vec[1];
    P.rh = W.vec[2];
    P.p[0] = W.vec[3];
    P.p[1] = W.vec[4];
    P.v[0] = W.vec[5];
    P.v[1] = W.vec[6];
    P.s = W.vec[7];
    P.t = W.vec[8];
    P.r64 = W.r64;
    P.st = W.st;
    P.part = W.part;
    P.arrive = W.arrive;
    P.chunk0 = 0;
    P.nchunk = nchunk;
    P.rtol = opts->rtol;
    P.inner_rtol = mixed ? opts->inner_rtol : 0.0;
    P.maxit = opts->maxit;
    P.inner_maxit = mixed ? opts->inner_maxit : opts->maxit;
    P.max_outer = mixed ? opts->max_outer : 1000;
    P.precond = opts->precond == 1 ? 1 : 0;
    MVGD_CUDA_TRY(cudaMemcpyAsync(W.prob, &P, sizeof(Prob), cudaMemcpyHostToDevice, s));
    k_fill_chunks<<<(nchunk + 255) / 256, 256, 0, s>>>(W.chunk_prob, nchunk, 0);
    k_init_states<<<1, 32, 0, s>>>(W.st, Q, W.arrive, W.bar, W.ctl_words, Q);

    Ctl ctl;
    ctl.bar.count = W.bar;
    ctl.bar.gen = W.bar + 1;
    ctl.err = W.ctl_words;
    ctl.active = W.ctl_words + 1;
    ctl.stop = W.ctl_words + 2;
    ctl.cancel = cancel;
    ctl.limit = 20000000ll;  // polls of >= 32 ns each: seconds, never reached by co-resident blocks
    // every inner iteration and every restart is one pass of the three phases
    long long budget = (long long)opts->maxit + 2ll * (P.max_outer + 2) + 4;
    if (budget > (1ll << 30)) budget = 1ll << 30;
    mvgd_status st = mixed ? dispatch_q<true>(Q, W.prob, W.chunk_prob, nchunk, ctl, (int)budget, s)
                           : dispatch_q<false>(Q, W.prob, W.chunk_prob, nchunk, ctl, (int)budget, s);
    if (st != MVGD_OK) return st;
    if (L->order) {
        int gb = (int)((n * Q + 255) / 256);
        if (gb > 8192) gb = 8192;
        k_scatter_rows<<<gb, 256, 0, s>>>(W.us, L->order, n, Q, u);
    }
    k_finish<<<1, 32, 0, s>>>(W.st, Q, W.ctl_words, host_info ? W.info : info);
    MVGD_CUDA_TRY(cudaGetLastError());
    if (!host_info) return MVGD_OK;
    MVGD_CUDA_TRY(cudaMemcpyAsync(info, W.info, sizeof(mvgd_solve_info) * Q, cudaMemcpyDeviceToHost, s));
    MVGD_CUDA_TRY(cudaStreamSynchronize(s));
    int worst = MVGD_OK;
    for (int q = 0; q < Q; q++)
        if (info[q].status != MVGD_OK && worst == MVGD_OK) worst = info[q].status;
    return (mvgd_status)worst;
}
