// Aggregation multigrid hierarchy of sigma I - L and its standalone V-cycle.
//
// The paper solves its MVGD systems with algebraic multigrid and reports its
// CPU time growing about linearly with N (Sec. 4.2, the timing table), without
// naming the variant.  This is plain aggregation (Braess 1995) on the
// stored row order, whose consecutive rows are spatial neighbours (the kNN
// step sorts points by cell along a Z-order curve):
//   * aggregate I of level l is rows kAmgAgg*I .. kAmgAgg*I + kAmgAgg-1;
//   * level l+1 is the Galerkin product P^T A_l P (entry (I, J) sums a_ij over
//     the rows of aggregate I and the columns of aggregate J), computed in
//     FP64 one warp per coarse row, with a fixed summation order;
//   * the first level with at most kAmgCoarsest rows is inverted by
//     Gauss-Jordan elimination with partial pivoting (FP32, one block),
//     refined by two Newton-Schulz steps in FP64;
//   * smoothing is a Jacobi step x += d (b - A x) with d_i = omega / a_ii on
//     rows with a strong diagonal (a_ii > theta sum_j |a_ij|; omega = 0.9,
//     theta = 0.3) and the l1 scaling d_i = 1 / sum_j |a_ij| (Baker, Falgout,
//     Kolev, Yang 2011), positive whatever the sign pattern, on the others:
//     MVGD rows with few neighbours on irregular samples can have a small or
//     negative diagonal.  Against l1-Jacobi everywhere this took 15-30 % off
//     the preconditioned iteration counts (K 12 and 20, 7k-262k points).
// Everything the V-cycle reads is FP32; the FP64 Galerkin values stay
// available for inspection.
#include <cooperative_groups.h>
#include <limits.h>

#include <algorithm>
#include <string.h>

#include "vcycle.cuh"

namespace mvgd {
namespace {

struct AmgLayout {
    AmgHeader* hdr;
    AmgHeader h;  // host copy of the pointers and sizes
};

AmgLayout amg_layout(void* ws, int64_t n, int k) {
    AmgLayout A;
    memset(&A.h, 0, sizeof(A.h));
    Carver cv(ws);
    A.hdr = cv.take<AmgHeader>(1);
    int64_t sizes[kAmgMaxLevels];
    const int nlev = amg_levels(n, sizes);
    A.h.nlev = nlev;
    A.h.k = k;
    A.h.n = n;
    for (int l = 0; l < nlev; l++) {
        const int64_t nl = sizes[l], np = n_padded(nl);
        AmgLevel& L = A.h.lv[l];
        L.n = nl;
        if (l == 0) {
            L.val = cv.take<float>(np * (k + 1));
        } else {
            L.col = cv.take<int32_t>(np * kAmgStride);
            L.val = cv.take<float>(np * kAmgStride);
            L.val64 = cv.take<double>(np * kAmgStride);
            L.cnt = cv.take<int32_t>(np);
            L.sw = cv.take<int32_t>(np / kSlice);
            L.rs = cv.take<float>(np);
        }
        L.dinv = cv.take<float>(np);
    }
    const int64_t nc = nlev > 0 ? sizes[nlev - 1] : 0;
    A.h.nc = nc;
    A.h.dense = cv.take<float>(nc * nc);
    A.h.cinv = cv.take<float>(nc * nc);
    A.h.piv = cv.take<int32_t>(nc);
    A.h.dense64 = cv.take<double>(nc * nc);
    A.h.cinv64 = cv.take<double>(nc * nc);
    A.h.ns_x = cv.take<double>(nc * nc);
    A.h.ns_t = cv.take<double>(nc * nc);
    A.h.bytes = cv.used;
    return A;
}

// Where the set-up reads the operator's own weights (FP64, or hi + lo).
struct OpView {
    const int32_t* col;
    const void* val;
    const float* val_lo;
    int prec;
};

__device__ __forceinline__ double op_weight(const OpView& O, int64_t idx) {
    return O.prec == MVGD_FP64 ? static_cast<const double*>(O.val)[idx]
                               : (double)static_cast<const float*>(O.val)[idx] + (double)O.val_lo[idx];
}

__global__ void k_amg_header(AmgHeader h, AmgHeader* dst) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = h;
}

// Level 0: FP32 copy of the weights and the smoother's scaling of sigma I - L.
__global__ void k_amg_level0(const AmgHeader* __restrict__ Hp, OpView O) {
    const AmgHeader& H = *Hp;
    const int k = H.k, m = k + 1;
    const double sigma = H.sigma;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < H.n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
        double l1 = 0.0, diag = 0.0;
        for (int s = 0; s < m; s++) {
            const int64_t idx = vb + (int64_t)s * kSlice;
            const double w = op_weight(O, idx);
            // FP64 weights round to nearest; the mixed format's hi is already that rounding
            H.lv[0].val[idx] = O.prec == MVGD_FP64 ? (float)w : static_cast<const float*>(O.val)[idx];
            if (s == 0) diag = sigma - w;
            l1 += s == 0 ? fabs(sigma - w) : fabs(w);
        }
        H.lv[0].dinv[r] = amg_smoother_scale(diag, l1);
    }
}

constexpr int kPerLane = kAmgAgg * kAmgStride / kWarp;  // entries a lane holds while coarsening

// Level l+1 from level l, one warp per coarse row I: gather the entries of
// the aggregate's rows, then emit distinct aggregate columns in increasing
// order, each with the FP64 sum of its entries (per-lane sums in entry order,
// then a butterfly over the warp: the same order on every run).  Each lane
// first sorts its entries by (column, slot) and adds up its equal columns
// once, so the merge over columns moves values instead of adding them: the
// GPU's FP64 rate made those predicated adds (one per entry and column) the
// kernel's cost.
__global__ void k_amg_coarsen(const AmgHeader* Hp, OpView O, int l) {
    const AmgHeader& H = *Hp;
    const AmgLevel& F = H.lv[l];
    const AmgLevel& Cl = H.lv[l + 1];
    const int lane = (int)lane_id();
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / kWarp);
    const int k = H.k;
    const int W = (l == 0) ? k + 1 : kAmgStride;  // entry slots per fine row
    for (int64_t I = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp; I < Cl.n; I += warps) {
        int key[kPerLane];
        double v[kPerLane];
#pragma unroll
        for (int t = 0; t < kPerLane; t++) {
            key[t] = INT_MAX;
            v[t] = 0.0;
            const int e = t * kWarp + lane;
            const int f = e / W, s = e % W;
            const int64_t i = I * kAmgAgg + f;
            if (f >= kAmgAgg || i >= F.n) continue;
            if (l == 0) {
                const int64_t vb = (i / kSlice) * (int64_t)(kSlice * (k + 1)) + (i % kSlice);
                const double w = op_weight(O, vb + (int64_t)s * kSlice);
                if (s == 0) {
                    key[t] = (int)(i / kAmgAgg);
                    v[t] = H.sigma - w;
                } else {
                    const int64_t j = O.col[(i / kSlice) * (int64_t)(kSlice * k) + (int64_t)(s - 1) * kSlice + (i % kSlice)];
                    key[t] = (int)(j / kAmgAgg);
                    v[t] = -w;
                }
            } else if (s < F.cnt[i]) {
                const int64_t idx = (i / kSlice) * (int64_t)(kSlice * kAmgStride) + (int64_t)s * kSlice + (i % kSlice);
                key[t] = F.col[idx] / kAmgAgg;
                v[t] = F.val64[idx];
            }
        }
        // sort the lane's entries by (column, slot): an odd-even transposition network
        int tt[kPerLane];
#pragma unroll
        for (int t = 0; t < kPerLane; t++) tt[t] = t;
#pragma unroll
        for (int ph = 0; ph < kPerLane; ph++)
#pragma unroll
            for (int i = ph & 1; i + 1 < kPerLane; i += 2) {
                const bool sw = key[i] > key[i + 1] || (key[i] == key[i + 1] && tt[i] > tt[i + 1]);
                const int ka = key[i], ta = tt[i];
                const double va = v[i];
                key[i] = sw ? key[i + 1] : ka;
                tt[i] = sw ? tt[i + 1] : ta;
                v[i] = sw ? v[i + 1] : va;
                key[i + 1] = sw ? ka : key[i + 1];
                tt[i + 1] = sw ? ta : tt[i + 1];
                v[i + 1] = sw ? va : v[i + 1];
            }
        // the lane's sum of each column, in slot order, left on its last entry
#pragma unroll
        for (int t = 1; t < kPerLane; t++)
            if (key[t] != INT_MAX && key[t] == key[t - 1]) {
                v[t] = v[t - 1] + v[t];
                key[t - 1] = INT_MAX;
            }
        const int64_t ob = (I / kSlice) * (int64_t)(kSlice * kAmgStride) + (I % kSlice);
        int out = 0;
        double l1 = 0.0, rsum = 0.0, diag = 0.0;
        while (true) {
            int mine = INT_MAX;
#pragma unroll
            for (int t = 0; t < kPerLane; t++) mine = min(mine, key[t]);
            int m = mine;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (m == INT_MAX) break;
            double part = 0.0;  // at most one entry of the lane holds column m now
#pragma unroll
            for (int t = 0; t < kPerLane; t++)
                if (key[t] == m) {
                    part = v[t];
                    key[t] = INT_MAX;
                }
            const double tot = warp_sum(part);
            if (out < kAmgStride && lane == 0) {
                Cl.col[ob + (int64_t)out * kSlice] = m;
                Cl.val64[ob + (int64_t)out * kSlice] = tot;
                Cl.val[ob + (int64_t)out * kSlice] = (float)tot;
            }
            l1 += fabs(tot);
            rsum += tot;
            if (m == I) diag = tot;
            out++;
        }
        if (lane == 0) {
            if (out > kAmgStride) atomicCAS((int*)&Hp->status, 0, (int)MVGD_EDEGENERATE);
            atomicMax((int*)&Hp->width_max, out);
            const int c = min(out, kAmgStride);
            Cl.cnt[I] = c;
            Cl.dinv[I] = amg_smoother_scale(diag, l1);
            Cl.rs[I] = (float)rsum;
        }
        // padding: (own row, 0) up to the full stride, so slice loops need no bounds
        for (int s = min(out, kAmgStride) + lane; s < kAmgStride; s += kWarp) {
            Cl.col[ob + (int64_t)s * kSlice] = (int32_t)I;
            Cl.val64[ob + (int64_t)s * kSlice] = 0.0;
            Cl.val[ob + (int64_t)s * kSlice] = 0.0f;
        }
    }
}

// Widest row of each 32-row slice of level l (>= 1).
__global__ void k_amg_slice_width(const AmgHeader* __restrict__ Hp, int l) {
    const AmgLevel& L = Hp->lv[l];
    const int64_t ns = (L.n + kSlice - 1) / kSlice;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < ns; s += (int64_t)gridDim.x * blockDim.x) {
        int w = 0;
        for (int64_t r = s * kSlice; r < (s + 1) * kSlice && r < L.n; r++) w = max(w, L.cnt[r]);
        L.sw[s] = w;
    }
}

// The coarsest level as dense FP32 and FP64 matrices (both zeroed first).
__global__ void k_amg_dense(const AmgHeader* __restrict__ Hp, OpView O) {
    const AmgHeader& H = *Hp;
    const int m = H.nlev - 1;
    const int64_t nc = H.nc;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nc; r += (int64_t)gridDim.x * blockDim.x) {
        float* row = H.dense + r * nc;
        double* row64 = H.dense64 + r * nc;
        if (m == 0) {
            const int k = H.k;
            const int64_t vb = (r / kSlice) * (int64_t)(kSlice * (k + 1)) + (r % kSlice);
            row64[r] = H.sigma - op_weight(O, vb);
            row[r] = (float)row64[r];
            for (int s = 0; s < k; s++) {
                const int64_t j = O.col[(r / kSlice) * (int64_t)(kSlice * k) + (int64_t)s * kSlice + (r % kSlice)];
                row64[j] = -op_weight(O, vb + (int64_t)(s + 1) * kSlice);
                row[j] = (float)row64[j];
            }
        } else {
            const AmgLevel& L = H.lv[m];
            const int64_t b = (r / kSlice) * (int64_t)(kSlice * kAmgStride) + (r % kSlice);
            for (int s = 0; s < L.cnt[r]; s++) {
                const int64_t e = b + (int64_t)s * kSlice;
                row64[L.col[e]] = L.val64[e];
                row[L.col[e]] = L.val[e];
            }
        }
    }
}

// cinv64 = the FP32 inverse (column-major) in FP64, row-major.
__global__ void k_amg_promote(const AmgHeader* __restrict__ Hp) {
    const int64_t n = Hp->nc;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x)
        Hp->cinv64[e] = (double)Hp->cinv[(e % n) * n + e / n];
}

// C = diag I + scale (A B) for small n x n row-major FP64 matrices: one block
// per 32 x 32 tile of C, 32-wide k tiles staged in shared memory.  A Newton-
// Schulz step X <- X (2I - A X) is two of these.
constexpr int kGemmTile = 32;
__global__ void __launch_bounds__(256) k_amg_dgemm(int n, const double* __restrict__ A, const double* __restrict__ B,
                                                   double* __restrict__ Cm, double diag, double scale) {
    __shared__ double As[kGemmTile][kGemmTile + 1], Bs[kGemmTile][kGemmTile + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads, 4 rows each
    const int row0 = blockIdx.y * kGemmTile, col = blockIdx.x * kGemmTile + tx;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += kGemmTile) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int r = ty + 8 * u;
            As[r][tx] = (row0 + r < n && k0 + tx < n) ? A[(int64_t)(row0 + r) * n + k0 + tx] : 0.0;
            Bs[r][tx] = (k0 + r < n && col < n) ? B[(int64_t)(k0 + r) * n + col] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kGemmTile; kk++) {
            const double b = Bs[kk][tx];
#pragma unroll
            for (int u = 0; u < 4; u++) acc[u] = fma(As[ty + 8 * u][kk], b, acc[u]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++) {
        const int r = row0 + ty + 8 * u;
        if (r < n && col < n) Cm[(int64_t)r * n + col] = scale * acc[u] + (r == col ? diag : 0.0);
    }
}

// Gauss-Jordan inversion in place with partial pivoting.  Step k picks the
// largest |a_ik|, i >= k (lowest i on ties), swaps rows k and p, and replaces
// a by the matrix of the eliminated system; the column swaps are undone in
// reverse order at the end (the classical in-place form).
constexpr int kInvThreads = 1024;
constexpr int kInvWarps = kInvThreads / 32;

// The matrix is held in shared memory: a cluster of up to 8 CTAs (one an
// SM), CTA q holding rows q*rows .. q*rows + rows - 1 (rows * n * 4 bytes
// <= 128 KB).  Each step the CTAs publish their column-k pivot candidate,
// every CTA reads all of them through distributed shared memory and picks the
// same pivot (largest magnitude, lowest row on a tie), the owners swap rows k
// and p, every CTA copies the pivot row, and each eliminates its own rows.
// One block sweeping a 256 KB matrix through L2 every step took about 2 ms
// for 256 rows.
__global__ void __launch_bounds__(kInvThreads) k_amg_invert_cluster(AmgHeader* Hp, int rows) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), ncta = (int)cl.num_blocks();
    const int n = (int)Hp->nc;
    extern __shared__ float smf[];
    float* A = smf;               // [rows][n] this CTA's rows
    float* rowk = A + rows * n;   // [n] the scaled pivot row
    float* tmp = rowk + n;        // [n] a row arriving in a swap
    __shared__ float bv[kInvWarps], cand_v;
    __shared__ int bi[kInvWarps], cand_i, piv_k, bad;
    __shared__ int col_of[kAmgCoarsest];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int r0 = rank * rows, r1 = min(n, r0 + rows);
    float* a = Hp->dense;
    for (int e = tid; e < (r1 - r0) * n; e += kInvThreads) A[e] = a[(int64_t)r0 * n + e];
    if (tid == 0) bad = 0;
    cl.sync();
    for (int k = 0; k < n; k++) {
        // this CTA's pivot candidate in column k
        float best = -1.0f;
        int bidx = INT_MAX;
        for (int i = max(k, r0) + tid; i < r1; i += kInvThreads) {
            const float v = fabsf(A[(i - r0) * n + k]);
            if (v > best) { best = v; bidx = i; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
        }
        if (lane == 0) { bv[wid] = best; bi[wid] = bidx; }
        __syncthreads();
        if (tid == 0) {
            float b = -1.0f;
            int p = INT_MAX;
            for (int w = 0; w < kInvWarps; w++)
                if (bv[w] > b || (bv[w] == b && bi[w] < p)) { b = bv[w]; p = bi[w]; }
            cand_v = b;
            cand_i = p;
        }
        cl.sync();
        // every CTA takes the same pivot from all candidates
        if (tid == 0) {
            float b = -1.0f;
            int p = INT_MAX;
            for (int q = 0; q < ncta; q++) {
                const float v = *cl.map_shared_rank(&cand_v, q);
                const int i = *cl.map_shared_rank(&cand_i, q);
                if (v > b || (v == b && i < p)) { b = v; p = i; }
            }
            if (!(b > 0.0f) || !isfinite(b)) bad = 1;
            piv_k = p == INT_MAX ? k : p;
            if (rank == 0) Hp->piv[k] = piv_k;
        }
        __syncthreads();
        if (bad) break;  // the same decision in every CTA
        const int p = piv_k;
        const int ok = k / rows, op = p / rows;
        if (p != k) {  // rows k and p trade places: each owner fetches the other row first
            if (rank == ok)
                for (int j = tid; j < n; j += kInvThreads) tmp[j] = cl.map_shared_rank(A, op)[(p - op * rows) * n + j];
            if (rank == op && op != ok)
                for (int j = tid; j < n; j += kInvThreads) tmp[j] = cl.map_shared_rank(A, ok)[(k - ok * rows) * n + j];
            if (rank == op && op == ok)
                for (int j = tid; j < n; j += kInvThreads) {
                    const float t = A[(k - r0) * n + j];
                    A[(k - r0) * n + j] = A[(p - r0) * n + j];
                    A[(p - r0) * n + j] = t;
                }
            cl.sync();
            if (op != ok) {
                if (rank == ok) for (int j = tid; j < n; j += kInvThreads) A[(k - r0) * n + j] = tmp[j];
                if (rank == op) for (int j = tid; j < n; j += kInvThreads) A[(p - r0) * n + j] = tmp[j];
            }
            cl.sync();
        }
        // the pivot row, scaled, in every CTA
        const float* src = cl.map_shared_rank(A, ok) + (k - ok * rows) * n;
        const float inv = 1.0f / src[k];
        for (int j = tid; j < n; j += kInvThreads) rowk[j] = (j == k) ? inv : src[j] * inv;
        cl.sync();  // every CTA has its copy before the owner overwrites row k
        for (int i = r0 + wid; i < r1; i += kInvWarps) {
            float* row = A + (i - r0) * n;
            if (i == k) {
                for (int j = lane; j < n; j += 32) row[j] = rowk[j];
            } else {
                const float cik = row[k];
#pragma unroll 4
                for (int j = lane; j < n; j += 32) row[j] = (j == k) ? -cik * inv : fmaf(-cik, rowk[j], row[j]);
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (rank == 0 && tid == 0) atomicCAS((int*)&Hp->status, 0, (int)MVGD_EDEGENERATE);
        cl.sync();
        return;
    }
    for (int e = tid; e < (r1 - r0) * n; e += kInvThreads) a[(int64_t)r0 * n + e] = A[e];
    cl.sync();  // the rows of every CTA are in global memory
    if (rank != 0) return;
    if (tid == 0) {
        for (int c = 0; c < n; c++) col_of[c] = c;
        for (int k = n - 1; k >= 0; k--) {
            const int p = Hp->piv[k], t = col_of[k];
            col_of[k] = col_of[p];
            col_of[p] = t;
        }
    }
    __syncthreads();
    for (int c = wid; c < n; c += kInvWarps)
        for (int r = lane; r < n; r += 32) Hp->cinv[c * n + r] = a[r * n + col_of[c]];  // column-major
}

int grid_for(int64_t threads) {
    int64_t g = (threads + 255) / 256;
    return (int)(g > 16384 ? 16384 : (g < 1 ? 1 : g));
}

// ---------------------------------------------------------------------------
// Standalone V-cycle (stored order): one kernel per step.
// ---------------------------------------------------------------------------
struct ApplyVecs {
    float* y[kAmgMaxLevels];
    float* r[kAmgMaxLevels];
    float* b[kAmgMaxLevels];  // b[0] unused: level 0 reads the FP64 input
    float* x[kAmgMaxLevels];  // x[0] unused: level 0 writes the FP64 output
    size_t bytes;
};

ApplyVecs apply_layout(void* ws, int64_t n, int Q) {
    ApplyVecs V;
    memset(&V, 0, sizeof(V));
    int64_t sizes[kAmgMaxLevels];
    const int nlev = amg_levels(n, sizes);
    Carver cv(ws);
    for (int l = 0; l < nlev; l++) {
        const int64_t m = n_padded(sizes[l]) * Q;
        V.y[l] = cv.take<float>(m);
        V.r[l] = cv.take<float>(m);
        if (l > 0) {
            V.b[l] = cv.take<float>(m);
            V.x[l] = cv.take<float>(m);
        }
    }
    V.bytes = cv.used;
    return V;
}

// Rows of a level in whole warps: rows past the end only join the shuffles.
__global__ void k_vpre(const AmgHeader* __restrict__ Hp, const double* __restrict__ b, int Q, float* y0) {
    const AmgHeader& H = *Hp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < H.n * Q; e += (int64_t)gridDim.x * blockDim.x)
        y0[e] = H.lv[0].dinv[e / Q] * (float)b[e];
}

// Blocks of kApplyThreads threads take kApplyThreads / G consecutive rows at a
// time (G lanes a row, amg_group; level 0: G = 1), like the solver's steps.
constexpr int kApplyThreads = 256;

__global__ void __launch_bounds__(kApplyThreads) k_vdown(const AmgHeader* __restrict__ Hp, int l,
                                                         const double* __restrict__ b0, int Q, ApplyVecs V) {
    __shared__ float agg[kApplyThreads / kAmgAgg];
    const AmgHeader& H = *Hp;
    const int64_t nl = H.lv[l].n;
    const int G = l == 0 ? 1 : amg_group(nl);
    const int64_t rows = kApplyThreads / G;
    const float* Y = V.y[l];
    const bool last = (l + 1 == H.nlev - 1);
    // block-uniform loop: every thread reaches the barriers of agg_sum
    for (int64_t c = blockIdx.x; c * rows < nl; c += gridDim.x) {
        const int64_t r = c * rows + threadIdx.x / G;
        const bool valid = r < nl;
        for (int q = 0; q < Q; q++) {
            const float bi = valid ? (l == 0 ? (float)b0[r * Q + q] : V.b[l][r * Q + q]) : 0.0f;
            const float yi = valid ? Y[r * Q + q] : 0.0f;
            vdown_row(H, l, G, r, valid, Q, q, bi, yi, [&](int64_t j) { return Y[j * Q + q]; }, V.r[l], V.b[l + 1],
                      last ? nullptr : V.y[l + 1], [&](float xi, auto&& xv) { return a0_row(H, r, xi, xv); }, agg);
        }
    }
}

__global__ void k_vcoarse(const AmgHeader* __restrict__ Hp, const double* __restrict__ b0, double* x0, int Q,
                          ApplyVecs V) {
    const AmgHeader& H = *Hp;
    const int m = H.nlev - 1;
    const int64_t rho = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kWarp;
    if (rho >= H.nc) return;  // warp-uniform
    for (int q = 0; q < Q; q++) {
        float x;
        if (m == 0) x = coarse_row(H, rho, [&](int64_t c) { return (float)b0[c * Q + q]; });
        else x = coarse_row(H, rho, [&](int64_t c) { return V.b[m][c * Q + q]; });
        if (lane_id() == 0) {
            if (m == 0) x0[rho * Q + q] = (double)x;
            else V.x[m][rho * Q + q] = x;
        }
    }
}

__global__ void __launch_bounds__(kApplyThreads) k_vup(const AmgHeader* __restrict__ Hp, int l, double* x0, int Q,
                                                       ApplyVecs V) {
    const AmgHeader& H = *Hp;
    const int64_t nl = H.lv[l].n;
    const int G = l == 0 ? 1 : amg_group(nl);
    const int64_t rows = kApplyThreads / G;
    const float* Xc = V.x[l + 1];
    for (int64_t c = blockIdx.x; c * rows < nl; c += gridDim.x) {
        const int64_t r = c * rows + threadIdx.x / G;
        const bool valid = r < nl;
        for (int q = 0; q < Q; q++) {
            const float x = vup_row(H, l, G, r, valid, valid ? V.y[l][r * Q + q] : 0.0f,
                                    valid ? V.r[l][r * Q + q] : 0.0f, [&](int64_t J) { return Xc[J * Q + q]; },
                                    [&](float xi, auto&& xv) { return a0_row(H, r, xi, xv); });
            if (!valid || (threadIdx.x & (G - 1)) != 0) continue;
            if (l == 0) x0[r * Q + q] = (double)x;
            else V.x[l][r * Q + q] = x;
        }
    }
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_amg_workspace_bytes(int64_t n, int32_t k) {
    if (n < 1 || k < kMinK || k > kMaxK || amg_levels(n, nullptr) == 0) return 0;
    return amg_layout(nullptr, n, k).h.bytes;
}

MVGD_API mvgd_status mvgd_amg_setup(const mvgd_ell* L, double sigma, void* amg_ws, size_t amg_bytes,
                                    mvgd_stream_t stream) {
    if (!L || !amg_ws || !L->col || !L->val || L->n < 2 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK)
        return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!aligned(amg_ws) || !aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo)) return MVGD_EINVAL;
    if (!(sigma == sigma)) return MVGD_EINVAL;
    if (amg_levels(L->n, nullptr) == 0) return MVGD_EINVAL;
    AmgLayout A = amg_layout(amg_ws, L->n, L->k);
    if (amg_bytes < A.h.bytes) return MVGD_EWORKSPACE;
    A.h.sigma = sigma;
    A.h.col0 = L->col;
    A.h.val0 = L->val;
    A.h.val0_lo = L->val_lo;
    A.h.prec0 = L->prec;
    A.h.status = MVGD_OK;
    A.h.width_max = 0;
    cudaStream_t s = (cudaStream_t)stream;
    OpView O{L->col, L->val, L->val_lo, L->prec};
    k_amg_header<<<1, 1, 0, s>>>(A.h, A.hdr);
    k_amg_level0<<<grid_for(L->n), 256, 0, s>>>(A.hdr, O);
    for (int l = 0; l + 1 < A.h.nlev; l++) {
        const int64_t nc = A.h.lv[l + 1].n;
        k_amg_coarsen<<<grid_for(nc * kWarp), 256, 0, s>>>(A.hdr, O, l);
        k_amg_slice_width<<<grid_for(nc / kSlice + 1), 256, 0, s>>>(A.hdr, l + 1);
    }
    const int64_t nc = A.h.nc;
    MVGD_CUDA_TRY(cudaMemsetAsync(A.h.dense, 0, sizeof(float) * nc * nc, s));
    MVGD_CUDA_TRY(cudaMemsetAsync(A.h.dense64, 0, sizeof(double) * nc * nc, s));
    k_amg_dense<<<grid_for(nc), 256, 0, s>>>(A.hdr, O);
    {
        // rows a CTA holds: the matrix in at most 8 CTAs' shared memory (128 KB of rows each)
        const int rows = (int)std::min<int64_t>(nc, 32768 / nc);
        const int ncta = (int)((nc + rows - 1) / rows);
        const size_t smem = sizeof(float) * ((size_t)rows * nc + 2 * nc);
        MVGD_CUDA_TRY(cudaFuncSetAttribute(k_amg_invert_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)ncta);
        cfg.blockDim = dim3(kInvThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)ncta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        MVGD_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_amg_invert_cluster, A.hdr, rows));
    }
    // two Newton-Schulz steps X <- X (2I - A X) in FP64 from the FP32 inverse: its
    // residual (~1e-5) squares each step, to the FP64 level
    k_amg_promote<<<grid_for(nc * nc), 256, 0, s>>>(A.hdr);
    const dim3 gg((unsigned)((nc + kGemmTile - 1) / kGemmTile), (unsigned)((nc + kGemmTile - 1) / kGemmTile));
    double* X = A.h.cinv64;
    double* Xn = A.h.ns_x;
    for (int step = 0; step < 2; step++) {
        k_amg_dgemm<<<gg, 256, 0, s>>>((int)nc, A.h.dense64, X, A.h.ns_t, 2.0, -1.0);  // T = 2I - A X
        k_amg_dgemm<<<gg, 256, 0, s>>>((int)nc, X, A.h.ns_t, Xn, 0.0, 1.0);          // X' = X T
        double* t = X;
        X = Xn;
        Xn = t;
    }
    // after an even number of steps the result is back in cinv64
    return launch_status();
}

MVGD_API mvgd_status mvgd_amg_describe(const void* amg_ws, int32_t level, mvgd_amg_info* out) {
    if (!amg_ws || !out || !aligned(amg_ws)) return MVGD_EINVAL;
    AmgHeader h;
    MVGD_CUDA_TRY(cudaMemcpy(&h, amg_ws, sizeof(h), cudaMemcpyDeviceToHost));
    if (level < 0 || level >= h.nlev) return MVGD_EINVAL;
    const AmgLevel& L = h.lv[level];
    memset(out, 0, sizeof(*out));
    out->levels = h.nlev;
    out->status = h.status;
    out->width_max = h.width_max;
    out->n = L.n;
    out->stride = level == 0 ? h.k + 1 : kAmgStride;
    out->col = level == 0 ? h.col0 : L.col;
    out->val = L.val;
    out->val64 = L.val64;
    out->cnt = L.cnt;
    out->dinv = L.dinv;
    out->cinv = level == h.nlev - 1 ? h.cinv : nullptr;
    out->cinv64 = level == h.nlev - 1 ? h.cinv64 : nullptr;
    return MVGD_OK;
}

MVGD_API size_t mvgd_amg_apply_workspace_bytes(int64_t n, int32_t nrhs) {
    if (n < 1 || nrhs < 1 || nrhs > 8 || amg_levels(n, nullptr) == 0) return 0;
    return apply_layout(nullptr, n, nrhs).bytes;
}

MVGD_API mvgd_status mvgd_amg_apply(const void* amg_ws, int64_t n, int32_t nrhs, const double* b, double* x,
                                    void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!amg_ws || !b || !x || !ws || n < 1 || nrhs < 1 || nrhs > 8) return MVGD_EINVAL;
    if (!aligned(amg_ws) || !aligned(b) || !aligned(x) || !aligned(ws)) return MVGD_EINVAL;
    int64_t sizes[kAmgMaxLevels];
    const int nlev = amg_levels(n, sizes);
    if (nlev == 0) return MVGD_EINVAL;
    ApplyVecs V = apply_layout(ws, n, nrhs);
    if (ws_bytes < V.bytes) return MVGD_EWORKSPACE;
    const AmgHeader* H = static_cast<const AmgHeader*>(amg_ws);
    cudaStream_t s = (cudaStream_t)stream;
    const int m = nlev - 1;
    if (m > 0) k_vpre<<<grid_for(n * nrhs), 256, 0, s>>>(H, b, nrhs, V.y[0]);
    for (int l = 0; l < m; l++) k_vdown<<<grid_for(n_padded(sizes[l])), kApplyThreads, 0, s>>>(H, l, b, nrhs, V);
    k_vcoarse<<<grid_for(sizes[m] * kWarp), 256, 0, s>>>(H, b, x, nrhs, V);
    for (int l = m - 1; l >= 0; l--) k_vup<<<grid_for(n_padded(sizes[l])), kApplyThreads, 0, s>>>(H, l, x, nrhs, V);
    return launch_status();
}
