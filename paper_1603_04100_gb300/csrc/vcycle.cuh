// Row steps of one V(1,1)-cycle of the aggregation multigrid hierarchy (FP32),
// shared by the standalone application (amg.cu) and the persistent solver
// (solve.cu).  One lane per row; a warp holds 32 consecutive rows of a level,
// so the 8 rows of an aggregate sit in 8 consecutive lanes and restriction is
// a shuffle sum inside each group of 8.  Vectors are [rows][Q] FP32,
// right-hand sides interleaved.
//
// With A_l the level-l matrix, d_l its l1-Jacobi scaling and P the
// piecewise-constant prolongation, the cycle on b_0 is
//   down (l = 0 .. m-1): y_l = d_l b_l,  r_l = b_l - A_l y_l,  b_{l+1} = P^T r_l
//   coarsest:            x_m = A_m^-1 b_m
//   up   (l = m-1 .. 0): x_l = y_l + P x_{l+1} + d_l (r_l - A_l P x_{l+1})
// which is y_l + P x_{l+1} followed by one l1-Jacobi step on b_l, since
// b_l - A_l (y_l + P x_{l+1}) = r_l - A_l P x_{l+1}.
#pragma once

#include "amg.cuh"

namespace mvgd {

// Every product below is taken in difference form, sum_j a_ij (x_j - x_i) +
// (sum_j a_ij) x_i, with the row sum exact: rows of L sum to zero, so level 0
// is sigma x_i - sum_s w_s (x_j - x_i), and a Galerkin row sums to sigma times
// its aggregate's size.  In FP32 the smooth components of a residual b - A y
// -- the ones the coarse levels exist to remove -- are tiny differences of
// terms of size h^-2 |y|; summed in the standard form they lose about
// h^-2 / lambda_smooth times the FP32 rounding (at 1M points, ~1e-3
// relative), which made the cycle a poor, slightly nonlinear preconditioner
// (BiCGSTAB needed 457 iterations in an FP32 emulation, 195 with an FP64
// cycle); in difference form the FP32 cycle stays within a few % of FP64.

// Level-0 product with the operator's FP32 weights, x given by `xv(j)`.
template <typename XV>
__device__ __forceinline__ float a0_row(const AmgHeader& H, int64_t r, float xi, XV&& xv) {
    const int k = H.k, m = k + 1;
    const float* w = H.lv[0].val + (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
    const int32_t* c = H.col0 + (r / kSlice) * (int64_t)(kSlice * k) + (r % kSlice);
    float acc = 0.0f;
#pragma unroll 4
    for (int s = 0; s < k; s++) acc = fmaf(w[(s + 1) * kSlice], xv((int64_t)c[s * kSlice]) - xi, acc);
    return (float)H.sigma * xi - acc;
}

// The same product from a staged slice: colS [k][32] columns, w [k+1][32]
// weights (slot 0 = the row itself), lane = the row's place in its slice.
template <typename XV>
__device__ __forceinline__ float a0_row_staged(const int* colS, const float* w, int lane, int k, float sigma, float xi,
                                               XV&& xv) {
    float acc = 0.0f;
#pragma unroll 4
    for (int s = 0; s < k; s++)
        acc = fmaf(w[(s + 1) * kSlice + lane], xv((int64_t)colS[s * kSlice + lane]) - xi, acc);
    return sigma * xi - acc;
}

// Row j of an [n][Q] array into x[0..QT) (zeros past Q).  When Q == QT is 2,
// 4 or 8 the row is one or two aligned vector loads (workspace arrays start on
// 256 bytes), else Q scalar loads: a gather of all right-hand sides at a
// neighbour costs one memory instruction instead of Q.
template <int QT, typename T>
__device__ __forceinline__ void load_row(const T* X, int64_t j, int Q, T (&x)[QT]) {
    if constexpr (QT == 2 && sizeof(T) == 4) {
        if (Q == 2) {
            const float2 v = reinterpret_cast<const float2*>(X)[j];
            x[0] = v.x;
            x[1] = v.y;
            return;
        }
    } else if constexpr ((QT == 4 || QT == 8) && sizeof(T) == 4) {
        if (Q == QT) {
#pragma unroll
            for (int h = 0; h < QT / 4; h++) {
                const float4 v = reinterpret_cast<const float4*>(X)[j * (QT / 4) + h];
                x[4 * h] = v.x;
                x[4 * h + 1] = v.y;
                x[4 * h + 2] = v.z;
                x[4 * h + 3] = v.w;
            }
            return;
        }
    } else if constexpr (QT >= 2 && QT <= 8 && (QT & (QT - 1)) == 0 && sizeof(T) == 8) {
        if (Q == QT) {
#pragma unroll
            for (int h = 0; h < QT / 2; h++) {
                const double2 v = reinterpret_cast<const double2*>(X)[j * (QT / 2) + h];
                x[2 * h] = v.x;
                x[2 * h + 1] = v.y;
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < QT; q++) x[q] = q < Q ? X[j * Q + q] : T(0);
}

// Level-0 products of every right-hand side from a staged slice (colS [k][32]
// columns, w [k+1][32] weights, slot 0 = the row itself): out[q] = sigma xi[q]
// - sum_s w_s (x_j[q] - xi[q]), the neighbours' rows read by `xrow(j, x)`.
// Each q's operations are those of a0_row_staged, in the same order.
template <int QT, typename XR>
__device__ __forceinline__ void a0_rows_staged(const int* colS, const float* w, int lane, int k, float sigma,
                                               const float (&xi)[QT], float (&out)[QT], XR&& xrow) {
    float acc[QT];
#pragma unroll
    for (int q = 0; q < QT; q++) acc[q] = 0.0f;
#pragma unroll 4
    for (int s = 0; s < k; s++) {
        float xj[QT];
        xrow((int64_t)colS[s * kSlice + lane], xj);
        const float ws = w[(s + 1) * kSlice + lane];
#pragma unroll
        for (int q = 0; q < QT; q++) acc[q] = fmaf(ws, xj[q] - xi[q], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < QT; q++) out[q] = sigma * xi[q] - acc[q];
}

// Level-l (>= 1) product with the explicit Galerkin matrix, row r taken by the
// G lanes of its group (groups aligned in the warp).  The sum is split over
// V = amg_group(n_l) virtual lanes (V a multiple of G, M = V / G <= 8 of them a
// lane): virtual lane v adds the row's slots v, v + V, v + 2V, ... in order,
// and a butterfly over the V virtual lanes (offsets 1, 2, 4, ...) adds them.
// Lane j of the group holds virtual lanes j, j + G, ...; the butterfly's
// offsets below G are shuffles, the others adds inside the lane -- the same
// operations in the same order for every G, so the result depends on V (the
// request's level size) alone, and every lane of the group returns it.
// Padding slots are (own row, 0).  Lanes of invalid rows return 0 but take
// part in the shuffles.
template <int M, int QT, typename XR>
__device__ __forceinline__ void al_rows_m(const AmgLevel& Lv, int64_t r, bool valid, int G, const float (&xi)[QT],
                                          XR&& xrow, float (&out)[QT]) {
    const int V = M * G;
    float acc[M][QT];
#pragma unroll
    for (int m = 0; m < M; m++)
#pragma unroll
        for (int q = 0; q < QT; q++) acc[m][q] = 0.0f;
    if (valid) {
        const int j = (int)(lane_id() & (G - 1));
        const int64_t base = (r / kSlice) * (int64_t)(kSlice * kAmgStride) + (r % kSlice);
        // the slice's widest row, rounded up to whole groups of V slots: every row
        // is padded with (own row, 0) to the full stride, whose terms add exact zeros
        const int w = (Lv.sw[r / kSlice] + V - 1) & ~(V - 1);
        constexpr int kUnroll = M >= 4 ? 1 : 4 / M;  // about four slots in flight a lane
#pragma unroll kUnroll
        for (int s0 = 0; s0 < w; s0 += V) {
#pragma unroll
            for (int m = 0; m < M; m++) {
                const int64_t e = base + (int64_t)(s0 + j + m * G) * kSlice;
                const float a = Lv.val[e];
                float x[QT];
                xrow((int64_t)Lv.col[e], x);  // every right-hand side of the neighbour at once
#pragma unroll
                for (int q = 0; q < QT; q++) acc[m][q] = fmaf(a, x[q] - xi[q], acc[m][q]);
            }
        }
    }
    for (int o = 1; o < G; o <<= 1)
#pragma unroll
        for (int m = 0; m < M; m++)
#pragma unroll
            for (int q = 0; q < QT; q++) acc[m][q] += __shfl_xor_sync(0xffffffffu, acc[m][q], o);
#pragma unroll
    for (int d = 1; d < M; d <<= 1)
#pragma unroll
        for (int m = 0; m < M; m++)
            if ((m & d) == 0)
#pragma unroll
                for (int q = 0; q < QT; q++) {
                    const float t = acc[m][q] + acc[m + d][q];
                    acc[m][q] = t;
                    acc[m + d][q] = t;
                }
    const float rs = valid ? Lv.rs[r] : 0.0f;
#pragma unroll
    for (int q = 0; q < QT; q++) out[q] = valid ? fmaf(rs, xi[q], acc[0][q]) : 0.0f;
}

// Products of every right-hand side at once: out[q] = (A_l x_q)[r], the
// neighbours' rows read by `xrow(j, x)`; each q's operations are those of a
// single product, in the same order.
template <int QT, typename XR>
__device__ __forceinline__ void al_rows(const AmgLevel& Lv, int64_t r, bool valid, int G, const float (&xi)[QT],
                                        XR&& xrow, float (&out)[QT]) {
    // M = V / G <= kAmgMaxPerLane / QT (amg_lanes): no larger case is instantiated
    constexpr int kMmax = kAmgMaxPerLane / QT > 1 ? kAmgMaxPerLane / QT : 1;
    const int M = amg_group(Lv.n) / G;  // warp-uniform
    if (kMmax >= 8 && M >= 8) al_rows_m<(kMmax >= 8 ? 8 : 1), QT>(Lv, r, valid, G, xi, xrow, out);
    else if (kMmax >= 4 && M >= 4) al_rows_m<(kMmax >= 4 ? 4 : 1), QT>(Lv, r, valid, G, xi, xrow, out);
    else if (kMmax >= 2 && M >= 2) al_rows_m<(kMmax >= 2 ? 2 : 1), QT>(Lv, r, valid, G, xi, xrow, out);
    else al_rows_m<1, QT>(Lv, r, valid, G, xi, xrow, out);
}

template <typename XV>
__device__ __forceinline__ float al_row(const AmgLevel& Lv, int64_t r, bool valid, int G, float xi, XV&& xv) {
    const float x1[1] = {xi};
    float o1[1];
    al_rows<1>(Lv, r, valid, G, x1, [&](int64_t j, float (&x)[1]) { x[0] = xv(j); }, o1);
    return o1[0];
}

// Sum of a value over the 8 rows of each aggregate, rows of G lanes each,
// returned to the lanes of the aggregate's first row (((v0+v1)+(v2+v3))+
// ((v4+v5)+(v6+v7)) for every G).  Up to G = 4 an aggregate lies in one warp
// and the sum is a butterfly; above, it spans warps and goes through `agg`
// (kThreads / G floats of shared memory) between two block barriers, so every
// thread of the block must call it.
__device__ __forceinline__ float agg_sum(float v, int G, float* agg) {
    if (G <= 4) {
        for (int o = G; o < kAmgAgg * G; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    const int i = (int)threadIdx.x / G;  // the row's place in the block
    if ((threadIdx.x & (G - 1)) == 0) agg[i] = v;
    __syncthreads();
    const float* a = agg + (i & ~(kAmgAgg - 1));
    v = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    __syncthreads();
    return v;
}

// Down step of level l for right-hand side q of row r (G lanes a row; level 0
// takes G = 1).  `b` is the row's own right-hand side (level 0: the Krylov
// vector, rounded to FP32), `y_of(j)` the pre-smoothed y_l at any row j
// (already stored: level 0 by the step that formed b_0, level >= 1 by the
// restriction that formed b_l).  Writes r_l, and b_{l+1}, y_{l+1} of the
// aggregate (the first lane of its first row).  `a0(xi, xv)` is the level-0
// product (from global memory or a staged slice).  With G >= 8 every thread
// of the block calls it (see agg_sum).
// The rest of a down step once the row's residual res = b - A_l y is known.
__device__ __forceinline__ void vdown_finish(const AmgHeader& H, int l, int G, int64_t r, bool valid, int Q, int q,
                                             float res, float* R, float* Bn, float* Yn, float* agg) {
    const bool lead = (lane_id() & (G - 1)) == 0;
    if (!valid) res = 0.0f;  // rows past the end contribute 0
    if (valid && lead) R[r * Q + q] = res;
    const float bc = agg_sum(res, G, agg);
    if (valid && lead && (r % kAmgAgg) == 0) {
        const int64_t I = r / kAmgAgg;
        Bn[I * Q + q] = bc;
        if (Yn) Yn[I * Q + q] = H.lv[l + 1].dinv[I] * bc;
    }
}

template <typename YOF, typename A0>
__device__ __forceinline__ void vdown_row(const AmgHeader& H, int l, int G, int64_t r, bool valid, int Q, int q,
                                          float b, float yi, YOF&& y_of, float* R, float* Bn, float* Yn, A0&& a0,
                                          float* agg) {
    float res = 0.0f;
    if (l == 0) {
        if (valid) res = b - a0(yi, y_of);
    } else {
        res = b - al_row(H.lv[l], r, valid, G, yi, y_of);
    }
    vdown_finish(H, l, G, r, valid, Q, q, res, R, Bn, Yn, agg);
}

// Up step of level l: x_l = y_l + P x_{l+1} + d_l (r_l - A_l P x_{l+1}), for
// row r of G lanes (level 0: G = 1); every lane of a valid row returns x.
template <typename XC, typename A0>
__device__ __forceinline__ float vup_row(const AmgHeader& H, int l, int G, int64_t r, bool valid, float yi, float ri,
                                         XC&& xc_of, A0&& a0) {
    const float xc = valid ? xc_of(r / kAmgAgg) : 0.0f;
    auto pxc = [&](int64_t j) { return xc_of(j / kAmgAgg); };
    float apx;
    if (l == 0) apx = valid ? a0(xc, pxc) : 0.0f;
    else apx = al_row(H.lv[l], r, valid, G, xc, pxc);
    return valid ? yi + xc + H.lv[l].dinv[r] * (ri - apx) : 0.0f;
}

// Coarsest solve, one warp per row rho: x[rho] = sum_c X[rho][c] b[c] with X
// the FP64 inverse (row-major, lanes along the row) and the sum in FP64.  An
// FP32 product with the inverse carries cond(A_c) ~ 1e4 times the FP32
// rounding (about 1e-3 relative at 1M points), which cost the outer Krylov
// solve ~20 % more iterations; in FP64 the cost is ~8 FP64 FMAs per lane.
template <typename BOF>
__device__ __forceinline__ float coarse_row(const AmgHeader& H, int64_t rho, BOF&& b_of) {
    const int64_t nc = H.nc;
    const double* row = H.cinv64 + rho * nc;
    double acc = 0.0;
    for (int64_t c = lane_id(); c < nc; c += kWarp) acc = fma(row[c], (double)b_of(c), acc);
    return (float)warp_sum(acc);
}

}  // namespace mvgd
