// Aggregation multigrid hierarchy of sigma I - L: the layout shared by its
// set-up (amg.cu) and the V-cycle phases of the persistent solver (solve.cu).
#pragma once

#include "common.cuh"

namespace mvgd {

constexpr int kAmgAgg = MVGD_AMG_AGG;            // rows per aggregate (consecutive in stored order)
constexpr int kAmgCoarsest = MVGD_AMG_COARSEST;  // a level this small is solved exactly
constexpr int kAmgStride = MVGD_AMG_MAX_WIDTH;   // slots per coarse row in the sliced layout
constexpr int kAmgMaxLevels = 12;

// The smoother's scaling of a row with diagonal a_ii and l1 norm sum_j |a_ij|
// (FP64, rounded once): omega / a_ii on a strong diagonal, else the l1 scaling.
__host__ __device__ inline float amg_smoother_scale(double diag, double l1) {
    if (diag > MVGD_AMG_JACOBI_THETA * l1) return (float)(MVGD_AMG_JACOBI_OMEGA / diag);
    return l1 > 0.0 ? (float)(1.0 / l1) : 1.0f;
}

// One level.  Level 0 is the operator itself: its neighbour columns (the
// operator's `col`, K slots) and an FP32 copy of its weights ([n_pad][K+1],
// slot 0 = the point itself), so that A x = sigma x_i - (w_0 x_i + sum_s w_s x_j).
// Levels >= 1 hold A explicitly: per row `cnt` entries (column, value) sorted
// by column, padded to the slice's widest row with (own index, 0).
struct AmgLevel {
    int64_t n;
    int32_t* col;    // level >= 1: [n_pad][kAmgStride] sliced
    float* val;      // level 0: [n_pad][K+1]; level >= 1: [n_pad][kAmgStride]
    double* val64;   // level >= 1: FP64 values (the Galerkin sums before rounding)
    int32_t* cnt;    // level >= 1: [n] entries per row
    int32_t* sw;     // level >= 1: [n_pad / 32] widest row of each slice
    float* dinv;     // [n] the smoother's scaling (amg_smoother_scale)
    float* rs;       // level >= 1: [n] row sums sum_j a_ij (FP64 sums, rounded once)
};

struct AmgHeader {
    int32_t nlev;       // levels, the coarsest included (>= 1)
    int32_t k;          // K of the operator
    int32_t status;     // MVGD_OK, or why set-up failed (device-written)
    int32_t width_max;  // widest coarse row (device-written)
    int64_t n;          // rows of level 0
    double sigma;
    const int32_t* col0;  // the operator's columns (level 0)
    AmgLevel lv[kAmgMaxLevels];
    const void* val0;   // the operator's weights (FP64, or FP32 hi) and
    const float* val0_lo;  //   lo (mixed format), for an exact coarsest residual on one-level hierarchies
    int32_t prec0, pad0;
    float* dense;       // [nc][nc] the coarsest level as a dense matrix (FP32, set-up scratch)
    float* cinv;        // [nc][nc] its FP32 Gauss-Jordan inverse, column-major: cinv[c * nc + r] = (A_c^-1)[r][c]
    double* dense64;    // [nc][nc] the coarsest level, FP64 row-major
    double* cinv64;     // [nc][nc] the inverse after two Newton-Schulz steps in FP64, row-major (what the cycle uses)
    double* ns_x;       // [nc][nc] set-up scratch
    double* ns_t;       // [nc][nc] set-up scratch
    int32_t* piv;       // [nc] set-up scratch
    int64_t nc;         // rows of the coarsest level
    size_t bytes;       // whole hierarchy
};

// Lanes of a row of level l >= 1 in a V-cycle step.  A coarse row holds 10-60
// entries; one lane per row makes each step a chain of that many dependent L2
// round trips on a level too small to fill the GPU, so a level of `rows` rows
// takes amg_group(rows) lanes a row: the largest power of two <= 32 that keeps
// rows x G within one pass of 152 SMs x 3 blocks x 256 threads.
//  - The product's arithmetic follows V = amg_group(n_l) of the request's own
//    level ("virtual lanes", al_row), so a request's result does not depend on
//    what else shares the launch.
//  - The lanes that take a row in a launch are G = max(amg_group(launch's rows
//    at level l), V Q / kAmgMaxPerLane) <= V (Q: the launch's widest request,
//    whose right-hand sides a lane takes at once): a batch of small requests
//    is not cut into units of a few rows each, and no lane holds more than
//    kAmgMaxPerLane partial sums.  Alone with one right-hand side, G = V.
// A block of 256 threads takes 256 / G rows: always whole aggregates.
constexpr int kAmgMaxPerLane = 8;
constexpr int64_t kAmgLanesOnePass = 152 * 3 * 256;
__host__ __device__ inline int amg_group(int64_t rows) {
    int g = 1;
    while (g < 32 && rows * 2 * g <= kAmgLanesOnePass) g *= 2;
    return g;
}
__host__ __device__ inline int amg_lanes(int launch_group, int64_t own_rows, int nrhs) {
    const int v = amg_group(own_rows);
    // virtual lanes a lane holds, times the right-hand sides it takes at once, <= kAmgMaxPerLane
    const int per_lane = kAmgMaxPerLane / nrhs > 1 ? kAmgMaxPerLane / nrhs : 1;
    const int g = v / per_lane;
    return launch_group > g ? (launch_group < v ? launch_group : v) : (g > 1 ? g : 1);
}

// Level sizes for a fine size n: n_0 = n, n_{l+1} = ceil(n_l / kAmgAgg) while
// n_l > kAmgCoarsest.  Returns the level count (0 if it would exceed the maximum).
__host__ __device__ inline int amg_levels(int64_t n, int64_t* sizes) {
    int l = 0;
    int64_t m = n;
    while (true) {
        if (l >= kAmgMaxLevels) return 0;
        if (sizes) sizes[l] = m;
        l++;
        if (m <= kAmgCoarsest) return l;
        m = (m + kAmgAgg - 1) / kAmgAgg;
    }
}

}  // namespace mvgd
