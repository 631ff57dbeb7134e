// MVGD row assembly (Sec. 2 and Sec. 3.1), FP64, one thread per point.
//
// FP64 issues at 1/56 of the FP32 rate on this part, and a warp instruction
// costs the same whether 1 or 32 lanes are active, so every FP64 step runs
// lane-parallel over 32 independent points.  Each lane keeps its (k+1) x 7
// design matrix [1, xi, eta, xi^2, xi eta, eta^2 | zeta] in shared memory,
// laid out lane-contiguously (element e of lane l at e * 32 + l) so every
// access is a conflict-free 256-byte wavefront.  One block = one warp = one
// 32-row slice of the sliced ELL output, so every store is coalesced.
//
// Per point:
//   offsets d_s = p_j - p_i of the k neighbours;
//   barycenter and covariance of N(i); cyclic Jacobi -> e_x (largest),
//   e_y (middle), e_z (smallest eigenvalue);
//   h by the chosen rule; h-scaled local coordinates (xi, eta, zeta);
//   Householder QR of the design matrix over p_i and N(i), applied to zeta;
//   surface coefficients a~ = R^-1 Q^T zeta; metric and A_1..A_5 at the
//   origin (from Eq. 1 for a graph surface);
//   the row in closed form: with c~ = (2(A3+A5), A1 h, A2 h, 2 A3, A4, 2 A5),
//   y = Q R^-T c~ equals P~^T c~ for the projector P~ of the h-scaled fit, and
//   w = y / h^2 except w_self = (y_0 - 2(A3+A5)) / h^2 -- the centred
//   differences on the 3x3 virtual grid of spacing h of a quadratic U(x,y),
//   with U_i in place of U(0,0).
//
// The FP32_REFINE format (weights stored as FP32 hi + lo) is assembled by an
// FP32 path instead (assemble_lane_mixed): the same steps with the
// neighbourhood arithmetic in double-float on the FP32 pipe (df.cuh) and FP64
// kept for the eigenvectors of the 3x3 covariance:
//   offsets p_j - p_i in FP64 (exact for nearby points), then split into
//   double-float; barycenter, mean distance and covariance in double-float;
//   an FP32 Jacobi frame polished by FP64 Jacobi sweeps on Q^T C Q;
//   local coordinates centred at p_i and scaled by h in double-float;
//   the least squares through the normal equations G = V^T V, formed from the
//   double-float moments sum xi^a eta^b (a + b <= 4) and sum xi^a eta^b zeta,
//   solved with an FP32 Cholesky factor of G and refined with double-float
//   residuals until the correction is below 2^-44 of the solution:
//   a~ = G^-1 V^T zeta, then g = G^-1 c~ and y = V g (= Q R^-T c~);
//   the weights y / h^2 come out as the (hi, lo) pair itself.
// In h-scaled coordinates cond(V) is small (about 6 typically, below 100 on
// the workloads' clouds), so G's FP32 factor contracts the error by about
// cond(G) 2^-24 per step and the double-float residuals carry the result to
// within about cond(G) 2^-48 of the exact solution.  A row whose G has a
// 1-norm condition number above 4096 (or its factor a tiny pivot), whose
// refinement does not settle, or with a non-finite value or an invalid
// neighbour index is handed to the FP64 path (k_assemble_fix), which also
// sets its row_status.
#include <vector>

#include "common.cuh"
#include "df.cuh"
#include "frame.cuh"

namespace mvgd {
namespace {

constexpr int kCols = 7;

struct AsmArgs {
    const double* pts;
    int64_t n;
    int k;
    const int32_t* nbr;
    const int32_t* order;   // stored row -> point
    const int32_t* inv;     // point -> stored row (only with order)
    int delta_kind, delta_m;
    double delta_scale;
    int variant;  // mvgd_row_variant
    int prec;
    int32_t* col;
    void* val;
    float* val_lo;
    double* h_out;
    uint8_t* status;
    int32_t* bad_rows;
    int arith;              // 1: FP64 arithmetic for the FP32_REFINE format too
    int kcap;               // the K a warp's shared memory is sized for (>= k)
    int2* fix;              // FP32 path: (item, row) handed to the FP64 path
    int32_t* nfix;
};

// Stored row `row` of one cloud's operator in FP64, by this lane (its design
// matrix lives in the lane's column of the warp's shared memory).
__device__ __noinline__ void assemble_lane(const AsmArgs& A, int64_t row) {
    extern __shared__ double sm[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int k = A.k, m = k + 1;
    double* smw = sm + (size_t)(threadIdx.x / kWarp) * (size_t)(A.kcap + 1) * kCols * kWarp;  // this warp's part
    // element (r, c) of this lane's design matrix
#define VM(r, c) smw[((r) * kCols + (c)) * kWarp + lane]

    const int64_t i = A.order ? (int64_t)A.order[row] : row;
    const double px = A.pts[3 * i], py = A.pts[3 * i + 1], pz = A.pts[3 * i + 2];
    const int32_t* nb = A.nbr + i * k;

    // offsets and barycenter of N(i); an index outside [0, n) marks the row
    // non-finite and is read as the point itself
    double cx = 0, cy = 0, cz = 0;
    bool idx_ok = true;
    for (int s = 0; s < k; s++) {
        int64_t j = nb[s];
        if (j < 0 || j >= A.n) { idx_ok = false; j = i; }
        double dx = A.pts[3 * j] - px, dy = A.pts[3 * j + 1] - py, dz = A.pts[3 * j + 2] - pz;
        VM(s + 1, 0) = dx;
        VM(s + 1, 1) = dy;
        VM(s + 1, 2) = dz;
        cx += dx; cy += dy; cz += dz;
    }
    const double rk = 1.0 / (double)k;
    cx *= rk; cy *= rk; cz *= rk;
    double C[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double hsum = 0;
    for (int s = 0; s < k; s++) {
        double dx = VM(s + 1, 0), dy = VM(s + 1, 1), dz = VM(s + 1, 2);
        if (s < A.delta_m) hsum += sqrt(dx * dx + dy * dy + dz * dz);
        dx -= cx; dy -= cy; dz -= cz;
        C[0][0] += dx * dx; C[0][1] += dx * dy; C[0][2] += dx * dz;
        C[1][1] += dy * dy; C[1][2] += dy * dz; C[2][2] += dz * dz;
    }
    C[1][0] = C[0][1]; C[2][0] = C[0][2]; C[2][1] = C[1][2];
    double V[3][3], ev[3];
    jacobi3(C, V, ev);
    int imax = 0, imin = 0;
    for (int a = 1; a < 3; a++) {
        if (ev[a] > ev[imax]) imax = a;
        if (ev[a] < ev[imin]) imin = a;
    }
    if (imax == imin) imin = (imax + 1) % 3;
    const int imid = 3 - imax - imin;
    const double ex0 = V[0][imax], ex1 = V[1][imax], ex2 = V[2][imax];
    const double ey0 = V[0][imid], ey1 = V[1][imid], ey2 = V[2][imid];
    const double ez0 = V[0][imin], ez1 = V[1][imin], ez2 = V[2][imin];

    // local coordinates; quarter-range extents
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int s = 1; s <= k; s++) {
        double dx = VM(s, 0), dy = VM(s, 1), dz = VM(s, 2);
        double lx = dx * ex0 + dy * ex1 + dz * ex2;
        double ly = dx * ey0 + dy * ey1 + dz * ey2;
        double lz = dx * ez0 + dy * ez1 + dz * ez2;
        VM(s, 0) = lx; VM(s, 1) = ly; VM(s, 2) = lz;
        x0 = fmin(x0, lx); x1 = fmax(x1, lx);
        y0 = fmin(y0, ly); y1 = fmax(y1, ly);
    }
    double h = (A.delta_kind == MVGD_DELTA_QUARTER_RANGE) ? fmin(0.25 * (x1 - x0), 0.25 * (y1 - y0))
                                                          : hsum / (double)A.delta_m;
    h *= A.delta_scale;
    const double ih = 1.0 / h;

    // design matrix in h units: row 0 is p_i itself
    VM(0, 0) = 1.0;
    for (int c = 1; c < kCols; c++) VM(0, c) = 0.0;
    for (int s = 1; s <= k; s++) {
        double xi = VM(s, 0) * ih, eta = VM(s, 1) * ih, zeta = VM(s, 2) * ih;
        VM(s, 0) = 1.0; VM(s, 1) = xi; VM(s, 2) = eta;
        VM(s, 3) = xi * xi; VM(s, 4) = xi * eta; VM(s, 5) = eta * eta;
        VM(s, 6) = zeta;
    }

    // Householder QR; v_k stored below the diagonal with v_k[k] kept in vk[k]
    double rd[6], vk[6], bk[6];
    for (int kc = 0; kc < 6; kc++) {
        double sig = 0;
        for (int r = kc; r < m; r++) { double a = VM(r, kc); sig += a * a; }
        double xk = VM(kc, kc);
        double alpha = (xk > 0) ? -sqrt(sig) : sqrt(sig);
        double den = sig - xk * alpha;     // v^T v / 2
        double beta = den > 0 ? 1.0 / den : 0.0;
        double v0 = xk - alpha;
        for (int c = kc + 1; c < kCols; c++) {
            double sdot = v0 * VM(kc, c);
            for (int r = kc + 1; r < m; r++) sdot += VM(r, kc) * VM(r, c);
            sdot *= beta;
            VM(kc, c) -= sdot * v0;
            for (int r = kc + 1; r < m; r++) VM(r, c) -= sdot * VM(r, kc);
        }
        rd[kc] = alpha;
        vk[kc] = v0;
        bk[kc] = beta;
    }
    double rmin = fabs(rd[0]);
    for (int c = 1; c < 6; c++) rmin = fmin(rmin, fabs(rd[c]));
    int st = (rmin < 1e-10 * fabs(rd[0])) ? 1 : 0;

    // a~ = R^-1 (Q^T zeta); only a~_1..a~_5 are needed
    double at[6];
    for (int r = 5; r >= 1; r--) {
        double s = VM(r, 6);
        for (int c = r + 1; c < 6; c++) s -= VM(r, c) * at[c];
        at[r] = s / rd[r];
    }
    const double zx = at[1], zy = at[2];
    const double zxx = 2.0 * at[3] * ih, zxy = at[4] * ih, zyy = 2.0 * at[5] * ih;
    const double W = 1.0 + zx * zx + zy * zy;
    const double iW = 1.0 / W;
    const double g11 = (1.0 + zy * zy) * iW, g12 = -zx * zy * iW, g22 = (1.0 + zx * zx) * iW;
    const double Hs = g11 * zxx + 2.0 * g12 * zxy + g22 * zyy;
    const double A1 = -Hs * zx * iW, A2 = -Hs * zy * iW, A3 = g11, A4 = 2.0 * g12, A5 = g22;
    // the least-squares comparator drops the centre-value term: c~_0 = 0 and no
    // self correction, which leaves the LB of the fitted quadratic itself
    const double c0 = A.variant == MVGD_ROW_LS ? 0.0 : 2.0 * (A3 + A5);
    const double ct[6] = {c0, A1 * h, A2 * h, 2.0 * A3, A4, 2.0 * A5};

    // t = R^-T c~ (forward substitution), y = Q [t; 0]
    double t[6];
    for (int r = 0; r < 6; r++) {
        double s = ct[r];
        for (int c = 0; c < r; c++) s -= VM(c, r) * t[c];
        t[r] = s / rd[r];
    }
    for (int r = 0; r < m; r++) VM(r, 6) = (r < 6) ? t[r] : 0.0;
    for (int kc = 5; kc >= 0; kc--) {
        double sdot = vk[kc] * VM(kc, 6);
        for (int r = kc + 1; r < m; r++) sdot += VM(r, kc) * VM(r, 6);
        sdot *= bk[kc];
        VM(kc, 6) -= sdot * vk[kc];
        for (int r = kc + 1; r < m; r++) VM(r, 6) -= sdot * VM(r, kc);
    }
    const double ih2 = ih * ih;
    bool finite = isfinite(h) && h > 0;
    if (A.prec == MVGD_FP64) {
        double* vo = static_cast<double*>(A.val);
        for (int r = 0; r < m; r++) {
            double w = (r == 0 ? VM(0, 6) - c0 : VM(r, 6)) * ih2;
            finite = finite && isfinite(w);
            vo[sell_index(row, r, m)] = w;
        }
    } else {
        float* vo = static_cast<float*>(A.val);
        for (int r = 0; r < m; r++) {
            double w = (r == 0 ? VM(0, 6) - c0 : VM(r, 6)) * ih2;
            finite = finite && isfinite(w);
            float hi = __double2float_rn(w);
            vo[sell_index(row, r, m)] = hi;
            A.val_lo[sell_index(row, r, m)] = __double2float_rn(w - (double)hi);
        }
    }
    for (int s = 0; s < k; s++) {
        int32_t j = nb[s];
        if (j < 0 || j >= A.n) j = (int32_t)i;
        A.col[sell_index(row, s, k)] = A.inv ? A.inv[j] : j;
    }
    if (!finite || !idx_ok) st = 2;
    if (A.h_out) A.h_out[i] = h;
    if (A.status) A.status[i] = (uint8_t)st;
    if (st && A.bad_rows) atomicAdd(A.bad_rows, 1);
#undef VM
}

// ---------------------------------------------------------------------------
// The FP32 path of the FP32_REFINE format (see the head of this file).
// ---------------------------------------------------------------------------
constexpr int kMixCols = 6;              // per neighbour: three double-float values
constexpr int kRefineSteps = 4;          // refinement steps of each 6x6 solve
constexpr float kPivotFloor = 0x1p-16f;  // Cholesky pivot / diagonal below this: FP64 path
constexpr float kCondCap = 4096.0f;      // 1-norm condition number of G above this: FP64 path
constexpr float kSettled = 0x1p-30f;     // last correction / solution above this: FP64 path

// Index of the moment sum xi^a eta^b (a + b <= 4) among the 15 moments.
__host__ __device__ constexpr int moment_index(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }
// Exponents of the quadratic basis [1, xi, eta, xi^2, xi eta, eta^2].
__host__ __device__ constexpr int mono_a(int p) { return p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0); }
__host__ __device__ constexpr int mono_b(int p) { return p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0); }

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // packed lower, j <= i

// FP32 Cholesky G = L L^T of the hi parts of a symmetric 6x6 (packed lower).
// False when a pivot falls below kPivotFloor of its diagonal entry.
__device__ __forceinline__ bool chol6(const df (&G)[21], float (&L)[21]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        float d = G[tri(j, j)].hi;
#pragma unroll
        for (int q = 0; q < j; q++) d = fmaf(-L[tri(j, q)], L[tri(j, q)], d);
        ok = ok && (d > kPivotFloor * G[tri(j, j)].hi);
        const float ljj = sqrtf(fmaxf(d, 1e-30f));
        L[tri(j, j)] = ljj;
        const float inv = 1.0f / ljj;
#pragma unroll
        for (int i = j + 1; i < 6; i++) {
            float t = G[tri(i, j)].hi;
#pragma unroll
            for (int q = 0; q < j; q++) t = fmaf(-L[tri(i, q)], L[tri(j, q)], t);
            L[tri(i, j)] = t * inv;
        }
    }
    return ok;
}

// x = (L L^T)^-1 r in FP32.
__device__ __forceinline__ void chol6_solve(const float (&L)[21], const float (&r)[6], float (&x)[6]) {
    float z[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
        float t = r[i];
#pragma unroll
        for (int q = 0; q < i; q++) t = fmaf(-L[tri(i, q)], z[q], t);
        z[i] = t / L[tri(i, i)];
    }
#pragma unroll
    for (int i = 5; i >= 0; i--) {
        float t = z[i];
#pragma unroll
        for (int q = i + 1; q < 6; q++) t = fmaf(-L[tri(q, i)], x[q], t);
        x[i] = t / L[tri(i, i)];
    }
}

// The 1-norm condition number |G|_1 |G^-1|_1 of the hi parts, G^-1 column by
// column from the FP32 factor.  It sets the accuracy the double-float
// residuals can reach, about cond(G) 2^-48 of the solution.
__device__ __forceinline__ float cond1_6(const df (&G)[21], const float (&L)[21]) {
    float gn = 0.0f, gin = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; j++) {
        float e[6], x[6], cs = 0.0f, ci = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; i++) {
            e[i] = i == j ? 1.0f : 0.0f;
            cs += fabsf(G[i >= j ? tri(i, j) : tri(j, i)].hi);
        }
        chol6_solve(L, e, x);
#pragma unroll
        for (int i = 0; i < 6; i++) ci += fabsf(x[i]);
        gn = fmaxf(gn, cs);
        gin = fmaxf(gin, ci);
    }
    return gn * gin;
}

// Solves G x = rhs: the FP32 factor's solution, then kRefineSteps corrections
// from double-float residuals rhs - G x.  False when the last correction is
// still above kSettled of the solution (the factor does not contract).
__device__ __forceinline__ bool solve6_refined(const df (&G)[21], const float (&L)[21], const df (&rhs)[6],
                                               df (&x)[6]) {
    float r[6], d[6];
#pragma unroll
    for (int p = 0; p < 6; p++) r[p] = rhs[p].hi;
    chol6_solve(L, r, d);
#pragma unroll
    for (int p = 0; p < 6; p++) x[p] = df_make(d[p]);
    float last = 0.0f, xmax = 0.0f;
#pragma unroll 1
    for (int it = 0; it < kRefineSteps; it++) {
#pragma unroll
        for (int p = 0; p < 6; p++) {
            df t = rhs[p];
#pragma unroll
            for (int q = 0; q < 6; q++) t = df_sub(t, df_mul(G[p >= q ? tri(p, q) : tri(q, p)], x[q]));
            r[p] = t.hi;
        }
        chol6_solve(L, r, d);
        last = 0.0f;
        xmax = 0.0f;
#pragma unroll
        for (int p = 0; p < 6; p++) {
            x[p] = df_add(x[p], df_make(d[p]));
            last = fmaxf(last, fabsf(d[p]));
            xmax = fmaxf(xmax, fabsf(x[p].hi));
        }
    }
    return last <= kSettled * xmax;
}

// Stored row `row` of one cloud's operator in the FP32_REFINE format by the
// FP32 path, by this lane.  Returns false (having written nothing) when the
// row must be assembled by the FP64 path instead.
__device__ __noinline__ bool assemble_lane_mixed(const AsmArgs& A, int64_t row) {
    extern __shared__ float smf[];
    const int lane = threadIdx.x & (kWarp - 1);
    const int k = A.k, m = k + 1;
    float* smw = smf + (size_t)(threadIdx.x / kWarp) * (size_t)A.kcap * kMixCols * kWarp;  // this warp's part
    // element (s, c) of this lane's neighbour table
#define MF(s, c) smw[((s) * kMixCols + (c)) * kWarp + lane]
    const int64_t i = A.order ? (int64_t)A.order[row] : row;
    const int32_t* nb = A.nbr + i * k;
    const double px = A.pts[3 * i], py = A.pts[3 * i + 1], pz = A.pts[3 * i + 2];

    // offsets d_s = p_j - p_i (FP64, then double-float), barycenter of N(i),
    // mean distance to the delta_m nearest
    df cx = df_make(0.f), cy = df_make(0.f), cz = df_make(0.f), hsum = df_make(0.f);
    for (int s = 0; s < k; s++) {
        const int64_t j = nb[s];
        if (j < 0 || j >= A.n) return false;  // the FP64 path marks the row
        const df dx = df_from_double(A.pts[3 * j] - px), dy = df_from_double(A.pts[3 * j + 1] - py),
                 dz = df_from_double(A.pts[3 * j + 2] - pz);
        MF(s, 0) = dx.hi; MF(s, 1) = dx.lo;
        MF(s, 2) = dy.hi; MF(s, 3) = dy.lo;
        MF(s, 4) = dz.hi; MF(s, 5) = dz.lo;
        cx = df_add(cx, dx); cy = df_add(cy, dy); cz = df_add(cz, dz);
        if (s < A.delta_m)
            hsum = df_add(hsum, df_sqrt(df_add(df_add(df_mul(dx, dx), df_mul(dy, dy)), df_mul(dz, dz))));
    }
    const df kk = df_make((float)k);
    cx = df_div(cx, kk); cy = df_div(cy, kk); cz = df_div(cz, kk);
    df C00 = df_make(0.f), C01 = C00, C02 = C00, C11 = C00, C12 = C00, C22 = C00;
    for (int s = 0; s < k; s++) {
        const df ex = df_sub({MF(s, 0), MF(s, 1)}, cx), ey = df_sub({MF(s, 2), MF(s, 3)}, cy),
                 ez = df_sub({MF(s, 4), MF(s, 5)}, cz);
        C00 = df_fma(C00, ex, ex); C01 = df_fma(C01, ex, ey); C02 = df_fma(C02, ex, ez);
        C11 = df_fma(C11, ey, ey); C12 = df_fma(C12, ey, ez); C22 = df_fma(C22, ez, ez);
    }

    // frame: FP32 Jacobi, its eigenvectors orthonormalised in FP64, the covariance
    // rotated into them and finished by FP64 Jacobi sweeps (the FP64 eigen step)
    double E[3][3], ev[3];
    {
        float Cf[3][3] = {{C00.hi, C01.hi, C02.hi}, {C01.hi, C11.hi, C12.hi}, {C02.hi, C12.hi, C22.hi}};
        float Vf[3][3], wf[3];
        jacobi3f(Cf, Vf, wf);
        double Q[3][3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) Q[r][c] = (double)Vf[r][c];
        const double n0 = rsqrt(Q[0][0] * Q[0][0] + Q[1][0] * Q[1][0] + Q[2][0] * Q[2][0]);
        for (int r = 0; r < 3; r++) Q[r][0] *= n0;
        const double d01 = Q[0][0] * Q[0][1] + Q[1][0] * Q[1][1] + Q[2][0] * Q[2][1];
        for (int r = 0; r < 3; r++) Q[r][1] -= d01 * Q[r][0];
        const double n1 = rsqrt(Q[0][1] * Q[0][1] + Q[1][1] * Q[1][1] + Q[2][1] * Q[2][1]);
        for (int r = 0; r < 3; r++) Q[r][1] *= n1;
        Q[0][2] = Q[1][0] * Q[2][1] - Q[2][0] * Q[1][1];
        Q[1][2] = Q[2][0] * Q[0][1] - Q[0][0] * Q[2][1];
        Q[2][2] = Q[0][0] * Q[1][1] - Q[1][0] * Q[0][1];
        const double C[3][3] = {{df_to_double(C00), df_to_double(C01), df_to_double(C02)},
                                {df_to_double(C01), df_to_double(C11), df_to_double(C12)},
                                {df_to_double(C02), df_to_double(C12), df_to_double(C22)}};
        double T[3][3], B[3][3], W[3][3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) T[r][c] = C[r][0] * Q[0][c] + C[r][1] * Q[1][c] + C[r][2] * Q[2][c];
        for (int r = 0; r < 3; r++)
            for (int c = r; c < 3; c++)
                B[r][c] = B[c][r] = Q[0][r] * T[0][c] + Q[1][r] * T[1][c] + Q[2][r] * T[2][c];
        jacobi3(B, W, ev);
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) E[r][c] = Q[r][0] * W[0][c] + Q[r][1] * W[1][c] + Q[r][2] * W[2][c];
    }
    int imax = 0, imin = 0;
    for (int a = 1; a < 3; a++) {
        if (ev[a] > ev[imax]) imax = a;
        if (ev[a] < ev[imin]) imin = a;
    }
    if (imax == imin) imin = (imax + 1) % 3;
    const int imid = 3 - imax - imin;
    const df ex0 = df_from_double(E[0][imax]), ex1 = df_from_double(E[1][imax]), ex2 = df_from_double(E[2][imax]);
    const df ey0 = df_from_double(E[0][imid]), ey1 = df_from_double(E[1][imid]), ey2 = df_from_double(E[2][imid]);
    const df ez0 = df_from_double(E[0][imin]), ez1 = df_from_double(E[1][imin]), ez2 = df_from_double(E[2][imin]);

    // local coordinates centred at p_i; quarter-range extents
    df x0 = df_make(3e38f), x1 = df_make(-3e38f), y0 = x0, y1 = x1;
    for (int s = 0; s < k; s++) {
        const df dx = {MF(s, 0), MF(s, 1)}, dy = {MF(s, 2), MF(s, 3)}, dz = {MF(s, 4), MF(s, 5)};
        const df lx = df_add(df_add(df_mul(dx, ex0), df_mul(dy, ex1)), df_mul(dz, ex2));
        const df ly = df_add(df_add(df_mul(dx, ey0), df_mul(dy, ey1)), df_mul(dz, ey2));
        const df lz = df_add(df_add(df_mul(dx, ez0), df_mul(dy, ez1)), df_mul(dz, ez2));
        MF(s, 0) = lx.hi; MF(s, 1) = lx.lo;
        MF(s, 2) = ly.hi; MF(s, 3) = ly.lo;
        MF(s, 4) = lz.hi; MF(s, 5) = lz.lo;
        if (df_less(lx, x0)) x0 = lx;
        if (df_less(x1, lx)) x1 = lx;
        if (df_less(ly, y0)) y0 = ly;
        if (df_less(y1, ly)) y1 = ly;
    }
    df h;
    if (A.delta_kind == MVGD_DELTA_QUARTER_RANGE) {
        const df rx = df_mul_f(df_sub(x1, x0), 0.25f), ry = df_mul_f(df_sub(y1, y0), 0.25f);
        h = df_less(rx, ry) ? rx : ry;
    } else {
        h = df_div(hsum, df_make((float)A.delta_m));
    }
    h = df_mul(h, df_from_double(A.delta_scale));
    if (!(h.hi > 0.0f) || !df_isfinite(h)) return false;
    const df ih = df_div(df_make(1.0f), h);

    // moments of the h-scaled design rows (the self row adds 1 to the count)
    df M[15], Z[6];
#pragma unroll
    for (int q = 0; q < 15; q++) M[q] = df_make(0.f);
#pragma unroll
    for (int q = 0; q < 6; q++) Z[q] = df_make(0.f);
    M[0] = df_make((float)m);
    for (int s = 0; s < k; s++) {
        const df xi = df_mul({MF(s, 0), MF(s, 1)}, ih), eta = df_mul({MF(s, 2), MF(s, 3)}, ih),
                 zeta = df_mul({MF(s, 4), MF(s, 5)}, ih);
        MF(s, 0) = xi.hi; MF(s, 1) = xi.lo;
        MF(s, 2) = eta.hi; MF(s, 3) = eta.lo;
        const df x2 = df_mul(xi, xi), xy = df_mul(xi, eta), y2 = df_mul(eta, eta);
        M[1] = df_add(M[1], xi); M[2] = df_add(M[2], eta);
        M[3] = df_add(M[3], x2); M[4] = df_add(M[4], xy); M[5] = df_add(M[5], y2);
        M[6] = df_fma(M[6], x2, xi); M[7] = df_fma(M[7], x2, eta);
        M[8] = df_fma(M[8], xi, y2); M[9] = df_fma(M[9], y2, eta);
        M[10] = df_fma(M[10], x2, x2); M[11] = df_fma(M[11], x2, xy); M[12] = df_fma(M[12], x2, y2);
        M[13] = df_fma(M[13], xy, y2); M[14] = df_fma(M[14], y2, y2);
        Z[0] = df_add(Z[0], zeta); Z[1] = df_fma(Z[1], xi, zeta); Z[2] = df_fma(Z[2], eta, zeta);
        Z[3] = df_fma(Z[3], x2, zeta); Z[4] = df_fma(Z[4], xy, zeta); Z[5] = df_fma(Z[5], y2, zeta);
    }
    df G[21];
#pragma unroll
    for (int p = 0; p < 6; p++)
#pragma unroll
        for (int q = 0; q <= p; q++) G[tri(p, q)] = M[moment_index(mono_a(p) + mono_a(q), mono_b(p) + mono_b(q))];
    float L[21];
    if (!chol6(G, L) || !(cond1_6(G, L) <= kCondCap)) return false;

    // surface fit a~ = G^-1 V^T zeta, then the metric and A_1..A_5 at the origin
    df at[6];
    if (!solve6_refined(G, L, Z, at)) return false;
    const df one = df_make(1.0f);
    const df zx = at[1], zy = at[2];
    const df zxx = df_mul(df_mul_f(at[3], 2.0f), ih), zxy = df_mul(at[4], ih),
             zyy = df_mul(df_mul_f(at[5], 2.0f), ih);
    const df zx2 = df_mul(zx, zx), zy2 = df_mul(zy, zy);
    const df iW = df_div(one, df_add(one, df_add(zx2, zy2)));
    const df g11 = df_mul(df_add(one, zy2), iW), g12 = df_neg(df_mul(df_mul(zx, zy), iW));
    const df g22 = df_mul(df_add(one, zx2), iW);
    const df Hs = df_add(df_add(df_mul(g11, zxx), df_mul_f(df_mul(g12, zxy), 2.0f)), df_mul(g22, zyy));
    const df A1 = df_neg(df_mul(df_mul(Hs, zx), iW)), A2 = df_neg(df_mul(df_mul(Hs, zy), iW));
    // the least-squares comparator drops the centre-value term (c~_0 = 0, no self correction)
    const df c0 = A.variant == MVGD_ROW_LS ? df_make(0.f) : df_mul_f(df_add(g11, g22), 2.0f);
    const df ct[6] = {c0, df_mul(A1, h), df_mul(A2, h), df_mul_f(g11, 2.0f), df_mul_f(g12, 2.0f),
                      df_mul_f(g22, 2.0f)};

    // g = G^-1 c~; the row is y = V g scaled by 1/h^2, with the self correction
    df g[6];
    if (!solve6_refined(G, L, ct, g)) return false;
    const df ih2 = df_mul(ih, ih);
    const df w0 = df_mul(df_sub(g[0], c0), ih2);
    bool finite = df_isfinite(w0);
    for (int s = 0; s < k; s++) {
        const df xi = {MF(s, 0), MF(s, 1)}, eta = {MF(s, 2), MF(s, 3)};
        df y = df_add(g[0], df_add(df_mul(xi, g[1]), df_mul(eta, g[2])));
        y = df_add(y, df_add(df_mul(df_mul(xi, xi), g[3]),
                             df_add(df_mul(df_mul(xi, eta), g[4]), df_mul(df_mul(eta, eta), g[5]))));
        const df w = df_mul(y, ih2);
        finite = finite && df_isfinite(w);
        MF(s, 4) = w.hi;
        MF(s, 5) = w.lo;
    }
    if (!finite) return false;
    float* vo = static_cast<float*>(A.val);
    vo[sell_index(row, 0, m)] = w0.hi;
    A.val_lo[sell_index(row, 0, m)] = w0.lo;
    for (int s = 0; s < k; s++) {
        vo[sell_index(row, s + 1, m)] = MF(s, 4);
        A.val_lo[sell_index(row, s + 1, m)] = MF(s, 5);
        const int32_t j = nb[s];
        A.col[sell_index(row, s, k)] = A.inv ? A.inv[j] : j;
    }
    if (A.h_out) A.h_out[i] = df_to_double(h);
    if (A.status) A.status[i] = 0;
#undef MF
    return true;
}

// A stored row of cloud `item`; padding rows are zero.  MODE 0: the FP64
// path; 1: the FP32 path (rows it hands over go to the fix list); 2: by the
// cloud's format (batches).
template <int MODE>
__device__ __forceinline__ void assemble_row(const AsmArgs& A, int64_t row, int item) {
    if (row >= A.n) {  // padding row of the last slice
        const int k = A.k, m = k + 1;
        for (int s = 0; s < k; s++) A.col[sell_index(row, s, k)] = 0;
        if (A.prec == MVGD_FP64) {
            double* v = static_cast<double*>(A.val);
            for (int s = 0; s <= k; s++) v[sell_index(row, s, m)] = 0.0;
        } else {
            float* v = static_cast<float*>(A.val);
            for (int s = 0; s <= k; s++) {
                v[sell_index(row, s, m)] = 0.0f;
                A.val_lo[sell_index(row, s, m)] = 0.0f;
            }
        }
        return;
    }
    if (MODE == 1 || (MODE == 2 && A.prec == MVGD_FP32_REFINE && !A.arith)) {
        if (!assemble_lane_mixed(A, row)) {
            const int pos = atomicAdd(A.nfix, 1);
            A.fix[pos] = make_int2(item, (int)row);
        }
        return;
    }
    assemble_lane(A, row);
}

// A warp per 32-row slice, blockDim.x / 32 warps a block (the launch's tuning).
template <int MODE>
__global__ void __launch_bounds__(256) k_assemble(AsmArgs A) {
    const int64_t slice = (int64_t)blockIdx.x * (blockDim.x / kWarp) + threadIdx.x / kWarp;
    if (slice * kSlice >= n_padded(A.n)) return;
    assemble_row<MODE>(A, slice * kSlice + (threadIdx.x & (kWarp - 1)), 0);
}

// The rows the FP32 path handed over, by the FP64 path: a lane per row.
__global__ void __launch_bounds__(32) k_assemble_fix(AsmArgs A) {
    const int32_t count = *A.nfix;
    for (int64_t e0 = blockIdx.x * (int64_t)kWarp; e0 < count; e0 += (int64_t)gridDim.x * kWarp) {
        const int64_t e = e0 + threadIdx.x;
        if (e < count) assemble_lane(A, A.fix[e].y);
    }
}

// Batched: many uneven clouds in one launch.  The work items are
// (cloud, slice) pairs; block b takes the cloud whose slice range holds b.
struct AsmItem {
    AsmArgs a;
    int64_t slice0;  // first global slice of this cloud
};

__device__ __forceinline__ int item_of_slice(const AsmItem* __restrict__ items, int count, int64_t b) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last item with slice0 <= b
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].slice0 <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(32) k_assemble_batch(const AsmItem* __restrict__ items, int count) {
    const int64_t b = blockIdx.x;
    const int it = item_of_slice(items, count, b);
    const AsmArgs A = items[it].a;
    assemble_row<2>(A, (b - items[it].slice0) * kSlice + threadIdx.x, it);
}

__global__ void __launch_bounds__(32) k_assemble_batch_fix(const AsmItem* __restrict__ items, const int2* fix,
                                                           const int32_t* nfix) {
    const int32_t count = *nfix;
    for (int64_t e0 = blockIdx.x * (int64_t)kWarp; e0 < count; e0 += (int64_t)gridDim.x * kWarp) {
        const int64_t e = e0 + threadIdx.x;
        if (e < count) {
            const int2 f = fix[e];
            assemble_lane(items[f.x].a, f.y);
        }
    }
}

constexpr int kAsmGroup = 48;
struct AsmGroup {
    AsmItem item[kAsmGroup];
    int count;
};

// Copies a group of descriptors (kernel parameters, so the batch is
// capturable in a graph) into the device table.
__global__ void k_put_items(AsmGroup G, AsmItem* dst) {
    for (int i = threadIdx.x; i < G.count; i += blockDim.x) dst[i] = G.item[i];
}

__global__ void k_invert_order(const int32_t* __restrict__ order, int64_t n, int32_t* __restrict__ inv) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        inv[order[r]] = (int32_t)r;
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_ell_bytes(int64_t n, int32_t k, int32_t prec, int32_t which) {
    if (n <= 0 || k < 1) return 0;
    int64_t np = n_padded(n);
    switch (which) {
        case MVGD_ELL_COL: return align_up(sizeof(int32_t) * np * k);
        case MVGD_ELL_VAL:
            return align_up((prec == MVGD_FP64 ? sizeof(double) : sizeof(float)) * np * (k + 1));
        case MVGD_ELL_VAL_LO: return prec == MVGD_FP32_REFINE ? align_up(sizeof(float) * np * (k + 1)) : 0;
        default: return 0;
    }
}

namespace mvgd {
namespace {

// Workspace of one cloud: the inverse order and the FP32 path's hand-over
// list (with its counter).
struct AsmWs {
    int32_t* inv;
    int2* fix;
    int32_t* nfix;
    size_t bytes;
};

AsmWs asm_ws(void* base, int64_t n) {
    Carver cv(base);
    AsmWs w;
    w.inv = cv.take<int32_t>((size_t)n);
    w.fix = cv.take<int2>((size_t)n);
    w.nfix = cv.take<int32_t>(1);
    w.bytes = cv.used;
    return w;
}

size_t smem_fp64(int k) { return sizeof(double) * (size_t)(k + 1) * kCols * kWarp; }
size_t smem_mixed(int k) { return sizeof(float) * (size_t)k * kMixCols * kWarp; }

// The FP32 path needs an overdetermined fit: with k < kMinKMixed the 6-unknown
// fit over k + 1 points is square or nearly so, its conditioning is beyond
// what double-float residuals settle, and the rows use FP64 arithmetic.
constexpr int kMinKMixed = 8;

bool fp32_path(const mvgd_ell& L, const mvgd_delta_rule& rule) {
    return L.prec == MVGD_FP32_REFINE && rule.arith == 0 && L.k >= kMinKMixed;
}

constexpr int kFixBlocks = 152;  // grid of the hand-over kernels (a warp each)

}  // namespace
}  // namespace mvgd

MVGD_API size_t mvgd_assemble_workspace_bytes(int64_t n) {
    return n > 0 ? asm_ws(nullptr, n).bytes : 0;
}

MVGD_API mvgd_status mvgd_assemble(const double* pts, int64_t n, int32_t k, const int32_t* nbr,
                                   mvgd_delta_rule rule, mvgd_ell* L, double* h, uint8_t* row_status,
                                   int32_t* bad_rows, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!pts || !nbr || !L || n < 2 || n >= (1ll << 31) || k < kMinK || k > kMaxK || k >= n)
        return MVGD_EINVAL;
    if (L->n != n || L->k != k || !L->col || !L->val) return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (rule.kind != MVGD_DELTA_QUARTER_RANGE && rule.kind != MVGD_DELTA_MEAN_NN) return MVGD_EINVAL;
    if (rule.kind == MVGD_DELTA_MEAN_NN && (rule.m < 1 || rule.m > k)) return MVGD_EINVAL;
    if (!(rule.scale > 0)) return MVGD_EINVAL;
    if (rule.variant != MVGD_ROW_MVGD && rule.variant != MVGD_ROW_LS) return MVGD_EINVAL;
    if (rule.arith != 0 && rule.arith != 1) return MVGD_EINVAL;
    if (!aligned(pts) || !aligned(nbr) || !aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo) ||
        !aligned(L->order) || !aligned(h) || !aligned(row_status) || !aligned(bad_rows) || !aligned(ws))
        return MVGD_EINVAL;
    const bool mixed = fp32_path(*L, rule);
    if ((L->order || mixed) && (!ws || ws_bytes < mvgd_assemble_workspace_bytes(n))) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const AsmWs W = asm_ws(ws, n);
    AsmArgs A;
    A.pts = pts; A.n = n; A.k = k; A.nbr = nbr; A.order = L->order;
    A.inv = L->order ? W.inv : nullptr;
    A.delta_kind = rule.kind;
    A.delta_m = rule.kind == MVGD_DELTA_MEAN_NN ? rule.m : 0;
    A.delta_scale = rule.scale;
    A.variant = rule.variant;
    A.prec = L->prec;
    A.col = L->col; A.val = L->val; A.val_lo = L->val_lo;
    A.h_out = h; A.status = row_status; A.bad_rows = bad_rows;
    A.arith = rule.arith;
    A.kcap = k;
    A.fix = mixed ? W.fix : nullptr;
    A.nfix = mixed ? W.nfix : nullptr;
    if (bad_rows) MVGD_CUDA_TRY(cudaMemsetAsync(bad_rows, 0, sizeof(int32_t), s));
    int gb = (int)((n + 255) / 256);
    if (gb > 4096) gb = 4096;
    if (L->order) k_invert_order<<<gb, 256, 0, s>>>(L->order, n, W.inv);
    const int64_t nslices = n_padded(n) / kSlice;
    // warps a block: the launch's tuning for the FP32 path (15 KB of shared memory a
    // warp); the FP64 arithmetic keeps one (38 KB a warp: more would only cost
    // resident warps)
    int wpb = mixed ? tuned_assemble_warps() : 1;
    const size_t per_warp = mixed ? smem_mixed(k) : smem_fp64(k);
    while (wpb > 1 && per_warp * wpb > (size_t)(200 << 10)) wpb >>= 1;
    const unsigned blocks = (unsigned)((nslices + wpb - 1) / wpb);
    if (mixed) {
        MVGD_CUDA_TRY(cudaMemsetAsync(W.nfix, 0, sizeof(int32_t), s));
        const size_t sm = per_warp * wpb;
        MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_assemble<1><<<blocks, kWarp * wpb, sm, s>>>(A);
        const size_t sf = smem_fp64(k);
        MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
        k_assemble_fix<<<kFixBlocks, kWarp, sf, s>>>(A);
    } else {
        const size_t sf = per_warp * wpb;
        MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
        k_assemble<0><<<blocks, kWarp * wpb, sf, s>>>(A);
    }
    return launch_status();
}

MVGD_API size_t mvgd_assemble_batch_workspace_bytes(const int64_t* n, int32_t count) {
    if (!n || count < 1) return 0;
    size_t b = align_up(sizeof(AsmItem) * (size_t)count);
    int64_t total = 0;
    for (int i = 0; i < count; i++) {
        if (n[i] <= 0) continue;
        b += align_up(sizeof(int32_t) * (size_t)n[i]);
        total += n[i];
    }
    return b + align_up(sizeof(int2) * (size_t)(total > 0 ? total : 1)) + align_up(sizeof(int32_t));
}

MVGD_API mvgd_status mvgd_assemble_batch(const mvgd_assemble_item* items, int32_t count, mvgd_delta_rule rule,
                                         int32_t* bad_rows, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!items || count < 1 || !ws || !aligned(ws) || !aligned(bad_rows)) return MVGD_EINVAL;
    if (rule.kind != MVGD_DELTA_QUARTER_RANGE && rule.kind != MVGD_DELTA_MEAN_NN) return MVGD_EINVAL;
    if (!(rule.scale > 0)) return MVGD_EINVAL;
    if (rule.variant != MVGD_ROW_MVGD && rule.variant != MVGD_ROW_LS) return MVGD_EINVAL;
    if (rule.arith != 0 && rule.arith != 1) return MVGD_EINVAL;
    std::vector<int64_t> ns((size_t)count);
    int kmax = 0;
    bool any_mixed = false, any_fp64 = false;
    for (int i = 0; i < count; i++) {
        const mvgd_assemble_item& it = items[i];
        const mvgd_ell& L = it.L;
        const int64_t n = L.n;
        const int k = L.k;
        if (!it.pts || !it.nbr || n < 2 || n >= (1ll << 31) || k < kMinK || k > kMaxK || k >= n) return MVGD_EINVAL;
        if (!L.col || !L.val || (L.prec != MVGD_FP64 && L.prec != MVGD_FP32_REFINE)) return MVGD_EINVAL;
        if (L.prec == MVGD_FP32_REFINE && !L.val_lo) return MVGD_EINVAL;
        if (rule.kind == MVGD_DELTA_MEAN_NN && (rule.m < 1 || rule.m > k)) return MVGD_EINVAL;
        if (!aligned(it.pts) || !aligned(it.nbr) || !aligned(L.col) || !aligned(L.val) || !aligned(L.val_lo) ||
            !aligned(L.order) || !aligned(it.h) || !aligned(it.row_status))
            return MVGD_EINVAL;
        ns[(size_t)i] = n;
        if (k > kmax) kmax = k;
        if (fp32_path(L, rule)) any_mixed = true;
        else any_fp64 = true;
    }
    if (ws_bytes < mvgd_assemble_batch_workspace_bytes(ns.data(), count)) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (bad_rows) MVGD_CUDA_TRY(cudaMemsetAsync(bad_rows, 0, sizeof(int32_t), s));
    Carver cv(ws);
    AsmItem* table = cv.take<AsmItem>(count);
    std::vector<int32_t*> invs((size_t)count);
    int64_t total = 0;
    for (int i = 0; i < count; i++) {
        invs[(size_t)i] = cv.take<int32_t>((size_t)ns[(size_t)i]);
        total += ns[(size_t)i];
    }
    int2* fix = cv.take<int2>((size_t)total);
    int32_t* nfix = cv.take<int32_t>(1);
    MVGD_CUDA_TRY(cudaMemsetAsync(nfix, 0, sizeof(int32_t), s));
    int64_t slices = 0;
    AsmGroup G;
    G.count = 0;
    int group_start = 0;
    for (int i = 0; i < count; i++) {
        const mvgd_assemble_item& it = items[i];
        const mvgd_ell& L = it.L;
        int32_t* inv = invs[(size_t)i];
        if (L.order) {
            int gb = (int)((L.n + 255) / 256);
            if (gb > 4096) gb = 4096;
            k_invert_order<<<gb, 256, 0, s>>>(L.order, L.n, inv);
        }
        const bool mixed = fp32_path(L, rule);
        AsmItem& a = G.item[G.count++];
        a.a.pts = it.pts;
        a.a.n = L.n;
        a.a.k = L.k;
        a.a.nbr = it.nbr;
        a.a.order = L.order;
        a.a.inv = L.order ? inv : nullptr;
        a.a.delta_kind = rule.kind;
        a.a.delta_m = rule.kind == MVGD_DELTA_MEAN_NN ? rule.m : 0;
        a.a.delta_scale = rule.scale;
        a.a.variant = rule.variant;
        a.a.prec = L.prec;
        a.a.col = L.col;
        a.a.val = L.val;
        a.a.val_lo = L.val_lo;
        a.a.h_out = it.h;
        a.a.status = it.row_status;
        a.a.bad_rows = bad_rows;
        a.a.arith = mixed ? 0 : 1;  // an FP32_REFINE item below kMinKMixed takes the FP64 path
        a.a.kcap = kmax;
        a.a.fix = mixed ? fix : nullptr;
        a.a.nfix = mixed ? nfix : nullptr;
        a.slice0 = slices;
        slices += n_padded(L.n) / kSlice;
        if (G.count == kAsmGroup || i == count - 1) {
            k_put_items<<<1, 64, 0, s>>>(G, table + group_start);
            group_start += G.count;
            G.count = 0;
        }
    }
    if (slices >= (1ll << 31)) return MVGD_EINVAL;
    const size_t sf = smem_fp64(kmax), sm = smem_mixed(kmax);
    const size_t smem = any_fp64 ? (sf > sm ? sf : sm) : sm;
    MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_assemble_batch<<<(unsigned)slices, kWarp, smem, s>>>(table, count);
    if (any_mixed) {
        MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble_batch_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
        k_assemble_batch_fix<<<kFixBlocks, kWarp, sf, s>>>(table, fix, nfix);
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// Sign pattern of the assembled rows (Sec. 3.2, Sec. 4.1): the rows sum to
// zero, so a row whose neighbour weights are all >= 0 gives sigma I - L a
// diagonally dominant row with non-positive off-diagonal entries (the
// M-matrix pattern).  Integer counts, summed with atomics: exact.
// ---------------------------------------------------------------------------
namespace mvgd {
namespace {

__global__ void k_row_signs(mvgd_ell L, unsigned long long* counts) {
    const int k = L.k, m = k + 1;
    unsigned long long pattern = 0, negative = 0, self_nonneg = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
        auto weight = [&](int s) {
            const int64_t e = vb + (int64_t)s * kSlice;
            return L.prec == MVGD_FP64 ? static_cast<const double*>(L.val)[e]
                                       : (double)static_cast<const float*>(L.val)[e] + (double)L.val_lo[e];
        };
        int neg = 0;
        for (int s = 1; s < m; s++) neg += weight(s) < 0.0 ? 1 : 0;
        pattern += neg == 0 ? 1 : 0;
        negative += (unsigned long long)neg;
        self_nonneg += weight(0) >= 0.0 ? 1 : 0;
    }
    pattern = warp_sum(pattern);
    negative = warp_sum(negative);
    self_nonneg = warp_sum(self_nonneg);
    if (lane_id() == 0) {
        atomicAdd(&counts[0], pattern);
        atomicAdd(&counts[1], negative);
        atomicAdd(&counts[2], self_nonneg);
    }
}

}  // namespace
}  // namespace mvgd

MVGD_API mvgd_status mvgd_row_signs(const mvgd_ell* L, int64_t* counts, mvgd_stream_t stream) {
    if (!L || !counts || !L->val || L->n < 1 || L->k < kMinK || L->k > kMaxK) return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!aligned(L->val) || !aligned(L->val_lo) || (reinterpret_cast<uintptr_t>(counts) & 7) != 0)
        return MVGD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MVGD_CUDA_TRY(cudaMemsetAsync(counts, 0, 3 * sizeof(int64_t), s));
    const int64_t blocks = (L->n + 255) / 256;
    k_row_signs<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(
        *L, reinterpret_cast<unsigned long long*>(counts));
    return launch_status();
}

// ---------------------------------------------------------------------------
// Dirichlet boundary rows (open surfaces, Sec. 3.1): U = g is enforced at the
// boundary points and the MVGD row kept at the interior points.
// ---------------------------------------------------------------------------
namespace mvgd {
namespace {

__global__ void k_dirichlet_rows(mvgd_ell L, const uint8_t* __restrict__ boundary, int32_t* count) {
    const int m = L.k + 1;
    int mine = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = L.order ? (int64_t)L.order[r] : r;
        if (!boundary[p]) continue;
        const int64_t vb = (r / kSlice) * (int64_t)(kSlice * m) + (r % kSlice);
        for (int s = 0; s < m; s++) {
            const int64_t e = vb + (int64_t)s * kSlice;
            if (L.prec == MVGD_FP64) {
                static_cast<double*>(L.val)[e] = 0.0;
            } else {
                static_cast<float*>(L.val)[e] = 0.0f;
                L.val_lo[e] = 0.0f;
            }
        }
        mine++;
    }
    mine = warp_sum(mine);
    if (count && lane_id() == 0 && mine) atomicAdd(count, mine);
}

}  // namespace
}  // namespace mvgd

MVGD_API mvgd_status mvgd_dirichlet_rows(mvgd_ell* L, const uint8_t* boundary, int32_t* count,
                                         mvgd_stream_t stream) {
    if (!L || !boundary || !L->val || L->n < 1 || L->n >= (1ll << 31) || L->k < kMinK || L->k > kMaxK)
        return MVGD_EINVAL;
    if (L->prec != MVGD_FP64 && L->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (L->prec == MVGD_FP32_REFINE && !L->val_lo) return MVGD_EINVAL;
    if (!aligned(L->val) || !aligned(L->val_lo) || (reinterpret_cast<uintptr_t>(count) & 3) != 0)
        return MVGD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (count) MVGD_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int32_t), s));
    const int64_t blocks = (L->n + 255) / 256;
    k_dirichlet_rows<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(*L, boundary, count);
    return launch_status();
}
