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
#include "common.cuh"
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
};

// One 32-row slice of one cloud's operator (one warp, one row per lane).
__device__ __forceinline__ void assemble_slice(const AsmArgs& A, int64_t slice) {
    extern __shared__ double sm[];
    const int lane = threadIdx.x;
    const int64_t row = slice * kSlice + lane;
    const int k = A.k, m = k + 1;
    // element (r, c) of this lane's design matrix
#define VM(r, c) sm[((r) * kCols + (c)) * kWarp + lane]

    if (row >= A.n) {  // padding row of the last slice
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

__global__ void __launch_bounds__(32) k_assemble(AsmArgs A) { assemble_slice(A, blockIdx.x); }

// Batched: many uneven clouds in one launch.  The work items are
// (cloud, slice) pairs; block b takes the cloud whose slice range holds b.
struct AsmItem {
    AsmArgs a;
    int64_t slice0;  // first global slice of this cloud
};

__global__ void __launch_bounds__(32) k_assemble_batch(const AsmItem* __restrict__ items, int count) {
    const int64_t b = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {  // last item with slice0 <= b
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].slice0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const AsmArgs A = items[lo].a;
    assemble_slice(A, b - items[lo].slice0);
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

MVGD_API size_t mvgd_assemble_workspace_bytes(int64_t n) {
    return n > 0 ? align_up(sizeof(int32_t) * n) : 0;
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
    if (!aligned(pts) || !aligned(nbr) || !aligned(L->col) || !aligned(L->val) || !aligned(L->val_lo) ||
        !aligned(L->order) || !aligned(h) || !aligned(row_status) || !aligned(bad_rows) || !aligned(ws))
        return MVGD_EINVAL;
    if (L->order && (!ws || ws_bytes < mvgd_assemble_workspace_bytes(n))) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    AsmArgs A;
    A.pts = pts; A.n = n; A.k = k; A.nbr = nbr; A.order = L->order;
    A.inv = L->order ? static_cast<int32_t*>(ws) : nullptr;
    A.delta_kind = rule.kind;
    A.delta_m = rule.kind == MVGD_DELTA_MEAN_NN ? rule.m : 0;
    A.delta_scale = rule.scale;
    A.variant = rule.variant;
    A.prec = L->prec;
    A.col = L->col; A.val = L->val; A.val_lo = L->val_lo;
    A.h_out = h; A.status = row_status; A.bad_rows = bad_rows;
    if (bad_rows) MVGD_CUDA_TRY(cudaMemsetAsync(bad_rows, 0, sizeof(int32_t), s));
    if (L->order) {
        int gb = (int)((n + 255) / 256);
        if (gb > 4096) gb = 4096;
        k_invert_order<<<gb, 256, 0, s>>>(L->order, n, const_cast<int32_t*>(A.inv));
    }
    size_t smem = sizeof(double) * (size_t)(k + 1) * kCols * kWarp;
    MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int64_t nslices = n_padded(n) / kSlice;
    k_assemble<<<(unsigned)nslices, kWarp, smem, s>>>(A);
    return launch_status();
}

MVGD_API size_t mvgd_assemble_batch_workspace_bytes(const int64_t* n, int32_t count) {
    if (!n || count < 1) return 0;
    size_t b = align_up(sizeof(AsmItem) * (size_t)count);
    for (int i = 0; i < count; i++) b += n[i] > 0 ? align_up(sizeof(int32_t) * (size_t)n[i]) : 0;
    return b;
}

MVGD_API mvgd_status mvgd_assemble_batch(const mvgd_assemble_item* items, int32_t count, mvgd_delta_rule rule,
                                         int32_t* bad_rows, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!items || count < 1 || !ws || !aligned(ws) || !aligned(bad_rows)) return MVGD_EINVAL;
    if (rule.kind != MVGD_DELTA_QUARTER_RANGE && rule.kind != MVGD_DELTA_MEAN_NN) return MVGD_EINVAL;
    if (!(rule.scale > 0)) return MVGD_EINVAL;
    if (rule.variant != MVGD_ROW_MVGD && rule.variant != MVGD_ROW_LS) return MVGD_EINVAL;
    size_t need = align_up(sizeof(AsmItem) * (size_t)count);
    int kmax = 0;
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
        need += align_up(sizeof(int32_t) * (size_t)n);
        if (k > kmax) kmax = k;
    }
    if (ws_bytes < need) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (bad_rows) MVGD_CUDA_TRY(cudaMemsetAsync(bad_rows, 0, sizeof(int32_t), s));
    Carver cv(ws);
    AsmItem* table = cv.take<AsmItem>(count);
    int64_t slices = 0;
    AsmGroup G;
    G.count = 0;
    int group_start = 0;
    for (int i = 0; i < count; i++) {
        const mvgd_assemble_item& it = items[i];
        const mvgd_ell& L = it.L;
        int32_t* inv = cv.take<int32_t>((size_t)L.n);
        if (L.order) {
            int gb = (int)((L.n + 255) / 256);
            if (gb > 4096) gb = 4096;
            k_invert_order<<<gb, 256, 0, s>>>(L.order, L.n, inv);
        }
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
        a.slice0 = slices;
        slices += n_padded(L.n) / kSlice;
        if (G.count == kAsmGroup || i == count - 1) {
            k_put_items<<<1, 64, 0, s>>>(G, table + group_start);
            group_start += G.count;
            G.count = 0;
        }
    }
    size_t smem = sizeof(double) * (size_t)(kmax + 1) * kCols * kWarp;
    MVGD_CUDA_TRY(cudaFuncSetAttribute(k_assemble_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (slices >= (1ll << 31)) return MVGD_EINVAL;
    k_assemble_batch<<<(unsigned)slices, kWarp, smem, s>>>(table, count);
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
