// Neumann boundary by reflection (Sec. 3.1).
//
// mvgd_neumann_ghosts: every interior point whose K nearest neighbours include
// a boundary point is mirrored through the boundary.  Its closest boundary
// point p_b carries a frame: e2 the surface normal (smallest eigenvector of
// the covariance of p_b's K neighbours), e1 the boundary tangent (a quadratic
// curve (xi, eta(xi), zeta(xi)) fitted through p_b and its kb nearest boundary
// points, xi along their principal axis), made orthogonal to e2, and
// e3 = e1 x e2, the boundary's normal in the tangent plane.  The ghost is
// p - 2 ((p - p_b).e3) e3.  The output cloud Q lists the interior points (in
// point order) and then the ghosts (in the order of the points they mirror).
//
// mvgd_neumann_fold: after kNN and assembly over Q, keeps the rows of the
// interior points (in the stored order of Q's operator, so the rows stay in
// their spatial order) and points every ghost column at the interior point it
// mirrors: with U(ghost) = U(point) the two weights act on one unknown.
//
// Kernels: flag scans (three launches each, fixed order), one thread per
// boundary point for the frames, one thread per flagged point for the
// closest boundary point (brute force over the boundary, which is a curve:
// O(sqrt n) points), one thread per kept row for the fold.
#include "common.cuh"
#include "frame.cuh"

namespace mvgd {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;                       // flags per thread
constexpr int kScanTile = kScanThreads * kScanPer;  // flags per block
constexpr int kMaxKb = 16;

// ---------------------------------------------------------------------------
// Exclusive prefix counts of byte flags: pos[i] = #{j < i : f[j] != 0}, *total.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int& block_total) {
    const int lane = (int)lane_id(), wid = threadIdx.x / kWarp;
    int incl = v;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == kWarp - 1) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x / kWarp;
        int t = lane < nw ? warp_tot[lane] : 0;
        int ti = t;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < nw) warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == nw - 1) warp_tot[kWarp] = ti;
    }
    __syncthreads();
    const int out = warp_tot[wid] + incl - v;
    block_total = warp_tot[kWarp];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(kScanThreads) k_flag_tiles(const uint8_t* __restrict__ f, int64_t n,
                                                             int32_t* __restrict__ tiles) {
    __shared__ int wt[kWarp + 1];
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanPer;
    int c = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; e++) c += (base + e < n && f[base + e]) ? 1 : 0;
    int tot = 0;
    block_exclusive_scan(c, wt, tot);
    if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

// One block: exclusive scan of the tile counts in place, the sum into *total.
__global__ void __launch_bounds__(kScanThreads) k_tile_offsets(int32_t* __restrict__ tiles, int64_t ntiles,
                                                               int32_t* __restrict__ total) {
    __shared__ int wt[kWarp + 1];
    int carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int v = i < ntiles ? tiles[i] : 0;
        int tot = 0;
        const int ex = block_exclusive_scan(v, wt, tot);
        if (i < ntiles) tiles[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_flag_positions(const uint8_t* __restrict__ f, int64_t n,
                                                                 const int32_t* __restrict__ tiles,
                                                                 int32_t* __restrict__ pos) {
    __shared__ int wt[kWarp + 1];
    const int64_t base = blockIdx.x * (int64_t)kScanTile + threadIdx.x * kScanPer;
    uint8_t fl[kScanPer];
    int c = 0;
#pragma unroll
    for (int e = 0; e < kScanPer; e++) {
        fl[e] = (base + e < n && f[base + e]) ? 1 : 0;
        c += fl[e];
    }
    int tot = 0;
    int p = tiles[blockIdx.x] + block_exclusive_scan(c, wt, tot);
#pragma unroll
    for (int e = 0; e < kScanPer; e++) {
        if (base + e < n) pos[base + e] = p;
        p += fl[e];
    }
}

int64_t scan_tiles(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

void scan_flags(const uint8_t* f, int64_t n, int32_t* pos, int32_t* tiles, int32_t* total, cudaStream_t s) {
    const int64_t nt = scan_tiles(n);
    k_flag_tiles<<<(unsigned)nt, kScanThreads, 0, s>>>(f, n, tiles);
    k_tile_offsets<<<1, kScanThreads, 0, s>>>(tiles, nt, total);
    k_flag_positions<<<(unsigned)nt, kScanThreads, 0, s>>>(f, n, tiles, pos);
}

// ---------------------------------------------------------------------------
// Ghosts
// ---------------------------------------------------------------------------
// Squared distance with the kNN step's key expression (no contraction).
__device__ __forceinline__ double dist2(const double* a, const double* b) {
    const double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__global__ void k_neumann_flags(const uint8_t* __restrict__ boundary, const int32_t* __restrict__ nbr, int64_t n,
                                int k, uint8_t* __restrict__ fi, uint8_t* __restrict__ fb, uint8_t* __restrict__ fm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const bool bnd = boundary[i] != 0;
        bool near = false;
        if (!bnd)
            for (int s = 0; s < k; s++) near |= boundary[nbr[i * k + s]] != 0;
        fi[i] = bnd ? 0 : 1;
        fb[i] = bnd ? 1 : 0;
        fm[i] = near ? 1 : 0;
    }
}

__global__ void k_neumann_compact(const double* __restrict__ pts, int64_t n, const uint8_t* __restrict__ fi,
                                  const int32_t* __restrict__ pos_i, const int32_t* __restrict__ pos_b,
                                  double* __restrict__ q, int32_t* __restrict__ q_src, int32_t* __restrict__ interior,
                                  int32_t* __restrict__ bidx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (fi[i]) {
            const int32_t p = pos_i[i];
            q[3 * (int64_t)p + 0] = pts[3 * i + 0];
            q[3 * (int64_t)p + 1] = pts[3 * i + 1];
            q[3 * (int64_t)p + 2] = pts[3 * i + 2];
            q_src[p] = p;
            interior[p] = (int32_t)i;
        } else {
            bidx[pos_b[i]] = (int32_t)i;
        }
    }
}

__device__ __forceinline__ int argmin3(const double w[3]) {
    return w[0] <= w[1] ? (w[0] <= w[2] ? 0 : 2) : (w[1] <= w[2] ? 1 : 2);
}
__device__ __forceinline__ int argmax3(const double w[3]) {
    return w[0] >= w[1] ? (w[0] >= w[2] ? 0 : 2) : (w[1] >= w[2] ? 1 : 2);
}

// Covariance (about the mean) of cnt offsets d[j] = p_j - origin.
__device__ void covariance(const double (*d)[3], int cnt, double C[3][3]) {
    double mu[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < cnt; j++)
        for (int c = 0; c < 3; c++) mu[c] += d[j][c];
    for (int c = 0; c < 3; c++) mu[c] /= cnt;
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) C[r][c] = 0.0;
    for (int j = 0; j < cnt; j++) {
        const double e[3] = {d[j][0] - mu[0], d[j][1] - mu[1], d[j][2] - mu[2]};
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) C[r][c] += e[r] * e[c];
    }
}

// e3 of every boundary point (one thread each); bad frames counted in *bad.
__global__ void k_boundary_frames(const double* __restrict__ pts, const int32_t* __restrict__ nbr, int k,
                                  const int32_t* __restrict__ bidx, const int32_t* __restrict__ nb_ptr, int kb,
                                  double* __restrict__ e3, int32_t* __restrict__ bad) {
    const int nb = *nb_ptr;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int64_t ib = bidx[b];
    const double* P = pts + 3 * ib;
    double d[kMaxK > kMaxKb ? kMaxK + 1 : kMaxKb + 1][3];
    double C[3][3], V[3][3], w[3];
    // e2: the surface normal from the K neighbours in the whole cloud
    for (int s = 0; s < k; s++) {
        const double* Q = pts + 3 * (int64_t)nbr[ib * k + s];
        for (int c = 0; c < 3; c++) d[s][c] = Q[c] - P[c];
    }
    covariance(d, k, C);
    jacobi3(C, V, w);
    int j = argmin3(w);
    double e2[3] = {V[0][j], V[1][j], V[2][j]};
    // the kb nearest boundary points (key: squared distance, then index)
    const int kbe = kb < nb - 1 ? kb : nb - 1;
    double bd[kMaxKb];
    int32_t bi[kMaxKb];
    int have = 0;
    for (int c = 0; c < (kbe >= 2 ? nb : 0); c++) {
        const int32_t ic = bidx[c];
        if (ic == ib) continue;
        const double dd = dist2(pts + 3 * (int64_t)ic, P);
        if (have == kbe && !(dd < bd[kbe - 1])) continue;  // bidx ascending: an equal key loses
        int at = have < kbe ? have++ : kbe - 1;
        while (at > 0 && dd < bd[at - 1]) {
            bd[at] = bd[at - 1];
            bi[at] = bi[at - 1];
            at--;
        }
        bd[at] = dd;
        bi[at] = ic;
    }
    bool ok = kbe >= 2;
    double out[3] = {0.0, 0.0, 0.0};
    if (ok) {
        // principal axis t and the other two axes u, v of p_b and its boundary neighbours
        d[0][0] = d[0][1] = d[0][2] = 0.0;
        for (int s = 0; s < kbe; s++)
            for (int c = 0; c < 3; c++) d[s + 1][c] = pts[3 * (int64_t)bi[s] + c] - P[c];
        const int cnt = kbe + 1;
        covariance(d, cnt, C);
        jacobi3(C, V, w);
        const int it = argmax3(w);
        const int iu = it == 0 ? 1 : 0;
        const int iv = 3 - it - iu;
        const double t[3] = {V[0][it], V[1][it], V[2][it]};
        const double u[3] = {V[0][iu], V[1][iu], V[2][iu]};
        const double v[3] = {V[0][iv], V[1][iv], V[2][iv]};
        // least squares eta, zeta ~ a0 + a1 xi + a2 xi^2, xi scaled by its largest magnitude
        double xs = 0.0;
        for (int s = 0; s < cnt; s++) xs = fmax(xs, fabs(d[s][0] * t[0] + d[s][1] * t[1] + d[s][2] * t[2]));
        double G[3][5];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 5; c++) G[r][c] = 0.0;
        for (int s = 0; s < cnt; s++) {
            const double xi = (d[s][0] * t[0] + d[s][1] * t[1] + d[s][2] * t[2]) / xs;
            const double ph[3] = {1.0, xi, xi * xi};
            const double eta = d[s][0] * u[0] + d[s][1] * u[1] + d[s][2] * u[2];
            const double zeta = d[s][0] * v[0] + d[s][1] * v[1] + d[s][2] * v[2];
            for (int r = 0; r < 3; r++) {
                for (int c = 0; c < 3; c++) G[r][c] += ph[r] * ph[c];
                G[r][3] += ph[r] * eta;
                G[r][4] += ph[r] * zeta;
            }
        }
        // Gaussian elimination with partial pivoting on the 3x3 normal equations, two right-hand sides
        const double g00 = fabs(G[0][0]);
        for (int c = 0; c < 3 && ok; c++) {
            int pr = c;
            for (int r = c + 1; r < 3; r++)
                if (fabs(G[r][c]) > fabs(G[pr][c])) pr = r;
            if (!(fabs(G[pr][c]) > 1e-12 * g00)) {
                ok = false;
                break;
            }
            if (pr != c)
                for (int e = 0; e < 5; e++) {
                    const double tmp = G[c][e];
                    G[c][e] = G[pr][e];
                    G[pr][e] = tmp;
                }
            for (int r = c + 1; r < 3; r++) {
                const double f = G[r][c] / G[c][c];
                for (int e = c; e < 5; e++) G[r][e] -= f * G[c][e];
            }
        }
        if (ok) {
            double a[3][2];
            for (int h = 0; h < 2; h++)
                for (int r = 2; r >= 0; r--) {
                    double acc = G[r][3 + h];
                    for (int c = r + 1; c < 3; c++) acc -= G[r][c] * a[c][h];
                    a[r][h] = acc / G[r][r];
                }
            const double s_eta = a[1][0] / xs, s_zeta = a[1][1] / xs;
            double e1[3];
            for (int c = 0; c < 3; c++) e1[c] = t[c] + s_eta * u[c] + s_zeta * v[c];
            const double dp = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
            for (int c = 0; c < 3; c++) e1[c] -= dp * e2[c];
            const double n1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
            ok = n1 > 0.0 && isfinite(n1);
            if (ok) {
                for (int c = 0; c < 3; c++) e1[c] /= n1;
                out[0] = e1[1] * e2[2] - e1[2] * e2[1];
                out[1] = e1[2] * e2[0] - e1[0] * e2[2];
                out[2] = e1[0] * e2[1] - e1[1] * e2[0];
                const double n3 = sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
                ok = n3 > 0.0 && isfinite(n3);
                for (int c = 0; c < 3; c++) out[c] = ok ? out[c] / n3 : 0.0;
            }
        }
    }
    if (!ok) {
        atomicAdd(bad, 1);
        out[0] = out[1] = out[2] = 0.0;
    }
    for (int c = 0; c < 3; c++) e3[3 * (int64_t)b + c] = out[c];
}

__global__ void k_ghosts(const double* __restrict__ pts, int64_t n, const uint8_t* __restrict__ fm,
                         const int32_t* __restrict__ pos_i, const int32_t* __restrict__ pos_g,
                         const int32_t* __restrict__ bidx, const int32_t* __restrict__ counts,
                         const double* __restrict__ e3, double* __restrict__ q, int32_t* __restrict__ q_src,
                         int32_t* __restrict__ ghost_bnd, double* __restrict__ ghost_dist) {
    const int ni = counts[0], nb = counts[2];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!fm[i]) continue;
        const double* P = pts + 3 * i;
        double best = INFINITY;
        int bb = 0;
        for (int b = 0; b < nb; b++) {  // bidx ascending: the first minimum has the lowest index
            const double dd = dist2(pts + 3 * (int64_t)bidx[b], P);
            if (dd < best) {
                best = dd;
                bb = b;
            }
        }
        const double* B = pts + 3 * (int64_t)bidx[bb];
        const double* e = e3 + 3 * (int64_t)bb;
        const double s = (P[0] - B[0]) * e[0] + (P[1] - B[1]) * e[1] + (P[2] - B[2]) * e[2];
        const int64_t g = pos_g[i];
        const int64_t at = ni + g;
        for (int c = 0; c < 3; c++) q[3 * at + c] = P[c] - 2.0 * s * e[c];
        q_src[at] = pos_i[i];
        ghost_bnd[g] = bidx[bb];
        ghost_dist[g] = 2.0 * fabs(s);
    }
}

struct GhostLayout {
    size_t fi, fb, fm, pos_i, pos_b, pos_g, tiles, cnt, bidx, e3, total;
};

GhostLayout ghost_layout(int64_t n) {
    GhostLayout l{};
    size_t o = 0;
    l.fi = o; o += align_up(n);
    l.fb = o; o += align_up(n);
    l.fm = o; o += align_up(n);
    l.pos_i = o; o += align_up(4 * (size_t)n);
    l.pos_b = o; o += align_up(4 * (size_t)n);
    l.pos_g = o; o += align_up(4 * (size_t)n);
    l.tiles = o; o += align_up(4 * (size_t)scan_tiles(n));
    l.cnt = o; o += align_up(4 * 4);
    l.bidx = o; o += align_up(4 * (size_t)n);
    l.e3 = o; o += align_up(24 * (size_t)n);
    l.total = o;
    return l;
}

// out = the caller's counts [interior, ghosts, boundary points, bad frames] from the
// scan totals [interior, boundary points, ghosts, bad frames]
__global__ void k_neumann_counts(const int32_t* __restrict__ cnt, int32_t* __restrict__ out) {
    if (threadIdx.x == 0) {
        out[0] = cnt[0];
        out[1] = cnt[2];
        out[2] = cnt[1];
        out[3] = cnt[3];
    }
}

// ---------------------------------------------------------------------------
// Fold
// ---------------------------------------------------------------------------
__global__ void k_fold_keep(const int32_t* __restrict__ order, int64_t nq, int64_t ni, uint8_t* __restrict__ keep,
                            int32_t* __restrict__ inv) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nq; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t qp = order ? order[r] : (int32_t)r;
        keep[r] = qp < ni ? 1 : 0;
        inv[qp] = (int32_t)r;
    }
}

__global__ void k_fold_rows(mvgd_ell LQ, const int32_t* __restrict__ q_src, const uint8_t* __restrict__ keep,
                            const int32_t* __restrict__ newidx, const int32_t* __restrict__ inv, mvgd_ell LI) {
    const int k = LQ.k, m = k + 1;
    const int64_t npad = n_padded(LI.n);
    int32_t* order_out = const_cast<int32_t*>(LI.order);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < LQ.n; r += (int64_t)gridDim.x * blockDim.x) {
        if (!keep[r]) continue;
        const int64_t rn = newidx[r];
        order_out[rn] = LQ.order ? LQ.order[r] : (int32_t)r;
        for (int s = 0; s < k; s++) {
            const int32_t c = LQ.col[sell_index(r, s, k)];
            const int32_t qp = LQ.order ? LQ.order[c] : c;
            LI.col[sell_index(rn, s, k)] = newidx[inv[q_src[qp]]];
        }
        for (int s = 0; s < m; s++) {
            const int64_t a = sell_index(r, s, m), b = sell_index(rn, s, m);
            if (LQ.prec == MVGD_FP64) {
                static_cast<double*>(LI.val)[b] = static_cast<const double*>(LQ.val)[a];
            } else {
                static_cast<float*>(LI.val)[b] = static_cast<const float*>(LQ.val)[a];
                LI.val_lo[b] = LQ.val_lo[a];
            }
        }
    }
    // padding rows: zero weights, column 0
    for (int64_t r = LI.n + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < npad;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int s = 0; s < k; s++) LI.col[sell_index(r, s, k)] = 0;
        for (int s = 0; s < m; s++) {
            const int64_t b = sell_index(r, s, m);
            if (LQ.prec == MVGD_FP64) {
                static_cast<double*>(LI.val)[b] = 0.0;
            } else {
                static_cast<float*>(LI.val)[b] = 0.0f;
                LI.val_lo[b] = 0.0f;
            }
        }
    }
}

// c[p] = sum over the ghost columns s of interior row p of w_s |p - ghost| g(p_b)
__global__ void k_neumann_rhs(mvgd_ell LQ, int64_t ni, const double* __restrict__ dist,
                              const int32_t* __restrict__ bnd, const double* __restrict__ g, double* __restrict__ c) {
    const int k = LQ.k, m = k + 1;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < LQ.n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t qp = LQ.order ? LQ.order[r] : (int32_t)r;
        if (qp >= ni) continue;
        double acc = 0.0;
        for (int s = 0; s < k; s++) {
            const int32_t cc = LQ.col[sell_index(r, s, k)];
            const int64_t q2 = LQ.order ? LQ.order[cc] : cc;
            if (q2 < ni) continue;
            const int64_t t = q2 - ni;
            const int64_t e = sell_index(r, s + 1, m);
            const double w = LQ.prec == MVGD_FP64
                                 ? static_cast<const double*>(LQ.val)[e]
                                 : (double)static_cast<const float*>(LQ.val)[e] + (double)LQ.val_lo[e];
            acc += w * dist[t] * g[bnd[t]];
        }
        c[qp] = acc;
    }
}

struct FoldLayout {
    size_t keep, newidx, inv, tiles, cnt, total;
};

FoldLayout fold_layout(int64_t nq) {
    FoldLayout l{};
    size_t o = 0;
    l.keep = o; o += align_up(nq);
    l.newidx = o; o += align_up(4 * (size_t)nq);
    l.inv = o; o += align_up(4 * (size_t)nq);
    l.tiles = o; o += align_up(4 * (size_t)scan_tiles(nq));
    l.cnt = o; o += align_up(4);
    l.total = o;
    return l;
}

unsigned grid_for(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_neumann_ghosts_workspace_bytes(int64_t n) {
    if (n < 2 || n >= (1ll << 30)) return 0;
    return ghost_layout(n).total;
}

MVGD_API mvgd_status mvgd_neumann_ghosts(const double* pts, int64_t n, int32_t k, const int32_t* nbr,
                                         const uint8_t* boundary, int32_t kb, double* q, int32_t* q_src,
                                         int32_t* interior, int32_t* ghost_bnd, double* ghost_dist,
                                         int32_t* counts, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!pts || !nbr || !boundary || !q || !q_src || !interior || !ghost_bnd || !ghost_dist || !counts || !ws)
        return MVGD_EINVAL;
    if (n < 2 || n >= (1ll << 30) || k < kMinK || k > kMaxK || k >= n || kb < 2 || kb > kMaxKb) return MVGD_EINVAL;
    if (!aligned(pts) || !aligned(nbr) || !aligned(q) || !aligned(q_src) || !aligned(interior) ||
        !aligned(ghost_bnd) || !aligned(ghost_dist) || !aligned(ws) || (reinterpret_cast<uintptr_t>(counts) & 3))
        return MVGD_EINVAL;
    if (ws_bytes < mvgd_neumann_ghosts_workspace_bytes(n)) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const GhostLayout L = ghost_layout(n);
    char* base = static_cast<char*>(ws);
    uint8_t* fi = reinterpret_cast<uint8_t*>(base + L.fi);
    uint8_t* fb = reinterpret_cast<uint8_t*>(base + L.fb);
    uint8_t* fm = reinterpret_cast<uint8_t*>(base + L.fm);
    int32_t* pos_i = reinterpret_cast<int32_t*>(base + L.pos_i);
    int32_t* pos_b = reinterpret_cast<int32_t*>(base + L.pos_b);
    int32_t* pos_g = reinterpret_cast<int32_t*>(base + L.pos_g);
    int32_t* tiles = reinterpret_cast<int32_t*>(base + L.tiles);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + L.cnt);  // interior, boundary, ghosts, bad frames
    int32_t* bidx = reinterpret_cast<int32_t*>(base + L.bidx);
    double* e3 = reinterpret_cast<double*>(base + L.e3);
    MVGD_CUDA_TRY(cudaMemsetAsync(cnt, 0, 4 * sizeof(int32_t), s));
    const unsigned g = grid_for(n);
    k_neumann_flags<<<g, 256, 0, s>>>(boundary, nbr, n, k, fi, fb, fm);
    scan_flags(fi, n, pos_i, tiles, cnt + 0, s);
    scan_flags(fb, n, pos_b, tiles, cnt + 1, s);
    scan_flags(fm, n, pos_g, tiles, cnt + 2, s);
    k_neumann_compact<<<g, 256, 0, s>>>(pts, n, fi, pos_i, pos_b, q, q_src, interior, bidx);
    // one thread per boundary point; launched for n (the count is on the device)
    k_boundary_frames<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(pts, nbr, k, bidx, cnt + 1, kb, e3, cnt + 3);
    // the caller's counts: interior points, ghosts, boundary points, bad frames
    k_neumann_counts<<<1, 32, 0, s>>>(cnt, counts);
    k_ghosts<<<g, 256, 0, s>>>(pts, n, fm, pos_i, pos_g, bidx, counts, e3, q, q_src, ghost_bnd, ghost_dist);
    return launch_status();
}

MVGD_API size_t mvgd_neumann_fold_workspace_bytes(int64_t nq) {
    if (nq < 1 || nq >= (1ll << 31)) return 0;
    return fold_layout(nq).total;
}

MVGD_API mvgd_status mvgd_neumann_fold(const mvgd_ell* LQ, const int32_t* q_src, mvgd_ell* LI, void* ws,
                                       size_t ws_bytes, mvgd_stream_t stream) {
    if (!LQ || !LI || !q_src || !ws || !LQ->col || !LQ->val || !LI->col || !LI->val || !LI->order)
        return MVGD_EINVAL;
    if (LQ->n < 1 || LQ->n >= (1ll << 31) || LI->n < 1 || LI->n > LQ->n || LQ->k < kMinK || LQ->k > kMaxK ||
        LI->k != LQ->k || LI->prec != LQ->prec)
        return MVGD_EINVAL;
    if (LQ->prec != MVGD_FP64 && LQ->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (LQ->prec == MVGD_FP32_REFINE && (!LQ->val_lo || !LI->val_lo)) return MVGD_EINVAL;
    if (!aligned(LQ->col) || !aligned(LQ->val) || !aligned(LQ->val_lo) || !aligned(LQ->order) ||
        !aligned(LI->col) || !aligned(LI->val) || !aligned(LI->val_lo) || !aligned(LI->order) || !aligned(q_src) ||
        !aligned(ws))
        return MVGD_EINVAL;
    if (ws_bytes < mvgd_neumann_fold_workspace_bytes(LQ->n)) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const FoldLayout F = fold_layout(LQ->n);
    char* base = static_cast<char*>(ws);
    uint8_t* keep = reinterpret_cast<uint8_t*>(base + F.keep);
    int32_t* newidx = reinterpret_cast<int32_t*>(base + F.newidx);
    int32_t* inv = reinterpret_cast<int32_t*>(base + F.inv);
    int32_t* tiles = reinterpret_cast<int32_t*>(base + F.tiles);
    int32_t* cnt = reinterpret_cast<int32_t*>(base + F.cnt);
    const unsigned g = grid_for(LQ->n);
    k_fold_keep<<<g, 256, 0, s>>>(LQ->order, LQ->n, LI->n, keep, inv);
    scan_flags(keep, LQ->n, newidx, tiles, cnt, s);
    k_fold_rows<<<g, 256, 0, s>>>(*LQ, q_src, keep, newidx, inv, *LI);
    return launch_status();
}

MVGD_API mvgd_status mvgd_neumann_rhs(const mvgd_ell* LQ, int64_t n_interior, const double* ghost_dist,
                                      const int32_t* ghost_bnd, const double* g, double* c, mvgd_stream_t stream) {
    if (!LQ || !ghost_dist || !ghost_bnd || !g || !c || !LQ->col || !LQ->val) return MVGD_EINVAL;
    if (LQ->n < 1 || LQ->n >= (1ll << 31) || n_interior < 1 || n_interior > LQ->n || LQ->k < kMinK ||
        LQ->k > kMaxK)
        return MVGD_EINVAL;
    if (LQ->prec != MVGD_FP64 && LQ->prec != MVGD_FP32_REFINE) return MVGD_EINVAL;
    if (LQ->prec == MVGD_FP32_REFINE && !LQ->val_lo) return MVGD_EINVAL;
    if (!aligned(ghost_dist) || !aligned(ghost_bnd) || !aligned(g) || !aligned(c) || !aligned(LQ->col) ||
        !aligned(LQ->val) || !aligned(LQ->val_lo) || !aligned(LQ->order))
        return MVGD_EINVAL;
    k_neumann_rhs<<<grid_for(LQ->n), 256, 0, (cudaStream_t)stream>>>(*LQ, n_interior, ghost_dist, ghost_bnd, g, c);
    return launch_status();
}
