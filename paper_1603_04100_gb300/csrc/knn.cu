// kNN on a periodic cell grid (Sec. 2: N(i) = the K nearest neighbours).
//
// Build: bounding box -> cell edge s (given, or estimated from the surface area
// covered by a 64^3 occupancy bitmap) -> every point gets integer cell
// coordinates c = floor((p - lo) / s) and a bucket = Morton code of
// (c mod M) with power-of-two wrap sizes M per axis, so that at most ~2n
// buckets exist whatever the extent; a counting sort groups points by bucket.
// Any block of <= M consecutive cells per axis maps to distinct buckets, so a
// query scans each bucket at most once; points of far cells that share a
// bucket are merely extra candidates.
//
// Query (one warp per point, points visited in bucket order for locality):
//   1. the 27 (then 125, ...) cells around the query are turned into bucket
//      ranges; lanes take candidates 32 at a time from the concatenated ranges;
//   2. FP32 screen: squared distances from FP32 copies of the coordinates,
//      a running top-32 list kept sorted across lanes by bitonic merges;
//   3. exact re-rank: FP64 keys fl(fl(fl(dx dx) + fl(dy dy)) + fl(dz dz)) of
//      the 32 kept candidates, bitonic sort by (key, index);
//   4. guards: the K-th exact distance must be inside the scanned block
//      (else the ring grows) and below the smallest distance any screened-out
//      candidate can have given the FP32 error bound (else the scan is redone
//      with exact keys).  Both bounds are evaluated with directed rounding.
#include <cfloat>
#include <mutex>

#include "common.cuh"

namespace mvgd {
namespace {

constexpr int kOccBits = 64;                 // occupancy bitmap edge
constexpr int kOccWords = kOccBits * kOccBits * kOccBits / 32;
constexpr int kBboxBlocks = 512;
constexpr int kScanTile = 2048;
constexpr int kQueryWarps = 8;

struct KnnParams {
    double lo[3];
    double ext[3];
    double s, inv_s;
    int D[3];       // cells per axis
    int Mb[3];      // log2 of the wrap per axis
    int nbuckets;
    int pad;
    float s_f;      // cell edge in FP32
    float ext_f;    // largest extent in FP32
    float eps_abs;  // bound on |d_fp32 - d_exact| from rounding the coordinates
    float margin;   // bound on the error of FP32 cell-boundary positions
};

struct Key {
    uint64_t a;  // distance bits (FP32 or FP64, non-negative so integer order = value order)
    uint32_t b;  // point index
};

__device__ __forceinline__ bool key_less(const Key& x, const Key& y) {
    return x.a < y.a || (x.a == y.a && x.b < y.b);
}
__device__ __forceinline__ Key key_shfl_xor(const Key& k, int m) {
    Key o;
    o.a = shfl_xor_u64(k.a, m);
    o.b = __shfl_xor_sync(0xffffffffu, k.b, m);
    return o;
}
__device__ __forceinline__ Key key_shfl(const Key& k, int src) {
    Key o;
    o.a = shfl_u64(k.a, src);
    o.b = __shfl_sync(0xffffffffu, k.b, src);
    return o;
}
__device__ __forceinline__ Key key_empty() { return Key{~0ull, 0xffffffffu}; }

// Ascending bitonic sort of one key per lane.
__device__ __forceinline__ void warp_sort(Key& k) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            Key o = key_shfl_xor(k, stride);
            bool up = (lane & size) == 0 || size == 32;
            bool lower = (lane & stride) == 0;
            bool o_less = key_less(o, k);
            // lower element keeps the min when ascending
            if ((lower == up) ? o_less : !o_less) k = o;
        }
    }
}

// list (ascending) <- the 32 smallest of list and chunk (chunk sorted ascending).
__device__ __forceinline__ void warp_merge(Key& list, Key chunk) {
    const unsigned lane = lane_id();
    Key rev = key_shfl(chunk, 31 - lane);
    if (key_less(rev, list)) list = rev;
#pragma unroll
    for (int stride = 16; stride > 0; stride >>= 1) {
        Key o = key_shfl_xor(list, stride);
        bool lower = (lane & stride) == 0;
        bool o_less = key_less(o, list);
        if (lower ? o_less : !o_less) list = o;
    }
}

__host__ __device__ inline uint32_t morton_bucket(uint32_t x, uint32_t y, uint32_t z, const int* Mb) {
    uint32_t out = 0;
    int bit = 0;
    int top = Mb[0] > Mb[1] ? Mb[0] : Mb[1];
    top = top > Mb[2] ? top : Mb[2];
    for (int t = 0; t < top; t++) {
        if (t < Mb[0]) out |= ((x >> t) & 1u) << bit++;
        if (t < Mb[1]) out |= ((y >> t) & 1u) << bit++;
        if (t < Mb[2]) out |= ((z >> t) & 1u) << bit++;
    }
    return out;
}

__device__ inline int cell_of(double x, double lo, double inv_s, int D) {
    double t = floor((x - lo) * inv_s);
    if (!(t >= 0.0)) t = 0.0;
    if (t > (double)(D - 1)) t = (double)(D - 1);
    return (int)t;
}

// ---------------------------------------------------------------------------
// Build kernels
// ---------------------------------------------------------------------------
__global__ void k_bbox_partial(const double* __restrict__ pts, int64_t n, double* __restrict__ part) {
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            double v = pts[3 * i + a];
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    __shared__ double sm[6][32];
    for (int a = 0; a < 3; a++) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    int w = threadIdx.x / 32, nw = blockDim.x / 32;
    if (lane_id() == 0)
        for (int a = 0; a < 3; a++) { sm[a][w] = mn[a]; sm[3 + a][w] = mx[a]; }
    __syncthreads();
    if (threadIdx.x < 6) {
        double v = sm[threadIdx.x][0];
        for (int q = 1; q < nw; q++)
            v = threadIdx.x < 3 ? fmin(v, sm[threadIdx.x][q]) : fmax(v, sm[threadIdx.x][q]);
        part[blockIdx.x * 6 + threadIdx.x] = v;
    }
}

__global__ void k_bbox_final(const double* __restrict__ part, int nparts, KnnParams* P) {
    if (threadIdx.x != 0) return;
    double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (int b = 0; b < nparts; b++)
        for (int a = 0; a < 3; a++) {
            mn[a] = fmin(mn[a], part[b * 6 + a]);
            mx[a] = fmax(mx[a], part[b * 6 + 3 + a]);
        }
    for (int a = 0; a < 3; a++) {
        P->lo[a] = mn[a];
        P->ext[a] = mx[a] - mn[a];
    }
}

__global__ void k_occupancy(const double* __restrict__ pts, int64_t n, const KnnParams* __restrict__ P,
                            unsigned* __restrict__ bits) {
    double e = fmax(P->ext[0], fmax(P->ext[1], P->ext[2]));
    double inv = e > 0 ? (double)kOccBits / e : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        for (int a = 0; a < 3; a++) {
            int t = (int)((pts[3 * i + a] - P->lo[a]) * inv);
            c[a] = t < 0 ? 0 : (t >= kOccBits ? kOccBits - 1 : t);
        }
        unsigned cell = (c[2] * kOccBits + c[1]) * kOccBits + c[0];
        atomicOr(&bits[cell >> 5], 1u << (cell & 31));
    }
}

// Cell edge, grid dimensions and wrap sizes.
__global__ void k_params(const unsigned* __restrict__ bits, int64_t n, int k, double cell_size,
                         int nbuckets_max, KnnParams* P) {
    __shared__ unsigned long long occ;
    if (threadIdx.x == 0) occ = 0;
    __syncthreads();
    if (cell_size <= 0) {
        unsigned long long c = 0;
        for (int w = threadIdx.x; w < kOccWords; w += blockDim.x) c += __popc(bits[w]);
        atomicAdd(&occ, c);
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double e = fmax(P->ext[0], fmax(P->ext[1], P->ext[2]));
    double s = cell_size;
    if (s <= 0) {
        // surface-area estimate: occupied cells x cell area / mean |n|_1 of a surface
        double s0 = e / kOccBits;
        double area = (double)occ * s0 * s0 / 1.5;
        double rk = sqrt((double)k * area / (3.141592653589793 * (double)n));
        s = 1.25 * rk * (cell_size < 0 ? -cell_size : 1.0);  // a negative cell_size scales the estimate
    }
    if (!(s > 0) || !isfinite(s)) s = e > 0 ? e : 1.0;
    if (e > 0 && s < e * 1e-6) s = e * 1e-6;   // keep cell coordinates below 2^20
    double inv_s = 1.0 / s;
    int Mb[3];
    for (int a = 0; a < 3; a++) {
        double d = floor(P->ext[a] * inv_s) + 1.0;
        if (d > 1048576.0) d = 1048576.0;
        P->D[a] = (int)d;
        int b = 0;
        while ((1 << b) < P->D[a] && b < 20) b++;
        Mb[a] = b < 2 ? 2 : b;  // wrap >= 4 so a 3-cell block never aliases
    }
    while (Mb[0] + Mb[1] + Mb[2] > 2 && (1ll << (Mb[0] + Mb[1] + Mb[2])) > nbuckets_max) {
        int a = (Mb[0] >= Mb[1] && Mb[0] >= Mb[2]) ? 0 : (Mb[1] >= Mb[2] ? 1 : 2);
        if (Mb[a] <= 2) break;
        Mb[a]--;
    }
    for (int a = 0; a < 3; a++) P->Mb[a] = Mb[a];
    P->nbuckets = 1 << (Mb[0] + Mb[1] + Mb[2]);
    P->s = s;
    P->inv_s = inv_s;
    P->s_f = (float)s;
    P->ext_f = (float)e;
    // |fl32(x - lo) - (x - lo)| <= 2^-24 e per coordinate, for both points: the
    // distance moves by at most 2 sqrt(3) 2^-24 e; rounded up generously.
    P->eps_abs = (float)(4.0 * e * 5.9604644775390625e-08) + 1e-30f;
    P->margin = (float)(8.0 * e * 5.9604644775390625e-08 + 4.0 * s * 5.9604644775390625e-08) + 1e-30f;
}

__global__ void k_count(const double* __restrict__ pts, int64_t n, const KnnParams* __restrict__ P,
                        int* __restrict__ counts, int* __restrict__ pbucket, int* __restrict__ prank,
                        uint32_t* __restrict__ pcell) {
    const KnnParams p = *P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int c[3];
        for (int a = 0; a < 3; a++) c[a] = cell_of(pts[3 * i + a], p.lo[a], p.inv_s, p.D[a]);
        uint32_t b = morton_bucket(c[0] & ((1u << p.Mb[0]) - 1), c[1] & ((1u << p.Mb[1]) - 1),
                                   c[2] & ((1u << p.Mb[2]) - 1), p.Mb);
        pbucket[i] = (int)b;
        prank[i] = atomicAdd(&counts[b], 1);
        for (int a = 0; a < 3; a++) pcell[3 * i + a] = (uint32_t)c[a];
    }
}

// Exclusive scan in three passes (tile sums, scan of sums, add).
__global__ void k_scan_tiles(int* __restrict__ a, int len, int* __restrict__ sums) {
    __shared__ int sh[kScanTile];
    int base = blockIdx.x * kScanTile;
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
        sh[t] = (base + t < len) ? a[base + t] : 0;
    __syncthreads();
    // Hillis-Steele on 2048 elements with 1024 threads, 2 elements each
    for (int off = 1; off < kScanTile; off <<= 1) {
        int v0 = 0, v1 = 0;
        int t0 = threadIdx.x, t1 = threadIdx.x + blockDim.x;
        if (t0 >= off) v0 = sh[t0 - off];
        if (t1 >= off) v1 = sh[t1 - off];
        __syncthreads();
        sh[t0] += v0;
        sh[t1] += v1;
        __syncthreads();
    }
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < len) a[base + t] = (t == 0 ? 0 : sh[t - 1]);
    if (threadIdx.x == 0) sums[blockIdx.x] = sh[kScanTile - 1];
}

__global__ void k_scan_sums(int* __restrict__ sums, int ntiles) {
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int t = 0; t < ntiles; t++) {
        int v = sums[t];
        sums[t] = acc;
        acc += v;
    }
}

__global__ void k_scan_add(int* __restrict__ a, int len, const int* __restrict__ sums, int total_at,
                           int64_t n) {
    int base = blockIdx.x * kScanTile;
    int add = sums[blockIdx.x];
    for (int t = threadIdx.x; t < kScanTile; t += blockDim.x)
        if (base + t < len) a[base + t] += add;
    if (blockIdx.x == 0 && threadIdx.x == 0) a[total_at] = (int)n;
}

__global__ void k_scatter(const double* __restrict__ pts, int64_t n, const KnnParams* __restrict__ P,
                          const int* __restrict__ start, const int* __restrict__ pbucket,
                          const int* __restrict__ prank, float4* __restrict__ sorted,
                          int* __restrict__ order) {
    const KnnParams p = *P;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int pos = start[pbucket[i]] + prank[i];
        float4 v;
        v.x = (float)(pts[3 * i + 0] - p.lo[0]);
        v.y = (float)(pts[3 * i + 1] - p.lo[1]);
        v.z = (float)(pts[3 * i + 2] - p.lo[2]);
        v.w = __int_as_float((int)i);
        sorted[pos] = v;
        order[pos] = (int)i;
    }
}

// Order points inside each bucket by index (warp per bucket, buckets of <= 32
// points; larger ones keep arrival order), so that `order` is reproducible.
__global__ void k_sort_buckets(const int* __restrict__ start, int nbuckets, float4* __restrict__ sorted,
                               int* __restrict__ order) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32;
    int nwarps = gridDim.x * blockDim.x / 32;
    unsigned lane = lane_id();
    for (int b = warp; b < nbuckets; b += nwarps) {
        int beg = start[b], cnt = start[b + 1] - beg;
        if (cnt <= 1 || cnt > 32) continue;
        Key k = key_empty();
        float4 v = make_float4(0, 0, 0, 0);
        if ((int)lane < cnt) {
            v = sorted[beg + lane];
            k.a = (uint32_t)__float_as_int(v.w);
            k.b = lane;
        }
        warp_sort(k);
        float4 w;
        w.x = __shfl_sync(0xffffffffu, v.x, k.b & 31);
        w.y = __shfl_sync(0xffffffffu, v.y, k.b & 31);
        w.z = __shfl_sync(0xffffffffu, v.z, k.b & 31);
        w.w = __shfl_sync(0xffffffffu, v.w, k.b & 31);
        if ((int)lane < cnt) {
            sorted[beg + lane] = w;
            order[beg + lane] = __float_as_int(w.w);
        }
    }
}

// ---------------------------------------------------------------------------
// The row order exported to callers: every point along one Z-order curve of
// the bounding cube (21 bits per axis), ties by index.  Consecutive points of
// this order are spatial neighbours at every scale down to a few points --
// which the kNN's hashed cell buckets are not where the hash wraps around the
// grid -- and aggregation multigrid, which groups consecutive rows, relies on
// it.  A stable LSD radix sort of (key, index) pairs, 8 bits per pass.
// ---------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixTile = 4096;  // elements per block: 16 rounds of 256
constexpr int kRadixWarps = kRadixThreads / 32;

__device__ __forceinline__ uint64_t spread3_21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__global__ void k_zorder_keys(const double* __restrict__ pts, int64_t n, const KnnParams* __restrict__ P,
                              uint64_t* __restrict__ key, int* __restrict__ val) {
    const KnnParams p = *P;
    const double e = fmax(p.ext[0], fmax(p.ext[1], p.ext[2]));
    const double scale = e > 0.0 ? 2097152.0 / e : 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = 0;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double t = (pts[3 * i + a] - p.lo[a]) * scale;
            t = t < 0.0 ? 0.0 : (t > 2097151.0 ? 2097151.0 : t);
            k |= spread3_21((uint32_t)t) << a;
        }
        key[i] = k;
        val[i] = (int)i;
    }
}

// Digit histogram of each tile, stored digit-major: counts[digit * nblocks + block].
__global__ void __launch_bounds__(kRadixThreads) k_radix_count(const uint64_t* __restrict__ key, int64_t n, int shift,
                                                               int* __restrict__ counts) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    const int64_t end = base + kRadixTile < n ? base + kRadixTile : n;
    for (int64_t i = base + threadIdx.x; i < end; i += kRadixThreads) atomicAdd(&h[(key[i] >> shift) & 255u], 1);
    __syncthreads();
    counts[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: the tile is read in order (round by round, thread by thread),
// and each element goes after every earlier element of its digit.
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                                 const int* __restrict__ vin, int64_t n, int shift,
                                                                 const int* __restrict__ offs,
                                                                 uint64_t* __restrict__ kout, int* __restrict__ vout) {
    __shared__ int run[256];
    __shared__ int wcnt[kRadixWarps][256];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    run[tid] = offs[tid * gridDim.x + blockIdx.x];
    for (int w = 0; w < kRadixWarps; w++) wcnt[w][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRadixTile;
    for (int round = 0; round < kRadixTile / kRadixThreads; round++) {
        const int64_t i = base + (int64_t)round * kRadixThreads + tid;
        const bool valid = i < n;
        const uint64_t k = valid ? kin[i] : 0;
        const int v = valid ? vin[i] : 0;
        const unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
        __syncthreads();
        int tot = 0;
        for (int w = 0; w < kRadixWarps; w++) {  // exclusive prefix over warps, digit tid
            const int c = wcnt[w][tid];
            wcnt[w][tid] = tot;
            tot += c;
        }
        __syncthreads();
        if (valid) {
            const int pos = run[d] + wcnt[wid][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        run[tid] += tot;
        for (int w = 0; w < kRadixWarps; w++) wcnt[w][tid] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Query
// ---------------------------------------------------------------------------
struct AxisRange {
    int first, len;  // first cell (or residue 0) and count
    bool full;       // all residues visited
};

__device__ __forceinline__ double exact_d2(const double* __restrict__ pts, int i, int j) {
    double dx = __dsub_rn(pts[3 * (int64_t)j + 0], pts[3 * (int64_t)i + 0]);
    double dy = __dsub_rn(pts[3 * (int64_t)j + 1], pts[3 * (int64_t)i + 1]);
    double dz = __dsub_rn(pts[3 * (int64_t)j + 2], pts[3 * (int64_t)i + 2]);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Scan the block of ring R around cell c; returns the running list.
template <bool EXACT>
__device__ Key scan_block(const double* __restrict__ pts, const float4* __restrict__ sorted,
                          const int* __restrict__ start, const KnnParams& p, const AxisRange* ax,
                          int i, float qx, float qy, float qz) {
    const unsigned lane = lane_id();
    Key list = key_empty();
    const int ncell = ax[0].len * ax[1].len * ax[2].len;
    const uint32_t mask[3] = {(1u << p.Mb[0]) - 1, (1u << p.Mb[1]) - 1, (1u << p.Mb[2]) - 1};
    for (int cb = 0; cb < ncell; cb += 32) {
        int cid = cb + (int)lane;
        int beg = 0, cnt = 0;
        if (cid < ncell) {
            int tx = cid % ax[0].len;
            int ty = (cid / ax[0].len) % ax[1].len;
            int tz = cid / (ax[0].len * ax[1].len);
            uint32_t bx = (uint32_t)(ax[0].first + tx) & mask[0];
            uint32_t by = (uint32_t)(ax[1].first + ty) & mask[1];
            uint32_t bz = (uint32_t)(ax[2].first + tz) & mask[2];
            uint32_t b = morton_bucket(bx, by, bz, p.Mb);
            beg = start[b];
            cnt = start[b + 1] - beg;
        }
        // inclusive prefix of counts across lanes
        int off = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, off, o);
            if ((int)lane >= o) off += v;
        }
        const int total = __shfl_sync(0xffffffffu, off, 31);
        for (int t = 0; t < total; t += 32) {
            int c = t + (int)lane;
            Key key = key_empty();
            // owning lane: smallest l with off[l] > c (all lanes take part in the shuffles)
            int l = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                int probe = __shfl_sync(0xffffffffu, off, l + step - 1);
                if (probe <= c) l += step;
            }
            int lb = __shfl_sync(0xffffffffu, beg, l & 31);
            int lo = __shfl_sync(0xffffffffu, off, l & 31) - __shfl_sync(0xffffffffu, cnt, l & 31);
            if (c < total) {
                int pos = lb + (c - lo);
                float4 v = __ldg(&sorted[pos]);
                int j = __float_as_int(v.w);
                if (j != i) {
                    if (EXACT) {
                        key.a = (uint64_t)__double_as_longlong(exact_d2(pts, i, j));
                    } else {
                        float dx = v.x - qx, dy = v.y - qy, dz = v.z - qz;
                        float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                        key.a = (uint32_t)__float_as_int(d2);
                    }
                    key.b = (uint32_t)j;
                }
            }
            // merge only if some candidate beats the current 32nd entry
            Key worst = key_shfl(list, 31);
            if (__any_sync(0xffffffffu, key_less(key, worst))) {
                warp_sort(key);
                warp_merge(list, key);
            }
        }
    }
    return list;
}

__global__ void __launch_bounds__(kQueryWarps * 32)
k_query(const double* __restrict__ pts, int64_t n, int k, const KnnParams* __restrict__ P,
        const float4* __restrict__ sorted, const int* __restrict__ start, const int* __restrict__ order,
        const uint32_t* __restrict__ pcell, int32_t* __restrict__ nbr) {
    const KnnParams p = *P;
    const unsigned lane = lane_id();
    const int64_t nwarps = (int64_t)gridDim.x * kQueryWarps;
    for (int64_t q = blockIdx.x * (int64_t)kQueryWarps + threadIdx.x / 32; q < n; q += nwarps) {
        const float4 me = __ldg(&sorted[q]);
        const int i = order[q];
        const float qv[3] = {me.x, me.y, me.z};
        int c[3] = {(int)pcell[3 * (int64_t)i], (int)pcell[3 * (int64_t)i + 1],
                    (int)pcell[3 * (int64_t)i + 2]};
        bool exact_mode = false;
        Key best = key_empty();
        // rings double until the k-th distance is inside the block; a block of
        // more than M cells per axis visits each residue once, so every scan is
        // bounded by the bucket count and the loop by log2 of the grid size
        for (int R = 1;;) {
            AxisRange ax[3];
            bool all_full = true;
            float guard = FLT_MAX;
            for (int a = 0; a < 3; a++) {
                int a0 = c[a] - R, a1 = c[a] + R;
                bool lo_open = a0 > 0, hi_open = a1 < p.D[a] - 1;
                if (a0 < 0) a0 = 0;
                if (a1 > p.D[a] - 1) a1 = p.D[a] - 1;
                int len = a1 - a0 + 1, M = 1 << p.Mb[a];
                ax[a].full = len > M;
                ax[a].first = ax[a].full ? 0 : a0;
                ax[a].len = ax[a].full ? M : len;
                if (lo_open || hi_open) all_full = false;
                // distance from the query to the faces of the block (FP32, rounded down)
                if (lo_open) guard = fminf(guard, __fsub_rd(qv[a], __fmul_ru((float)a0, p.s_f)));
                if (hi_open) guard = fminf(guard, __fsub_rd(__fmul_rd((float)(a1 + 1), p.s_f), qv[a]));
            }
            guard = __fsub_rd(guard, p.margin);
            Key list = exact_mode ? scan_block<true>(pts, sorted, start, p, ax, i, me.x, me.y, me.z)
                                  : scan_block<false>(pts, sorted, start, p, ax, i, me.x, me.y, me.z);
            Key ex = list;
            if (!exact_mode && list.b != 0xffffffffu)
                ex.a = (uint64_t)__double_as_longlong(exact_d2(pts, i, (int)list.b));
            if (!exact_mode) warp_sort(ex);
            Key kth = key_shfl(ex, k - 1);
            bool have_k = kth.b != 0xffffffffu;
            double dk2 = have_k ? __longlong_as_double((long long)kth.a) : 0.0;
            float ub = __fsqrt_ru(__double2float_ru(dk2));
            bool cov_ok = have_k && (all_full || ub < guard);
            bool ex_ok = true;
            if (!exact_mode) {
                Key last = key_shfl(list, 31);
                if (last.b != 0xffffffffu) {
                    float d = __fsqrt_rd(__uint_as_float((uint32_t)last.a));
                    float lb = __fsub_rd(__fmul_rd(d, 1.0f - 8.0f * 5.9604645e-08f), p.eps_abs);
                    ex_ok = lb > ub;
                }
            }
            if (cov_ok && ex_ok) {
                best = ex;
                break;
            }
            if (!ex_ok && !exact_mode) {
                exact_mode = true;  // redo this ring with exact keys
                continue;
            }
            if (all_full) {  // fewer than k points: impossible after host checks
                best = ex;
                break;
            }
            R *= 2;
        }
        if ((int)lane < k) nbr[(int64_t)i * k + lane] = (int32_t)best.b;
    }
}

struct KnnLayout {
    KnnParams* params;
    double* bbox;
    unsigned* occ;
    int* start;       // nbuckets_max + 1
    int* sums;
    int* pbucket;
    int* prank;
    uint32_t* pcell;  // [n][3]
    float4* sorted;
    int* order;
    uint64_t* zkey[2];  // radix-sort buffers of the exported order
    int* zval[2];
    int* zcount;        // [256 * radix blocks + 1]
    int* zsums;
    size_t bytes;
    int nbuckets_max;
};

int bucket_budget(int64_t n) {
    int64_t b = 1024;
    while (b < 2 * n && b < (1ll << 26)) b <<= 1;
    return (int)b;
}

KnnLayout knn_layout(void* ws, int64_t n) {
    KnnLayout L;
    Carver cv(ws);
    L.nbuckets_max = bucket_budget(n);
    int ntiles = (L.nbuckets_max + 1 + kScanTile - 1) / kScanTile;
    L.params = cv.take<KnnParams>(1);
    L.bbox = cv.take<double>(kBboxBlocks * 6);
    L.occ = cv.take<unsigned>(kOccWords);
    L.start = cv.take<int>(L.nbuckets_max + 1);
    L.sums = cv.take<int>(ntiles);
    L.pbucket = cv.take<int>(n);
    L.prank = cv.take<int>(n);
    L.pcell = cv.take<uint32_t>(3 * n);
    L.sorted = cv.take<float4>(n);
    L.order = cv.take<int>(n);
    const int64_t rblocks = (n + kRadixTile - 1) / kRadixTile;
    for (int b = 0; b < 2; b++) {
        L.zkey[b] = cv.take<uint64_t>(n);
        L.zval[b] = cv.take<int>(n);
    }
    L.zcount = cv.take<int>(256 * rblocks + 1);
    L.zsums = cv.take<int>((256 * rblocks + kScanTile - 1) / kScanTile + 1);
    L.bytes = cv.used;
    return L;
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API size_t mvgd_knn_workspace_bytes(int64_t n, int32_t k) {
    (void)k;
    if (n <= 0) return 0;
    return knn_layout(nullptr, n).bytes;
}

MVGD_API mvgd_status mvgd_knn(const double* pts, int64_t n, int32_t k, int32_t* nbr, int32_t* order,
                              double cell_size, void* ws, size_t ws_bytes, mvgd_stream_t stream) {
    if (!pts || !nbr || !ws || n < 2 || n >= (1ll << 31) || k < 1 || k > kMaxK || k >= n)
        return MVGD_EINVAL;
    if (!aligned(pts) || !aligned(nbr) || !aligned(order) || !aligned(ws)) return MVGD_EINVAL;
    if (!(cell_size == cell_size)) return MVGD_EINVAL;
    KnnLayout L = knn_layout(ws, n);
    if (ws_bytes < L.bytes) return MVGD_EWORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    MVGD_CUDA_TRY(cudaGetDevice(&dev));
    MVGD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int tb = 256;
    int gb = (int)((n + tb - 1) / tb);
    if (gb > sms * 8) gb = sms * 8;
    int nb_box = gb < kBboxBlocks ? gb : kBboxBlocks;

    k_bbox_partial<<<nb_box, tb, 0, s>>>(pts, n, L.bbox);
    k_bbox_final<<<1, 32, 0, s>>>(L.bbox, nb_box, L.params);
    if (cell_size <= 0) {
        MVGD_CUDA_TRY(cudaMemsetAsync(L.occ, 0, sizeof(unsigned) * kOccWords, s));
        k_occupancy<<<gb, tb, 0, s>>>(pts, n, L.params, L.occ);
    }
    k_params<<<1, 256, 0, s>>>(L.occ, n, k, cell_size, L.nbuckets_max, L.params);
    MVGD_CUDA_TRY(cudaMemsetAsync(L.start, 0, sizeof(int) * (L.nbuckets_max + 1), s));
    k_count<<<gb, tb, 0, s>>>(pts, n, L.params, L.start, L.pbucket, L.prank, L.pcell);
    // scan over the whole budget; buckets past params->nbuckets stay empty
    int len = L.nbuckets_max;
    int ntiles = (len + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<ntiles, 1024, 0, s>>>(L.start, len, L.sums);
    k_scan_sums<<<1, 32, 0, s>>>(L.sums, ntiles);
    k_scan_add<<<ntiles, 1024, 0, s>>>(L.start, len, L.sums, len, n);
    k_scatter<<<gb, tb, 0, s>>>(pts, n, L.params, L.start, L.pbucket, L.prank, L.sorted, L.order);
    k_sort_buckets<<<sms * 8, 256, 0, s>>>(L.start, L.nbuckets_max, L.sorted, L.order);
    int qblocks = (int)((n + kQueryWarps - 1) / kQueryWarps);
    if (qblocks > sms * 16) qblocks = sms * 16;
    k_query<<<qblocks, kQueryWarps * 32, 0, s>>>(pts, n, k, L.params, L.sorted, L.start, L.order,
                                                 L.pcell, nbr);
    if (order) {
        const int rblocks = (int)((n + kRadixTile - 1) / kRadixTile);
        const int len = 256 * rblocks;
        const int st = (len + kScanTile - 1) / kScanTile;
        k_zorder_keys<<<gb, tb, 0, s>>>(pts, n, L.params, L.zkey[0], L.zval[0]);
        for (int pass = 0; pass < 8; pass++) {
            const int a = pass & 1;
            k_radix_count<<<rblocks, kRadixThreads, 0, s>>>(L.zkey[a], n, 8 * pass, L.zcount);
            k_scan_tiles<<<st, 1024, 0, s>>>(L.zcount, len, L.zsums);
            k_scan_sums<<<1, 32, 0, s>>>(L.zsums, st);
            k_scan_add<<<st, 1024, 0, s>>>(L.zcount, len, L.zsums, len, n);
            k_radix_scatter<<<rblocks, kRadixThreads, 0, s>>>(L.zkey[a], L.zval[a], n, 8 * pass, L.zcount,
                                                              L.zkey[a ^ 1], L.zval[a ^ 1]);
        }
        MVGD_CUDA_TRY(cudaMemcpyAsync(order, L.zval[0], sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    return launch_status();
}

// ---------------------------------------------------------------------------
// kNN for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc at all: code that is
// being recorded into a CUDA graph (an allocation would break the capture),
// latency-bound loops that must never wait on the allocator, and host
// applications or plug-in frameworks that own every device buffer and hand
// the library only its inputs and outputs.  For them the scratch that
// mvgd_knn takes from a caller workspace lives instead in one file-scope
// device array, reserved when the library's code is loaded on a GPU and held
// by every GPU that loads it until the process exits.  The array is sized for
// MVGD_KNN_NOALLOC_MAX_POINTS points; larger clouds are refused.
//
// In host code the array's name is only a host-side stand-in, never a device
// address, so its address is fetched with cudaGetSymbolAddress once per
// device, with that device current, on the first call made on that device;
// that first call should therefore come before any stream capture.  Every
// call on a device shares the one array: calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on it and must be
// serialised by the caller.  The array keeps the last call's contents; the
// kNN zeroes what it needs zeroed (bucket counts, occupancy bits) itself.
// ---------------------------------------------------------------------------
namespace mvgd {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // >= knn workspace of 65,536 points
static __device__ __align__(256) unsigned char g_knn_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

mvgd_status scratch_for_current_device(void** out) {
    int dev = 0;
    MVGD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MVGD_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_knn_scratch) != cudaSuccess || p == nullptr) return MVGD_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MVGD_OK;
}

}  // namespace
}  // namespace mvgd

MVGD_API mvgd_status mvgd_knn_noalloc(const double* pts, int64_t n, int32_t k, int32_t* nbr, int32_t* order,
                                      double cell_size, mvgd_stream_t stream) {
    if (n > MVGD_KNN_NOALLOC_MAX_POINTS || knn_layout(nullptr, n).bytes > kNoAllocScratchBytes) return MVGD_EINVAL;
    if (!pts || !nbr || n < 2 || k < 1 || k > kMaxK || k >= n) return MVGD_EINVAL;
    void* scratch = nullptr;
    mvgd_status st = scratch_for_current_device(&scratch);
    if (st != MVGD_OK) return st;
    return mvgd_knn(pts, n, k, nbr, order, cell_size, scratch, kNoAllocScratchBytes, stream);
}
