/*
 * mvgd.h -- C ABI of the GB300 (sm_103a) implementation of the Modified
 * Virtual Grid Difference (MVGD) discretisation of the Laplace-Beltrami
 * operator on point clouds (Wang, Leung & Zhao, arXiv:1603.04100), and of the
 * solve of (sigma I - L) u = f that the discretisation feeds.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, unless a
 *     comment says "host".  The library never allocates, frees or keeps
 *     caller memory; scratch comes from a caller buffer whose size the
 *     matching *_workspace_bytes() returns.  Device pointers must be 256-byte
 *     aligned (every PyTorch allocation is); otherwise MVGD_EINVAL.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default
 *     stream) and the call returns without waiting, except where a comment
 *     says it synchronises.
 *   - Errors are returned as mvgd_status; nothing aborts, traps or throws.
 *     Argument errors are detected on the host before anything is enqueued.
 *   - Points are FP64 [n][3] row-major.  Indices are int32 (n < 2^31).
 *   - 5 <= k <= 31 neighbours (the quadratic fit has 6 unknowns and uses the
 *     point itself plus its k neighbours), and k < n.
 */
#ifndef MVGD_H
#define MVGD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mvgd_stream_t; /* identical to cudaStream_t */

typedef enum {
    MVGD_OK = 0,
    MVGD_EINVAL = 1,      /* bad size, null or misaligned pointer, k out of range */
    MVGD_EWORKSPACE = 2,  /* workspace smaller than *_workspace_bytes() */
    MVGD_EDEGENERATE = 3, /* at least one row has a rank-deficient fit (row_status) */
    MVGD_ENOCONV = 4,     /* solver reached maxit above the tolerance */
    MVGD_EBREAKDOWN = 5,  /* Krylov breakdown that restarts did not cure */
    MVGD_ENONFINITE = 6,  /* non-finite input or intermediate value */
    MVGD_ECANCELLED = 7,  /* a host-set cancel word stopped the device loop */
    MVGD_ETIMEOUT = 8,    /* a bounded device-side wait gave up */
    MVGD_ECUDA = 9        /* a CUDA runtime call failed */
} mvgd_status;

/* Human-readable name of a status (static storage). */
const char *mvgd_status_string(mvgd_status s);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t mvgd_version(void);

/* ------------------------------------------------------------------------
 * kNN -- Sec. 2: N(i) = the k nearest neighbours of p_i in R^3.
 *
 * nbr[i][0..k-1] (out, int32 [n][k]) are the k indices j != i with the
 * smallest key (d2_ij, j), ascending, where
 *     d2_ij = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)),  dx = fl(x_j - x_i), ...
 * in IEEE FP64 round-to-nearest without contraction; equal keys are broken by
 * the lower index.  The result is exact: identical to a brute-force search.
 *
 * order (optional out, int32 [n]) receives a locality order of the points
 * (the cell order of the search grid); pass it to mvgd_assemble so that the
 * solver works on rows whose neighbours are close in memory.
 *
 * cell_size > 0 fixes the edge of the search grid's cells; 0 picks one from
 * an estimate of the k-th neighbour distance, and a negative value picks
 * -cell_size times that estimate (what a tuner varies).  Results never depend
 * on it, only the speed does.
 * ------------------------------------------------------------------------ */
size_t mvgd_knn_workspace_bytes(int64_t n, int32_t k);
mvgd_status mvgd_knn(const double *pts, int64_t n, int32_t k, int32_t *nbr, int32_t *order,
                     double cell_size, void *workspace, size_t workspace_bytes,
                     mvgd_stream_t stream);

/* The same kNN for callers that cannot allocate device memory -- code being
 * recorded into a CUDA graph, where a cudaMalloc would break the capture;
 * loops that must never wait on the allocator; host frameworks that own every
 * device buffer and pass only inputs and outputs.  (The paper has no
 * counterpart: this is an interface variant, not part of the method.)
 * The call allocates nothing: its scratch is one static device array of the
 * library, sized for MVGD_KNN_NOALLOC_MAX_POINTS points and held by every GPU
 * that loads the library until the process exits.  n above that maximum
 * returns MVGD_EINVAL before touching the device.  The first call on a device
 * looks up the array's device address (set-up, once per device), so make it
 * before any stream capture.  All calls on a device share the array: calls
 * whose work may overlap on the GPU (unordered streams) race on it and must be
 * serialised by the caller.  Results are identical to mvgd_knn.  The looked-up
 * address is cached per device for the life of the process; after
 * cudaDeviceReset the cache is stale, so do not call this entry point again in
 * a process that has reset a device it used. */
#define MVGD_KNN_NOALLOC_MAX_POINTS 65536
mvgd_status mvgd_knn_noalloc(const double *pts, int64_t n, int32_t k, int32_t *nbr, int32_t *order,
                             double cell_size, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Assembly -- Sec. 2 and Sec. 3.1.  Row i of L approximates the LB operator at
 * p_i as a combination of U_i and the values at its k neighbours:
 *   PCA frame of N(i) (z axis = smallest eigenvalue), local coordinates
 *   centred at p_i, least-squares quadratics z(x,y) and U(x,y) over p_i and
 *   N(i) (Eq. 2, Eq. 4), metric coefficients A_1..A_5 of Eq. 3 at the origin,
 *   centred differences of U(x,y) on the 3x3 virtual grid of spacing h with
 *   the centre node replaced by U_i (Eq. 7 and the 2-D rule of Sec. 3.1).
 *
 * Grid spacing h (Sec. 3.1):
 *   MVGD_DELTA_QUARTER_RANGE: h = min(range of x_j, range of y_j) / 4 over N(i)
 *   MVGD_DELTA_MEAN_NN:       h = mean |p_j - p_i| over the m nearest (1 <= m <= k)
 *   both multiplied by `scale` (> 0).
 * ------------------------------------------------------------------------ */
typedef enum { MVGD_DELTA_QUARTER_RANGE = 0, MVGD_DELTA_MEAN_NN = 1 } mvgd_delta_kind;

typedef struct {
    int32_t kind;     /* mvgd_delta_kind */
    int32_t m;        /* MEAN_NN only */
    double scale;     /* 1.0 = the paper's rule */
    int32_t variant;  /* mvgd_row_variant; 0 (zero-initialised) = MVGD */
    int32_t arith;    /* 0: the arithmetic of the storage format (below); 1: FP64
                         arithmetic for MVGD_FP32_REFINE too */
} mvgd_delta_rule;

/* Which row the assembly forms.  MVGD_ROW_MVGD is the method (Sec. 3.1).
 * MVGD_ROW_LS is the comparator of Sec. 2: the LB of the local least-squares
 * quadratic itself, w = A1 U_x + A2 U_y + A3 U_xx + A4 U_xy + A5 U_yy from the
 * fit's derivatives at the origin, without the centre value substituted on the
 * virtual grid.  Both rows sum to zero; they differ by
 * 2 (A3 + A5) / h^2 (P_00 - e_self). */
typedef enum { MVGD_ROW_MVGD = 0, MVGD_ROW_LS = 1 } mvgd_row_variant;

typedef enum {
    MVGD_FP64 = 0,        /* weights FP64; plain FP64 SpMV and Krylov */
    MVGD_FP32_REFINE = 1  /* weights as FP32 hi + FP32 lo (hi + lo = the FP64 weight to
                             ~2^-48 relative); FP32 inner Krylov on hi, FP64 residual on hi+lo */
} mvgd_precision;

/* Arithmetic of the assembly.  MVGD_FP64 rows are formed in FP64 (the local
 * fit by Householder QR).  MVGD_FP32_REFINE rows are formed on the FP32 pipe
 * unless rule.arith == 1: offsets p_j - p_i in FP64, then covariance and
 * h-scaled local coordinates in double-float (pairs of FP32 numbers, about 48
 * bits), the 3x3 eigenvectors
 * from an FP32 Jacobi polished by FP64 Jacobi sweeps, and the least-squares
 * fits through normal equations solved with an FP32 Cholesky factor and
 * refined from double-float residuals (for k >= 8: a fit over fewer points is
 * square or nearly so and always uses FP64); the hi + lo weights then agree with the
 * FP64 arithmetic's to about cond(V)^2 2^-48 (cond(V) of the h-scaled design
 * matrix, typically below 100).  A row whose factor is nearly singular or whose
 * refinement does not settle is formed in FP64 instead, so row_status and the
 * rank test are those of the FP64 arithmetic. */

/* Sparse operator in sliced ELL form, slice height 32.  Row r (0 <= r < n)
 * of the stored matrix is point order[r] (order == NULL: point r).  Element
 * (r, s) of a [.][w] array lives at  (r / 32) * (32 * w) + s * 32 + (r % 32),
 * and arrays are sized for n_pad = 32 * ceil(n / 32) rows.
 *   col  int32 [n_pad][k]:   stored-row index of neighbour s of row r
 *   val  [n_pad][k+1]:       slot 0 = self weight, slot s+1 = weight of col[s];
 *                            double (MVGD_FP64) or float hi (MVGD_FP32_REFINE)
 *   val_lo float [n_pad][k+1] (MVGD_FP32_REFINE only), hi + lo = the weight
 * Padding rows hold zero weights and point to row 0.  All five pointers
 * are caller-owned device memory; sizes from mvgd_ell_bytes(). */
typedef struct {
    int64_t n;
    int32_t k;
    int32_t prec;          /* mvgd_precision */
    const int32_t *order;  /* [n] or NULL; read by mvgd_assemble and mvgd_solve */
    int32_t *col;
    void *val;
    float *val_lo;
} mvgd_ell;

enum { MVGD_ELL_COL = 0, MVGD_ELL_VAL = 1, MVGD_ELL_VAL_LO = 2 };
size_t mvgd_ell_bytes(int64_t n, int32_t k, int32_t prec, int32_t which);

/* Fills L->col, L->val (and L->val_lo).  h (optional out, double [n], point
 * order) receives the grid spacing; row_status (optional out, uint8 [n],
 * point order) 0 = ok, 1 = rank-deficient fit (|R_kk| < 1e-10 |R_00| in
 * h-scaled coordinates), 2 = non-finite value; bad_rows (optional out, one
 * device int32, zeroed by this call) counts the rows with status != 0.
 * Asynchronous: check row_status / bad_rows after the stream has run.
 * The workspace (size from mvgd_assemble_workspace_bytes) is needed when
 * L->order is set (the inverse order that maps neighbour indices to stored
 * rows) or when the rows are formed on the FP32 pipe (the list of rows
 * handed to the FP64 arithmetic). */
size_t mvgd_assemble_workspace_bytes(int64_t n);
mvgd_status mvgd_assemble(const double *pts, int64_t n, int32_t k, const int32_t *nbr,
                          mvgd_delta_rule rule, mvgd_ell *L, double *h, uint8_t *row_status,
                          int32_t *bad_rows, void *workspace, size_t workspace_bytes,
                          mvgd_stream_t stream);

/* Batched assembly: many clouds (uneven sizes, any k and precision each) in
 * ONE launch whose work items are (cloud, 32-row slice) pairs.  Each item's
 * arrays follow the rules of mvgd_assemble; bad_rows (optional device int32)
 * counts rows with status != 0 over the whole batch.  The workspace holds the
 * descriptor table and the inverse orders (size from
 * mvgd_assemble_batch_workspace_bytes with the items' point counts). */
typedef struct {
    const double *pts;     /* [n][3] */
    const int32_t *nbr;    /* [n][k] from mvgd_knn */
    mvgd_ell L;            /* n, k, prec, order and the output arrays */
    double *h;             /* optional [n] */
    uint8_t *row_status;   /* optional [n] */
} mvgd_assemble_item;
size_t mvgd_assemble_batch_workspace_bytes(const int64_t *n, int32_t count);
mvgd_status mvgd_assemble_batch(const mvgd_assemble_item *items, int32_t count, mvgd_delta_rule rule,
                                int32_t *bad_rows, void *workspace, size_t workspace_bytes,
                                mvgd_stream_t stream);

/* Sign pattern of an assembled operator's rows (Sec. 3.2 and Sec. 4.1).  The
 * rows sum to zero, so a row whose K neighbour weights are all >= 0 makes
 * sigma I - L diagonally dominant with non-positive off-diagonal entries: the
 * M-matrix pattern the paper's MVGD is built to favour over the plain
 * least-squares row.  counts: DEVICE int64 [3] (8-byte aligned), overwritten:
 *   [0] rows whose neighbour weights are all >= 0,
 *   [1] neighbour weights < 0, over all rows,
 *   [2] rows whose self weight w_0 is >= 0 (a Laplacian row has w_0 < 0).
 * Weights are FP64, or hi + lo evaluated in FP64.  Padding rows are not counted.
 * Asynchronous; MVGD_EINVAL on a null pointer or out-of-range sizes. */
mvgd_status mvgd_row_signs(const mvgd_ell *L, int64_t *counts, mvgd_stream_t stream);

/* Dirichlet boundary rows for point clouds of open surfaces (Sec. 3.1): the
 * condition U = g is enforced at the boundary points and the MVGD row kept at
 * every interior point, whose neighbours may include boundary points.  Zeroes
 * every weight (self included) of the rows of the points flagged in boundary,
 * so that row of sigma I - L becomes sigma e_r; the caller puts sigma g_i
 * into f at those points.
 *   boundary: DEVICE uint8 [n] in point order (nonzero = boundary point);
 *             stored row r is point L->order[r] (or r without an order).
 *   count:    optional DEVICE int32, overwritten with the number of rows zeroed
 *             (4-byte aligned).
 * Call after mvgd_assemble and before mvgd_amg_setup / mvgd_solve.
 * Asynchronous; MVGD_EINVAL on a null operator or mask, or out-of-range sizes. */
mvgd_status mvgd_dirichlet_rows(mvgd_ell *L, const uint8_t *boundary, int32_t *count, mvgd_stream_t stream);

/* Neumann boundary by reflection (Sec. 3.1), homogeneous condition dU/dn = 0.
 * The unknowns are the interior points.  An interior point whose K nearest
 * neighbours include a boundary point is mirrored through the boundary at its
 * closest boundary point p_b (key: squared distance, then index), in the frame
 *   e2 = surface normal at p_b (smallest eigenvector of the covariance of p_b's
 *        K neighbours), e1 = boundary tangent at p_b (quadratic fit of the curve
 *        through p_b and its kb nearest boundary points, along their principal
 *        axis), made orthogonal to e2, e3 = e1 x e2;
 * the ghost is p - 2 ((p - p_b).e3) e3.  Three calls make the operator:
 *   1. mvgd_neumann_ghosts writes the cloud Q = interior points (point order)
 *      followed by the ghosts (in the order of the points they mirror);
 *   2. mvgd_knn and mvgd_assemble run on Q (any stored order);
 *   3. mvgd_neumann_fold keeps the interior rows of Q's operator, in its stored
 *      order, and maps every column to the interior point it stands for; a
 *      column may then repeat, or equal its own row (a point next to its ghost).
 * The folded operator's rows sum to zero as before, so every product, solve,
 * multigrid set-up and eigensolver call takes it as it is.
 *
 * mvgd_neumann_ghosts:
 *   pts [n][3], nbr [n][k] (mvgd_knn of the whole cloud), boundary uint8 [n]:
 *            DEVICE, point order
 *   kb       boundary neighbours of the tangent fit, 2 <= kb <= 16 (fewer when
 *            the boundary has fewer points)
 *   q        DEVICE double [2 n][3] out: Q, n_interior + n_ghost rows written
 *   q_src    DEVICE int32 [2 n] out: the interior position each point of Q
 *            stands for (itself for the interior points)
 *   interior DEVICE int32 [n] out: point index of each interior position
 *   ghost_bnd, ghost_dist  DEVICE int32 / double [n] out: per ghost, the
 *            boundary point used and |p - ghost| (for an inhomogeneous
 *            condition U(ghost) = U(p) + |p - ghost| g(p_b))
 *   counts   DEVICE int32 [4] out: n_interior, n_ghost, n_boundary, and the
 *            boundary points whose frame failed (fewer than 3 boundary points,
 *            a singular tangent fit, e1 parallel to e2; their e3 is zero, so
 *            their ghosts coincide with their points)
 * Workspace mvgd_neumann_ghosts_workspace_bytes(n).  Asynchronous.
 *
 * mvgd_neumann_fold:
 *   LQ       Q's operator (n = n_interior + n_ghost, optional order)
 *   q_src    as written by mvgd_neumann_ghosts
 *   LI       out: n = n_interior, the same k and prec as LQ, arrays from
 *            mvgd_ell_bytes(n_interior, ...); LI->order must point to DEVICE
 *            int32 [n_interior] that the call fills (stored row -> interior
 *            position).  Padding rows get zero weights and column 0.
 * Workspace mvgd_neumann_fold_workspace_bytes(LQ->n).  Asynchronous. */
size_t mvgd_neumann_ghosts_workspace_bytes(int64_t n);
mvgd_status mvgd_neumann_ghosts(const double *pts, int64_t n, int32_t k, const int32_t *nbr,
                                const uint8_t *boundary, int32_t kb, double *q, int32_t *q_src, int32_t *interior,
                                int32_t *ghost_bnd, double *ghost_dist, int32_t *counts, void *workspace,
                                size_t workspace_bytes, mvgd_stream_t stream);
size_t mvgd_neumann_fold_workspace_bytes(int64_t nq);
mvgd_status mvgd_neumann_fold(const mvgd_ell *LQ, const int32_t *q_src, mvgd_ell *LI, void *workspace,
                              size_t workspace_bytes, mvgd_stream_t stream);
/* mvgd_neumann_rhs: an inhomogeneous condition dU/dn = g (n the boundary's
 * outward normal in the tangent plane) sets U(ghost) = U(p) + |p - ghost| g(p_b)
 * (Sec. 3.1).  The known part moves to the right-hand side: the folded system
 * for (sigma I - L) u = f is (sigma I - L_folded) u = f + c with
 *   c[i] = sum over the ghost neighbours s of interior row i of w_s |p - ghost_s| g(p_b(s)),
 * read from Q's operator before the fold (a column whose Q point is >= n_interior
 * is a ghost).  ghost_dist, ghost_bnd as written by mvgd_neumann_ghosts; g
 * DEVICE double [n] in the ORIGINAL cloud's point order (read at the boundary
 * points); c DEVICE double [n_interior] out, interior positions.  Asynchronous. */
mvgd_status mvgd_neumann_rhs(const mvgd_ell *LQ, int64_t n_interior, const double *ghost_dist,
                             const int32_t *ghost_bnd, const double *g, double *c, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Sets of vectors, for the subspace iteration behind the lowest eigenpairs of
 * the LB operator (Sec. 4.3).  A set of p vectors of length n (FP64, DEVICE,
 * 256-byte aligned) is stored in blocks of w interleaved columns (1 <= w <= 8),
 * each block a right-hand-side array [n][w] of mvgd_solve / mvgd_spmv:
 *   element (r, c) at (c / w) * n * w + r * w + (c % w);  p, q multiples of w, <= 128.
 * mvgd_block_gram: G = X^T Y (p x q, row-major, DEVICE) summed in a fixed
 *   order (256 row ranges, each in row order, then the ranges in order), so the
 *   result does not depend on the GPU; ws sized by mvgd_block_gram_workspace_bytes.
 * mvgd_block_combine: Y = X C with C p x q row-major (DEVICE); X and Y distinct.
 * Both asynchronous; MVGD_EINVAL on bad shapes or pointers.
 * ------------------------------------------------------------------------ */
size_t mvgd_block_gram_workspace_bytes(int32_t p, int32_t q);
mvgd_status mvgd_block_gram(const double *X, int32_t p, const double *Y, int32_t q, int64_t n, int32_t w,
                            double *G, void *ws, size_t ws_bytes, mvgd_stream_t stream);
mvgd_status mvgd_block_combine(const double *X, int32_t p, const double *C, int32_t q, int64_t n, int32_t w,
                               double *Y, mvgd_stream_t stream);
/* Host-side p x p steps of the same eigensolver (HOST pointers, row-major,
 * synchronous, p <= 128; the paper's eigs does the same on the projected
 * matrices of its Arnoldi process):
 * mvgd_block_chol_inverse: Rinv = R^-1 for the upper-triangular Cholesky factor
 *   R^T R = (G + G^T) / 2 of a Gram matrix G (the orthonormalisation
 *   X = Y R^-1).  MVGD_EDEGENERATE if G is not positive definite.
 * mvgd_ritz_values: the p eigenvalues (re[i] + i im[i], complex pairs adjacent)
 *   of a general real matrix H -- the Ritz values of the projected operator
 *   X^T L X -- by Householder reduction to Hessenberg form and Francis
 *   double-shift QR (Golub and Van Loan, Algorithms 7.4.2, 7.5.1-7.5.2).
 *   MVGD_ENONFINITE for a non-finite entry, MVGD_ENOCONV if a block does not
 *   deflate within 60 p steps. */
mvgd_status mvgd_block_chol_inverse(const double *G, int32_t p, double *Rinv);
mvgd_status mvgd_ritz_values(const double *H, int32_t p, double *re, double *im);
/* mvgd_block_zero_rows: X(r, c) = 0 for all c at the rows r with mask[r] != 0
 * (DEVICE uint8 [n], the set's row order); keeps a subspace off Dirichlet rows. */
mvgd_status mvgd_block_zero_rows(double *X, int32_t p, int64_t n, int32_t w, const uint8_t *mask,
                                 mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Conditioning of the stored system (Sec. 4.1): the Gauss-Seidel iteration
 * matrix T = M^-1 N of A = sigma I - L, split A = M + N with M the lower
 * triangle including the diagonal and N the strictly upper triangle, both in
 * STORED row order (the order the operator's rows are kept in).  A Gauss-Seidel
 * sweep converges from every start iff the spectral radius of T is below 1.
 *
 * mvgd_gs_power runs `iters` steps of the power iteration
 *   x_0 = x0 / ||x0||_2,   y_t = T x_t,   nu[t] = ||y_t||_2,   x_{t+1} = y_t / nu[t]
 * in one cooperative launch.  nu[t] tends to |lambda_max(T)| when that
 * eigenvalue is real and simple; with a complex pair (or +-lambda) on top, nu
 * oscillates and the geometric mean of nu over a window converges instead.
 * Each T x is N x followed by the forward substitution M y = N x: warps take
 * rows in increasing order from a ticket counter, and a row waits (bounded) on
 * a flag of each lower neighbour written by the warp that computed it, so
 * there is no level schedule; every row's sums are over its own slots in slot
 * order, and the norms are reduced in a fixed order, so results repeat bit for
 * bit.  A neighbour column equal to the row itself adds to the diagonal.
 *   L       the operator (MVGD_FP64, or FP32_REFINE read as hi + lo in FP64)
 *   x0      DEVICE double [n], stored order, not all zero
 *   nu      DEVICE double [iters] out
 *   x       DEVICE double [n] out: x_iters (unit norm), stored order; may be x0
 *   status  DEVICE int32 [1] out: MVGD_OK, MVGD_ENONFINITE (zero or non-finite
 *           norm: a zero diagonal of A, or x0 = 0) or MVGD_ETIMEOUT (a bounded
 *           wait gave up)
 * Workspace: mvgd_gs_power_workspace_bytes(n, iters).  1 <= iters <= 2^20;
 * n < 2^31. */
size_t mvgd_gs_power_workspace_bytes(int64_t n, int32_t iters);
mvgd_status mvgd_gs_power(const mvgd_ell *L, double sigma, const double *x0, int32_t iters, double *nu, double *x,
                          int32_t *status, void *workspace, size_t workspace_bytes, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Operator application (the product every Krylov step repeats, Sec. 3.1 and
 * Sec. 4.2):  y = alpha * (sigma x - L x) + beta * y  for nrhs right-hand
 * sides stored interleaved, x and y [n][nrhs] in STORED row order.
 *   MVGD_SPMV_F64:      val double, x/y double
 *   MVGD_SPMV_F32:      val hi,     x/y float, rows evaluated in difference form
 *                       sum_s w_s (x_col - x_row), the self weight taken as
 *                       minus the sum of the others (rows of L sum to zero)
 *   MVGD_SPMV_F64_HILO: val hi + lo in FP64 arithmetic, x/y double
 * 1 <= nrhs <= 8.  When beta == 0, y is not read.
 * ------------------------------------------------------------------------ */
enum { MVGD_SPMV_F64 = 0, MVGD_SPMV_F32 = 1, MVGD_SPMV_F64_HILO = 2 };
mvgd_status mvgd_spmv(const mvgd_ell *L, int32_t mode, int32_t nrhs, double sigma, double alpha,
                      const void *x, double beta, void *y, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Solve (sigma I - L) u = f (Sec. 4.2; the paper uses AMG, this library a
 * device-resident Krylov method) for nrhs right-hand sides, f and u FP64
 * [n][nrhs] in POINT order (the solver applies L->order itself).  u holds the
 * initial guess on entry.
 *   L->prec == MVGD_FP64:        BiCGSTAB in FP64 to ||f - A u|| <= rtol ||f||.
 *   L->prec == MVGD_FP32_REFINE: iterative refinement -- FP64 residual on hi+lo,
 *                                 inner FP32 BiCGSTAB on hi to inner_rtol, FP64
 *                                 update of u -- until the FP64 residual meets rtol.
 * All iterations run in one persistent device kernel; no host round trip.
 * info (out, [nrhs]): if it is host memory the call synchronises the stream
 * and returns the worst per-RHS status; if device memory, the call is
 * asynchronous and returns MVGD_OK after enqueueing.
 * cancel (optional, device or mapped host int32): when it becomes non-zero the
 * device loop stops at the next iteration with MVGD_ECANCELLED.
 * ------------------------------------------------------------------------ */
typedef struct {
    double rtol;         /* relative residual target, e.g. 1e-8 */
    int32_t maxit;       /* cap on Krylov iterations (inner ones included) */
    int32_t inner_maxit; /* FP32_REFINE: cap per inner solve */
    double inner_rtol;   /* FP32_REFINE: inner relative tolerance, e.g. 1e-3 (with the multigrid
                            preconditioner fewer Krylov iterations in all than 1e-4 or 1e-5) */
    int32_t max_outer;   /* FP32_REFINE: cap on refinement steps */
    int32_t precond;     /* 0 = none; 1 = left scaling of each row of the Krylov system by
                            1 / (|sigma| + sum_s |w_s|) (row equilibration: always positive,
                            unlike the Jacobi divisor sigma - w_self, which can vanish on rows
                            of irregular samples that are not diagonally dominant);
                            2 = right preconditioning by one aggregation-multigrid V-cycle
                            (see mvgd_amg_setup) */
    const void *amg;     /* precond == 2: the hierarchy from mvgd_amg_setup for this operator
                            and sigma (DEVICE).  mvgd_solve builds one in its own workspace
                            when this is NULL; mvgd_request_init requires it. */
} mvgd_solve_opts;

typedef struct {
    int32_t iters;       /* Krylov iterations (all inner ones) */
    int32_t outer;       /* refinement steps (FP32_REFINE), restarts (FP64) */
    double relres;       /* final ||f - A u||_2 / ||f||_2 in FP64 */
    int32_t status;      /* mvgd_status */
    int32_t reserved;
} mvgd_solve_info;

/* Workspace of mvgd_solve.  With precond == 2 it includes room for the
 * hierarchy; a call given opts->amg needs that much less
 * (mvgd_amg_workspace_bytes(n, k) rounded up to 256). */
size_t mvgd_solve_workspace_bytes(int64_t n, int32_t k, int32_t nrhs, int32_t prec, int32_t precond);
mvgd_status mvgd_solve(const mvgd_ell *L, int32_t nrhs, double sigma, const double *f, double *u,
                       const mvgd_solve_opts *opts, mvgd_solve_info *info, const int32_t *cancel,
                       void *workspace, size_t workspace_bytes, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Aggregation multigrid.  The paper solves its systems with algebraic
 * multigrid (Sec. 4.2, whose timing table grows about linearly in N)
 * without naming a variant.  Here: plain aggregation on the stored row order
 * (consecutive rows are spatial neighbours after the kNN step's cell sort).
 *   - aggregate I of a level = its MVGD_AMG_AGG consecutive rows I*AGG ..;
 *   - next level = Galerkin product P^T A P, P piecewise constant (FP64 sums,
 *     kept as FP32 for the cycle);
 *   - the first level with <= MVGD_AMG_COARSEST rows is inverted
 *     (Gauss-Jordan with partial pivoting in FP32, then two Newton-Schulz
 *     steps in FP64) and solved by an FP64 product with that inverse;
 *   - one V(1,1)-cycle in FP32 with Jacobi smoothing x += d (b - A x):
 *     d_i = MVGD_AMG_JACOBI_OMEGA / a_ii on rows with a strong diagonal
 *     (a_ii > MVGD_AMG_JACOBI_THETA sum_j |a_ij|), the l1 scaling
 *     d_i = 1 / sum_j |a_ij| on the others (MVGD rows with few neighbours on
 *     irregular samples can have a small or negative diagonal).
 * mvgd_amg_workspace_bytes: bytes of the hierarchy of an n-row operator with
 *   K neighbours (0 if n or K is out of range).
 * mvgd_amg_setup: builds the hierarchy of sigma I - L in amg_ws (DEVICE,
 *   caller-owned, 256-byte aligned).  L must outlive it.  Asynchronous; what
 *   only the device can find -- a coarse row wider than MVGD_AMG_MAX_WIDTH
 *   (a row order that is not spatially coherent) or a singular coarsest
 *   level -- is reported as MVGD_EDEGENERATE by mvgd_amg_describe.
 * mvgd_amg_describe (synchronous): one level's size and DEVICE arrays, for
 *   inspection.  Levels >= 1 are sliced like the operator (element (r, s) of
 *   a width-w array at (r/32)*32*w + 32*s + r%32) with w = stride.
 * mvgd_amg_apply: x = one V-cycle applied to b (FP64 [n][nrhs], DEVICE,
 *   stored order); ws sized by mvgd_amg_apply_workspace_bytes.  Asynchronous.
 * ------------------------------------------------------------------------ */
#define MVGD_AMG_AGG 8
#define MVGD_AMG_COARSEST 512
#define MVGD_AMG_MAX_WIDTH 64
#define MVGD_AMG_JACOBI_OMEGA 0.9
#define MVGD_AMG_JACOBI_THETA 0.3

typedef struct {
    int64_t n;             /* rows of this level */
    int32_t levels;        /* levels in the hierarchy, the coarsest included */
    int32_t stride;        /* slots per row: K + 1 at level 0, MVGD_AMG_MAX_WIDTH above */
    int32_t status;        /* MVGD_OK or MVGD_EDEGENERATE (whole hierarchy) */
    int32_t width_max;     /* widest coarse row found (whole hierarchy) */
    const int32_t *col;    /* level 0: the operator's col; above: [n_pad][stride] columns */
    const float *val;      /* FP32 values (level 0: the operator's weights, slot 0 = self) */
    const double *val64;   /* levels >= 1: FP64 Galerkin sums */
    const int32_t *cnt;    /* levels >= 1: entries of each row (sorted by column) */
    const float *dinv;     /* [n] the smoother's scaling d_i (FP64 choice, rounded once) */
    const float *cinv;     /* coarsest level only: [n][n] FP32 Gauss-Jordan inverse, column-major (element (r, c) at c*n + r) */
    const double *cinv64;  /* coarsest level only: [n][n] refined FP64 inverse, row-major (used by the cycle) */
} mvgd_amg_info;

size_t mvgd_amg_workspace_bytes(int64_t n, int32_t k);
mvgd_status mvgd_amg_setup(const mvgd_ell *L, double sigma, void *amg_ws, size_t amg_bytes, mvgd_stream_t stream);
mvgd_status mvgd_amg_describe(const void *amg_ws, int32_t level, mvgd_amg_info *out);
size_t mvgd_amg_apply_workspace_bytes(int64_t n, int32_t nrhs);
mvgd_status mvgd_amg_apply(const void *amg_ws, int64_t n, int32_t nrhs, const double *b, double *x, void *ws,
                           size_t ws_bytes, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Requests: the same solve (Sec. 4.2) split so that many systems advance in
 * one persistent launch (uneven clouds batched together, and requests that
 * join or leave between launches).  A request's whole solver state -- Krylov
 * vectors, per-RHS scalars, reduction partials -- lives in its own
 * caller-owned workspace; the operator L it was initialised with must stay
 * alive until mvgd_request_finish.  Results of a request do not depend on
 * which other requests share a launch: every reduction runs per request in a
 * fixed order over fixed 256-row chunks.
 *
 * mvgd_request_init: gathers f (and u0, or zeros if u0 == NULL) into stored
 *   order and sets every right-hand side to its first restart.  Asynchronous.
 * mvgd_iterate: advances the listed requests (host array of descriptors;
 *   all of one precision and one preconditioner kind, the `precond` each was
 *   initialised with) by at
 *   most max_iterations Krylov iterations in one cooperative launch; requests
 *   whose right-hand sides are all done cost nothing.  ctl_ws (size from
 *   mvgd_iterate_workspace_bytes for at least this many requests and rows)
 *   holds the launch's tables and barrier.  Asynchronous; a set cancel word
 *   stops the launch after the current iteration.
 * mvgd_request_finish: writes u (FP64 [n][nrhs], point order) and info
 *   (DEVICE [nrhs]); a right-hand side not yet done reports MVGD_ENOCONV,
 *   or MVGD_ECANCELLED / MVGD_ETIMEOUT if a launch was cut short.
 * ------------------------------------------------------------------------ */
size_t mvgd_request_workspace_bytes(int64_t n, int32_t k, int32_t nrhs, int32_t prec, int32_t precond);
mvgd_status mvgd_request_init(void *req_workspace, size_t req_bytes, const mvgd_ell *L, int32_t nrhs,
                              double sigma, const double *f, const double *u0, const mvgd_solve_opts *opts,
                              mvgd_stream_t stream);
size_t mvgd_iterate_workspace_bytes(int32_t max_requests, int64_t max_total_rows);
typedef struct {
    void *workspace;  /* the request's workspace, as given to mvgd_request_init */
    int64_t n;        /* rows of its operator */
    int32_t nrhs;     /* its right-hand sides */
    int32_t k;        /* K of its operator (sizes the launch's shared-memory staging) */
} mvgd_request;
mvgd_status mvgd_iterate(const mvgd_request *reqs, int32_t count, int32_t prec, int32_t precond,
                         int32_t max_iterations, const int32_t *cancel, void *ctl_workspace, size_t ctl_bytes,
                         mvgd_stream_t stream);
mvgd_status mvgd_request_finish(void *req_workspace, int64_t n, int32_t nrhs, double *u,
                                mvgd_solve_info *info, mvgd_stream_t stream);
/* done (out, DEVICE int32 [count]): 1 where every right-hand side of the
 * request has finished (converged or stopped with a status), else 0.  A cheap
 * check between mvgd_iterate launches.  Asynchronous. */
mvgd_status mvgd_request_poll(void *const *reqs, int32_t count, int32_t *done, mvgd_stream_t stream);

/* ------------------------------------------------------------------------
 * Step trace (diagnostics; no counterpart in the paper).  When enabled, the
 * persistent solver stamps the device clock (ns) after every grid-wide step:
 * entry = code << 48 | (time & 2^48-1), code = Krylov phase 0..4 (PRE_A, A,
 * PRE_B, B, C; the multigrid flow has no C step: its B ends an iteration and
 * the next PRE_A forms the new residual), or
 * 0x1000 | side << 8 | kind << 4 | level for a multigrid step
 * (side 0: the cycle on p, 1: on s; kind 0 down, 1 coarsest, 2 up).  Process-
 * wide, one device; entries past 65,536 wrap.  Both calls synchronise.
 * mvgd_trace_enable: on != 0 clears the trace and turns it on for launches
 *   made from now on; 0 turns it off.
 * mvgd_trace_read: copies up to max entries to host memory; returns the count
 *   (-1 on error).
 * ------------------------------------------------------------------------ */
mvgd_status mvgd_trace_enable(int32_t on);
int32_t mvgd_trace_read(uint64_t *out, int32_t max);

/* ------------------------------------------------------------------------
 * Bounded device-side waits (liveness; the paper has no counterpart).  The
 * persistent kernels wait on one another: the grid barriers of the solver
 * (mvgd_solve, mvgd_iterate) and of mvgd_gs_power, and the row flags of
 * mvgd_gs_power's forward substitution.  Every such wait polls at most a
 * limited number of times; a wait that runs out sets MVGD_ETIMEOUT, every
 * other block of the launch then stops at its next wait, the launch ends, and
 * the status reaches the caller through mvgd_solve_info / the status word.
 * The context stays usable and the next call on the same workspace runs
 * normally (each launch resets its barrier and flags).
 * mvgd_set_wait_limit: polls a wait may take before it gives up, for launches
 *   made from now on, process-wide (a poll is one L2 round trip, about
 *   0.5-1 us).  0 restores each kernel's default (seconds: never reached by
 *   co-resident blocks that make progress).  MVGD_EINVAL if polls < 0.
 * mvgd_test_withhold_arrival: a test control for those paths.  on != 0 arms
 *   it for exactly one launch: in the next solver launch block 0 leaves its
 *   arrival at the first grid barrier out, and in the next mvgd_gs_power
 *   launch row 0's flag of the first step is never published.  Nothing else
 *   ends those waits, so they run out at the limit and the launch returns
 *   MVGD_ETIMEOUT; no memory is touched that a normal launch would not touch.
 *   on == 0 disarms it.  Host-side only; returns MVGD_OK.
 * ------------------------------------------------------------------------ */
mvgd_status mvgd_set_wait_limit(int64_t polls);
mvgd_status mvgd_test_withhold_arrival(int32_t on);

/* ------------------------------------------------------------------------
 * Launch shapes (for a tuner; the paper has no counterpart).  Process-wide,
 * for launches made from now on; they change the speed of a call, never its
 * results (the solver's reductions run over fixed chunks whatever the grid,
 * and every assembled row is one lane's work whatever the block).
 *   solver_blocks_per_sm: resident blocks per SM of the persistent solver
 *     (0: as many as fit, the default; otherwise at most that many);
 *   stage_buffers: operator slices a solver warp keeps in flight, 1 (default)
 *     or 2 (used only when the shared memory allows it; 0 = 1);
 *   assemble_warps: warps per block of the FP32 assembly path, 1 (default),
 *     2, 4 or 8 (fewer when the shared memory would not fit; 0 = 1); the FP64
 *     arithmetic always takes one.
 * MVGD_EINVAL for a value out of range.  Host-side only. */
mvgd_status mvgd_set_launch_tuning(int32_t solver_blocks_per_sm, int32_t stage_buffers, int32_t assemble_warps);

#ifdef __cplusplus
}
#endif
#endif /* MVGD_H */
