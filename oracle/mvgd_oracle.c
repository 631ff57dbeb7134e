/*
 * mvgd_oracle.c -- plain, slow, FP64 CPU restatement of the Modified Virtual
 * Grid Difference (MVGD) discretisation of the Laplace-Beltrami operator on
 * point clouds (Wang, Leung & Zhao, arXiv:1603.04100).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction,
 * so every expression rounds in the order written).  OpenMP only splits the
 * independent per-point loops and the vector loops of the solvers.
 *
 * Every function names the passage of the paper it follows.  Readings taken
 * where the paper is silent:
 *   - N(i) excludes p_i; PCA uses the K neighbours (Sec. 2, barycenter over K);
 *     the quadratic fits use p_i together with its K neighbours (the normal
 *     matrix of Sec. 2 has K+1 in its corner).
 *   - local coordinates are centred at p_i (Sec. 2); the LB expansion is
 *     evaluated at the local origin.
 *   - A_1..A_5 (Eq. 3, not printed) follow from Eq. 1 for a graph surface:
 *     Delta U = g^{ab} U_ab - (g^{ab} z_ab / W) (grad z . grad U), W = 1+|grad z|^2.
 *   - the 2-D virtual grid is the 3x3 grid of spacing h in the local x,y plane;
 *     D_xy uses the four corner nodes.
 *   - the kNN key is fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)), ties by index.
 *   - least squares are unweighted (the explicit system of Sec. 2).
 * Parity of this file is pinned by the tests in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 64
#define OR_MAXM (OR_MAXK + 1)

int or_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* kNN (Sec. 2: "K nearest neighbors"), by brute force: the definition.      */
/* ------------------------------------------------------------------------ */

static double or_dist2(const double *a, const double *b)
{
    double dx = b[0] - a[0];
    double dy = b[1] - a[1];
    double dz = b[2] - a[2];
    double s = dx * dx + dy * dy;
    s = s + dz * dz;
    return s;
}

/* (d, j) < (e, k) lexicographically */
static int or_key_less(double d, int32_t j, double e, int32_t k)
{
    return d < e || (d == e && j < k);
}

/* insert (d, j) into the ascending list (kd, kj) of length *len <= k */
static void or_list_insert(double *kd, int32_t *kj, int *len, int k, double d, int32_t j)
{
    int pos = *len;
    if (pos == k) {
        if (!or_key_less(d, j, kd[k - 1], kj[k - 1])) return;
        pos = k - 1;
    } else {
        (*len)++;
    }
    while (pos > 0 && or_key_less(d, j, kd[pos - 1], kj[pos - 1])) {
        kd[pos] = kd[pos - 1];
        kj[pos] = kj[pos - 1];
        pos--;
    }
    kd[pos] = d;
    kj[pos] = j;
}

int or_knn_brute(const double *pts, int64_t n, int k, int32_t *nbr)
{
    if (k < 1 || k > OR_MAXK || k >= n) return 1;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double kd[OR_MAXK];
        int32_t kj[OR_MAXK];
        int len = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            or_list_insert(kd, kj, &len, k, or_dist2(pts + 3 * i, pts + 3 * j), (int32_t)j);
        }
        memcpy(nbr + i * k, kj, sizeof(int32_t) * k);
    }
    return 0;
}

/* Same result as or_knn_brute (tests check equality), found with a uniform
 * grid: rings of cells are searched until the K-th distance is inside the
 * searched block.  Used only to time the CPU baseline at large N. */
int or_knn_grid(const double *pts, int64_t n, int k, int32_t *nbr)
{
    if (k < 1 || k > OR_MAXK || k >= n) return 1;
    double lo[3] = {pts[0], pts[1], pts[2]}, hi[3] = {pts[0], pts[1], pts[2]};
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            if (pts[3 * i + a] < lo[a]) lo[a] = pts[3 * i + a];
            if (pts[3 * i + a] > hi[a]) hi[a] = pts[3 * i + a];
        }
    double ext = 0;
    for (int a = 0; a < 3; a++) ext = fmax(ext, hi[a] - lo[a]);
    if (ext <= 0) ext = 1;
    double cells_wanted = (double)n / 2.0 + 1.0;
    double s = ext / cbrt(cells_wanted);
    int64_t dim[3];
    for (int a = 0; a < 3; a++) {
        dim[a] = (int64_t)floor((hi[a] - lo[a]) / s) + 1;
        if (dim[a] < 1) dim[a] = 1;
    }
    int64_t ncell = dim[0] * dim[1] * dim[2];
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *cellof = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *sorted = malloc(sizeof(int64_t) * (size_t)n);
    int64_t *fill = calloc((size_t)ncell, sizeof(int64_t));
    if (!start || !cellof || !sorted || !fill) {
        free(start); free(cellof); free(sorted); free(fill);
        return 2;
    }
    for (int64_t i = 0; i < n; i++) {
        int64_t c[3];
        for (int a = 0; a < 3; a++) {
            c[a] = (int64_t)floor((pts[3 * i + a] - lo[a]) / s);
            if (c[a] >= dim[a]) c[a] = dim[a] - 1;
            if (c[a] < 0) c[a] = 0;
        }
        cellof[i] = (c[2] * dim[1] + c[1]) * dim[0] + c[0];
        start[cellof[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; i++) sorted[start[cellof[i]] + fill[cellof[i]]++] = i;
    free(fill);

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        double kd[OR_MAXK];
        int32_t kj[OR_MAXK];
        int64_t c[3];
        for (int a = 0; a < 3; a++) {
            c[a] = (int64_t)floor((pts[3 * i + a] - lo[a]) / s);
            if (c[a] >= dim[a]) c[a] = dim[a] - 1;
            if (c[a] < 0) c[a] = 0;
        }
        for (int64_t ring = 1;; ring++) {
            int len = 0, whole = 1;
            int64_t a0[3], a1[3];
            for (int a = 0; a < 3; a++) {
                a0[a] = c[a] - ring; a1[a] = c[a] + ring;
                if (a0[a] < 0) a0[a] = 0; else whole = 0;
                if (a1[a] > dim[a] - 1) a1[a] = dim[a] - 1; else whole = 0;
            }
            for (int64_t z = a0[2]; z <= a1[2]; z++)
                for (int64_t y = a0[1]; y <= a1[1]; y++)
                    for (int64_t x = a0[0]; x <= a1[0]; x++) {
                        int64_t cc = (z * dim[1] + y) * dim[0] + x;
                        for (int64_t t = start[cc]; t < start[cc + 1]; t++) {
                            int64_t j = sorted[t];
                            if (j == i) continue;
                            or_list_insert(kd, kj, &len, k, or_dist2(pts + 3 * i, pts + 3 * j),
                                           (int32_t)j);
                        }
                    }
            /* every point outside the block is farther than ring*s - rounding */
            double guard = (double)ring * s * (1.0 - 1e-9);
            if (whole || (len == k && kd[k - 1] < guard * guard)) {
                memcpy(nbr + i * k, kj, sizeof(int32_t) * k);
                break;
            }
        }
    }
    free(start); free(cellof); free(sorted);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Local PCA frame (Sec. 2): cyclic Jacobi for the 3x3 covariance.           */
/* ------------------------------------------------------------------------ */

/* Eigen-decomposition of symmetric a (3x3, row-major, overwritten).
 * On return v columns are eigenvectors, w eigenvalues (unsorted). */
static void or_jacobi3(double a[3][3], double v[3][3], double w[3])
{
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) v[r][c] = (r == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 64; sweep++) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-40 * dia || off == 0.0) break;
        for (int p = 0; p < 2; p++)
            for (int q = p + 1; q < 3; q++) {
                if (a[p][q] == 0.0) continue;
                /* Golub & Van Loan, symmetric Schur 2x2 */
                double tau = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double cs = 1.0 / sqrt(1.0 + t * t);
                double sn = t * cs;
                /* a <- J^T a J with J = rotation in the (p, q) plane */
                for (int k = 0; k < 3; k++) {
                    double akp = a[k][p], akq = a[k][q];
                    a[k][p] = cs * akp - sn * akq;
                    a[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; k++) {
                    double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = cs * apk - sn * aqk;
                    a[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 3; k++) {
                    double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = cs * vkp - sn * vkq;
                    v[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    for (int k = 0; k < 3; k++) w[k] = a[k][k];
}

/* ------------------------------------------------------------------------ */
/* Householder QR least squares (textbook; Golub & Van Loan Alg. 5.2.1).     */
/* a: m x 6 row-major (overwritten by R in its upper rows), rhs: m x nr      */
/* row-major, overwritten by Q^T rhs.  Returns min |R_kk| / |R_00|.           */
/* ------------------------------------------------------------------------ */
static double or_house_qr(double *a, int m, double *rhs, int nr)
{
    const int nc = 6;
    for (int k = 0; k < nc; k++) {
        double nrm = 0;
        for (int r = k; r < m; r++) nrm += a[r * nc + k] * a[r * nc + k];
        nrm = sqrt(nrm);
        if (nrm == 0.0) continue;
        double alpha = (a[k * nc + k] > 0) ? -nrm : nrm;
        double v[OR_MAXM];
        for (int r = 0; r < m; r++) v[r] = 0;
        v[k] = a[k * nc + k] - alpha;
        for (int r = k + 1; r < m; r++) v[r] = a[r * nc + k];
        double vtv = 0;
        for (int r = k; r < m; r++) vtv += v[r] * v[r];
        if (vtv == 0.0) continue;
        double beta = 2.0 / vtv;
        for (int c = k; c < nc; c++) {
            double s = 0;
            for (int r = k; r < m; r++) s += v[r] * a[r * nc + c];
            s *= beta;
            for (int r = k; r < m; r++) a[r * nc + c] -= s * v[r];
        }
        for (int c = 0; c < nr; c++) {
            double s = 0;
            for (int r = k; r < m; r++) s += v[r] * rhs[r * nr + c];
            s *= beta;
            for (int r = k; r < m; r++) rhs[r * nr + c] -= s * v[r];
        }
    }
    double r00 = fabs(a[0]), rmin = INFINITY;
    for (int k = 0; k < nc; k++) rmin = fmin(rmin, fabs(a[k * nc + k]));
    return (r00 > 0) ? rmin / r00 : 0.0;
}

/* back substitution R x = y for the 6x6 upper triangle of a (row stride 6),
 * nr right-hand sides stored row-major in y (first 6 rows), result in x */
static void or_back_subst(const double *a, const double *y, int nr, double *x)
{
    for (int c = 0; c < nr; c++)
        for (int k = 5; k >= 0; k--) {
            double s = y[k * nr + c];
            for (int l = k + 1; l < 6; l++) s -= a[k * 6 + l] * x[l * nr + c];
            x[k * nr + c] = s / a[k * 6 + k];
        }
}

/* monomials of Eq. 2 / Eq. 4 in the order of the unknown vector b of Sec. 2:
 * (1, x, y, x^2, x y, y^2) */
static void or_monomials(double x, double y, double *v)
{
    v[0] = 1.0; v[1] = x; v[2] = y; v[3] = x * x; v[4] = x * y; v[5] = y * y;
}

/* The normal-equation matrix A of Sec. 2 for points (x_j, y_j), j = 0..m-1,
 * entry by entry as printed (the [4][5] entry is sum x y^3 by symmetry with
 * [5][4]; the print shows x y^2). */
void or_normal_matrix(const double *x, const double *y, int m, double *A)
{
    double s[5][5];
    memset(s, 0, sizeof s);
    for (int j = 0; j < m; j++) {
        double px = 1;
        for (int a = 0; a <= 4; a++) {
            double py = 1;
            for (int b = 0; a + b <= 4; b++) {
                s[a][b] += px * py;
                py *= y[j];
            }
            px *= x[j];
        }
    }
    /* rows as printed; s[a][b] = sum x^a y^b */
    const int ex[6][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}};
    for (int r = 0; r < 6; r++)
        for (int c = 0; c < 6; c++)
            A[r * 6 + c] = s[ex[r][0] + ex[c][0]][ex[r][1] + ex[c][1]];
}

/* ------------------------------------------------------------------------ */
/* MVGD row at one point (Sec. 3.1 with Sec. 2).                              */
/* ------------------------------------------------------------------------ */

enum { OR_DELTA_QUARTER_RANGE = 0, OR_DELTA_MEAN_NN = 1 };
enum { OR_VARIANT_MVGD = 0, OR_VARIANT_LS = 1 };

typedef struct {
    double A[5];      /* A_1 .. A_5 of Eq. 3 */
    double h;         /* virtual grid spacing */
    double normal[3]; /* e_z */
    double gap;       /* (lambda_1 - lambda_2) / lambda_1 of the tangent pair */
    double rank;      /* min |R_kk| / |R_00| of the scaled design matrix */
} or_diag;

/* w: out [k+1] (slot 0 = p_i, slot s+1 = nbr[s]); p00: optional out [k+1],
 * the functional giving b_00 = U^{(i)}(0,0).  Returns status: 0 ok,
 * 1 rank-deficient fit, 2 non-finite value. */
static int or_row(const double *pts, int k, const int32_t *nb, const double *pi, int delta_kind,
                  int delta_m, double delta_scale, int variant, double *w, double *p00,
                  or_diag *dg)
{
    const int m = k + 1;
    double d[OR_MAXK][3];
    for (int s = 0; s < k; s++)
        for (int a = 0; a < 3; a++) d[s][a] = pts[3 * (int64_t)nb[s] + a] - pi[a];

    /* barycenter and covariance of N(i) (Sec. 2) */
    double c[3] = {0, 0, 0};
    for (int s = 0; s < k; s++)
        for (int a = 0; a < 3; a++) c[a] += d[s][a];
    for (int a = 0; a < 3; a++) c[a] /= k;
    double C[3][3] = {{0}};
    for (int s = 0; s < k; s++)
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) C[a][b] += (d[s][a] - c[a]) * (d[s][b] - c[b]);

    /* eigenvectors: z axis = smallest eigenvalue, x = largest, y = middle */
    double V[3][3], ev[3];
    or_jacobi3(C, V, ev);
    int imax = 0, imin = 0;
    for (int a = 1; a < 3; a++) {
        if (ev[a] > ev[imax]) imax = a;
        if (ev[a] < ev[imin]) imin = a;
    }
    if (imax == imin) imin = (imax + 1) % 3;
    int imid = 3 - imax - imin;
    double ex[3], ey[3], ez[3];
    for (int a = 0; a < 3; a++) { ex[a] = V[a][imax]; ey[a] = V[a][imid]; ez[a] = V[a][imin]; }

    /* local coordinates centred at p_i; p_i itself is the origin */
    double lx[OR_MAXM], ly[OR_MAXM], lz[OR_MAXM];
    lx[0] = ly[0] = lz[0] = 0.0;
    for (int s = 0; s < k; s++) {
        lx[s + 1] = d[s][0] * ex[0] + d[s][1] * ex[1] + d[s][2] * ex[2];
        ly[s + 1] = d[s][0] * ey[0] + d[s][1] * ey[1] + d[s][2] * ey[2];
        lz[s + 1] = d[s][0] * ez[0] + d[s][1] * ez[1] + d[s][2] * ez[2];
    }

    /* grid spacing h (Sec. 3.1) */
    double h;
    if (delta_kind == OR_DELTA_QUARTER_RANGE) {
        double x0 = lx[1], x1 = lx[1], y0 = ly[1], y1 = ly[1];
        for (int s = 2; s <= k; s++) {
            x0 = fmin(x0, lx[s]); x1 = fmax(x1, lx[s]);
            y0 = fmin(y0, ly[s]); y1 = fmax(y1, ly[s]);
        }
        h = fmin(0.25 * (x1 - x0), 0.25 * (y1 - y0));
    } else {
        double acc = 0;
        for (int s = 0; s < delta_m; s++)
            acc += sqrt(d[s][0] * d[s][0] + d[s][1] * d[s][1] + d[s][2] * d[s][2]);
        h = acc / delta_m;
    }
    h *= delta_scale;

    /* design matrix over p_i and N(i) in units of h: a change of monomial
     * basis that leaves the least-squares fit unchanged */
    double Vd[OR_MAXM * 6], Vz[OR_MAXM * 6];
    double rhs_z[OR_MAXM], rhs_u[OR_MAXM * OR_MAXM];
    for (int r = 0; r < m; r++) {
        or_monomials(lx[r] / h, ly[r] / h, Vd + 6 * r);
        rhs_z[r] = lz[r] / h;
        for (int q = 0; q < m; q++) rhs_u[r * m + q] = (r == q) ? 1.0 : 0.0;
    }
    memcpy(Vz, Vd, sizeof(double) * 6 * m);

    /* surface fit z^{(i)} (Eq. 2): coefficients a~ in units of h */
    double at[6];
    double rank = or_house_qr(Vz, m, rhs_z, 1);
    or_back_subst(Vz, rhs_z, 1, at);
    /* function fit U^{(i)} (Eq. 4): P~ (6 x m), column q = fit of the unit vector e_q */
    double Pt[6 * OR_MAXM];
    or_house_qr(Vd, m, rhs_u, m);
    or_back_subst(Vd, rhs_u, m, Pt);

    /* derivatives of z^{(i)} at the local origin (Eq. 6), back in length units */
    double zx = at[1], zy = at[2];
    double zxx = 2.0 * at[3] / h, zxy = at[4] / h, zyy = 2.0 * at[5] / h;
    /* metric of Eq. 5, its inverse, and the coefficients of Eq. 3 */
    double W = 1.0 + zx * zx + zy * zy;
    double g11 = (1.0 + zy * zy) / W, g12 = -zx * zy / W, g22 = (1.0 + zx * zx) / W;
    double Hs = g11 * zxx + 2.0 * g12 * zxy + g22 * zyy;
    double A1 = -Hs * zx / W, A2 = -Hs * zy / W, A3 = g11, A4 = 2.0 * g12, A5 = g22;

    if (variant == OR_VARIANT_LS) {
        /* derivatives of the least-squares polynomial at the origin (Sec. 2):
         * U_x = b10, U_y = b01, U_xx = 2 b20, U_xy = b11, U_yy = 2 b02 */
        for (int q = 0; q < m; q++) {
            double bx = Pt[1 * m + q] / h, by = Pt[2 * m + q] / h;
            double bxx = 2.0 * Pt[3 * m + q] / (h * h), bxy = Pt[4 * m + q] / (h * h);
            double byy = 2.0 * Pt[5 * m + q] / (h * h);
            w[q] = A1 * bx + A2 * by + A3 * bxx + A4 * bxy + A5 * byy;
        }
    } else {
        /* values of U^{(i)} on the virtual grid nodes (i h, j h), i, j in {-1,0,1}:
         * each is a linear functional of (U_i, U_nbr) (Sec. 3.1) */
        double G[3][3][OR_MAXM];
        for (int gi = -1; gi <= 1; gi++)
            for (int gj = -1; gj <= 1; gj++) {
                double mono[6];
                or_monomials((double)gi, (double)gj, mono);
                for (int q = 0; q < m; q++) {
                    double s = 0;
                    for (int t = 0; t < 6; t++) s += mono[t] * Pt[t * m + q];
                    G[gi + 1][gj + 1][q] = s;
                }
            }
        /* modified centred differences: the centre node takes U_i itself
         * (Eq. 7 in each direction; the mixed term from the corners) */
        for (int q = 0; q < m; q++) {
            double ui = (q == 0) ? 1.0 : 0.0;
            double Dx = (G[2][1][q] - G[0][1][q]) / (2.0 * h);
            double Dy = (G[1][2][q] - G[1][0][q]) / (2.0 * h);
            double Dxx = (G[2][1][q] - 2.0 * ui + G[0][1][q]) / (h * h);
            double Dyy = (G[1][2][q] - 2.0 * ui + G[1][0][q]) / (h * h);
            double Dxy = (G[2][2][q] - G[2][0][q] - G[0][2][q] + G[0][0][q]) / (4.0 * h * h);
            w[q] = A1 * Dx + A2 * Dy + A3 * Dxx + A4 * Dxy + A5 * Dyy;
        }
    }
    if (p00)
        for (int q = 0; q < m; q++) p00[q] = Pt[q];
    if (dg) {
        dg->A[0] = A1; dg->A[1] = A2; dg->A[2] = A3; dg->A[3] = A4; dg->A[4] = A5;
        dg->h = h;
        for (int a = 0; a < 3; a++) dg->normal[a] = ez[a];
        dg->gap = (ev[imax] > 0) ? (ev[imax] - ev[imid]) / ev[imax] : 0.0;
        dg->rank = rank;
    }
    int status = (rank < 1e-10) ? 1 : 0;
    for (int q = 0; q < m; q++)
        if (!isfinite(w[q])) status = 2;
    if (!isfinite(h) || h <= 0) status = 2;
    return status;
}

/* Whole operator.  val: [n][k+1] row-major, slot 0 = self.  diag: optional
 * [n][11] = (A1..A5, h, normal xyz, gap, rank).  p00: optional [n][k+1]. */
int or_assemble(const double *pts, int64_t n, int k, const int32_t *nbr, int delta_kind,
                int delta_m, double delta_scale, int variant, double *val, uint8_t *status,
                double *diag, double *p00)
{
    if (k < 5 || k > OR_MAXK || k >= n) return 1;
    if (delta_kind == OR_DELTA_MEAN_NN && (delta_m < 1 || delta_m > k)) return 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(| : bad)
    for (int64_t i = 0; i < n; i++) {
        or_diag dg;
        int st = or_row(pts, k, nbr + i * k, pts + 3 * i, delta_kind, delta_m, delta_scale, variant,
                        val + i * (k + 1), p00 ? p00 + i * (k + 1) : NULL, &dg);
        if (status) status[i] = (uint8_t)st;
        if (diag) {
            double *o = diag + 11 * i;
            for (int a = 0; a < 5; a++) o[a] = dg.A[a];
            o[5] = dg.h;
            o[6] = dg.normal[0]; o[7] = dg.normal[1]; o[8] = dg.normal[2];
            o[9] = dg.gap; o[10] = dg.rank;
        }
        bad |= (st != 0);
    }
    return bad ? 3 : 0;
}

/* ------------------------------------------------------------------------ */
/* Operator application and solvers for (sigma I - L) u = f (Sec. 4.2).      */
/* ------------------------------------------------------------------------ */

/* y = alpha (sigma x - L x) + beta y; x, y: [n][nr] */
void or_spmv(const double *val, const int32_t *nbr, int64_t n, int k, int nr, double sigma,
             double alpha, const double *x, double beta, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int c = 0; c < nr; c++) {
            double lx = val[i * (k + 1)] * x[i * nr + c];
            for (int s = 0; s < k; s++)
                lx += val[i * (k + 1) + 1 + s] * x[(int64_t)nbr[i * k + s] * nr + c];
            double out = alpha * (sigma * x[i * nr + c] - lx);
            if (beta != 0.0) out += beta * y[i * nr + c];
            y[i * nr + c] = out;
        }
}

static double or_dot(const double *a, const double *b, int64_t n)
{
    double s = 0;
#pragma omp parallel for schedule(static) reduction(+ : s)
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* A x for one right-hand side, A = sigma I - L */
static void or_apply(const double *val, const int32_t *nbr, int64_t n, int k, double sigma,
                     const double *x, double *y)
{
    or_spmv(val, nbr, n, k, 1, sigma, 1.0, x, 0.0, y);
}

/* BiCGSTAB (van der Vorst 1992), unpreconditioned, zero-aware initial guess
 * in x.  Stops when ||f - A x||_2 / ||f||_2 <= rtol (recursive residual,
 * verified against the true residual at exit).  info: [iters, relres]. */
int or_bicgstab(const double *val, const int32_t *nbr, int64_t n, int k, double sigma,
                const double *f, double *x, double rtol, int maxit, double *info)
{
    double *r = malloc(sizeof(double) * n), *rh = malloc(sizeof(double) * n);
    double *p = calloc(n, sizeof(double)), *v = calloc(n, sizeof(double));
    double *s = malloc(sizeof(double) * n), *t = malloc(sizeof(double) * n);
    if (!r || !rh || !p || !v || !s || !t) return 2;
    or_apply(val, nbr, n, k, sigma, x, r);
    for (int64_t i = 0; i < n; i++) { r[i] = f[i] - r[i]; rh[i] = r[i]; }
    double fn = sqrt(or_dot(f, f, n));
    if (fn == 0) fn = 1;
    double rho = 1, alpha = 1, omega = 1;
    double rn = sqrt(or_dot(r, r, n));
    int it = 0, status = 1;
    for (int restart = 0; restart < 50 && status == 1; restart++) {
        for (; it < maxit; it++) {
            if (rn / fn <= rtol) { status = 0; break; }
            double rho1 = or_dot(rh, r, n);
            if (rho1 == 0) break; /* breakdown: restart from the true residual */
            double beta = (rho1 / rho) * (alpha / omega);
            for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            or_apply(val, nbr, n, k, sigma, p, v);
            double rv = or_dot(rh, v, n);
            if (rv == 0) break;
            alpha = rho1 / rv;
            for (int64_t i = 0; i < n; i++) s[i] = r[i] - alpha * v[i];
            or_apply(val, nbr, n, k, sigma, s, t);
            double tt = or_dot(t, t, n);
            omega = (tt > 0) ? or_dot(t, s, n) / tt : 0.0;
            for (int64_t i = 0; i < n; i++) x[i] += alpha * p[i] + omega * s[i];
            for (int64_t i = 0; i < n; i++) r[i] = s[i] - omega * t[i];
            rho = rho1;
            rn = sqrt(or_dot(r, r, n));
            if (omega == 0) { it++; break; }
        }
        /* true residual: exit test and restart point */
        or_apply(val, nbr, n, k, sigma, x, r);
        for (int64_t i = 0; i < n; i++) { r[i] = f[i] - r[i]; rh[i] = r[i]; p[i] = 0; v[i] = 0; }
        rn = sqrt(or_dot(r, r, n));
        rho = alpha = omega = 1;
        if (rn / fn <= rtol) status = 0;
        else if (it >= maxit) break;
        else status = 1;
    }
    info[0] = it;
    info[1] = rn / fn;
    free(r); free(rh); free(p); free(v); free(s); free(t);
    return status;
}

/* Restarted GMRES(m) with modified Gram-Schmidt Arnoldi and Givens rotations
 * (Saad & Schultz 1986).  info: [iters, relres]. */
int or_gmres(const double *val, const int32_t *nbr, int64_t n, int k, double sigma,
             const double *f, double *x, double rtol, int maxit, int restart, double *info)
{
    if (restart < 1) restart = 30;
    double *Vb = malloc(sizeof(double) * n * (restart + 1));
    double *H = calloc((size_t)(restart + 1) * restart, sizeof(double));
    double *cs = malloc(sizeof(double) * restart), *sn = malloc(sizeof(double) * restart);
    double *g = malloc(sizeof(double) * (restart + 1)), *w = malloc(sizeof(double) * n);
    if (!Vb || !H || !cs || !sn || !g || !w) return 2;
    double fn = sqrt(or_dot(f, f, n));
    if (fn == 0) fn = 1;
    int it = 0, status = 1;
    double rn = 0;
    while (it < maxit) {
        or_apply(val, nbr, n, k, sigma, x, w);
        for (int64_t i = 0; i < n; i++) w[i] = f[i] - w[i];
        rn = sqrt(or_dot(w, w, n));
        if (rn / fn <= rtol) { status = 0; break; }
        for (int64_t i = 0; i < n; i++) Vb[i] = w[i] / rn;
        for (int j = 0; j <= restart; j++) g[j] = 0;
        g[0] = rn;
        int j;
        for (j = 0; j < restart && it < maxit; j++, it++) {
            or_apply(val, nbr, n, k, sigma, Vb + (int64_t)j * n, w);
            for (int l = 0; l <= j; l++) {
                double hl = or_dot(w, Vb + (int64_t)l * n, n);
                H[l * restart + j] = hl;
                for (int64_t i = 0; i < n; i++) w[i] -= hl * Vb[(int64_t)l * n + i];
            }
            double hn = sqrt(or_dot(w, w, n));
            H[(j + 1) * restart + j] = hn;
            if (hn > 0)
                for (int64_t i = 0; i < n; i++) Vb[(int64_t)(j + 1) * n + i] = w[i] / hn;
            for (int l = 0; l < j; l++) {
                double a = H[l * restart + j], b = H[(l + 1) * restart + j];
                H[l * restart + j] = cs[l] * a + sn[l] * b;
                H[(l + 1) * restart + j] = -sn[l] * a + cs[l] * b;
            }
            double a = H[j * restart + j], b = H[(j + 1) * restart + j];
            double den = sqrt(a * a + b * b);
            cs[j] = (den > 0) ? a / den : 1.0;
            sn[j] = (den > 0) ? b / den : 0.0;
            H[j * restart + j] = den;
            H[(j + 1) * restart + j] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) / fn <= rtol || hn == 0) { j++; it++; break; }
        }
        /* y = H^{-1} g, x += V y */
        double y[1024];
        for (int l = j - 1; l >= 0; l--) {
            double s = g[l];
            for (int q = l + 1; q < j; q++) s -= H[l * restart + q] * y[q];
            y[l] = s / H[l * restart + l];
        }
        for (int l = 0; l < j; l++)
            for (int64_t i = 0; i < n; i++) x[i] += y[l] * Vb[(int64_t)l * n + i];
    }
    or_apply(val, nbr, n, k, sigma, x, w);
    for (int64_t i = 0; i < n; i++) w[i] = f[i] - w[i];
    rn = sqrt(or_dot(w, w, n));
    if (rn / fn <= rtol) status = 0;
    info[0] = it;
    info[1] = rn / fn;
    free(Vb); free(H); free(cs); free(sn); free(g); free(w);
    return status;
}

/* ------------------------------------------------------------------------ */
/* 1-D Laplacian on a line (Sec. 3.2): least-squares quadratic T^{(0)} over   */
/* samples x_q (one of them the centre x = 0 at index c), then either the LS  */
/* second derivative 2 a_2 or the modified centred difference with the       */
/* centre value T_0 (Eq. 7).  w: out [m].                                    */
/* ------------------------------------------------------------------------ */
int or_line_weights(const double *xs, int m, int c, double h, int variant, double *w)
{
    if (m < 3 || m > OR_MAXM || c < 0 || c >= m) return 1;
    /* normal equations of the quadratic fit, solved by Gaussian elimination
     * with partial pivoting on [A | B], B = Vandermonde^T */
    double A[3][3] = {{0}}, B[3][OR_MAXM];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < m; q++) B[r][q] = pow(xs[q], r);
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++)
            for (int q = 0; q < m; q++) A[r][s] += pow(xs[q], r + s);
    for (int col = 0; col < 3; col++) {
        int piv = col;
        for (int r = col + 1; r < 3; r++)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0) return 2;
        for (int s = 0; s < 3; s++) { double t = A[col][s]; A[col][s] = A[piv][s]; A[piv][s] = t; }
        for (int q = 0; q < m; q++) { double t = B[col][q]; B[col][q] = B[piv][q]; B[piv][q] = t; }
        for (int r = col + 1; r < 3; r++) {
            double f = A[r][col] / A[col][col];
            for (int s = col; s < 3; s++) A[r][s] -= f * A[col][s];
            for (int q = 0; q < m; q++) B[r][q] -= f * B[col][q];
        }
    }
    double a[3][OR_MAXM];
    for (int q = 0; q < m; q++)
        for (int r = 2; r >= 0; r--) {
            double s = B[r][q];
            for (int t = r + 1; t < 3; t++) s -= A[r][t] * a[t][q];
            a[r][q] = s / A[r][r];
        }
    for (int q = 0; q < m; q++) {
        if (variant == OR_VARIANT_LS) {
            w[q] = 2.0 * a[2][q];
        } else {
            double tp = a[0][q] + a[1][q] * h + a[2][q] * h * h;   /* T^{(0)}(h) */
            double tm = a[0][q] - a[1][q] * h + a[2][q] * h * h;   /* T^{(0)}(-h) */
            double t0 = (q == c) ? 1.0 : 0.0;                       /* T_0 */
            w[q] = (tp - 2.0 * t0 + tm) / (h * h);
        }
    }
    return 0;
}
