// Host-side dense kernels of the subspace eigensolver (Sec. 4.3): the p x p
// steps between the device's block operations, p <= 128.
//
//   mvgd_block_chol_inverse: R^-1 for the Cholesky factor R^T R = (G + G^T)/2
//     of a Gram matrix (the orthonormalisation X = Y R^-1 of the basis);
//   mvgd_ritz_values: the eigenvalues of the projected matrix H = X^T L X,
//     real and nonsymmetric, by Householder reduction to upper Hessenberg form
//     followed by Francis double-shift QR steps with deflation (Golub and Van
//     Loan, Matrix Computations, Algorithms 7.4.2 and 7.5.1-7.5.2).
// Plain FP64 host code: the matrices are tiny, the device would only wait.
#include <math.h>
#include <string.h>

#include <vector>

#include "common.cuh"

namespace mvgd {
namespace {

constexpr int kMaxRitz = 128;

// Eigenvalues of the 2x2 block [[a, b], [c, d]].
void eig2(double a, double b, double c, double d, double* r0, double* i0, double* r1, double* i1) {
    const double p = 0.5 * (a - d);
    const double bc = b * c;
    const double disc = p * p + bc;
    const double mid = 0.5 * (a + d);
    if (disc >= 0.0) {
        // the root of larger magnitude first, the other from the product (no cancellation)
        const double s = sqrt(disc);
        const double z = p + (p >= 0.0 ? s : -s);
        const double e0 = d + z;
        const double e1 = (z != 0.0) ? d - bc / z : d;
        *r0 = e0; *i0 = 0.0;
        *r1 = e1; *i1 = 0.0;
    } else {
        const double w = sqrt(-disc);
        *r0 = mid; *i0 = w;
        *r1 = mid; *i1 = -w;
    }
}

// Reduces the n x n row-major matrix a to upper Hessenberg form in place by
// Householder similarity transforms.
void hessenberg(int n, double* a) {
    std::vector<double> v((size_t)n);
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;  // length of the column part below the diagonal
        double scale = 0.0;
        for (int i = 0; i < m; i++) scale += fabs(a[(k + 1 + i) * n + k]);
        if (scale == 0.0) continue;
        double norm2 = 0.0;
        for (int i = 0; i < m; i++) {
            v[i] = a[(k + 1 + i) * n + k] / scale;
            norm2 += v[i] * v[i];
        }
        double alpha = sqrt(norm2);
        if (v[0] > 0.0) alpha = -alpha;
        v[0] -= alpha;
        double vv = 0.0;
        for (int i = 0; i < m; i++) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double beta = 2.0 / vv;
        // left: rows k+1.., every column from k
        for (int j = k; j < n; j++) {
            double s = 0.0;
            for (int i = 0; i < m; i++) s += v[i] * a[(k + 1 + i) * n + j];
            s *= beta;
            for (int i = 0; i < m; i++) a[(k + 1 + i) * n + j] -= s * v[i];
        }
        // right: columns k+1.., every row
        for (int i = 0; i < n; i++) {
            double s = 0.0;
            for (int j = 0; j < m; j++) s += a[i * n + k + 1 + j] * v[j];
            s *= beta;
            for (int j = 0; j < m; j++) a[i * n + k + 1 + j] -= s * v[j];
        }
        a[(k + 1) * n + k] = alpha * scale;
        for (int i = 1; i < m; i++) a[(k + 1 + i) * n + k] = 0.0;
    }
}

// Applies the 3x3 (or 2x2 when r == 2) Householder reflector I - beta u u^T
// with u = (1, u1, u2) to rows k..k+r-1 (columns c0..c1) and to columns
// k..k+r-1 (rows r0..r1) of the Hessenberg matrix a.
void reflect(int n, double* a, int k, int r, double u1, double u2, double beta, int c0, int c1, int r0, int r1) {
    for (int j = c0; j <= c1; j++) {
        double s = a[k * n + j] + u1 * a[(k + 1) * n + j] + (r == 3 ? u2 * a[(k + 2) * n + j] : 0.0);
        s *= beta;
        a[k * n + j] -= s;
        a[(k + 1) * n + j] -= s * u1;
        if (r == 3) a[(k + 2) * n + j] -= s * u2;
    }
    for (int i = r0; i <= r1; i++) {
        double s = a[i * n + k] + u1 * a[i * n + k + 1] + (r == 3 ? u2 * a[i * n + k + 2] : 0.0);
        s *= beta;
        a[i * n + k] -= s;
        a[i * n + k + 1] -= s * u1;
        if (r == 3) a[i * n + k + 2] -= s * u2;
    }
}

// Householder vector u = (1, u1, u2) and beta of the reflector mapping
// (x, y, z) onto a multiple of e_1; false when (x, y, z) = 0.
bool house3(double x, double y, double z, double* u1, double* u2, double* beta) {
    const double sc = fabs(x) + fabs(y) + fabs(z);
    if (sc == 0.0) return false;
    x /= sc; y /= sc; z /= sc;
    double alpha = sqrt(x * x + y * y + z * z);
    if (x > 0.0) alpha = -alpha;
    const double v0 = x - alpha;  // |v0| >= |x|, never zero
    *u1 = y / v0;
    *u2 = z / v0;
    *beta = 2.0 / (1.0 + *u1 * *u1 + *u2 * *u2);
    return true;
}

// Eigenvalues of an upper Hessenberg matrix by Francis double-shift QR.
// Returns false if a block does not deflate within the iteration cap.
bool francis(int n, double* a, double* wr, double* wi) {
    const double eps = 2.220446049250313e-16;
    double anorm = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = (i > 0 ? i - 1 : 0); j < n; j++) anorm += fabs(a[i * n + j]);
    int hi = n - 1;
    int iter = 0, total = 0;
    while (hi >= 0) {
        int l = hi;
        while (l > 0) {  // the lowest l with a negligible subdiagonal entry a(l, l-1)
            double s = fabs(a[(l - 1) * n + l - 1]) + fabs(a[l * n + l]);
            if (s == 0.0) s = anorm;
            if (fabs(a[l * n + l - 1]) <= eps * s) {
                a[l * n + l - 1] = 0.0;
                break;
            }
            l--;
        }
        if (l == hi) {  // a 1x1 block
            wr[hi] = a[hi * n + hi];
            wi[hi] = 0.0;
            hi--;
            iter = 0;
            continue;
        }
        if (l == hi - 1) {  // a 2x2 block
            eig2(a[(hi - 1) * n + hi - 1], a[(hi - 1) * n + hi], a[hi * n + hi - 1], a[hi * n + hi], &wr[hi - 1],
                 &wi[hi - 1], &wr[hi], &wi[hi]);
            hi -= 2;
            iter = 0;
            continue;
        }
        if (++total > 60 * n) return false;
        iter++;
        // shifts: the eigenvalues of the trailing 2x2 block (sum s, product t);
        // ad hoc shifts after 10 and 20 steps without deflation
        double s, t;
        if (iter == 10 || iter == 20) {
            const double w = fabs(a[hi * n + hi - 1]) + fabs(a[(hi - 1) * n + hi - 2]);
            s = 1.5 * w + a[hi * n + hi];
            t = w * w;
        } else {
            const double p = a[(hi - 1) * n + hi - 1], q = a[(hi - 1) * n + hi];
            const double r = a[hi * n + hi - 1], d = a[hi * n + hi];
            s = p + d;
            t = p * d - q * r;
        }
        // first column of (H - s1 I)(H - s2 I) restricted to the window
        double x = a[l * n + l] * a[l * n + l] + a[l * n + l + 1] * a[(l + 1) * n + l] - s * a[l * n + l] + t;
        double y = a[(l + 1) * n + l] * (a[l * n + l] + a[(l + 1) * n + l + 1] - s);
        double z = a[(l + 1) * n + l] * a[(l + 2) * n + l + 1];
        for (int k = l; k <= hi - 2; k++) {
            double u1, u2, beta;
            if (house3(x, y, z, &u1, &u2, &beta)) {
                const int c0 = k > l ? k - 1 : l;
                const int r1 = k + 3 < hi ? k + 3 : hi;
                reflect(n, a, k, 3, u1, u2, beta, c0, hi, l, r1);
            }
            x = a[(k + 1) * n + k];
            y = a[(k + 2) * n + k];
            if (k < hi - 2) z = a[(k + 3) * n + k];
            if (k > l) {  // the reflector annihilated the bulge in column k-1: clear its rounding residue
                a[(k + 1) * n + k - 1] = 0.0;
                a[(k + 2) * n + k - 1] = 0.0;
            }
        }
        // the last step is a 2x2 reflector on rows/columns hi-1, hi
        double u1, u2, beta;
        if (house3(x, y, 0.0, &u1, &u2, &beta)) reflect(n, a, hi - 1, 2, u1, 0.0, beta, hi - 2, hi, l, hi);
        a[hi * n + hi - 2] = 0.0;  // hi - 2 >= l here: the window holds at least 3 rows
    }
    return true;
}

}  // namespace
}  // namespace mvgd

using namespace mvgd;

MVGD_API mvgd_status mvgd_block_chol_inverse(const double* G, int32_t p, double* Rinv) {
    if (!G || !Rinv || p < 1 || p > kMaxRitz) return MVGD_EINVAL;
    std::vector<double> R((size_t)p * p, 0.0);
    // R^T R = (G + G^T) / 2, R upper triangular, row by row
    for (int i = 0; i < p; i++) {
        for (int j = i; j < p; j++) {
            double s = 0.5 * (G[i * p + j] + G[j * p + i]);
            for (int q = 0; q < i; q++) s -= R[q * p + i] * R[q * p + j];
            if (j == i) {
                if (!(s > 0.0) || !isfinite(s)) return MVGD_EDEGENERATE;
                R[i * p + i] = sqrt(s);
            } else {
                R[i * p + j] = s / R[i * p + i];
            }
        }
    }
    // R^-1 by back substitution, column by column (upper triangular)
    memset(Rinv, 0, sizeof(double) * (size_t)p * p);
    for (int c = 0; c < p; c++) {
        for (int i = c; i >= 0; i--) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int q = i + 1; q <= c; q++) s -= R[i * p + q] * Rinv[q * p + c];
            Rinv[i * p + c] = s / R[i * p + i];
        }
    }
    return MVGD_OK;
}

MVGD_API mvgd_status mvgd_ritz_values(const double* H, int32_t p, double* re, double* im) {
    if (!H || !re || !im || p < 1 || p > kMaxRitz) return MVGD_EINVAL;
    std::vector<double> a(H, H + (size_t)p * p);
    for (double v : a)
        if (!isfinite(v)) return MVGD_ENONFINITE;
    hessenberg(p, a.data());
    if (!francis(p, a.data(), re, im)) return MVGD_ENOCONV;
    return MVGD_OK;
}
