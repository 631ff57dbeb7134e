// Small dense kernels of the local frames (Sec. 2): the symmetric 3x3
// eigenproblem of a neighbourhood's covariance.
#pragma once

#include <cuda_runtime.h>

namespace mvgd {

// Cyclic Jacobi on a symmetric 3x3 matrix (a, upper part used).  Columns of v
// are the eigenvectors, w the eigenvalues.
__device__ inline void jacobi3(double a[3][3], double v[3][3], double w[3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) v[r][c] = (r == c) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 32; sweep++) {
        double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-40 * dia)) break;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            double apq = a[p][q];
            if (apq == 0.0) continue;
            double tau = (a[q][q] - a[p][p]) / (2.0 * apq);
            double t = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double c = rsqrt(1.0 + t * t);
            double s = t * c;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                double akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - s * akq;
                a[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                double apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - s * aqk;
                a[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                double vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    w[0] = a[0][0];
    w[1] = a[1][1];
    w[2] = a[2][2];
}

// The same cyclic Jacobi in FP32, stopped at FP32 accuracy: the starting
// frame that one or two FP64 sweeps then polish (the FP32 assembly path).
__device__ inline void jacobi3f(float a[3][3], float v[3][3], float w[3]) {
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) v[r][c] = (r == c) ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 16; sweep++) {
        const float off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const float dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (!(off > 1e-14f * dia)) break;
#pragma unroll
        for (int pq = 0; pq < 3; pq++) {
            const int p = pq == 2 ? 1 : 0;
            const int q = pq == 0 ? 1 : 2;
            const float apq = a[p][q];
            if (apq == 0.0f) continue;
            const float tau = (a[q][q] - a[p][p]) / (2.0f * apq);
            const float t = copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
            const float c = rsqrtf(1.0f + t * t);
            const float s = t * c;
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float akp = a[k][p], akq = a[k][q];
                a[k][p] = c * akp - s * akq;
                a[k][q] = s * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float apk = a[p][k], aqk = a[q][k];
                a[p][k] = c * apk - s * aqk;
                a[q][k] = s * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float vkp = v[k][p], vkq = v[k][q];
                v[k][p] = c * vkp - s * vkq;
                v[k][q] = s * vkp + c * vkq;
            }
        }
    }
    w[0] = a[0][0];
    w[1] = a[1][1];
    w[2] = a[2][2];
}

}  // namespace mvgd
