/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The exact E step: the Gaussian sums of Eq. 6 (M0, M1) and the numerator of
 * Eq. 9 (the kernel-weighted observation normals), evaluated directly in
 * O(N M) double-precision work.  The normalisation constant of the Gaussian
 * PDF is omitted as in Eq. 11 (Section 4.1); the outlier constant absorbs it
 * (or_outlier_constant).  This is the plain definition the lattice
 * approximates.
 */
#include "oracle.h"

#include <math.h>

void or_exact_sums_at(const double x[3], const float *Y, const float *Yn, int64_t N,
                      double sigma, double *M0, double M1[3], double Ns[3])
{
    const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
    double m0 = 0.0, m1[3] = {0, 0, 0}, ns[3] = {0, 0, 0};
    for (int64_t k = 0; k < N; ++k) {
        double d0 = x[0] - Y[4 * k], d1 = x[1] - Y[4 * k + 1], d2 = x[2] - Y[4 * k + 2];
        double g = exp(-(d0 * d0 + d1 * d1 + d2 * d2) * inv2s2);
        m0 += g;
        for (int c = 0; c < 3; ++c)
            m1[c] += g * (double)Y[4 * k + c];
        if (Yn)
            for (int c = 0; c < 3; ++c)
                ns[c] += g * (double)Yn[4 * k + c];
    }
    *M0 = m0;
    for (int c = 0; c < 3; ++c) {
        M1[c] = m1[c];
        Ns[c] = ns[c];
    }
}

void or_estep_exact(const float *X, int64_t M, const float *Y, const float *Yn,
                    int64_t N, double sigma, double *M0, double *M1, double *Ns)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double x[3] = {X[4 * i], X[4 * i + 1], X[4 * i + 2]}, ns[3];
        or_exact_sums_at(x, Y, Yn, N, sigma, M0 + i, M1 + 3 * i, ns);
        if (Yn && Ns)
            for (int c = 0; c < 3; ++c)
                Ns[3 * i + c] = ns[c];
    }
}
