/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * SE(3) exponential and logarithm for the twist update of Section 5, and a
 * Cholesky solve for the Gauss-Newton normal equations (Eq. 18, delta theta =
 * -A^{-1} b).
 *
 * Eq. 16 gives the first-order form T_new ~ (I + zeta^) T with
 * zeta = (alpha, beta, gamma, a, b, c); its upper-left block is I + [omega]_x
 * with omega = (alpha, beta, gamma).  The update applied here is the full
 * exponential of that same twist matrix, exp(zeta^) T, which stays on SE(3):
 *   R = I + A W + B W^2,  t = (I + B W + C W^2) v,  W = [omega]_x,
 *   A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3.
 * Series of A, B, C are used for th < 1e-3.
 */
#include "oracle.h"

#include <math.h>
#include <string.h>

static void skew(const double w[3], double W[9])
{
    W[0] = 0.0;   W[1] = -w[2]; W[2] = w[1];
    W[3] = w[2];  W[4] = 0.0;   W[5] = -w[0];
    W[6] = -w[1]; W[7] = w[0];  W[8] = 0.0;
}

static void mat3_mul(const double *a, const double *b, double *c)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
                s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
}

void or_se3_exp(const double zeta[6], double T[16])
{
    const double *w = zeta, *v = zeta + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-3) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    double W[9], W2[9];
    skew(w, W);
    mat3_mul(W, W, W2);
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * W[i] + B * W2[i];
        V[i] = I + B * W[i] + C * W2[i];
    }
    memset(T, 0, 16 * sizeof(double));
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            T[4 * i + j] = R[3 * i + j];
        T[4 * i + 3] = V[3 * i] * v[0] + V[3 * i + 1] * v[1] + V[3 * i + 2] * v[2];
    }
    T[15] = 1.0;
}

void or_se3_log(const double T[16], double zeta[6])
{
    double R[9], t[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = T[4 * i + j];
        t[i] = T[4 * i + 3];
    }
    double cth = 0.5 * (R[0] + R[4] + R[8] - 1.0);
    if (cth > 1.0)
        cth = 1.0;
    if (cth < -1.0)
        cth = -1.0;
    double th = acos(cth);
    double vee[3] = {R[7] - R[5], R[2] - R[6], R[3] - R[1]}; /* 2 sin(th) omega/th */
    double w[3];
    if (th < 1e-6) {
        for (int i = 0; i < 3; ++i)
            w[i] = 0.5 * vee[i];
    } else if (3.14159265358979323846 - th < 1e-4) {
        /* Near pi: R + I = 2 n n^T + O(pi - th); take the best-conditioned column. */
        int c = 0;
        for (int i = 1; i < 3; ++i)
            if (R[4 * i] > R[4 * c])
                c = i;
        double n[3];
        for (int i = 0; i < 3; ++i)
            n[i] = R[3 * i + c] + (i == c ? 1.0 : 0.0);
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        double sgn = (n[0] * vee[0] + n[1] * vee[1] + n[2] * vee[2]) < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < 3; ++i)
            w[i] = sgn * th * n[i] / nn;
    } else {
        double f = th / (2.0 * sin(th));
        for (int i = 0; i < 3; ++i)
            w[i] = f * vee[i];
    }
    /* v = V^{-1} t with V^{-1} = I - W/2 + k W^2, k = (1 - A/(2B)) / th^2. */
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double thw = sqrt(th2);
    double k;
    if (thw < 1e-3)
        k = 1.0 / 12.0 + th2 / 720.0;
    else {
        double A = sin(thw) / thw, B = (1.0 - cos(thw)) / th2;
        k = (1.0 - A / (2.0 * B)) / th2;
    }
    double W[9], W2[9];
    skew(w, W);
    mat3_mul(W, W, W2);
    for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int j = 0; j < 3; ++j) {
            double Vi = (i == j ? 1.0 : 0.0) - 0.5 * W[3 * i + j] + k * W2[3 * i + j];
            s += Vi * t[j];
        }
        zeta[i] = w[i];
        zeta[3 + i] = s;
    }
}

int or_cholesky_solve(int n, const double *A, const double *b, double *x)
{
    double L[64 * 64];
    if (n > 64)
        return 1;
    /* Scale-relative pivot floor: a pivot below it means "not positive definite". */
    double maxdiag = 0.0;
    for (int i = 0; i < n; ++i)
        if (A[i * n + i] > maxdiag)
            maxdiag = A[i * n + i];
    if (!(maxdiag > 0.0))
        return 1;
    const double floor_ = maxdiag * 1e-12;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k)
                s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > floor_))
                    return 1;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    }
    double y[64];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k)
            s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k)
            s -= L[k * n + i] * x[k];
        x[i] = s / L[i * n + i];
    }
    return 0;
}
