/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Node-graph deformable model (Section 5.2, Eq. 21).
 *
 * Nodes k = 0..K-1 have reference positions p_k and poses T_k in SE(3).  A
 * model point x_i_ref with nearest nodes N_i and fixed skinning weights w_ki
 * moves by the dual-quaternion blend of its nodes' poses (Eq. 21):
 *     T_i = normalized(sum_k w_ki dq(T_k)),   x_i = T_i x_i_ref,
 * each node's dual quaternion sign-aligned with that of the neighbour of
 * largest weight (the first such) before summing, the blend divided by the norm of its real part, and the
 * translation read as 2 (r0 d - d0 r + r x d) (Kavan et al.).
 *
 * The supplement the paper defers to is missing; these readings fill it:
 *   - parameters theta = one twist zeta_k per node, applied on the left,
 *     T_k <- exp(zeta_k^) T_k (world frame, (omega; v), as Eq. 16);
 *   - the twist of a point is the skinning-weighted sum of its nodes'
 *     twists, d zeta_i / d zeta_k = w_ki I_6 (the first-order DQB
 *     derivative, exact when the node poses agree), so the data term adds
 *     w_ai w_bi J_i^T J_i to block (a, b) and w_ai J_i^T r_i to g_a, with J_i
 *     and r_i the rigid model's point terms (Eq. 7 / Eq. 10, sqrt(W)/sigma
 *     weighted);
 *   - a regulariser keeps neighbouring nodes consistent: for every directed
 *     edge (j, k), r_jk = sqrt(lambda)/sigma (T_j p_k - T_k p_k), with
 *     d r_jk / d zeta_j = sqrt(lambda)/sigma [-[T_j p_k]_x, I] and
 *     d r_jk / d zeta_k = -sqrt(lambda)/sigma [-[T_k p_k]_x, I];
 *   - the Gauss-Newton system A dtheta = -g is solved by block-Jacobi
 *     preconditioned conjugate gradients with a fixed iteration count from
 *     dtheta = 0 (a block that is not positive definite is preconditioned
 *     by 1 / its largest diagonal entry);
 *   - every node is updated by its twist's exponential.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- quaternions and dual quaternions ------------------------------------ */

static void quat_mul(const double a[4], const double b[4], double c[4])
{
    /* (w1, v1)(w2, v2) = (w1 w2 - v1.v2, w1 v2 + w2 v1 + v1 x v2) */
    double t[4];
    t[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    t[1] = a[0] * b[1] + b[0] * a[1] + a[2] * b[3] - a[3] * b[2];
    t[2] = a[0] * b[2] + b[0] * a[2] + a[3] * b[1] - a[1] * b[3];
    t[3] = a[0] * b[3] + b[0] * a[3] + a[1] * b[2] - a[2] * b[1];
    memcpy(c, t, sizeof t);
}

/* Unit quaternion of a rotation matrix (the largest of w, x, y, z pivots). */
static void quat_from_R(const double T[16], double q[4])
{
    const double m00 = T[0], m01 = T[1], m02 = T[2];
    const double m10 = T[4], m11 = T[5], m12 = T[6];
    const double m20 = T[8], m21 = T[9], m22 = T[10];
    const double tr = m00 + m11 + m22;
    if (tr >= m00 && tr >= m11 && tr >= m22) {
        const double s = sqrt(1.0 + tr) * 2.0; /* 4 w */
        q[0] = 0.25 * s;
        q[1] = (m21 - m12) / s;
        q[2] = (m02 - m20) / s;
        q[3] = (m10 - m01) / s;
    } else if (m00 >= m11 && m00 >= m22) {
        const double s = sqrt(1.0 + m00 - m11 - m22) * 2.0; /* 4 x */
        q[0] = (m21 - m12) / s;
        q[1] = 0.25 * s;
        q[2] = (m01 + m10) / s;
        q[3] = (m02 + m20) / s;
    } else if (m11 >= m22) {
        const double s = sqrt(1.0 + m11 - m00 - m22) * 2.0; /* 4 y */
        q[0] = (m02 - m20) / s;
        q[1] = (m01 + m10) / s;
        q[2] = 0.25 * s;
        q[3] = (m12 + m21) / s;
    } else {
        const double s = sqrt(1.0 + m22 - m00 - m11) * 2.0; /* 4 z */
        q[0] = (m10 - m01) / s;
        q[1] = (m02 + m20) / s;
        q[2] = (m12 + m21) / s;
        q[3] = 0.25 * s;
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a)
        q[a] /= n;
}

void or_dq_from_T(const double T[16], double dq[8])
{
    /* real part q_r (rotation), dual part q_d = 1/2 (0, t) q_r */
    quat_from_R(T, dq);
    const double t[4] = {0.0, T[3], T[7], T[11]};
    quat_mul(t, dq, dq + 4);
    for (int a = 4; a < 8; ++a)
        dq[a] *= 0.5;
}

void or_T_from_dq(const double dq[8], double T[16])
{
    const double n = sqrt(dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2] + dq[3] * dq[3]);
    const double w = dq[0] / n, x = dq[1] / n, y = dq[2] / n, z = dq[3] / n;
    const double d0 = dq[4] / n, dx = dq[5] / n, dy = dq[6] / n, dz = dq[7] / n;
    T[0] = 1.0 - 2.0 * (y * y + z * z);
    T[1] = 2.0 * (x * y - w * z);
    T[2] = 2.0 * (x * z + w * y);
    T[4] = 2.0 * (x * y + w * z);
    T[5] = 1.0 - 2.0 * (x * x + z * z);
    T[6] = 2.0 * (y * z - w * x);
    T[8] = 2.0 * (x * z - w * y);
    T[9] = 2.0 * (y * z + w * x);
    T[10] = 1.0 - 2.0 * (x * x + y * y);
    /* t = 2 (r0 d - d0 r + r x d) */
    T[3] = 2.0 * (w * dx - d0 * x + (y * dz - z * dy));
    T[7] = 2.0 * (w * dy - d0 * y + (z * dx - x * dz));
    T[11] = 2.0 * (w * dz - d0 * z + (x * dy - y * dx));
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}

void or_dqb(const double *node_dq, const int32_t knn[4], const float w[4], double T[16])
{
    int ref = 0;
    for (int k = 1; k < 4; ++k)
        if (w[k] > w[ref])
            ref = k;
    const double *q0 = node_dq + 8 * (size_t)knn[ref];
    double b[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 4; ++k) {
        const double *q = node_dq + 8 * (size_t)knn[k];
        const double dot = q[0] * q0[0] + q[1] * q0[1] + q[2] * q0[2] + q[3] * q0[3];
        const double s = (dot < 0.0 ? -1.0 : 1.0) * (double)w[k];
        for (int a = 0; a < 8; ++a)
            b[a] += s * q[a];
    }
    or_T_from_dq(b, T);
}

static void node_dqs(int K, const double *node_T, double *dq)
{
    for (int k = 0; k < K; ++k)
        or_dq_from_T(node_T + 16 * (size_t)k, dq + 8 * (size_t)k);
}

int or_nodegraph_warp(const float *Xref, const int32_t *knn, const float *skw, int64_t M, int K,
                      const double *node_T, double *X)
{
    double *dq = (double *)malloc((size_t)K * 8 * sizeof(double));
    if (!dq)
        return OR_ENOMEM;
    node_dqs(K, node_T, dq);
    for (int64_t i = 0; i < M; ++i) {
        double T[16];
        or_dqb(dq, knn + 4 * i, skw + 4 * i, T);
        const float *p = Xref + 4 * i;
        for (int a = 0; a < 3; ++a)
            X[3 * i + a] = T[4 * a] * p[0] + T[4 * a + 1] * p[1] + T[4 * a + 2] * p[2] + T[4 * a + 3];
    }
    free(dq);
    return OR_OK;
}

/* ---- normal equations -------------------------------------------------------- */

static double *obs_values(const float *Y, const float *Yn, int64_t N, int vdim)
{
    double *V = (double *)malloc((size_t)N * vdim * sizeof(double));
    if (!V)
        return NULL;
    for (int64_t k = 0; k < N; ++k) {
        double *v = V + (size_t)vdim * k;
        v[0] = 1.0;
        for (int a = 0; a < 3; ++a)
            v[1 + a] = Y[4 * k + a];
        if (vdim == 7)
            for (int a = 0; a < 3; ++a)
                v[4 + a] = Yn[4 * k + a];
    }
    return V;
}

static void twist_jacobian(const double x[3], double s, double J[18])
{
    /* s [-[x]_x, I]: rows of d(exp(zeta) x)/d zeta at zeta = 0 */
    const double Jx[18] = {0.0, x[2], -x[1], 1.0, 0.0, 0.0,
                           -x[2], 0.0, x[0], 0.0, 1.0, 0.0,
                           x[1], -x[0], 0.0, 0.0, 0.0, 1.0};
    for (int a = 0; a < 18; ++a)
        J[a] = s * Jx[a];
}

/* A (6K x 6K, dense, row-major) and g (6K) at the node poses node_T, with the
 * E step taken on lattice `lat` (lattice back end) or the exact sums. */
static int normal_equations(const float *Xref, const int32_t *knn, const float *skw, int64_t M,
                            const or_nodegraph *ng, const float *Y, const float *Yn, int64_t N,
                            const or_lattice *lat, const or_options *opt, double sigma,
                            const double *node_T, double *A, double *g, int64_t *inliers,
                            double *cost, double *sum_w)
{
    const int K = ng->K;
    const size_t n = 6 * (size_t)K;
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    double *X = (double *)malloc((size_t)M * 3 * sizeof(double));
    if (!X)
        return OR_ENOMEM;
    int status = or_nodegraph_warp(Xref, knn, skw, M, K, node_T, X);
    if (status != OR_OK) {
        free(X);
        return status;
    }
    memset(A, 0, n * n * sizeof(double));
    memset(g, 0, n * sizeof(double));
    const double c_eff = or_outlier_constant(opt->w, N, M, sigma, opt->backend, opt->blur);
    *inliers = 0;
    *cost = 0.0;
    *sum_w = 0.0;
    /* data term */
    for (int64_t i = 0; i < M; ++i) {
        const double *x = X + 3 * i;
        double e[7] = {0, 0, 0, 0, 0, 0, 0};
        if (opt->backend == OR_LATTICE) {
            const float xf[4] = {(float)x[0], (float)x[1], (float)x[2], 0.0f};
            or_lattice_slice(lat, xf, 1, e);
        } else {
            double ns[3];
            or_exact_sums_at(x, Y, Yn, N, sigma, e, e + 1, ns);
            if (vdim == 7)
                for (int c = 0; c < 3; ++c)
                    e[4 + c] = ns[c];
        }
        double Ns[3] = {0, 0, 0};
        if (vdim == 7)
            for (int c = 0; c < 3; ++c)
                Ns[c] = e[4 + c];
        double W, r[3], J[18];
        const int rows = or_point_terms(x, e[0], e + 1, Ns, c_eff, sigma, opt->residual,
                                        opt->renormalize_normals, &W, r, J);
        if (rows == 0)
            continue;
        ++*inliers;
        *sum_w += W;
        double H[36] = {0}, h[6] = {0};
        for (int a = 0; a < rows; ++a) {
            *cost += r[a] * r[a];
            for (int p = 0; p < 6; ++p) {
                h[p] += J[6 * a + p] * r[a];
                for (int q = 0; q < 6; ++q)
                    H[6 * p + q] += J[6 * a + p] * J[6 * a + q];
            }
        }
        const int32_t *nb = knn + 4 * i;
        const float *wk = skw + 4 * i;
        for (int ka = 0; ka < 4; ++ka) {
            const size_t a0 = 6 * (size_t)nb[ka];
            for (int p = 0; p < 6; ++p)
                g[a0 + p] += (double)wk[ka] * h[p];
            for (int kb = 0; kb < 4; ++kb) {
                const size_t b0 = 6 * (size_t)nb[kb];
                const double wab = (double)wk[ka] * (double)wk[kb];
                for (int p = 0; p < 6; ++p)
                    for (int q = 0; q < 6; ++q)
                        A[(a0 + p) * n + b0 + q] += wab * H[6 * p + q];
            }
        }
    }
    /* regulariser */
    const double s = sqrt(ng->lambda) / sigma;
    for (int e = 0; e < ng->E; ++e) {
        const int j = ng->edges[2 * e], k = ng->edges[2 * e + 1];
        const double *Tj = node_T + 16 * (size_t)j, *Tk = node_T + 16 * (size_t)k;
        const double *pk = ng->node_pos + 3 * (size_t)k;
        double a[3], b[3], r[3];
        for (int c = 0; c < 3; ++c) {
            a[c] = Tj[4 * c] * pk[0] + Tj[4 * c + 1] * pk[1] + Tj[4 * c + 2] * pk[2] + Tj[4 * c + 3];
            b[c] = Tk[4 * c] * pk[0] + Tk[4 * c + 1] * pk[1] + Tk[4 * c + 2] * pk[2] + Tk[4 * c + 3];
            r[c] = s * (a[c] - b[c]);
        }
        double Jj[18], Jk[18];
        twist_jacobian(a, s, Jj);
        twist_jacobian(b, -s, Jk);
        const int idx[2] = {j, k};
        const double *Js[2] = {Jj, Jk};
        for (int u = 0; u < 2; ++u) {
            const size_t u0 = 6 * (size_t)idx[u];
            for (int p = 0; p < 6; ++p) {
                for (int c = 0; c < 3; ++c)
                    g[u0 + p] += Js[u][6 * c + p] * r[c];
                for (int v = 0; v < 2; ++v) {
                    const size_t v0 = 6 * (size_t)idx[v];
                    for (int q = 0; q < 6; ++q) {
                        double acc = 0.0;
                        for (int c = 0; c < 3; ++c)
                            acc += Js[u][6 * c + p] * Js[v][6 * c + q];
                        A[(u0 + p) * n + v0 + q] += acc;
                    }
                }
            }
        }
        *cost += r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    }
    free(X);
    return OR_OK;
}

int or_nodegraph_normal_equations(const float *Xref, const int32_t *knn, const float *skw,
                                  int64_t M, const or_nodegraph *ng, const float *Y,
                                  const float *Yn, int64_t N, const or_options *opt, double sigma,
                                  const double *node_T, double *A, double *g, or_report *rep)
{
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    or_lattice *lat = NULL;
    int status = OR_OK;
    if (opt->backend == OR_LATTICE) {
        double *V = obs_values(Y, Yn, N, vdim);
        lat = V ? or_lattice_build(Y, V, N, vdim, (float)sigma, &status) : NULL;
        free(V);
        if (!lat)
            return status != OR_OK ? status : OR_ENOMEM;
        if (opt->blur)
            or_lattice_blur(lat);
    }
    int64_t inl;
    double cost, sw;
    status = normal_equations(Xref, knn, skw, M, ng, Y, Yn, N, lat, opt, sigma, node_T, A, g, &inl,
                              &cost, &sw);
    if (rep) {
        memset(rep, 0, sizeof *rep);
        rep->last_inliers = inl;
        rep->last_cost = cost;
        rep->last_sum_w = sw;
    }
    or_lattice_free(lat);
    return status;
}

/* ---- block-Jacobi preconditioned conjugate gradients ------------------------ */

int or_pcg_block_jacobi(int nb, const double *A, const double *b, int iters, double *x)
{
    const size_t n = 6 * (size_t)nb;
    double *P = (double *)malloc((size_t)nb * 36 * sizeof(double));
    double *r = (double *)malloc(n * sizeof(double));
    double *z = (double *)malloc(n * sizeof(double));
    double *p = (double *)malloc(n * sizeof(double));
    double *Ap = (double *)malloc(n * sizeof(double));
    if (!P || !r || !z || !p || !Ap) {
        free(P); free(r); free(z); free(p); free(Ap);
        return OR_ENOMEM;
    }
    /* P_k = (A_kk)^-1 by Cholesky solves against the unit vectors */
    for (int k = 0; k < nb; ++k) {
        double D[36], e[6], col[6];
        double dmax = 0.0;
        for (int a = 0; a < 6; ++a)
            for (int c = 0; c < 6; ++c) {
                D[6 * a + c] = A[(6 * (size_t)k + a) * n + 6 * (size_t)k + c];
                if (a == c && D[6 * a + c] > dmax)
                    dmax = D[6 * a + c];
            }
        int ok = 1;
        for (int c = 0; c < 6 && ok; ++c) {
            for (int a = 0; a < 6; ++a)
                e[a] = (a == c) ? 1.0 : 0.0;
            if (or_cholesky_solve(6, D, e, col) != 0)
                ok = 0;
            else
                for (int a = 0; a < 6; ++a)
                    P[36 * (size_t)k + 6 * a + c] = col[a];
        }
        if (!ok)
            for (int a = 0; a < 36; ++a)
                P[36 * (size_t)k + a] = (a % 7 == 0) ? (dmax > 0.0 ? 1.0 / dmax : 1.0) : 0.0;
    }
    for (size_t i = 0; i < n; ++i) {
        x[i] = 0.0;
        r[i] = b[i];
    }
    double rz = 0.0;
    for (int k = 0; k < nb; ++k)
        for (int a = 0; a < 6; ++a) {
            double acc = 0.0;
            for (int c = 0; c < 6; ++c)
                acc += P[36 * (size_t)k + 6 * a + c] * r[6 * (size_t)k + c];
            z[6 * (size_t)k + a] = acc;
        }
    for (size_t i = 0; i < n; ++i) {
        p[i] = z[i];
        rz += r[i] * z[i];
    }
    for (int it = 0; it < iters; ++it) {
        if (!(rz > 0.0))
            break;
        double pAp = 0.0;
        for (size_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (size_t j = 0; j < n; ++j)
                acc += A[i * n + j] * p[j];
            Ap[i] = acc;
            pAp += p[i] * acc;
        }
        if (!(pAp > 0.0))
            break;
        const double alpha = rz / pAp;
        for (size_t i = 0; i < n; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        double rz_new = 0.0;
        for (int k = 0; k < nb; ++k)
            for (int a = 0; a < 6; ++a) {
                double acc = 0.0;
                for (int c = 0; c < 6; ++c)
                    acc += P[36 * (size_t)k + 6 * a + c] * r[6 * (size_t)k + c];
                z[6 * (size_t)k + a] = acc;
            }
        for (size_t i = 0; i < n; ++i)
            rz_new += r[i] * z[i];
        const double beta = rz_new / rz;
        for (size_t i = 0; i < n; ++i)
            p[i] = z[i] + beta * p[i];
        rz = rz_new;
    }
    free(P); free(r); free(z); free(p); free(Ap);
    return OR_OK;
}

/* ---- EM driver ----------------------------------------------------------------- */

static void mat4_mul(const double *a, const double *b, double *c)
{
    double t[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc += a[4 * i + k] * b[4 * k + j];
            t[4 * i + j] = acc;
        }
    memcpy(c, t, sizeof t);
}

int or_register_nodegraph(const float *Xref, const int32_t *knn, const float *skw, int64_t M,
                          const or_nodegraph *ng, const float *Y, const float *Yn, int64_t N,
                          const or_options *opt, double *node_T, or_report *rep)
{
    or_report dummy;
    if (!rep)
        rep = &dummy;
    memset(rep, 0, sizeof *rep);
    if (M <= 0 || N <= 0 || ng->K < 1 || ng->E < 0 || !(ng->lambda >= 0.0) || ng->pcg_iters < 0 ||
        opt->iters < 0 || !(opt->sigma_start > 0.0) || !(opt->sigma_end > 0.0) ||
        !(opt->w >= 0.0 && opt->w < 1.0))
        return OR_EINVAL;
    if (opt->residual == OR_PT2PL && !Yn)
        return OR_EINVAL;
    for (int64_t i = 0; i < 4 * M; ++i)
        if (knn[i] < 0 || knn[i] >= ng->K)
            return OR_EINVAL;
    for (int e = 0; e < 2 * ng->E; ++e)
        if (ng->edges[e] < 0 || ng->edges[e] >= ng->K)
            return OR_EINVAL;
    const size_t n = 6 * (size_t)ng->K;
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    float *sched = (float *)malloc((size_t)(opt->iters ? opt->iters : 1) * sizeof(float));
    double *V = obs_values(Y, Yn, N, vdim);
    double *A = (double *)malloc(n * n * sizeof(double));
    double *g = (double *)malloc(n * sizeof(double));
    double *dt = (double *)malloc(n * sizeof(double));
    if (!sched || !V || !A || !g || !dt) {
        free(sched); free(V); free(A); free(g); free(dt);
        return OR_ENOMEM;
    }
    or_sigma_schedule(opt->sigma_start, opt->sigma_end, opt->iters, sched);
    or_lattice *lat = NULL;
    float lat_sigma = 0.0f;
    int status = OR_OK;
    for (int it = 0; it < opt->iters; ++it) {
        const float sigf = sched[it];
        if (opt->backend == OR_LATTICE && (lat == NULL || sigf != lat_sigma)) {
            or_lattice_free(lat);
            lat = or_lattice_build(Y, V, N, vdim, sigf, &status);
            if (!lat || status != OR_OK)
                break;
            if (opt->blur)
                or_lattice_blur(lat);
            lat_sigma = sigf;
        }
        int64_t inl;
        double cost, sw;
        status = normal_equations(Xref, knn, skw, M, ng, Y, Yn, N, lat, opt, (double)sigf, node_T, A,
                                  g, &inl, &cost, &sw);
        if (status != OR_OK)
            break;
        rep->iters_run = it + 1;
        rep->last_inliers = inl;
        rep->last_cost = cost;
        rep->last_sum_w = sw;
        for (size_t i = 0; i < n; ++i)
            g[i] = -g[i];
        status = or_pcg_block_jacobi(ng->K, A, g, ng->pcg_iters, dt);
        if (status != OR_OK)
            break;
        double n2 = 0.0;
        for (int k = 0; k < ng->K; ++k) {
            double E[16];
            or_se3_exp(dt + 6 * (size_t)k, E);
            mat4_mul(E, node_T + 16 * (size_t)k, node_T + 16 * (size_t)k);
        }
        for (size_t i = 0; i < n; ++i)
            n2 += dt[i] * dt[i];
        rep->last_twist_norm = sqrt(n2);
        if (opt->stop_twist > 0.0 && rep->last_twist_norm < opt->stop_twist)
            break;
    }
    or_lattice_free(lat);
    free(sched); free(V); free(A); free(g); free(dt);
    return status;
}
