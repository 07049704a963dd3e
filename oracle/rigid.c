/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Rigid registration by EM (Section 3.1) with the twist Gauss-Newton M step
 * (Section 5), following the paper's steps in order:
 *
 *   for each EM iteration:
 *     E step   M0, M1 (Eq. 6) and, for point-to-plane, the normal sums of
 *              Eq. 9, at the model points x_i = T x_i_ref, either summed
 *              exactly or read off the permutohedral lattice built over the
 *              observation (Section 4, the augmentation of Eq. 13-14 making X
 *              a pure query).
 *     M step   one Gauss-Newton step on Eq. 7 (point-to-point) or Eq. 10
 *              (point-to-plane): A = sum J^T J, b = sum J^T r (Eq. 17-18),
 *              rigid model so d zeta / d theta = I (Section 5), and
 *              delta zeta = -A^{-1} b.
 *     update   T <- exp(delta zeta^) T (Eq. 16, applied as the exponential).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - dx/d zeta follows the twist matrix of Eq. 16: delta x = omega x x + v,
 *     i.e. [-[x]_x, I] (the prose "skew(x)" has the opposite sign).
 *   - The outlier constant c = w/(1-w) N/M of Eq. 7 belongs to normalised
 *     Gaussians; with the unnormalised kernel of Eq. 11 it becomes
 *     c sigma^3 G, G the kernel's integral in feature units.
 *   - Residuals carry Sigma^{-1/2} = 1/sigma (Eq. 7); Eq. 10 omits it, and it
 *     cancels in the rigid step anyway.
 *   - N_x of Eq. 9 is used as written (divided by M0, not unit-normalised)
 *     unless renormalize_normals is set.
 *   - A model point with M0 <= 0 has no defined target and is skipped.
 *   - One Gauss-Newton step per EM iteration; the lattice is rebuilt only when
 *     sigma changes (Section 3.2: the index is built once for a fixed sigma).
 *   - sigma as a decision variable (Section 3.3; its closed form is in the
 *     missing supplement), point-to-point: with the E step's posteriors
 *     P_ij = K_ij / (M0_i + c), maximising the expected complete-data
 *     log-likelihood sum_ij P_ij [-|x_i - y_j|^2 / (2 sigma^2) - 3 log sigma]
 *     over sigma gives
 *       sigma^2 = sum_i Q_i / (M0_i + c) / (3 sum_i W_i),
 *       Q_i = sum_j K_ij |x_i - y_j|^2 = M0_i |x_i|^2 - 2 x_i . M1_i + M2_i,
 *     M2_i = sum_j K_ij |y_j|^2 (one more splat channel, |y|^2), W_i as in
 *     Eq. 7.  It is taken from the same E step as the Gauss-Newton step (a
 *     conditional maximisation over sigma at the current pose), floored at
 *     sigma_end, rounded to float and used from the next iteration on.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

double or_outlier_constant(double w, int64_t N, int64_t M, double sigma, int backend, int blur)
{
    double c = (w / (1.0 - w)) * ((double)N / (double)M);
    return c * sigma * sigma * sigma * or_kernel_mass(backend, blur);
}

int or_point_terms(const double x[3], double M0, const double M1[3], const double Ns[3],
                   double c_eff, double sigma, int residual, int renormalize,
                   double *W, double *r, double *J)
{
    *W = 0.0;
    if (!(M0 > 0.0))
        return 0;
    double w = M0 / (M0 + c_eff);
    *W = w;
    double sw = sqrt(w) / sigma;
    double e[3];
    for (int a = 0; a < 3; ++a)
        e[a] = x[a] - M1[a] / M0; /* x minus the weight-averaged target */
    if (residual == OR_PT2PT) {
        /* r = sqrt(W)/sigma (x - t), dr/dzeta = sqrt(W)/sigma [-[x]_x, I]. */
        double Jx[3][6] = {
            {0.0, x[2], -x[1], 1.0, 0.0, 0.0},
            {-x[2], 0.0, x[0], 0.0, 1.0, 0.0},
            {x[1], -x[0], 0.0, 0.0, 0.0, 1.0},
        };
        for (int a = 0; a < 3; ++a) {
            r[a] = sw * e[a];
            for (int p = 0; p < 6; ++p)
                J[6 * a + p] = sw * Jx[a][p];
        }
        return 3;
    }
    double n[3];
    for (int a = 0; a < 3; ++a)
        n[a] = Ns[a] / M0;
    if (renormalize) {
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nn > 0.0))
            return 0;
        for (int a = 0; a < 3; ++a)
            n[a] /= nn;
    }
    /* r = sqrt(W)/sigma n.(x - t); n^T [-[x]_x, I] = [(x cross n)^T, n^T]. */
    r[0] = sw * (n[0] * e[0] + n[1] * e[1] + n[2] * e[2]);
    double xn[3] = {x[1] * n[2] - x[2] * n[1], x[2] * n[0] - x[0] * n[2], x[0] * n[1] - x[1] * n[0]};
    for (int a = 0; a < 3; ++a) {
        J[a] = sw * xn[a];
        J[3 + a] = sw * n[a];
    }
    return 1;
}

/* Points per fixed summation chunk of the Gauss-Newton sums, and the values
 * each chunk carries. */
#define GN_CHUNK 4096
#define GN_VALS 46

static void transform_point(const double T[16], const float *p, double x[3])
{
    for (int a = 0; a < 3; ++a)
        x[a] = T[4 * a] * p[0] + T[4 * a + 1] * p[1] + T[4 * a + 2] * p[2] + T[4 * a + 3];
}

static void mat4_mul(const double *a, const double *b, double *c)
{
    double t[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k)
                s += a[4 * i + k] * b[4 * k + j];
            t[4 * i + j] = s;
        }
    memcpy(c, t, sizeof t);
}

/* E-step sums for all model points at pose T; out is M x vdim. */
static int estep_at(const float *X, int64_t M, const float *Y, const float *Yn, int64_t N,
                    int backend, const or_lattice *lat, double sigma, const double T[16],
                    int vdim, double *out)
{
    float *xs = (float *)malloc((size_t)(M ? M : 1) * 4 * sizeof(float));
    if (!xs)
        return OR_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
        double x[3];
        transform_point(T, X + 4 * i, x);
        for (int a = 0; a < 3; ++a)
            xs[4 * i + a] = (float)x[a];
        xs[4 * i + 3] = 0.0f;
    }
    int status = OR_OK;
    if (backend == OR_LATTICE) {
        status = or_lattice_slice(lat, xs, M, out);
    } else {
        /* The exact sums use the double-precision moved points. */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < M; ++i) {
            double x[3], m0, m1[3], ns[3];
            transform_point(T, X + 4 * i, x);
            or_exact_sums_at(x, Y, Yn, N, sigma, &m0, m1, ns);
            out[i * vdim] = m0;
            for (int c = 0; c < 3; ++c)
                out[i * vdim + 1 + c] = m1[c];
            if (vdim == 7)
                for (int c = 0; c < 3; ++c)
                    out[i * vdim + 4 + c] = ns[c];
            if (vdim == 5) { /* M2 = sum_k K |y_k|^2 */
                const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
                double m2 = 0.0;
                for (int64_t k = 0; k < N; ++k) {
                    const double d0 = x[0] - Y[4 * k], d1 = x[1] - Y[4 * k + 1], d2 = x[2] - Y[4 * k + 2];
                    const double yy = (double)Y[4 * k] * Y[4 * k] + (double)Y[4 * k + 1] * Y[4 * k + 1] +
                                      (double)Y[4 * k + 2] * Y[4 * k + 2];
                    m2 += exp(-(d0 * d0 + d1 * d1 + d2 * d2) * inv2s2) * yy;
                }
                out[i * vdim + 4] = m2;
            }
        }
    }
    free(xs);
    return status;
}

/* Observation values [1, y (, n)] of Eq. 11's v_y, for splatting. */
static double *observation_values(const float *Y, const float *Yn, int64_t N, int vdim)
{
    double *V = (double *)malloc((size_t)(N ? N : 1) * vdim * sizeof(double));
    if (!V)
        return NULL;
    for (int64_t k = 0; k < N; ++k) {
        V[k * vdim] = 1.0;
        for (int c = 0; c < 3; ++c)
            V[k * vdim + 1 + c] = Y[4 * k + c];
        if (vdim == 7)
            for (int c = 0; c < 3; ++c)
                V[k * vdim + 4 + c] = Yn[4 * k + c];
        if (vdim == 5) /* |y|^2, for the sigma update */
            V[k * vdim + 4] = (double)Y[4 * k] * Y[4 * k] + (double)Y[4 * k + 1] * Y[4 * k + 1] +
                              (double)Y[4 * k + 2] * Y[4 * k + 2];
    }
    return V;
}

int or_estep(const float *X, int64_t M, const float *Y, const float *Yn, int64_t N,
             int backend, int blur, double sigma, const double T[16], double *out)
{
    const int vdim = Yn ? 7 : 4;
    or_lattice *lat = NULL;
    int status = OR_OK;
    if (backend == OR_LATTICE) {
        double *V = observation_values(Y, Yn, N, vdim);
        if (!V)
            return OR_ENOMEM;
        lat = or_lattice_build(Y, V, N, vdim, (float)sigma, &status);
        free(V);
        if (!lat)
            return status;
        if (blur)
            or_lattice_blur(lat);
    }
    int s2 = estep_at(X, M, Y, Yn, N, backend, lat, sigma, T, vdim, out);
    or_lattice_free(lat);
    return status != OR_OK ? status : s2;
}

/* The Gauss-Newton sums of Eq. 17-18 at pose T from the E-step sums es
 * (M x vdim): out = A (36, row-major), b (6), sum of weights, cost, inliers,
 * and the sigma moment sum_i Q_i / (M0_i + c) (update_sigma).  Each fixed
 * chunk of GN_CHUNK points is summed in point order, then the chunk sums in
 * chunk order -- the same result whatever the number of threads. */
static int gn_sums(const float *X, int64_t M, const double *es, int vdim, const double T[16],
                   double c_eff, double sigma, const or_options *opt, double out[GN_VALS])
{
    const int64_t nchunk = (M + GN_CHUNK - 1) / GN_CHUNK;
    double *part = (double *)calloc((size_t)(nchunk ? nchunk : 1) * GN_VALS, sizeof(double));
    if (!part)
        return OR_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t ch = 0; ch < nchunk; ++ch) {
        double *q = part + ch * GN_VALS; /* A (36), b (6), sum_w, cost, inliers, sum_q */
        const int64_t i1 = (ch + 1) * GN_CHUNK < M ? (ch + 1) * GN_CHUNK : M;
        for (int64_t i = ch * GN_CHUNK; i < i1; ++i) {
            double x[3];
            transform_point(T, X + 4 * i, x);
            const double *e = es + i * vdim;
            double Ns[3] = {0, 0, 0};
            if (vdim == 7)
                for (int c = 0; c < 3; ++c)
                    Ns[c] = e[4 + c];
            double Wt, r[3], J[18];
            int rows = or_point_terms(x, e[0], e + 1, Ns, c_eff, sigma, opt->residual,
                                      opt->renormalize_normals, &Wt, r, J);
            if (rows == 0)
                continue;
            q[44] += 1.0;
            q[42] += Wt;
            if (opt->update_sigma) { /* Q_i / (M0_i + c) */
                const double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
                const double xm = x[0] * e[1] + x[1] * e[2] + x[2] * e[3];
                q[45] += (e[0] * xx - 2.0 * xm + e[4]) / (e[0] + c_eff);
            }
            for (int a = 0; a < rows; ++a) {
                q[43] += r[a] * r[a];
                for (int p = 0; p < 6; ++p) {
                    q[36 + p] += J[6 * a + p] * r[a];
                    for (int qq = 0; qq < 6; ++qq)
                        q[6 * p + qq] += J[6 * a + p] * J[6 * a + qq];
                }
            }
        }
    }
    for (int v = 0; v < GN_VALS; ++v)
        out[v] = 0.0;
    for (int64_t ch = 0; ch < nchunk; ++ch) {
        const double *q = part + ch * GN_VALS;
        for (int v = 0; v < 36; ++v)
            out[v] += q[v];
        for (int p = 0; p < 6; ++p)
            out[36 + p] += q[36 + p];
        out[42] += q[42];
        out[43] += q[43];
        out[44] += q[44];
        out[45] += q[45];
    }
    free(part);
    return OR_OK;
}

int or_register_rigid(const float *X, int64_t M, const float *Y, const float *Yn,
                      int64_t N, const or_options *opt, double T[16], or_report *rep)
{
    or_report dummy;
    if (!rep)
        rep = &dummy;
    memset(rep, 0, sizeof *rep);
    if (M <= 0 || N <= 0 || opt->iters < 0 || !(opt->sigma_start > 0.0) ||
        !(opt->sigma_end > 0.0) || !(opt->w >= 0.0 && opt->w < 1.0))
        return OR_EINVAL;
    if (opt->residual == OR_PT2PL && !Yn)
        return OR_EINVAL;
    if (opt->update_sigma && (opt->residual != OR_PT2PT || opt->blur))
        return OR_EINVAL; /* the sigma update is derived for point-to-point without blur */
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : (opt->update_sigma ? 5 : 4);

    float *sched = (float *)malloc((size_t)(opt->iters ? opt->iters : 1) * sizeof(float));
    double *V = observation_values(Y, Yn, N, vdim);
    double *es = (double *)malloc((size_t)M * vdim * sizeof(double));
    if (!sched || !V || !es) {
        free(sched); free(V); free(es);
        return OR_ENOMEM;
    }
    or_sigma_schedule(opt->sigma_start, opt->sigma_end, opt->iters, sched);

    or_lattice *lat = NULL;
    float lat_sigma = 0.0f;
    int status = OR_OK;
    float sig_upd = (float)opt->sigma_start; /* the updated sigma (update_sigma) */
    for (int it = 0; it < opt->iters; ++it) {
        const float sigf = opt->update_sigma ? sig_upd : sched[it];
        rep->last_sigma = sigf;
        const double sigma = (double)sigf;
        if (opt->backend == OR_LATTICE && (lat == NULL || sigf != lat_sigma)) {
            or_lattice_free(lat);
            lat = or_lattice_build(Y, V, N, vdim, sigf, &status);
            if (!lat || status != OR_OK)
                break;
            if (opt->blur)
                or_lattice_blur(lat);
            lat_sigma = sigf;
        }
        status = estep_at(X, M, Y, Yn, N, opt->backend, lat, sigma, T, vdim, es);
        if (status != OR_OK)
            break;

        const double c_eff = or_outlier_constant(opt->w, N, M, sigma, opt->backend, opt->blur);
        double g[GN_VALS];
        status = gn_sums(X, M, es, vdim, T, c_eff, sigma, opt, g);
        if (status != OR_OK)
            break;
        double A[36], b[6];
        memcpy(A, g, sizeof A);
        memcpy(b, g + 36, sizeof b);
        const double sum_w = g[42], cost = g[43], sum_q = g[45];
        const int64_t inliers = (int64_t)g[44];
        if (opt->update_sigma && sum_w > 0.0) {
            /* the lattice kernel's per-axis variance is kappa sigma^2, not
             * sigma^2: the sigma at which it matches the residuals */
            const double kappa = opt->backend == OR_LATTICE ? or_lattice_kernel_variance() : 1.0;
            const double s2 = sum_q / (3.0 * sum_w * kappa);
            rep->sigma_next = sqrt(s2 > 0.0 ? s2 : 0.0);
            const double fl = opt->sigma_end;
            sig_upd = (float)(rep->sigma_next > fl ? rep->sigma_next : fl);
        }
        rep->iters_run = it + 1;
        rep->last_inliers = inliers;
        rep->last_sum_w = sum_w;
        rep->last_cost = cost;

        double nb[6], dz[6];
        for (int p = 0; p < 6; ++p)
            nb[p] = -b[p];
        if (or_cholesky_solve(6, A, nb, dz) != 0) {
            ++rep->degenerate_iters;
            continue;
        }
        double dT[16];
        or_se3_exp(dz, dT);
        mat4_mul(dT, T, T);
        double nrm = 0.0;
        for (int p = 0; p < 6; ++p)
            nrm += dz[p] * dz[p];
        rep->last_twist_norm = sqrt(nrm);
        if (opt->stop_twist > 0.0 && rep->last_twist_norm < opt->stop_twist)
            break;
    }
    or_lattice_free(lat);
    free(sched);
    free(V);
    free(es);
    return status;
}

/* One EM iteration's normal equations for a shard of the model (X, M points
 * of a model of M_total): the E step at sigma_start and pose T, the
 * Gauss-Newton sums with Eq. 7's outlier constant from M_total.  ne = A's
 * upper triangle row by row (21), b (6), sum of weights, cost, inliers. */
int or_rigid_normal_equations(const float *X, int64_t M, const float *Y, const float *Yn, int64_t N,
                              const or_options *opt, int64_t M_total, const double T[16], double ne[30])
{
    if (M <= 0 || N <= 0 || M_total < M || !(opt->sigma_start > 0.0) || !(opt->w >= 0.0 && opt->w < 1.0))
        return OR_EINVAL;
    if (opt->residual == OR_PT2PL && !Yn)
        return OR_EINVAL;
    if (opt->update_sigma)
        return OR_EINVAL;
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    const float sigf = (float)opt->sigma_start;
    const double sigma = (double)sigf;
    double *V = observation_values(Y, opt->residual == OR_PT2PL ? Yn : NULL, N, vdim);
    double *es = (double *)malloc((size_t)M * vdim * sizeof(double));
    if (!V || !es) {
        free(V);
        free(es);
        return OR_ENOMEM;
    }
    int status = OR_OK;
    or_lattice *lat = NULL;
    if (opt->backend == OR_LATTICE) {
        lat = or_lattice_build(Y, V, N, vdim, sigf, &status);
        if (lat && status == OR_OK && opt->blur)
            or_lattice_blur(lat);
    }
    if (status == OR_OK && (lat || opt->backend != OR_LATTICE))
        status = estep_at(X, M, Y, Yn, N, opt->backend, lat, sigma, T, vdim, es);
    double g[GN_VALS];
    if (status == OR_OK) {
        const double c_eff = or_outlier_constant(opt->w, N, M_total, sigma, opt->backend, opt->blur);
        status = gn_sums(X, M, es, vdim, T, c_eff, sigma, opt, g);
    }
    if (status == OR_OK) {
        int t = 0;
        for (int p = 0; p < 6; ++p)
            for (int q = p; q < 6; ++q)
                ne[t++] = g[6 * p + q];
        for (int p = 0; p < 6; ++p)
            ne[21 + p] = g[36 + p];
        ne[27] = g[42];
        ne[28] = g[43];
        ne[29] = g[44];
    }
    or_lattice_free(lat);
    free(V);
    free(es);
    return status;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
#else
    (void)n;
#endif
}

double or_align_error(const float *X, int64_t M, const double T[16], const double Tgt[16])
{
    double s = 0.0;
    for (int64_t i = 0; i < M; ++i) {
        double a[3], b[3];
        transform_point(T, X + 4 * i, a);
        transform_point(Tgt, X + 4 * i, b);
        s += sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                  (a[2] - b[2]) * (a[2] - b[2]));
    }
    return M ? s / (double)M : 0.0;
}
