/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Articulated registration (Section 5.1, Eq. 20, Algorithm 1).
 *
 * Kinematic tree: body 0 is the root, every other body b has a parent p(b) <
 * b.  A body's transform is
 *     T_b = T_{p(b)} * O_b * R(a_{j1}, q_{j1}) * R(a_{j2}, q_{j2}) * ...
 * (T_{p(0)} = the root pose, a 6-DOF SE(3) transform), where O_b is the fixed
 * offset of the body's joint frame in its parent's frame and the body's
 * revolute joints rotate about axes a_j given in the frame they act in.
 * Points are given in their body's frame: x_i = T_{b(i)} x_i_ref (Eq. 15).
 *
 * Motion parameters theta = (root twist (6), joint angles (n_joints)).  The
 * spatial velocity Jacobian of body b (Section 5.1: d zeta_b / d theta, world
 * frame, about the world origin, twist order (omega; v) as in Eq. 16):
 *   - root columns: the identity (the root update T_root <- exp(dz^) T_root
 *     moves every body by the same world twist);
 *   - joint j, for b in the subtree of the joint's body: (a_w; p_w x a_w),
 *     a_w the joint's world axis and p_w a world point on it (rotating by dq
 *     moves x by dq a_w x (x - p_w));
 *   - zero otherwise.
 * The normal equations follow Algorithm 1: per-body J^T J and J^T r sums over
 * the body's points first, then A = sum_b J_sp^T (J^T J)_b J_sp and
 * g = sum_b J_sp^T (J^T r)_b.  One Gauss-Newton step per EM
 * iteration, solved by Cholesky; the root is updated by the exponential, the
 * joints additively and clamped to their limits.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

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

/* Rotation by angle q about unit axis a (Rodrigues), as a 4x4 transform. */
static void axis_rotation(const double a[3], double q, double R[16])
{
    double c = cos(q), s = sin(q), v = 1.0 - c;
    memset(R, 0, 16 * sizeof(double));
    R[0] = c + a[0] * a[0] * v;
    R[1] = a[0] * a[1] * v - a[2] * s;
    R[2] = a[0] * a[2] * v + a[1] * s;
    R[4] = a[1] * a[0] * v + a[2] * s;
    R[5] = c + a[1] * a[1] * v;
    R[6] = a[1] * a[2] * v - a[0] * s;
    R[8] = a[2] * a[0] * v - a[1] * s;
    R[9] = a[2] * a[1] * v + a[0] * s;
    R[10] = c + a[2] * a[2] * v;
    R[15] = 1.0;
}

int or_fk(const or_kintree *t, const double root_T[16], const double *q, double *T,
          double *axis_w, double *point_w)
{
    int j = 0;
    for (int b = 0; b < t->nb; ++b) {
        double F[16];
        if (b == 0) {
            memcpy(F, root_T, sizeof F);
        } else {
            if (t->parent[b] < 0 || t->parent[b] >= b)
                return OR_EINVAL;
            memcpy(F, T + 16 * t->parent[b], sizeof F);
        }
        mat4_mul(F, t->offset + 16 * b, F);
        for (; j < t->nj && t->joint_body[j] == b; ++j) {
            const double *a = t->joint_axis + 3 * j;
            for (int r = 0; r < 3; ++r) {
                if (axis_w)
                    axis_w[3 * j + r] = F[4 * r] * a[0] + F[4 * r + 1] * a[1] + F[4 * r + 2] * a[2];
                if (point_w)
                    point_w[3 * j + r] = F[4 * r + 3];
            }
            double R[16];
            axis_rotation(a, q[j], R);
            mat4_mul(F, R, F);
        }
        memcpy(T + 16 * b, F, sizeof F);
    }
    return j == t->nj ? OR_OK : OR_EINVAL;
}

static int is_in_subtree(const or_kintree *t, int b, int a)
{
    for (int x = b; x >= 0; x = (x == 0) ? -1 : t->parent[x])
        if (x == a)
            return 1;
    return 0;
}

int or_spatial_jacobian(const or_kintree *t, const double *axis_w, const double *point_w, int b,
                        double *Jsp)
{
    const int nd = 6 + t->nj;
    memset(Jsp, 0, 6 * (size_t)nd * sizeof(double));
    for (int p = 0; p < 6; ++p)
        Jsp[p * nd + p] = 1.0;
    for (int j = 0; j < t->nj; ++j) {
        if (!is_in_subtree(t, b, t->joint_body[j]))
            continue;
        const double *a = axis_w + 3 * j, *pw = point_w + 3 * j;
        const double v[3] = {pw[1] * a[2] - pw[2] * a[1], pw[2] * a[0] - pw[0] * a[2],
                             pw[0] * a[1] - pw[1] * a[0]};
        for (int r = 0; r < 3; ++r) {
            Jsp[r * nd + 6 + j] = a[r];
            Jsp[(3 + r) * nd + 6 + j] = v[r];
        }
    }
    return OR_OK;
}

/* Observation values [1, y (, n)] for splatting. */
static double *obs_values(const float *Y, const float *Yn, int64_t N, int vdim)
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
    }
    return V;
}

/* Per-body sums (Algorithm 1, first part) at the current pose, then the
 * assembled A (nd x nd) and g (nd).  Returns the number of inliers via
 * *inliers and the weighted cost via *cost. */
static int normal_equations(const float *Xref, const int32_t *body, int64_t M, const or_kintree *t,
                            const float *Y, const float *Yn, int64_t N, const or_lattice *lat,
                            const or_options *opt, double sigma, const double *Tb,
                            const double *axis_w, const double *point_w, double *A, double *g,
                            int64_t *inliers, double *cost, double *sum_w)
{
    const int nd = 6 + t->nj;
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    double *H = (double *)calloc((size_t)t->nb * 36, sizeof(double));
    double *h = (double *)calloc((size_t)t->nb * 6, sizeof(double));
    double *Jsp = (double *)malloc(6 * (size_t)nd * sizeof(double));
    if (!H || !h || !Jsp) {
        free(H); free(h); free(Jsp);
        return OR_ENOMEM;
    }
    const double c_eff = or_outlier_constant(opt->w, N, M, sigma, opt->backend, opt->blur);
    *inliers = 0;
    *cost = 0.0;
    *sum_w = 0.0;
    int status = OR_OK;
    for (int64_t i = 0; i < M; ++i) {
        const int b = body[i];
        if (b < 0 || b >= t->nb) {
            status = OR_EINVAL;
            continue;
        }
        const double *T = Tb + 16 * b;
        const float *p = Xref + 4 * i;
        double x[3];
        for (int a = 0; a < 3; ++a)
            x[a] = T[4 * a] * p[0] + T[4 * a + 1] * p[1] + T[4 * a + 2] * p[2] + T[4 * a + 3];
        double e[7] = {0, 0, 0, 0, 0, 0, 0};
        if (opt->backend == OR_LATTICE) {
            float xf[4] = {(float)x[0], (float)x[1], (float)x[2], 0.0f};
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
        int rows = or_point_terms(x, e[0], e + 1, Ns, c_eff, sigma, opt->residual,
                                  opt->renormalize_normals, &W, r, J);
        if (rows == 0)
            continue;
        ++*inliers;
        *sum_w += W;
        for (int a = 0; a < rows; ++a) {
            *cost += r[a] * r[a];
            for (int pp = 0; pp < 6; ++pp) {
                h[6 * b + pp] += J[6 * a + pp] * r[a];
                for (int qq = 0; qq < 6; ++qq)
                    H[36 * b + 6 * pp + qq] += J[6 * a + pp] * J[6 * a + qq];
            }
        }
    }
    memset(A, 0, (size_t)nd * nd * sizeof(double));
    memset(g, 0, (size_t)nd * sizeof(double));
    for (int b = 0; b < t->nb; ++b) {
        or_spatial_jacobian(t, axis_w, point_w, b, Jsp);
        for (int i = 0; i < nd; ++i) {
            for (int pp = 0; pp < 6; ++pp) {
                const double jpi = Jsp[pp * nd + i];
                if (jpi == 0.0)
                    continue;
                g[i] += jpi * h[6 * b + pp];
                for (int qq = 0; qq < 6; ++qq) {
                    const double hq = jpi * H[36 * b + 6 * pp + qq];
                    if (hq == 0.0)
                        continue;
                    for (int j = 0; j < nd; ++j)
                        A[i * nd + j] += hq * Jsp[qq * nd + j];
                }
            }
        }
    }
    free(H); free(h); free(Jsp);
    return status;
}

int or_articulated_normal_equations(const float *Xref, const int32_t *body, int64_t M,
                                    const or_kintree *t, const float *Y, const float *Yn,
                                    int64_t N, const or_options *opt, double sigma,
                                    const double root_T[16], const double *q, double *A,
                                    double *g)
{
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    double *Tb = (double *)malloc((size_t)t->nb * 16 * sizeof(double));
    double *aw = (double *)malloc((size_t)(t->nj ? t->nj : 1) * 3 * sizeof(double));
    double *pw = (double *)malloc((size_t)(t->nj ? t->nj : 1) * 3 * sizeof(double));
    int status = (Tb && aw && pw) ? or_fk(t, root_T, q, Tb, aw, pw) : OR_ENOMEM;
    or_lattice *lat = NULL;
    if (status == OR_OK && opt->backend == OR_LATTICE) {
        double *V = obs_values(Y, Yn, N, vdim);
        lat = V ? or_lattice_build(Y, V, N, vdim, (float)sigma, &status) : NULL;
        free(V);
        if (lat && opt->blur)
            or_lattice_blur(lat);
    }
    if (status == OR_OK) {
        int64_t inl;
        double cost, sw;
        status = normal_equations(Xref, body, M, t, Y, Yn, N, lat, opt, sigma, Tb, aw, pw, A, g,
                                  &inl, &cost, &sw);
    }
    or_lattice_free(lat);
    free(Tb); free(aw); free(pw);
    return status;
}

int or_register_articulated(const float *Xref, const int32_t *body, int64_t M,
                            const or_kintree *t, const float *Y, const float *Yn, int64_t N,
                            const or_options *opt, double root_T[16], double *q, or_report *rep)
{
    or_report dummy;
    if (!rep)
        rep = &dummy;
    memset(rep, 0, sizeof *rep);
    if (M <= 0 || N <= 0 || t->nb < 1 || t->nj < 0 || 6 + t->nj > 64 || opt->iters < 0 ||
        !(opt->sigma_start > 0.0) || !(opt->sigma_end > 0.0) || !(opt->w >= 0.0 && opt->w < 1.0))
        return OR_EINVAL;
    if (opt->residual == OR_PT2PL && !Yn)
        return OR_EINVAL;
    const int nd = 6 + t->nj;
    const int vdim = (opt->residual == OR_PT2PL) ? 7 : 4;
    float *sched = (float *)malloc((size_t)(opt->iters ? opt->iters : 1) * sizeof(float));
    double *V = obs_values(Y, Yn, N, vdim);
    double *Tb = (double *)malloc((size_t)t->nb * 16 * sizeof(double));
    double *aw = (double *)malloc((size_t)(t->nj ? t->nj : 1) * 3 * sizeof(double));
    double *pw = (double *)malloc((size_t)(t->nj ? t->nj : 1) * 3 * sizeof(double));
    double *A = (double *)malloc((size_t)nd * nd * sizeof(double));
    double *g = (double *)malloc((size_t)nd * sizeof(double));
    double *dt = (double *)malloc((size_t)nd * sizeof(double));
    if (!sched || !V || !Tb || !aw || !pw || !A || !g || !dt) {
        free(sched); free(V); free(Tb); free(aw); free(pw); free(A); free(g); free(dt);
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
        status = or_fk(t, root_T, q, Tb, aw, pw);
        if (status != OR_OK)
            break;
        int64_t inl;
        double cost, sw;
        status = normal_equations(Xref, body, M, t, Y, Yn, N, lat, opt, (double)sigf, Tb, aw, pw,
                                  A, g, &inl, &cost, &sw);
        if (status != OR_OK)
            break;
        rep->iters_run = it + 1;
        rep->last_inliers = inl;
        rep->last_cost = cost;
        rep->last_sum_w = sw;
        for (int i = 0; i < nd; ++i)
            g[i] = -g[i];
        if (or_cholesky_solve(nd, A, g, dt) != 0) {
            ++rep->degenerate_iters;
            continue;
        }
        double E[16];
        or_se3_exp(dt, E);
        mat4_mul(E, root_T, root_T);
        for (int j = 0; j < t->nj; ++j) {
            q[j] += dt[6 + j];
            if (q[j] < t->q_min[j])
                q[j] = t->q_min[j];
            if (q[j] > t->q_max[j])
                q[j] = t->q_max[j];
        }
        double n2 = 0.0;
        for (int i = 0; i < nd; ++i)
            n2 += dt[i] * dt[i];
        rep->last_twist_norm = sqrt(n2);
        if (opt->stop_twist > 0.0 && rep->last_twist_norm < opt->stop_twist)
            break;
    }
    or_lattice_free(lat);
    free(sched); free(V); free(Tb); free(aw); free(pw); free(A); free(g); free(dt);
    return status;
}
