/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The permutohedral lattice for d-dimensional features (1 <= d <= 7), and the
 * feature-space E step of Eq. feature_estep (Section 3.3): the kernel is a
 * Gaussian in feature space with diagonal covariance Sigma_f, the values are
 * the observation's [1, y] (and its normals for point-to-plane).  Section 4.2
 * normalises features to identity covariance before filtering: g_c = f_c /
 * sigma_c.  The lattice construction is the d = 3 one of lattice.c written
 * for any d (Adams et al. 2010, which Section 4.2 adopts):
 *   - elevation z = alpha E g into the hyperplane sum(z) = 0 of R^(d+1), with
 *     z_j = sum_{i > j} c_i - j c_j, c_i = g_i alpha / sqrt(i (i+1)),
 *     alpha = sqrt(2/3) (d+1);
 *   - the nearest remainder-0 point (d+1) round(z_j / (d+1)), the ranks of the
 *     differences (descending, ties to the lower index), the repair of the
 *     coordinate sum, barycentric weights from the ranked differences and the
 *     d+1 vertices, vertex k having every coordinate congruent to k mod (d+1).
 * Every float step is one IEEE operation in a fixed order (compiled with
 * -ffp-contract=off); z / (d+1) is an IEEE division (for d = 3 it equals the
 * exact multiplication by 1/4 of lattice.c, so the two agree bit for bit).
 * Splat and slice sums are in double; the vertex set is kept key-sorted and
 * searched by bisection.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define DMAX (OR_FEATURE_DMAX + 1) /* largest lattice dimension */
#define KEY_LIMIT_D 1000000.0f

typedef struct {
    float z[DMAX];
    int32_t r0[DMAX];
    int32_t rank[DMAX];
    float b[DMAX];
    int32_t key[DMAX][DMAX]; /* key[k][j]: coordinate j of vertex k */
} simplex_d;

void or_feature_scale(int d, const float *sigma_f, float *scale)
{
    const double alpha = sqrt(2.0 / 3.0) * (double)(d + 1);
    for (int i = 1; i <= d; ++i)
        scale[i - 1] = (float)(alpha / sqrt((double)(i * (i + 1))) / (double)sigma_f[i - 1]);
}

/* Embed one d-dimensional feature; 0 if non-finite or out of the key range. */
static int embed_d(int d, const float *f, const float *s, simplex_d *o)
{
    const int D = d + 1;
    float c[DMAX];
    for (int i = 1; i <= d; ++i)
        c[i] = f[i - 1] * s[i - 1];
    float t = 0.0f;
    for (int i = d; i >= 1; --i) {
        o->z[i] = t - (float)i * c[i];
        t = t + c[i];
    }
    o->z[0] = t;
    for (int j = 0; j < D; ++j)
        if (!(fabsf(o->z[j]) < KEY_LIMIT_D))
            return 0;

    int sum = 0;
    for (int j = 0; j < D; ++j) {
        float q = rintf(o->z[j] / (float)D);
        o->r0[j] = (int32_t)q * D;
        sum += (int32_t)q;
    }
    float delta[DMAX];
    for (int j = 0; j < D; ++j)
        delta[j] = o->z[j] - (float)o->r0[j];
    for (int j = 0; j < D; ++j) {
        int r = 0;
        for (int k = 0; k < D; ++k)
            if (delta[k] > delta[j] || (k < j && delta[k] == delta[j]))
                ++r;
        o->rank[j] = r;
    }
    if (sum > D || sum < -D)
        return 0;
    if (sum > 0) {
        for (int j = 0; j < D; ++j) {
            if (o->rank[j] >= D - sum) {
                o->r0[j] -= D;
                o->rank[j] += sum - D;
            } else {
                o->rank[j] += sum;
            }
        }
    } else if (sum < 0) {
        for (int j = 0; j < D; ++j) {
            if (o->rank[j] < -sum) {
                o->r0[j] += D;
                o->rank[j] += D + sum;
            } else {
                o->rank[j] += sum;
            }
        }
    }
    float b[DMAX + 1];
    for (int k = 0; k <= D; ++k)
        b[k] = 0.0f;
    for (int j = 0; j < D; ++j) {
        float v = (o->z[j] - (float)o->r0[j]) / (float)D;
        b[D - 1 - o->rank[j]] += v;
        b[D - o->rank[j]] -= v;
    }
    b[0] = b[0] + (1.0f + b[D]);
    for (int k = 0; k < D; ++k)
        o->b[k] = b[k];
    for (int k = 0; k < D; ++k)
        for (int j = 0; j < D; ++j)
            o->key[k][j] = o->r0[j] + k - (o->rank[j] > D - 1 - k ? D : 0);
    return 1;
}

int or_feature_embed(const float *F, int64_t n, int d, const float *scale, int32_t *keys, float *bary)
{
    if (d < 1 || d > OR_FEATURE_DMAX)
        return OR_EINVAL;
    const int D = d + 1;
    int status = OR_OK;
    for (int64_t i = 0; i < n; ++i) {
        simplex_d sx;
        if (!embed_d(d, F + (size_t)d * i, scale, &sx)) {
            status = OR_EINVAL;
            memset(&sx, 0, sizeof sx);
        }
        for (int k = 0; k < D; ++k) {
            if (keys)
                for (int j = 0; j < D; ++j)
                    keys[((size_t)i * D + k) * D + j] = sx.key[k][j];
            if (bary)
                bary[(size_t)i * D + k] = sx.b[k];
        }
    }
    return status;
}

/* ---- the lattice over d-dimensional features: a key-sorted vertex array ---- */

struct or_flattice {
    int d, vdim;
    int64_t nv;
    float scale[OR_FEATURE_DMAX];
    int32_t *keys; /* nv x (d+1) */
    double *vals;  /* nv x vdim */
};

typedef struct {
    int32_t key[DMAX];
    int64_t src;
    int32_t k;
    float b;
} fentry;

static int g_cmp_dim; /* lattice dimension of the entries being sorted (qsort has no context) */

static int cmp_keyd(const int32_t *a, const int32_t *b, int D)
{
    for (int j = 0; j < D; ++j) {
        if (a[j] < b[j])
            return -1;
        if (a[j] > b[j])
            return 1;
    }
    return 0;
}

static int cmp_fentry(const void *pa, const void *pb)
{
    const fentry *a = (const fentry *)pa, *b = (const fentry *)pb;
    int c = cmp_keyd(a->key, b->key, g_cmp_dim);
    if (c)
        return c;
    if (a->src != b->src)
        return a->src < b->src ? -1 : 1;
    return a->k - b->k;
}

static int64_t find_vertex_d(const or_flattice *lat, const int32_t *key)
{
    const int D = lat->d + 1;
    int64_t lo = 0, hi = lat->nv - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = cmp_keyd(lat->keys + (size_t)D * mid, key, D);
        if (c == 0)
            return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

or_flattice *or_flattice_build(const float *F, int64_t n, int d, const float *scale, const double *V,
                               int vdim, int *status)
{
    *status = OR_OK;
    if (d < 1 || d > OR_FEATURE_DMAX) {
        *status = OR_EINVAL;
        return NULL;
    }
    const int D = d + 1;
    or_flattice *lat = (or_flattice *)calloc(1, sizeof *lat);
    if (!lat) {
        *status = OR_ENOMEM;
        return NULL;
    }
    lat->d = d;
    lat->vdim = vdim;
    memcpy(lat->scale, scale, (size_t)d * sizeof(float));
    fentry *e = (fentry *)malloc((size_t)(n ? n : 1) * D * sizeof *e);
    if (!e) {
        free(lat);
        *status = OR_ENOMEM;
        return NULL;
    }
    int64_t ne = 0;
    for (int64_t i = 0; i < n; ++i) {
        simplex_d sx;
        if (!embed_d(d, F + (size_t)d * i, scale, &sx)) {
            *status = OR_EINVAL;
            continue;
        }
        for (int k = 0; k < D; ++k) {
            memset(e[ne].key, 0, sizeof e[ne].key);
            memcpy(e[ne].key, sx.key[k], (size_t)D * sizeof(int32_t));
            e[ne].src = i;
            e[ne].k = k;
            e[ne].b = sx.b[k];
            ++ne;
        }
    }
    g_cmp_dim = D;
    qsort(e, (size_t)ne, sizeof *e, cmp_fentry);
    int64_t nv = 0;
    for (int64_t t = 0; t < ne; ++t)
        if (t == 0 || cmp_keyd(e[t].key, e[t - 1].key, D) != 0)
            ++nv;
    lat->nv = nv;
    lat->keys = (int32_t *)malloc((size_t)(nv ? nv : 1) * D * sizeof(int32_t));
    lat->vals = (double *)calloc((size_t)(nv ? nv : 1) * (size_t)vdim, sizeof(double));
    if (!lat->keys || !lat->vals) {
        free(e);
        or_flattice_free(lat);
        *status = OR_ENOMEM;
        return NULL;
    }
    int64_t v = -1;
    for (int64_t t = 0; t < ne; ++t) {
        if (t == 0 || cmp_keyd(e[t].key, e[t - 1].key, D) != 0) {
            ++v;
            memcpy(lat->keys + (size_t)D * v, e[t].key, (size_t)D * sizeof(int32_t));
        }
        for (int c = 0; c < vdim; ++c)
            lat->vals[v * vdim + c] += (double)e[t].b * V[e[t].src * vdim + c];
    }
    free(e);
    return lat;
}

int or_flattice_slice(const or_flattice *lat, const float *Q, int64_t m, double *out)
{
    const int d = lat->d, D = d + 1, vdim = lat->vdim;
    int status = OR_OK;
    for (int64_t i = 0; i < m; ++i) {
        for (int c = 0; c < vdim; ++c)
            out[i * vdim + c] = 0.0;
        simplex_d sx;
        if (!embed_d(d, Q + (size_t)d * i, lat->scale, &sx)) {
            status = OR_EINVAL;
            continue;
        }
        for (int k = 0; k < D; ++k) {
            int64_t v = find_vertex_d(lat, sx.key[k]);
            if (v < 0)
                continue;
            for (int c = 0; c < vdim; ++c)
                out[i * vdim + c] += (double)sx.b[k] * lat->vals[v * vdim + c];
        }
    }
    return status;
}

int64_t or_flattice_size(const or_flattice *lat) { return lat->nv; }

void or_flattice_vertices(const or_flattice *lat, int32_t *keys, double *vals)
{
    if (lat->nv == 0)
        return;
    memcpy(keys, lat->keys, (size_t)lat->nv * (lat->d + 1) * sizeof(int32_t));
    memcpy(vals, lat->vals, (size_t)lat->nv * lat->vdim * sizeof(double));
}

void or_flattice_free(or_flattice *lat)
{
    if (!lat)
        return;
    free(lat->keys);
    free(lat->vals);
    free(lat);
}

/* ---- the feature-space E step (Eq. feature_estep) -------------------------- */

int or_estep_features(const float *FX, int64_t M, const float *FY, int64_t N, int d, const float *sigma_f,
                      const float *Y, const float *Yn, int backend, double *out)
{
    if (d < 1 || d > OR_FEATURE_DMAX || M < 0 || N < 0)
        return OR_EINVAL;
    for (int c = 0; c < d; ++c)
        if (!(sigma_f[c] > 0.0f))
            return OR_EINVAL;
    const int vdim = Yn ? 7 : 4;
    if (backend == OR_EXACT) {
        /* K_ik = exp(-sum_c (f_xi,c - f_yk,c)^2 / (2 sigma_c^2)), double sums */
        for (int64_t i = 0; i < M; ++i) {
            double acc[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int64_t k = 0; k < N; ++k) {
                double q = 0.0;
                for (int c = 0; c < d; ++c) {
                    const double t = ((double)FX[(size_t)d * i + c] - (double)FY[(size_t)d * k + c]) / sigma_f[c];
                    q += t * t;
                }
                const double g = exp(-0.5 * q);
                acc[0] += g;
                for (int c = 0; c < 3; ++c)
                    acc[1 + c] += g * (double)Y[4 * k + c];
                if (Yn)
                    for (int c = 0; c < 3; ++c)
                        acc[4 + c] += g * (double)Yn[4 * k + c];
            }
            for (int c = 0; c < vdim; ++c)
                out[i * vdim + c] = acc[c];
        }
        return OR_OK;
    }
    float scale[OR_FEATURE_DMAX];
    or_feature_scale(d, sigma_f, scale);
    double *V = (double *)malloc((size_t)(N ? N : 1) * vdim * sizeof(double));
    if (!V)
        return OR_ENOMEM;
    for (int64_t k = 0; k < N; ++k) {
        V[k * vdim] = 1.0;
        for (int c = 0; c < 3; ++c)
            V[k * vdim + 1 + c] = Y[4 * k + c];
        if (Yn)
            for (int c = 0; c < 3; ++c)
                V[k * vdim + 4 + c] = Yn[4 * k + c];
    }
    int status = OR_OK;
    or_flattice *lat = or_flattice_build(FY, N, d, scale, V, vdim, &status);
    free(V);
    if (!lat)
        return status;
    const int st2 = or_flattice_slice(lat, FX, M, out);
    or_flattice_free(lat);
    return status != OR_OK ? status : st2;
}

double or_feature_kernel_mass(int d)
{
    /* Volume per lattice point of the union of remainder classes in the
     * hyperplane, (d+1)^(d - 1/2), over alpha^d (the elevation's scale). */
    const double alpha = sqrt(2.0 / 3.0) * (double)(d + 1);
    return pow((double)(d + 1), (double)d - 0.5) / pow(alpha, (double)d);
}
