/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Reference permutohedral lattice for d = 3 position features.
 *
 * Section 4.2 reviews the filter the paper builds on (Adams et al. 2010): a
 * d-dimensional feature is embedded in the (d+1)-dimensional hyperplane where
 * the permutohedral lattice lives, each value is splatted onto the vertices of
 * its enclosing simplex with barycentric weights, optionally blurred between
 * neighbouring lattice points, and sliced back with the same weights.  Eq. 13-14
 * (the augmentation [F_X, F_Y], [0, V_Y]) mean that only the observation cloud
 * carries values: slicing the model cloud is a pure query and lattice points
 * that no observation touched contribute zero.
 *
 * The geometry written out here:
 *   - Elevation: z = alpha * E f, E's columns the orthonormal basis
 *     (1,..,1,-i,0,..)/sqrt(i(i+1)), i = 1..d, of the hyperplane sum(z) = 0.
 *     alpha = sqrt(2/3)(d+1) sets the lattice scale so that splat-blur-slice
 *     approximates a unit-std Gaussian in feature units.
 *   - The lattice is the union over k = 0..d of the "remainder-k" integer
 *     points of the hyperplane (all coordinates congruent to k mod d+1).
 *   - The enclosing simplex: round z to the nearest remainder-0 point, rank
 *     the differences z - r0 (descending, ties to the lower index), repair the
 *     coordinate sum, and read the d+1 vertices and barycentric weights off
 *     the ranks.
 *
 * Float discipline: every step of the embedding is one IEEE float operation in
 * a fixed order (compile with -ffp-contract=off), with round-half-to-even
 * rounding, so that the integer keys are reproducible bit for bit.  Splat,
 * blur and slice sums are in double.  The vertex set is kept key-sorted and
 * searched by bisection: plain and obviously ordered, not fast.  Built with
 * OpenMP, the per-point loops run in parallel and the sort is chunked; every
 * sum keeps its order, so results are bit-identical to the serial build.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define LD 3          /* feature dimension d */
#define LD1 4         /* lattice dimension d + 1 */
#define KEY_LIMIT 1000000.0f /* |z_j| must stay below this (integer key range) */

void or_lattice_feature_scale(float sigma, float scale[3])
{
    const double alpha = sqrt(2.0 / 3.0) * (double)LD1;
    for (int i = 1; i <= LD; ++i)
        scale[i - 1] = (float)(alpha / sqrt((double)(i * (i + 1))) / (double)sigma);
}

typedef struct {
    float z[LD1];
    int32_t r0[LD1];
    int32_t rank[LD1];
    float b[LD1];
    int32_t key[LD1][LD1]; /* key[k][j]: coordinate j of vertex k */
} simplex;

/* Embed one point; returns 0 if a coordinate is non-finite or out of range. */
static int embed_point(const float p[3], const float s[3], simplex *o)
{
    float c[LD + 1];
    for (int i = 1; i <= LD; ++i)
        c[i] = p[i - 1] * s[i - 1];

    /* z_j = sum_{i > j} c_i - j c_j, accumulated from the last axis down. */
    float t = 0.0f;
    for (int i = LD; i >= 1; --i) {
        o->z[i] = t - (float)i * c[i];
        t = t + c[i];
    }
    o->z[0] = t;
    for (int j = 0; j < LD1; ++j)
        if (!(fabsf(o->z[j]) < KEY_LIMIT))
            return 0;

    /* Nearest remainder-0 point, coordinate by coordinate. */
    int sum = 0;
    for (int j = 0; j < LD1; ++j) {
        float q = rintf(o->z[j] * 0.25f);
        o->r0[j] = (int32_t)q * LD1;
        sum += (int32_t)q;
    }
    float delta[LD1];
    for (int j = 0; j < LD1; ++j)
        delta[j] = o->z[j] - (float)o->r0[j];

    /* Rank of each coordinate's difference, descending, ties to lower index. */
    for (int j = 0; j < LD1; ++j) {
        int r = 0;
        for (int k = 0; k < LD1; ++k)
            if (delta[k] > delta[j] || (k < j && delta[k] == delta[j]))
                ++r;
        o->rank[j] = r;
    }

    /* Repair the coordinate sum: move the sum coordinates with the smallest
     * (sum > 0) or largest (sum < 0) differences by one lattice step. */
    if (sum > LD1 || sum < -LD1)
        return 0;
    if (sum > 0) {
        for (int j = 0; j < LD1; ++j) {
            if (o->rank[j] >= LD1 - sum) {
                o->r0[j] -= LD1;
                o->rank[j] += sum - LD1;
            } else {
                o->rank[j] += sum;
            }
        }
    } else if (sum < 0) {
        for (int j = 0; j < LD1; ++j) {
            if (o->rank[j] < -sum) {
                o->r0[j] += LD1;
                o->rank[j] += LD1 + sum;
            } else {
                o->rank[j] += sum;
            }
        }
    }

    /* Barycentric weights from the ranked differences. */
    float b[LD1 + 1];
    for (int k = 0; k <= LD1; ++k)
        b[k] = 0.0f;
    for (int j = 0; j < LD1; ++j) {
        float v = (o->z[j] - (float)o->r0[j]) * 0.25f;
        b[LD1 - 1 - o->rank[j]] += v;
        b[LD1 - o->rank[j]] -= v;
    }
    b[0] = b[0] + (1.0f + b[LD1]);
    for (int k = 0; k < LD1; ++k)
        o->b[k] = b[k];

    /* Vertex k: all coordinates congruent to k mod (d+1). */
    for (int k = 0; k < LD1; ++k)
        for (int j = 0; j < LD1; ++j)
            o->key[k][j] = o->r0[j] + k - (o->rank[j] > LD1 - 1 - k ? LD1 : 0);
    return 1;
}

int or_lattice_embed(const float *P, int64_t n, float sigma, int32_t *keys,
                     float *bary, float *z, int32_t *rank)
{
    float s[3];
    or_lattice_feature_scale(sigma, s);
    int status = OR_OK;
    for (int64_t i = 0; i < n; ++i) {
        simplex sx;
        if (!embed_point(P + 4 * i, s, &sx)) {
            status = OR_EINVAL;
            memset(&sx, 0, sizeof sx);
        }
        for (int k = 0; k < LD1; ++k) {
            if (keys)
                for (int j = 0; j < LD1; ++j)
                    keys[(i * LD1 + k) * LD1 + j] = sx.key[k][j];
            if (bary)
                bary[i * LD1 + k] = sx.b[k];
            if (z)
                z[i * LD1 + k] = sx.z[k];
            if (rank)
                rank[i * LD1 + k] = sx.rank[k];
        }
    }
    return status;
}

/* ---- the lattice: a key-sorted vertex array -------------------------------- */

struct or_lattice {
    int64_t nv;
    int vdim;
    float scale[3];
    int32_t *keys;  /* nv x 4 */
    double *vals;   /* nv x vdim */
};

typedef struct {
    int32_t key[LD1];
    int64_t src;
    int32_t k;
    float b;
} splat_entry;

static int cmp_key(const int32_t *a, const int32_t *b)
{
    for (int j = 0; j < LD1; ++j) {
        if (a[j] < b[j])
            return -1;
        if (a[j] > b[j])
            return 1;
    }
    return 0;
}

static int cmp_entry(const void *pa, const void *pb)
{
    const splat_entry *a = (const splat_entry *)pa, *b = (const splat_entry *)pb;
    int c = cmp_key(a->key, b->key);
    if (c)
        return c;
    if (a->src != b->src)
        return a->src < b->src ? -1 : 1;
    return a->k - b->k;
}

/* Sorts the splat entries by (key, source point, vertex): a total order, so
 * the result does not depend on how the work is split.  Built with OpenMP,
 * chunks are sorted in parallel and merged pairwise; otherwise one qsort. */
static void sort_entries(splat_entry *e, int64_t n)
{
#ifdef _OPENMP
    const int64_t chunk = 16384;
    if (n > 2 * chunk) {
        const int64_t nc = (n + chunk - 1) / chunk;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t lo = c * chunk, hi = lo + chunk < n ? lo + chunk : n;
            qsort(e + lo, (size_t)(hi - lo), sizeof *e, cmp_entry);
        }
        splat_entry *tmp = (splat_entry *)malloc((size_t)n * sizeof *e);
        if (tmp) {
            splat_entry *src = e, *dst = tmp;
            for (int64_t w = chunk; w < n; w *= 2) {
                const int64_t np = (n + 2 * w - 1) / (2 * w);
#pragma omp parallel for schedule(dynamic, 1)
                for (int64_t q = 0; q < np; ++q) {
                    const int64_t lo = q * 2 * w;
                    const int64_t mid = lo + w < n ? lo + w : n, hi = lo + 2 * w < n ? lo + 2 * w : n;
                    int64_t a = lo, b = mid, o = lo;
                    while (a < mid && b < hi)
                        dst[o++] = cmp_entry(src + b, src + a) < 0 ? src[b++] : src[a++];
                    while (a < mid)
                        dst[o++] = src[a++];
                    while (b < hi)
                        dst[o++] = src[b++];
                }
                splat_entry *t = src;
                src = dst;
                dst = t;
            }
            if (src != e)
                memcpy(e, src, (size_t)n * sizeof *e);
            free(tmp);
            return;
        }
    }
#endif
    qsort(e, (size_t)n, sizeof *e, cmp_entry);
}

/* Index of key in the sorted vertex array, or -1. */
static int64_t find_vertex(const or_lattice *lat, const int32_t key[LD1])
{
    int64_t lo = 0, hi = lat->nv - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = cmp_key(lat->keys + LD1 * mid, key);
        if (c == 0)
            return mid;
        if (c < 0)
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

or_lattice *or_lattice_build(const float *P, const double *V, int64_t n, int vdim,
                             float sigma, int *status)
{
    *status = OR_OK;
    or_lattice *lat = (or_lattice *)calloc(1, sizeof *lat);
    if (!lat) {
        *status = OR_ENOMEM;
        return NULL;
    }
    lat->vdim = vdim;
    or_lattice_feature_scale(sigma, lat->scale);
    if (n == 0)
        return lat;

    splat_entry *e = (splat_entry *)malloc((size_t)n * LD1 * sizeof *e);
    if (!e) {
        free(lat);
        *status = OR_ENOMEM;
        return NULL;
    }
    /* Point i's entries go to slots 4 i .. 4 i + 3 (a point outside the key
     * range leaves them marked unused), then the used ones are packed in
     * point order: the same entry array for any number of threads. */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < n; ++i) {
        simplex sx;
        const int ok = embed_point(P + 4 * i, lat->scale, &sx);
        if (!ok)
            bad = 1;
        for (int k = 0; k < LD1; ++k) {
            splat_entry *t = e + LD1 * i + k;
            memcpy(t->key, sx.key[k], sizeof t->key);
            t->src = ok ? i : -1;
            t->k = k;
            t->b = ok ? sx.b[k] : 0.0f;
        }
    }
    if (bad)
        *status = OR_EINVAL;
    int64_t ne = 0;
    for (int64_t t = 0; t < n * LD1; ++t)
        if (e[t].src >= 0)
            e[ne++] = e[t];
    sort_entries(e, ne);

    int64_t nv = 0;
    for (int64_t t = 0; t < ne; ++t)
        if (t == 0 || cmp_key(e[t].key, e[t - 1].key) != 0)
            ++nv;
    lat->nv = nv;
    lat->keys = (int32_t *)malloc((size_t)(nv ? nv : 1) * LD1 * sizeof(int32_t));
    lat->vals = (double *)calloc((size_t)(nv ? nv : 1) * (size_t)vdim, sizeof(double));
    if (!lat->keys || !lat->vals) {
        free(e);
        or_lattice_free(lat);
        *status = OR_ENOMEM;
        return NULL;
    }
    int64_t v = -1;
    for (int64_t t = 0; t < ne; ++t) {
        if (t == 0 || cmp_key(e[t].key, e[t - 1].key) != 0) {
            ++v;
            memcpy(lat->keys + LD1 * v, e[t].key, LD1 * sizeof(int32_t));
        }
        for (int c = 0; c < vdim; ++c)
            lat->vals[v * vdim + c] += (double)e[t].b * V[e[t].src * vdim + c];
    }
    free(e);
    return lat;
}

void or_lattice_blur(or_lattice *lat)
{
    const int vdim = lat->vdim;
    double *next = (double *)malloc((size_t)(lat->nv ? lat->nv : 1) * vdim * sizeof(double));
    if (!next)
        return;
    for (int dir = 0; dir < LD1; ++dir) {
        /* Neighbour offset along lattice axis dir: +1 on every coordinate,
         * -d on coordinate dir (the coordinates still sum to zero). */
        int32_t off[LD1];
        for (int j = 0; j < LD1; ++j)
            off[j] = (j == dir) ? 1 - LD1 : 1;
        for (int64_t v = 0; v < lat->nv; ++v) {
            int32_t kp[LD1], km[LD1];
            for (int j = 0; j < LD1; ++j) {
                kp[j] = lat->keys[LD1 * v + j] + off[j];
                km[j] = lat->keys[LD1 * v + j] - off[j];
            }
            int64_t ip = find_vertex(lat, kp), im = find_vertex(lat, km);
            for (int c = 0; c < vdim; ++c) {
                double acc = lat->vals[v * vdim + c];
                if (im >= 0)
                    acc += 0.5 * lat->vals[im * vdim + c];
                if (ip >= 0)
                    acc += 0.5 * lat->vals[ip * vdim + c];
                next[v * vdim + c] = acc;
            }
        }
        memcpy(lat->vals, next, (size_t)lat->nv * vdim * sizeof(double));
    }
    free(next);
}

int or_lattice_slice(const or_lattice *lat, const float *Q, int64_t m, double *out)
{
    const int vdim = lat->vdim;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < m; ++i) {
        for (int c = 0; c < vdim; ++c)
            out[i * vdim + c] = 0.0;
        simplex sx;
        if (!embed_point(Q + 4 * i, lat->scale, &sx)) {
            bad = 1;
            continue;
        }
        for (int k = 0; k < LD1; ++k) {
            int64_t v = find_vertex(lat, sx.key[k]);
            if (v < 0)
                continue;
            for (int c = 0; c < vdim; ++c)
                out[i * vdim + c] += (double)sx.b[k] * lat->vals[v * vdim + c];
        }
    }
    return bad ? OR_EINVAL : OR_OK;
}

int64_t or_lattice_size(const or_lattice *lat) { return lat->nv; }
int or_lattice_vdim(const or_lattice *lat) { return lat->vdim; }

void or_lattice_vertices(const or_lattice *lat, int32_t *keys, double *vals)
{
    if (lat->nv == 0)
        return;
    memcpy(keys, lat->keys, (size_t)lat->nv * LD1 * sizeof(int32_t));
    memcpy(vals, lat->vals, (size_t)lat->nv * lat->vdim * sizeof(double));
}

void or_lattice_free(or_lattice *lat)
{
    if (!lat)
        return;
    free(lat->keys);
    free(lat->vals);
    free(lat);
}

double or_kernel_mass(int backend, int blur)
{
    const double pi = 3.14159265358979323846;
    if (backend == OR_EXACT)
        return pow(2.0 * pi, 1.5);
    /* Volume per lattice point of the union of remainder classes in the
     * hyperplane: (d+1)^(d-1/2); the elevation scales lengths by alpha. */
    const double alpha = sqrt(2.0 / 3.0) * (double)LD1;
    double g = pow((double)LD1, (double)LD - 0.5) / pow(alpha, (double)LD);
    if (blur)
        g *= pow(2.0, (double)LD1); /* each (1/2, 1, 1/2) pass doubles the mass */
    return g;
}

/* Per-axis variance, in units of sigma^2, of the unblurred splat+slice
 * kernel K(p, q) = sum_v b_v(p) b_v(q), averaged over positions p:
 * E_p[int K(p,q) |q - p|^2 dq] / (d int K) = 2 M2 / (d covol), where M2 =
 * int b_0(q) |q|^2 dq is the second moment of one vertex's hat (the first
 * moment vanishes: the triangulation is symmetric about a vertex).  The hat is
 * linear on the (d+1)! congruent simplices around the vertex, each of volume
 * covol / d!, and on a simplex with vertices 0, v_1..v_d the integral of
 * lambda_0 lambda_k lambda_l is d! vol (1 + [k == l]) / (d+3)!, so that
 * M2 = covol (|sum_k v_k|^2 + sum_k |v_k|^2) / ((d+2)(d+3)), the v_k the
 * canonical simplex's vertices in feature units (elevated coordinates over
 * alpha).  For d = 3 this is 1/4: the kernel is half as wide as the Gaussian
 * of the same sigma. */
double or_lattice_kernel_variance(void)
{
    const double alpha = sqrt(2.0 / 3.0) * (double)LD1;
    double sum[LD1] = {0, 0, 0, 0}, sq = 0.0;
    for (int k = 1; k < LD1; ++k)
        for (int j = 0; j < LD1; ++j) {
            /* canonical vertex k: k in its first LD1 - k coordinates, k - LD1 after */
            const double c = (j < LD1 - k) ? (double)k : (double)(k - LD1);
            sum[j] += c;
            sq += c * c;
        }
    double s2 = 0.0;
    for (int j = 0; j < LD1; ++j)
        s2 += sum[j] * sum[j];
    const double B = (s2 + sq) / (alpha * alpha);
    return 2.0 * B / ((double)LD * (LD + 2) * (LD + 3));
}

void or_sigma_schedule(double s0, double s1, int iters, float *out)
{
    for (int k = 0; k < iters; ++k) {
        if (iters == 1 || s0 == s1)
            out[k] = (float)s0;
        else
            out[k] = (float)(s0 * pow(s1 / s0, (double)k / (double)(iters - 1)));
    }
}
