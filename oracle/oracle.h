/*
 * FilterReg CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow restatement of what the registration hot path
 * computes, written from the paper (Gao & Tedrake, "FilterReg", CVPR 2019) and
 * from the permutohedral-lattice construction it cites (Adams et al. 2010).
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, constant or helper with the CUDA
 * library; the product path never calls it.
 *
 * Conventions
 *   - Point clouds are float[n][4] (x, y, z, unused), the same host layout the
 *     CUDA library takes, so one seeded array feeds both sides.
 *   - Poses are double[16], row-major 4x4 homogeneous transforms.
 *   - Twists are zeta = (omega; v) = (alpha, beta, gamma, a, b, c), rotation
 *     first, as in the twist linearisation of Section 5 (Eq. 16).
 *   - Sums of the E and M steps are in double.  The permutohedral embedding
 *     (elevation, rounding, rank sort, barycentric weights) is evaluated in
 *     float with no fused multiply-add, in a fixed operation order, because
 *     those float results decide integer lattice keys.
 *
 * Threads: built plain (liboracle.so) everything runs on one thread; built
 * with -fopenmp (liboracle_omp.so, the benchmark's all-core baseline) the
 * per-point loops of the rigid path run in parallel.  Every sum keeps a fixed
 * order (chunks of fixed size, reduced in chunk order), so the two builds
 * return bit-identical results.
 *
 * Parity status of each function is stated beside it; every function is
 * pinned by the CPU tests (tests/test_oracle_*.py) against closed forms,
 * invariants, library routines or brute force, except where marked
 * "parity unpinned".
 */
#ifndef FILTERREG_ORACLE_H
#define FILTERREG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_EDEGENERATE = 7 };
enum { OR_PT2PT = 0, OR_PT2PL = 1 };
enum { OR_EXACT = 0, OR_LATTICE = 1 };

typedef struct {
    int backend;             /* OR_EXACT (Eq. 6 summed directly) or OR_LATTICE (Section 4.2) */
    int residual;            /* OR_PT2PT (Eq. 7) or OR_PT2PL (Eq. 10) */
    int blur;                /* lattice only: 1 = blur along the 4 lattice axes */
    int iters;               /* EM iterations, one Gauss-Newton step each */
    double sigma_start;      /* isotropic kernel std-dev of the first iteration */
    double sigma_end;        /* of the last; geometric schedule in between */
    double w;                /* outlier ratio, 0 <= w < 1 (Section 3.1) */
    int renormalize_normals; /* pt2pl: 1 = unit-normalise N_x (Eq. 9 as written: 0) */
    double stop_twist;       /* stop once |delta zeta| < stop_twist (0 = never) */
    int update_sigma;        /* 1 = sigma re-estimated every iteration (Section 3.3's
                                sigma as a decision variable, point-to-point): sigma_start
                                starts it, sigma_end is its floor; 0 = the schedule */
} or_options;

typedef struct {
    int iters_run;
    int degenerate_iters;    /* iterations whose normal matrix was not positive definite */
    int64_t last_inliers;    /* model points with M0 > 0 in the last iteration */
    double last_sum_w;       /* sum of outlier weights in the last iteration */
    double last_cost;        /* sum of squared weighted residuals in the last iteration */
    double last_twist_norm;  /* |delta zeta| of the last applied update */
    double sigma_next;       /* update_sigma: the sigma the next iteration would use,
                                before the floor (otherwise 0) */
    double last_sigma;       /* sigma of the last iteration run */
} or_report;

/* ---- exact E step (Eq. 6, Eq. 9 numerator), unnormalised kernel ---------- */
/* M0[i] = sum_k exp(-|x_i - y_k|^2 / (2 sigma^2)), M1[i] = sum_k (..) y_k,
 * Ns[i] = sum_k (..) n_k.  Yn may be NULL (then Ns is not written).          */
void or_estep_exact(const float *X, int64_t M, const float *Y, const float *Yn,
                    int64_t N, double sigma, double *M0, double *M1, double *Ns);
/* The same sums at one double-precision position x. */
void or_exact_sums_at(const double x[3], const float *Y, const float *Yn, int64_t N,
                      double sigma, double *M0, double M1[3], double Ns[3]);

/* ---- permutohedral lattice, d = 3 (Section 4.2) -------------------------- */
/* Per-axis float feature scale alpha / sqrt(i (i+1)) / sigma, i = 1..3.       */
void or_lattice_feature_scale(float sigma, float scale[3]);

/* Embed n points: for each, the 4 vertices of its enclosing simplex as full
 * 4-coordinate integer keys (keys[i][k][j]), barycentric weights bary[i][k],
 * elevated coordinates z[i][j] and ranks rank[i][j] (each output nullable).
 * Returns OR_EINVAL if any coordinate is non-finite or beyond the key range.  */
int or_lattice_embed(const float *P, int64_t n, float sigma, int32_t *keys,
                     float *bary, float *z, int32_t *rank);

typedef struct or_lattice or_lattice;
/* Splat values V (n x vdim, double) of points P at scale sigma. */
or_lattice *or_lattice_build(const float *P, const double *V, int64_t n, int vdim,
                             float sigma, int *status);
void or_lattice_blur(or_lattice *lat);
/* Slice at m query points: out[i][c] = sum_k b_k table[key_k][c] (0 if absent). */
int or_lattice_slice(const or_lattice *lat, const float *Q, int64_t m, double *out);
int64_t or_lattice_size(const or_lattice *lat);
int or_lattice_vdim(const or_lattice *lat);
/* Vertex keys (nv x 4, all four coordinates) and values (nv x vdim), key-sorted. */
void or_lattice_vertices(const or_lattice *lat, int32_t *keys, double *vals);
void or_lattice_free(or_lattice *lat);

/* Integral of the unnormalised E-step kernel over feature space (unit sigma):
 * exact Gaussian (2 pi)^{3/2}; lattice splat+slice: volume per lattice vertex
 * in feature units; times the blur gain 2^4 when blurred.                    */
double or_kernel_mass(int backend, int blur);
/* Per-axis variance of the unblurred splat+slice kernel in units of sigma^2,
 * averaged over positions (1/4 for d = 3; the exact Gaussian's is 1).  The
 * sigma update divides by it, so that sigma is the width at which the kernel
 * actually used matches the residuals.                                        */
double or_lattice_kernel_variance(void);

/* Geometric sigma schedule: sigma_k = s0 (s1/s0)^{k/(iters-1)}, rounded to float. */
void or_sigma_schedule(double s0, double s1, int iters, float *out);

/* ---- M step pieces (Section 5) ------------------------------------------- */
void or_se3_exp(const double zeta[6], double T[16]);
void or_se3_log(const double T[16], double zeta[6]);
/* Solve A x = b for symmetric positive definite A (n x n, row-major) by
 * Cholesky.  Returns 0 on success, 1 if A is not positive definite.          */
int or_cholesky_solve(int n, const double *A, const double *b, double *x);

/* One model point's outlier weight, residual and twist Jacobian.
 * x: current position; M0, M1, Ns: its E-step sums; c_eff: outlier constant in
 * the kernel's own normalisation.  Returns the number of residual rows (3 for
 * pt2pt, 1 for pt2pl, 0 if M0 <= 0).  r[rows], J[rows][6] are sqrt(W)/sigma
 * weighted, so that A = sum J^T J and b = sum J^T r (Eq. 17-18).             */
int or_point_terms(const double x[3], double M0, const double M1[3], const double Ns[3],
                   double c_eff, double sigma, int residual, int renormalize,
                   double *W, double *r, double *J);

/* Outlier constant c = w/(1-w) N/M of Eq. 7, in the unnormalised kernel's
 * units: c * sigma^3 * G with G = or_kernel_mass(backend, blur).            */
double or_outlier_constant(double w, int64_t N, int64_t M, double sigma, int backend, int blur);

/* ---- rigid registration driver (EM of Section 3.1, M step of Section 5) --- */
int or_register_rigid(const float *X, int64_t M, const float *Y, const float *Yn,
                      int64_t N, const or_options *opt, double T[16], or_report *rep);

/* One EM iteration's normal equations of a shard X (M points) of a model of
 * M_total points at pose T and sigma = opt->sigma_start (Eq. 7's outlier
 * constant from M_total): ne = A's upper triangle row by row (21),
 * b = sum J^T r (6), sum of weights, cost, inliers -- additive over shards. */
int or_rigid_normal_equations(const float *X, int64_t M, const float *Y, const float *Yn, int64_t N,
                              const or_options *opt, int64_t M_total, const double T[16], double ne[30]);

/* E-step sums at the model points moved by T (lattice or exact back end), for
 * parity of a single E step: out is M x (1 + 3 [+ 3]) = [M0, M1, Ns].        */
int or_estep(const float *X, int64_t M, const float *Y, const float *Yn, int64_t N,
             int backend, int blur, double sigma, const double T[16], double *out);

/* ---- articulated model (Section 5.1, Eq. 20, Algorithm 1) -------------------
 * Body 0 is the root; parent[b] < b for b > 0.  T_b = T_parent(b) * offset_b *
 * R(a_j1, q_j1) * R(a_j2, q_j2) * ... over the joints of b (consecutive in the
 * joint arrays, ordered by body); the root's parent transform is the root
 * pose.  Joint axes are unit vectors in the frame each joint acts in.       */
typedef struct {
    int nb, nj;
    const int32_t *parent;     /* nb */
    const double *offset;      /* nb x 16, row-major */
    const int32_t *joint_body; /* nj, non-decreasing */
    const double *joint_axis;  /* nj x 3 */
    const double *q_min, *q_max; /* nj joint limits */
} or_kintree;

/* Forward kinematics: body transforms T (nb x 16) and each joint's world axis
 * and a world point on it (nj x 3 each; nullable). */
int or_fk(const or_kintree *t, const double root_T[16], const double *q, double *T,
          double *axis_w, double *point_w);
/* Spatial velocity Jacobian of body b: 6 x (6 + nj), row-major. */
int or_spatial_jacobian(const or_kintree *t, const double *axis_w, const double *point_w, int b,
                        double *Jsp);
/* One E step at (root_T, q) and the normal equations of Algorithm 1:
 * A ((6+nj) x (6+nj)) and g (6+nj), with A dtheta = -g the Gauss-Newton step. */
int or_articulated_normal_equations(const float *Xref, const int32_t *body, int64_t M,
                                    const or_kintree *t, const float *Y, const float *Yn,
                                    int64_t N, const or_options *opt, double sigma,
                                    const double root_T[16], const double *q, double *A,
                                    double *g);
/* Articulated EM registration; Xref in body frames, body[i] its body. */
int or_register_articulated(const float *Xref, const int32_t *body, int64_t M,
                            const or_kintree *t, const float *Y, const float *Yn, int64_t N,
                            const or_options *opt, double root_T[16], double *q, or_report *rep);

/* ---- node-graph deformable model (Section 5.2, Eq. 21) ----------------------
 * Nodes k = 0..K-1 with reference positions node_pos (K x 3) and poses
 * node_T (K x 16, row-major).  Model point i has 4 nearest nodes knn[i][0..3]
 * with skinning weights skw[i][0..3] (summing to 1).  Directed regulariser
 * edges (j, k) = edges[e][0..1], weight lambda.  The readings that fill the
 * missing supplement are stated in nodegraph.c.                               */
typedef struct {
    int K;
    const double *node_pos;    /* K x 3 */
    int E;
    const int32_t *edges;      /* E x 2 */
    double lambda;
    int pcg_iters;
} or_nodegraph;

/* Dual quaternion (q_r (w, x, y, z), q_d) of a rigid transform and back (the
 * latter normalises by |q_r|; translation 2 (r0 d - d0 r + r x d)). */
void or_dq_from_T(const double T[16], double dq[8]);
void or_T_from_dq(const double dq[8], double T[16]);
/* Dual-quaternion blend of the poses of nodes knn[0..3] (node_dq: K x 8),
 * signs aligned with the largest-weight neighbour's (the first such),
 * weights w (Eq. 21). */
void or_dqb(const double *node_dq, const int32_t knn[4], const float w[4], double T[16]);
/* Warped model points X (M x 3) at the node poses. */
int or_nodegraph_warp(const float *Xref, const int32_t *knn, const float *skw, int64_t M, int K,
                      const double *node_T, double *X);
/* One E step at node_T and the Gauss-Newton system: A (6K x 6K, dense) and
 * g (6K), A dtheta = -g.  rep (nullable) gets inliers, cost (data +
 * regulariser) and the weight sum. */
int or_nodegraph_normal_equations(const float *Xref, const int32_t *knn, const float *skw,
                                  int64_t M, const or_nodegraph *ng, const float *Y,
                                  const float *Yn, int64_t N, const or_options *opt, double sigma,
                                  const double *node_T, double *A, double *g, or_report *rep);
/* x = block-Jacobi PCG solution of A x = b after `iters` iterations from 0
 * (A: 6 nb x 6 nb dense, blocks of 6). */
int or_pcg_block_jacobi(int nb, const double *A, const double *b, int iters, double *x);
/* Node-graph EM registration: node_T in/out. */
int or_register_nodegraph(const float *Xref, const int32_t *knn, const float *skw, int64_t M,
                          const or_nodegraph *ng, const float *Y, const float *Yn, int64_t N,
                          const or_options *opt, double *node_T, or_report *rep);

/* Alignment error of Eq. 22: mean |(T - T_gt) x_ref|. */
double or_align_error(const float *X, int64_t M, const double T[16], const double Tgt[16]);

/* ---- feature-space E step (Eq. feature_estep), d-dimensional lattice ------
 * Features are rows of d floats (1 <= d <= OR_FEATURE_DMAX), the kernel a
 * Gaussian with diagonal covariance diag(sigma_f^2) in feature space.        */
#define OR_FEATURE_DMAX 7
/* Per-axis scale alpha / sqrt(i (i+1)) / sigma_f[i-1], alpha = sqrt(2/3)(d+1). */
void or_feature_scale(int d, const float *sigma_f, float *scale);
/* Vertices (keys[i][k][j], j < d+1) and barycentric weights of n features.  */
int or_feature_embed(const float *F, int64_t n, int d, const float *scale, int32_t *keys, float *bary);
typedef struct or_flattice or_flattice;
or_flattice *or_flattice_build(const float *F, int64_t n, int d, const float *scale, const double *V,
                               int vdim, int *status);
int or_flattice_slice(const or_flattice *lat, const float *Q, int64_t m, double *out);
int64_t or_flattice_size(const or_flattice *lat);
void or_flattice_vertices(const or_flattice *lat, int32_t *keys, double *vals);
void or_flattice_free(or_flattice *lat);
/* M0, M1 (and normal sums with Yn) at the model features FX, kernel over the
 * observation features FY: exact sums (OR_EXACT) or splat + slice on the
 * d-dimensional lattice (OR_LATTICE); out is M x 4 or M x 7.                 */
int or_estep_features(const float *FX, int64_t M, const float *FY, int64_t N, int d, const float *sigma_f,
                      const float *Y, const float *Yn, int backend, double *out);
/* Integral of the unnormalised splat+slice kernel in normalised feature units. */
double or_feature_kernel_mass(int d);

/* Threads the OpenMP build uses (1 for the plain build); set them (n > 0). */
int or_num_threads(void);
void or_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
