/*
 * filterreg.h -- C ABI of the GB300 (sm_103a) FilterReg hot path.
 *
 * FilterReg (Gao & Tedrake, CVPR 2019) registers a model cloud X (M points,
 * moved by the motion parameters) to an observation cloud Y (N points, fixed)
 * by EM on a Gaussian mixture induced by Y (Section 3.1).  The E step is
 * computed as Gaussian filtering on a permutohedral lattice built over Y
 * (Section 4), the M step as Gauss-Newton over twists (Section 5).
 *
 * Conventions shared by every entry point
 *   - Point clouds are float32 arrays of n rows of 4 floats (x, y, z, unused),
 *     16-byte aligned, row-major ("n x 4").  Normals use the same layout.
 *   - Pointers named d_* are DEVICE pointers on the context's device; h_*
 *     are host pointers (pinned host memory makes their copies asynchronous).
 *     The caller owns every buffer it passes; the library never frees them
 *     and keeps no reference after the call returns.
 *   - Poses are host double[16], row-major 4x4 homogeneous transforms with
 *     x_moved = T x; T_inout carries the initial guess in and the result out.
 *   - Twists are zeta = (omega; v) = (alpha, beta, gamma, a, b, c), rotation
 *     first, as in the twist matrix of Eq. 16.
 *   - Every call returns an fr_status, never aborts and never traps; a
 *     human-readable reason for the last failure is in fr_ctx_last_error().
 *     Device-side failures (hash overflow, out-of-range coordinates) are
 *     recorded in device flags and mapped to a status when the call returns.
 *   - Work is issued on the context's CUDA stream; every call that launches
 *     work synchronises that stream before it returns (so that device-side
 *     error flags are reported by the call that raised them).
 *   - Handles (fr_ctx, fr_lattice) are owned by the library and released by
 *     the matching *_destroy call.  A context must be used by one host thread
 *     at a time.
 *   - Registration calls take the method's scalar parameters -- the sigma
 *     schedule, the outlier ratio w, the EM iteration count, the residual,
 *     blur and storage -- in one fr_options struct (fr_options_default fills
 *     it) rather than as separate arguments, so that one struct describes a
 *     registration for the single, batched and served forms alike.
 */
#ifndef FILTERREG_H
#define FILTERREG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FR_API __attribute__((visibility("default")))
#else
#define FR_API
#endif

typedef enum {
    FR_OK = 0,
    FR_EINVAL = 1,         /* bad argument: null pointer, size < 1, sigma <= 0, w outside [0,1),
                              non-finite input, coordinate beyond the lattice key range */
    FR_ENOMEM = 2,         /* device or pinned-host allocation failed */
    FR_ECUDA = 3,          /* a CUDA runtime call failed (message in fr_ctx_last_error) */
    FR_ECAPACITY = 4,      /* lattice hash table full (capacity_hint too small) */
    FR_ETIMEOUT = 5,       /* a bounded device-side wait expired */
    FR_ENOTSUPPORTED = 6   /* option combination not implemented */
} fr_status;

typedef enum { FR_PT2PT = 0, FR_PT2PL = 1 } fr_residual;
typedef enum { FR_FP32 = 0, FR_BF16 = 1, FR_FP16 = 2 } fr_storage;

typedef struct fr_ctx fr_ctx;
typedef struct fr_lattice fr_lattice;

/* Options of one registration.  fr_options_default() fills the defaults in
 * brackets. */
typedef struct {
    int32_t residual;           /* FR_PT2PT: Eq. 7; FR_PT2PL: Eq. 9-10            [PT2PT] */
    int32_t blur;               /* 1 = blur the lattice along its 4 axes before
                                   slicing (Section 4.2 "Blur"); 0 = splat+slice [0]   */
    int32_t iters;              /* EM iterations, one Gauss-Newton step each     [30]  */
    float sigma_start;          /* kernel std-dev of the first iteration          [0.02]*/
    float sigma_end;            /* of the last; geometric schedule in between;
                                   equal to sigma_start = fixed sigma, lattice built
                                   once (Section 3.2)                              [0.02]*/
    float w;                    /* outlier ratio of Section 3.1, 0 <= w < 1       [0.1] */
    int32_t storage;            /* lattice values read by the slice: FR_FP32, or
                                   FR_BF16 / FR_FP16 16-byte records made from the
                                   float32 sums (see fr_estep_storage); the 16-bit
                                   modes take no blur (FR_ENOTSUPPORTED)          [FP32]*/
    int32_t kahan;              /* 1 = Kahan-compensated float partial sums       [0]   */
    int32_t renormalize_normals;/* pt2pl: unit-normalise N_x of Eq. 9             [0]   */
    float stop_twist;           /* stop once |delta zeta| < stop_twist (Section 6.1's
                                   termination); 0 = run all iterations           [0]   */
    int32_t use_graph;          /* replay the EM loop as one CUDA graph           [1]   */
    int32_t update_sigma;       /* 1 = sigma as a decision variable (Section 3.3):
                                   re-estimated after every E step as
                                   sigma^2 = sum_i Q_i / (M0_i + c) / (3 sum_i W_i),
                                   Q_i = sum_j K_ij |x_i - y_j|^2, starting at
                                   sigma_start and floored at sigma_end; the lattice
                                   is rebuilt every iteration.  Point-to-point,
                                   float32 storage, no blur, fr_register_rigid only
                                   (FR_ENOTSUPPORTED otherwise)                    [0]   */
} fr_options;

/* Per-call diagnostics (all nullable where passed). */
typedef struct {
    int32_t iters_run;          /* EM iterations executed */
    int32_t degenerate_iters;   /* iterations whose 6x6 normal matrix was not positive
                                   definite (pose left unchanged that iteration) */
    int64_t last_inliers;       /* model points with M0 > 0 in the last iteration */
    double last_sum_w;          /* sum of outlier weights M0/(M0+c), last iteration */
    double last_cost;           /* sum of squared weighted residuals, last iteration */
    double last_twist_norm;     /* |delta zeta| of the last applied update */
    int64_t lattice_vertices;   /* vertices of the last lattice built */
    int32_t lattice_builds;     /* lattices built during the call (1, or one per sigma) */
    int64_t lattice_vertices_sum; /* vertices summed over those builds */
    double last_sigma;          /* sigma of the last iteration run */
} fr_report;

/* Kernel classes of the per-kernel profile. */
/* FR_K_CONVERT: a launch that only converts (and builds) ahead of the first
 * step under 16-bit storage; later conversions run inside FR_K_STEP launches.
 * FR_K_NG_ASSEMBLE / FR_K_NG_SOLVE: a node-graph iteration's E step with the
 * assembly of A and g (point and edge kernels), and its PCG solve with the
 * node update (timed as spans of launches).  FR_K_SLICE: the feature-space
 * E step's slice (its build and clear count as FR_K_BUILD and FR_K_CLEAR). */
enum {
    FR_K_CLEAR = 0, FR_K_BUILD = 1, FR_K_BLUR = 2, FR_K_STEP = 3, FR_K_CONVERT = 4,
    FR_K_NG_ASSEMBLE = 5, FR_K_NG_SOLVE = 6, FR_K_SLICE = 7, FR_K_CLASSES = 8
};
typedef struct {
    int64_t launches[FR_K_CLASSES]; /* kernels of each class timed since the last reset */
    double total_ms[FR_K_CLASSES];  /* their summed durations (CUDA events) */
} fr_profile;

FR_API void fr_options_default(fr_options *opt);
FR_API const char *fr_status_string(fr_status s);

/* ---- context ---------------------------------------------------------------
 * fr_ctx_create: bind a context to CUDA device `device` and the stream
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).  The
 * context owns a growable device workspace (lattice hash tables, reduction
 * partials) and small pinned host buffers.  FR_ECUDA if the device cannot be
 * used.  fr_ctx_destroy frees everything the context allocated. */
FR_API fr_status fr_ctx_create(int device, void *cuda_stream, fr_ctx **out);
FR_API fr_status fr_ctx_destroy(fr_ctx *ctx);
FR_API fr_status fr_ctx_set_stream(fr_ctx *ctx, void *cuda_stream);
/* fr_ctx_set_workspace_limit: the most device memory (bytes) the lattice-table
 * arena of batched registrations may hold; 0 (the default) = no limit.  A
 * batched call whose tables would need more fails with FR_ENOMEM before it
 * allocates -- including the safe-size rerun of items whose compact tables
 * overflowed, which then report FR_ENOMEM in their own status field. */
FR_API fr_status fr_ctx_set_workspace_limit(fr_ctx *ctx, size_t bytes);
FR_API const char *fr_ctx_last_error(const fr_ctx *ctx);
/* Number of kernels this context has launched (graph replays count each node). */
FR_API int64_t fr_ctx_kernel_launches(const fr_ctx *ctx);
/* fr_ctx_set_profiling: when on, registrations record a CUDA event pair on
 * the context's stream around every kernel they launch (inside the replayed
 * graph as event nodes) and accumulate each kernel class's launch count and
 * duration; fr_ctx_profile copies the totals to *out and, if reset, zeroes
 * them.  Off by default. */
FR_API fr_status fr_ctx_set_profiling(fr_ctx *ctx, int on);
/* fr_debug_fail_allocations: host-side fault injection for testing error
 * paths -- of the library's next device allocations (any context, any
 * thread) the first `after` proceed and the `n` after them fail as on a full
 * device, so that the call making them returns FR_ENOMEM with whatever it had
 * allocated before; n = 0 clears.  Nothing faults on the GPU.  FR_EINVAL for
 * a negative argument. */
FR_API fr_status fr_debug_fail_allocations(int32_t after, int32_t n);
/* Bytes this context has copied host->device and device->host (all calls). */
FR_API fr_status fr_ctx_transfer_bytes(const fr_ctx *ctx, int64_t *h2d, int64_t *d2h);
FR_API fr_status fr_ctx_profile(fr_ctx *ctx, fr_profile *out, int reset);

/* ---- permutohedral lattice primitives (Section 4.2) -------------------------
 * The lattice lives in the (d+1) = 4 dimensional hyperplane sum(z) = 0.  A
 * position p is scaled to the feature f = p / sigma (identity covariance,
 * Section 4.1), elevated, and assigned the 4 vertices of its enclosing simplex
 * with barycentric weights.  Keys are the vertices' integer coordinates.
 */

/* fr_lattice_embed: for n points d_pos (n x 4), write the 4 vertex keys of each
 * point's enclosing simplex, all four integer coordinates, to d_keys
 * (int32, n x 4 x 4: [point][vertex k][coordinate j]; vertex k has every
 * coordinate congruent to k mod 4) and the barycentric weights to d_bary
 * (float, n x 4).  Either output may be NULL.  FR_EINVAL if a coordinate is
 * non-finite or |elevated coordinate| >= 1e6 (that point's outputs are 0). */
FR_API fr_status fr_lattice_embed(fr_ctx *ctx, const float *d_pos, int64_t n, float sigma,
                                  int32_t *d_keys, float *d_bary);

/* fr_lattice_build: create a lattice over n points d_pos (n x 4) at scale
 * sigma: the hash table of their simplex vertices (no values yet).  The table
 * holds max(capacity_hint, 8 n) slots rounded up to a power of two.  The
 * lattice keeps each point's vertex slots and weights for fr_lattice_splat.
 * FR_ECAPACITY if the table fills; FR_EINVAL as for fr_lattice_embed. */
FR_API fr_status fr_lattice_build(fr_ctx *ctx, const float *d_pos, int64_t n, float sigma,
                                  int64_t capacity_hint, fr_lattice **out);

/* fr_lattice_splat: zero the lattice values and splat the n x val_dim float
 * values d_vals (row stride val_dim, 1 <= val_dim <= 8) of the build points
 * onto their vertices with the barycentric weights ("Splat" of Section 4.2;
 * the observation's values [1, y, n_y] of Eq. 11). */
FR_API fr_status fr_lattice_splat(fr_ctx *ctx, fr_lattice *lat, const float *d_vals, int val_dim);

/* fr_lattice_blur: one (1/2, 1, 1/2) pass along each of the 4 lattice axes
 * ("Blur" of Section 4.2); vertices absent from the table contribute 0 and
 * are not created. */
FR_API fr_status fr_lattice_blur(fr_ctx *ctx, fr_lattice *lat);

/* fr_lattice_slice: for m query points d_query (m x 4), write
 * out[i][c] = sum_k b_k value[key_k][c] (absent vertices contribute 0) to
 * d_out (float, m x val_dim) ("Slice" of Section 4.2; with the augmentation of
 * Eq. 13-14 the queries are never inserted). */
FR_API fr_status fr_lattice_slice(fr_ctx *ctx, const fr_lattice *lat, const float *d_query,
                                  int64_t m, float *d_out);

/* fr_lattice_vertices: write the lattice's vertices, in unspecified order, as
 * int32 keys d_keys (capacity x 4, all four coordinates) and float values
 * d_vals (capacity x val_dim; nullable), and their count to *n_vertices
 * (host).  Synchronises the stream. */
FR_API fr_status fr_lattice_vertices(fr_ctx *ctx, const fr_lattice *lat, int32_t *d_keys,
                                     float *d_vals, int64_t *n_vertices);
/* Vertex count, table capacity and value width (host outputs, nullable). */
FR_API fr_status fr_lattice_info(fr_ctx *ctx, const fr_lattice *lat, int64_t *n_vertices,
                                 int64_t *capacity, int32_t *val_dim);
FR_API fr_status fr_lattice_destroy(fr_ctx *ctx, fr_lattice *lat);

/* ---- E step (Eq. 6 and Eq. 9 via Section 4) ---------------------------------
 * fr_estep: build the lattice over the observation d_Y (N x 4) at sigma with
 * values [1, y] (d_Yn == NULL) or [1, y, n_y] (d_Yn, N x 4), blur it if
 * `blur`, and slice it at the model points moved by T (host double[16]):
 * d_out (float, M x 4 or M x 7) = [M0, M1 (3) (, Nsum (3))] of Eq. 6 / Eq. 9's
 * numerator, with the Gaussian's normalisation omitted as in Eq. 11.  This is
 * the same build and slice the registration runs, exposed for checking. */
FR_API fr_status fr_estep(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                          const float *d_Yn, int64_t N, float sigma, int blur,
                          const double T[16], float *d_out);
/* fr_gauss_transform: the exact E step (Section 4.1's Gauss transform, the
 * sums the lattice approximates): at x_i = T x_i (T host double[16], NULL =
 * identity) M0_i = sum_j K_ij, M1_i = sum_j K_ij y_j and, with d_Yn, the
 * normal sums of Eq. 9, K_ij = exp(-|x_i - y_j|^2 / (2 sigma^2)) unnormalised
 * (Eq. 11), over every observation -- O(N M) float32 work (each thread sums
 * 256-observation tiles before adding them to its totals).  d_out (float,
 * M x 4 or M x 7, as fr_estep) is overwritten.  FR_EINVAL for invalid
 * clouds, sigma <= 0 or a non-finite pose.  Synchronises the stream. */
FR_API fr_status fr_gauss_transform(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                    const float *d_Yn, int64_t N, float sigma, const double T[16],
                                    float *d_out);
/* fr_estep_storage: fr_estep without blur, with the lattice values read by
 * the slice stored as `storage` (fr_storage).  FR_FP32 is fr_estep itself;
 * FR_BF16 / FR_FP16 keep the splat's float32 sums and, once the build is
 * complete, round each vertex's values to one 16-byte record
 * [W, sum b (y - p_v) (3), sum b n (3), 0] re-centred on the vertex position
 * p_v (FR_FP16 also scales by 2^-e, e >= 0 the least with N 2^-e <= 2^14);
 * the slice restores W p_v in float32.  The paper stores the lattice in
 * float32 (Section 4.2); this mode has no counterpart there.  FR_EINVAL for
 * an unknown storage value, otherwise as fr_estep. */
FR_API fr_status fr_estep_storage(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                  const float *d_Yn, int64_t N, float sigma, int32_t storage,
                                  const double T[16], float *d_out);

/* ---- sharded single registration (model points split across ranks) -----------
 * One rigid registration whose model X is partitioned across ranks (one
 * process per GPU), every rank holding the whole observation Y: the E step's
 * sums and the Gauss-Newton sums of Eq. 17-18 are sums over model points, so
 * each rank forms its shard's normal equations, one all-reduce adds them, and
 * every rank solves the same 6 x 6 system and makes the same update (Eq. 16,
 * Eq. 18).  The collective is the caller's (NCCL, MPI, gloo, ...), passed as a
 * callback; the library owns the EM loop.
 *
 * The FR_NE_VALS values of one shard's normal equations, in order: A's upper
 * triangle row by row (21: A[0][0..5], A[1][1..5], ..., A[5][5]), b =
 * sum J^T r (6), the sum of outlier weights M0/(M0+c), the cost sum r^2, and
 * the number of model points with M0 > 0 -- all additive over shards. */
#define FR_NE_VALS 30

/* Normal-equation provider: at pose T (host double[16]) and scale sigma,
 * write this rank's FR_NE_VALS values to ne; return 0 or an fr_status. */
typedef int (*fr_ne_fn)(const double T[16], float sigma, double *ne, void *user);
/* Sum of n doubles in place over the ranks of one registration; return 0 on
 * success.  Every rank must call its collective the same number of times. */
typedef int (*fr_allreduce_fn)(double *vals, int n, void *user);

/* fr_rigid_normal_equations: one EM iteration's E step (lattice over d_Y at
 * sigma = opt->sigma_start, sliced at T x) and the Gauss-Newton sums of the
 * model points d_X (M x 4, one shard of a model of M_total points: Eq. 7's
 * outlier constant c = w/(1-w) N / M_total) written to ne (host
 * double[FR_NE_VALS]).  Options as for fr_register_rigid (iters, sigma_end and
 * stop_twist ignored); FR_ENOTSUPPORTED with update_sigma; FR_EINVAL for
 * M_total < M or a non-finite pose.  Synchronises the stream. */
FR_API fr_status fr_rigid_normal_equations(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                           const float *d_Yn, int64_t N, const fr_options *opt, int64_t M_total,
                                           const double T[16], double ne[FR_NE_VALS]);

/* fr_rigid_solve_update: the M step from summed normal equations: delta zeta
 * = -A^-1 b (float64 LDL^T; a pivot at or below 1e-12 of A's largest diagonal
 * entry makes A count as singular), T_inout <- exp(delta zeta^) T_inout (Eq.
 * 16, Eq. 18); |delta zeta| to *twist_norm (nullable).  FR_EINVAL if A is
 * singular or not positive definite (T_inout unchanged).  Host only: needs
 * no GPU and no context. */
FR_API fr_status fr_rigid_solve_update(const double ne[FR_NE_VALS], double T_inout[16], double *twist_norm);

/* fr_em_sharded: the EM loop of a sharded registration on the host: for each
 * iteration k of opt's geometric sigma schedule (as fr_register_rigid), the
 * provider's normal equations at the current pose, the all-reduce (NULL: a
 * single rank), fr_rigid_solve_update (a singular system counts as a
 * degenerate iteration and leaves the pose), and the stop test |delta zeta| <
 * stop_twist.  report (nullable) gets iters_run, degenerate_iters,
 * last_inliers, last_sum_w, last_cost, last_twist_norm and last_sigma.  A
 * non-zero return of a callback ends the call with it (FR_ECUDA if it is not
 * an fr_status).  FR_EINVAL for invalid options; FR_ENOTSUPPORTED with
 * update_sigma. */
FR_API fr_status fr_em_sharded(fr_ne_fn ne_fn, void *ne_user, fr_allreduce_fn allreduce, void *ar_user,
                               const fr_options *opt, double T_inout[16], fr_report *report);

/* fr_register_rigid_sharded: fr_em_sharded with this context's GPU as the
 * provider (fr_rigid_normal_equations of this rank's shard d_X, M points of a
 * model of M_total).  The lattice is rebuilt every iteration. */
FR_API fr_status fr_register_rigid_sharded(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                           const float *d_Yn, int64_t N, const fr_options *opt, int64_t M_total,
                                           fr_allreduce_fn allreduce, void *ar_user, double T_inout[16],
                                           fr_report *report);

/* ---- feature-space E step (Section 3.3, Eq. feature_estep) -------------------
 * The E step's Gaussian over d-dimensional per-point features (1 <= d <= 7)
 * with diagonal covariance diag(sigma_f^2): K_ij = exp(-sum_c (fx_ic -
 * fy_jc)^2 / (2 sigma_f[c]^2)), unnormalised as in Eq. 11.  Features are
 * row-major float rows of d values (d_FX: M x d of the model, d_FY: N x d of
 * the observation, 4-byte aligned; positions, normals, colours or any
 * descriptor, already expressed in the frame the caller wants compared);
 * sigma_f is a host array of d positive floats.  Filtering follows Section
 * 4.2 on the (d+1)-dimensional permutohedral lattice: g = f / sigma_f is
 * elevated with alpha = sqrt(2/3) (d+1), the enclosing simplex found, the
 * observation splatted, the model sliced (no blur; queries insert nothing).
 */

/* fr_feature_embed: the d+1 vertex keys (int32, n x (d+1) x (d+1):
 * [row][vertex k][coordinate j], vertex k's coordinates all congruent to k
 * mod d+1) and barycentric weights (float, n x (d+1)) of n feature rows d_F.
 * Either output may be NULL.  FR_EINVAL for d outside [1, 7], a sigma_f entry
 * that is not finite and > 0, or a row with a non-finite value or an elevated
 * coordinate of magnitude >= 1e6 (>= 131000 for d = 7, whose packed key
 * fields are 18 bits); such rows' outputs are 0.  Synchronises the stream. */
FR_API fr_status fr_feature_embed(fr_ctx *ctx, const float *d_F, int64_t n, int32_t d, const float *sigma_f,
                                  int32_t *d_keys, float *d_bary);

/* fr_estep_features: build the lattice over the observation features d_FY
 * with values [1, y] (d_Yn == NULL) or [1, y, n_y] (d_Y, d_Yn: N x 4 float,
 * 16-byte aligned) and slice it at the model features d_FX: d_out (float,
 * M x 4, 16-byte aligned, or M x 7) = [M0, M1 (3) (, Nsum (3))], the
 * feature-space counterparts of Eq. 6 / Eq. 9's numerators.  The number of
 * lattice vertices goes to *n_vertices (host, nullable).  The context keeps
 * the table (2 (d+1) N slots rounded up to a power of two, 32-byte records,
 * 64-byte with normals) between calls and empties only the slots each call
 * claimed.  FR_EINVAL as for fr_feature_embed (rows out of range contribute
 * nothing and read 0) or for more than 2^27 table slots; FR_ECAPACITY if a
 * probe sequence runs past 512 slots; FR_ENOMEM past the workspace limit.
 * Synchronises the stream. */
FR_API fr_status fr_estep_features(fr_ctx *ctx, const float *d_FX, int64_t M, const float *d_FY, int64_t N,
                                   int32_t d, const float *sigma_f, const float *d_Y, const float *d_Yn,
                                   float *d_out, int64_t *n_vertices);

/* fr_gauss_transform_features: the same sums without the lattice, every
 * model-observation pair in float32 (O(N M) work; observation tiles summed
 * on their own before joining each model point's totals).  d_out as for
 * fr_estep_features (4-byte aligned suffices).  FR_EINVAL for invalid
 * arguments.  Synchronises the stream. */
FR_API fr_status fr_gauss_transform_features(fr_ctx *ctx, const float *d_FX, int64_t M, const float *d_FY,
                                             int64_t N, int32_t d, const float *sigma_f, const float *d_Y,
                                             const float *d_Yn, float *d_out);

/* ---- rigid registration (Sections 3.1, 3.3, 4, 5) ---------------------------
 * fr_register_rigid: run opt->iters EM iterations aligning the model d_X
 * (M x 4) to the observation d_Y (N x 4).  Each iteration: (re)build the
 * lattice over Y when sigma changed (values [1, y] or [1, y, n_y]), slice it
 * at x_i = T x_i (E step), weight each point by M0/(M0 + c) with
 * c = w/(1-w) N/M (Eq. 7), form point-to-point (Eq. 7) or point-to-plane
 * (Eq. 10, d_Yn required, N x 4 normals) residuals, reduce A = sum J^T J and
 * b = sum J^T r over twists (Eq. 17-18, rigid: d zeta / d theta = I), solve
 * delta zeta = -A^{-1} b in float64 on the device and update
 * T <- exp(delta zeta^) T.  T_inout (host) carries the initial pose in and
 * the result out; report (nullable) receives diagnostics.  Synchronises the
 * stream.  FR_EINVAL for bad arguments or out-of-range inputs.  The lattice
 * table starts at 3 N slots (a power of two, inserts bounded to 128 probes);
 * a registration whose table overflows is rerun from its initial pose at
 * 6 N slots, which holds every vertex (at most 4 N), so FR_ECAPACITY here
 * indicates a bug. */
FR_API fr_status fr_register_rigid(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                   const float *d_Yn, int64_t N, const fr_options *opt,
                                   double T_inout[16], fr_report *report);

/* fr_register_rigid_host: the same registration from HOST buffers h_X
 * (M x 4), h_Y (N x 4), h_Yn (N x 4, nullable): the inputs are copied to a
 * context-owned device staging area on the context's stream (asynchronously
 * when the host buffers are pinned), then registered as above. */
FR_API fr_status fr_register_rigid_host(fr_ctx *ctx, const float *h_X, int64_t M,
                                        const float *h_Y, const float *h_Yn, int64_t N,
                                        const fr_options *opt, double T_inout[16],
                                        fr_report *report);

/* ---- articulated registration (Section 5.1, Eq. 20, Algorithm 1) -----------
 * A kinematic tree: body 0 is the root; every other body b has a parent
 * parent[b] < b.  Body b's frame is
 *     T_b = T_parent(b) * offset_b * R(axis_j1, q_j1) * R(axis_j2, q_j2) ...
 * over the revolute joints that move b (consecutive entries of joint_body,
 * which is non-decreasing); the root's parent frame is the root pose.  The
 * motion parameters are the root pose (6 DOF, updated by the exponential of
 * its twist) and the joint angles (added, then clamped to [q_min, q_max]). */
typedef struct {
    int32_t n_bodies;           /* 1..32 */
    int32_t n_joints;           /* 0..32 */
    const int32_t *parent;      /* [n_bodies]; parent[0] is ignored */
    const double *offset;       /* [n_bodies][16], row-major */
    const int32_t *joint_body;  /* [n_joints], non-decreasing, each in [0, n_bodies) */
    const double *joint_axis;   /* [n_joints][3], unit, in the frame the joint acts in */
    const double *q_min;        /* [n_joints], radians */
    const double *q_max;        /* [n_joints], radians */
} fr_kintree;

/* fr_register_articulated: EM registration of an articulated model.  The
 * model points d_Xref (M x 4) are given in their bodies' frames, d_body
 * (int32, M) names each point's body (points sorted by body run faster);
 * the observation d_Y (N x 4, + normals d_Yn for FR_PT2PL).  Each iteration
 * slices the lattice over Y at x_i = T_b(i) x_i_ref, sums J^T J and J^T r
 * per body over the body twists (Algorithm 1), assembles the
 * (6 + n_joints)^2 normal equations with the spatial velocity Jacobians
 * (world-frame twists about the origin; identity for the root,
 * (a; p x a) for a joint of world axis a through world point p, on every
 * body under the joint), solves them in float64 and updates the root pose
 * and the joint angles (clamped).  root_T_inout (host double[16]) and
 * q_inout (host double[n_joints]) carry the initial and the final
 * parameters.  FR_EINVAL for an invalid tree or arguments;
 * FR_ENOTSUPPORTED for blur or Kahan sums (rigid path only).  Synchronises
 * the stream. */
FR_API fr_status fr_register_articulated(fr_ctx *ctx, const float *d_Xref, const int32_t *d_body,
                                         int64_t M, const fr_kintree *tree, const float *d_Y,
                                         const float *d_Yn, int64_t N, const fr_options *opt,
                                         double root_T_inout[16], double *q_inout,
                                         fr_report *report);

/* ---- batched articulated registration ----------------------------------------
 * One registration of a batched articulated call: clouds as for
 * fr_register_articulated (device pointers), the initial root pose in
 * root_T (row-major, replaced by the result) and the joint angles in the
 * caller's host array q (double[n_joints], replaced by the result); status
 * is written by the call. */
typedef struct fr_articulated_item {
    const float *d_Xref;    /* M x 4, in the bodies' frames */
    const int32_t *d_body;  /* M, body of each point */
    int64_t M;
    const float *d_Y;       /* N x 4 */
    const float *d_Yn;      /* N x 4 normals (FR_PT2PL) or NULL */
    int64_t N;
    double root_T[16];      /* in: initial root pose; out: result */
    double *q;              /* host double[n_joints]: in initial, out result */
    int32_t status;         /* out: FR_OK or this item's failure */
} fr_articulated_item;

#define FR_ART_BATCH_MAX 4096 /* items per call */
#define FR_ART_CONCURRENT 16  /* registrations in flight together */

/* fr_register_articulated_batch: n_items articulated registrations of one
 * kinematic tree (Section 5.1, Algorithm 1) with the same options, each
 * exactly as fr_register_articulated would run it, up to FR_ART_CONCURRENT
 * of them at once, each on a stream of its own owned by ctx (created on
 * first use, destroyed with ctx), so that one registration's serial solve
 * overlaps the others' point work.  The items' streams start after the work
 * queued on ctx's stream when the call is made.  An item whose table
 * overflows is rerun alone at the safe size.  Returns FR_OK when every item
 * succeeded, else the first failing item's status (its pose and angles are
 * left as given; items[b].status tells each); reports (n_items, may be NULL)
 * receive each item's report.  FR_EINVAL for invalid arguments (checked
 * before any work), FR_ENOTSUPPORTED as fr_register_articulated.
 * Synchronises the items' streams. */
FR_API fr_status fr_register_articulated_batch(fr_ctx *ctx, const fr_kintree *tree,
                                               fr_articulated_item *items, int32_t n_items,
                                               const fr_options *opt, fr_report *reports);

/* ---- batched rigid registration ---------------------------------------------
 * One registration of a batch.  Clouds as for fr_register_rigid (device
 * pointers for fr_register_rigid_batch, host pointers for
 * fr_register_rigid_batch_host); sigma_start/sigma_end/w replace the options'
 * values for this item; T carries the initial pose in and the result out;
 * status receives this item's outcome. */
typedef struct {
    const float *d_X;
    int64_t M;
    const float *d_Y;
    const float *d_Yn;
    int64_t N;
    float sigma_start, sigma_end, w;
    double T[16];
    fr_status status;
} fr_batch_item;

/* fr_register_rigid_batch: register n_items independent pairs together, each
 * exactly as fr_register_rigid would (Sections 3.1, 4, 5) but with one launch
 * per EM iteration for the whole batch: every item's step, next-sigma build
 * and clear run side by side, so that one item's float64 solve overlaps the
 * others' work.  Items may differ in size and sigma schedule; they share
 * opt->residual, iters, kahan, renormalize_normals and stop_twist (blur is
 * not supported: FR_ENOTSUPPORTED).  1 <= n_items <= 16384 (13107 with 16-bit
 * storage: a launch's block-to-role map indexes its segments with 16 bits).
 * reports (nullable) has n_items entries.  An item whose compact lattice
 * table overflows is rerun (from its initial pose) with the items that
 * overflowed, at the size that cannot.
 * Launch shapes come from the context's tuning table (fr_tune_*); the
 * call's launch sequence is captured once per shape (item sizes, iteration
 * count, options) into a CUDA graph that later calls replay with new
 * descriptors.
 * Returns FR_OK, or the status of the first failed item (each item's own
 * outcome is in its status field; failed items keep their input pose).
 * Synchronises the stream. */
FR_API fr_status fr_register_rigid_batch(fr_ctx *ctx, fr_batch_item *items, int n_items,
                                         const fr_options *opt, fr_report *reports);
/* The same with the items' clouds in host memory: they are copied into a
 * context-owned device staging area on the context's stream first -- by one
 * gather kernel reading across the host link when every cloud lies in
 * page-locked (pinned) host memory, else by one copy per cloud.  Launches
 * are replayed from a CUDA graph cached per launch shape, as below. */
FR_API fr_status fr_register_rigid_batch_host(fr_ctx *ctx, fr_batch_item *items, int n_items,
                                              const fr_options *opt, fr_report *reports);

/* ---- launch-shape tuning ------------------------------------------------------
 * The batched path and the server size their launches from a per-context
 * table with five size classes by a cloud's observation count N (<= 4096,
 * <= 16384, <= 65536, <= 262144, larger); a class holds the parameters below.
 * Systems choices only (the paper has no counterpart): every setting
 * computes the same registration, up to float32 summation order.
 *   step_points_per_thread   model points per thread of a batched step block
 *   build_points_per_thread  observation points per thread of a batched
 *                            build block
 *   table_slots_x2           a compact lattice table holds at least
 *                            table_slots_x2 / 2 slots per observation point
 *                            (rounded up to a power of two; too small a table
 *                            overflows and the item reruns at the safe size)
 *   serve_points_per_thread  points per thread of a server tick's step and
 *                            build blocks (short chains keep ticks short)
 * Defaults: 8, 8, 6, 2; fr_ctx_create loads the table file named by the
 * environment variable FR_TUNE_TABLE, if set and well formed.
 * fr_tune_get / fr_tune_set read / write the class
 * that n_points falls in (FR_EINVAL outside 1..64 points per thread or 2..12
 * slots); fr_tune_save writes the table as text (one class per line),
 * fr_tune_load reads such a file (FR_EINVAL if malformed, the table
 * unchanged). */
typedef struct {
    int32_t step_points_per_thread;
    int32_t build_points_per_thread;
    int32_t table_slots_x2;
    int32_t serve_points_per_thread;
} fr_tune_params;
#define FR_TUNE_CLASSES 5
FR_API fr_status fr_tune_get(const fr_ctx *ctx, int64_t n_points, fr_tune_params *out);
FR_API fr_status fr_tune_set(fr_ctx *ctx, int64_t n_points, const fr_tune_params *p);
FR_API fr_status fr_tune_save(const fr_ctx *ctx, const char *path);
FR_API fr_status fr_tune_load(fr_ctx *ctx, const char *path);
/* fr_autotune_batch: time candidate launch shapes on the caller's batch
 * (device pointers, as for fr_register_rigid_batch; the items' poses and
 * statuses are left untouched) and install the fastest in the size class of
 * the items' mean N.  objective FR_TUNE_THROUGHPUT chooses the batched
 * parameters (step / build points per thread, table slots) by the whole
 * batch's time; FR_TUNE_LATENCY chooses serve_points_per_thread by the time
 * of the same batch run with one shape for step and build blocks (a serving
 * tick).  Each candidate runs `reps` times (median of CUDA-event times on the
 * context's stream).  *best receives the installed parameters; best_ms and
 * default_ms (nullable) the times of the chosen and of the default shape. */
enum { FR_TUNE_THROUGHPUT = 0, FR_TUNE_LATENCY = 1 };
FR_API fr_status fr_autotune_batch(fr_ctx *ctx, const fr_batch_item *items, int n_items,
                                   const fr_options *opt, int objective, int reps,
                                   fr_tune_params *best, double *best_ms, double *default_ms);

/* ---- node-graph deformable model (Section 5.2, Eq. 21) ----------------------
 * Nodes k = 0..K-1 with reference positions p_k and poses T_k; model point i
 * moves by the dual-quaternion blend of its 4 nodes' poses with fixed
 * skinning weights (Eq. 21): x_i = normalized(sum_k w_ki dq(T_k)) x_i_ref,
 * the node dual quaternions sign-aligned with the largest-weight node's.
 * The supplement the paper defers to for the M step is not available; this
 * library reads it as: one twist per node, T_k <- exp(dzeta_k^) T_k; a
 * point's twist is the weighted sum of its nodes' (the first-order blend
 * derivative), so the rigid point terms (Eq. 7 / Eq. 10) enter block (a, b)
 * of A with weight w_a w_b; a regulariser adds, for every directed edge
 * (j, k), the residual sqrt(lambda)/sigma (T_j p_k - T_k p_k); the system is
 * solved by block-Jacobi preconditioned conjugate gradients, pcg_iters
 * iterations from zero, in float64 (blocks accumulated in float32). */
typedef struct fr_nodegraph fr_nodegraph;

/* Prepare a model on ctx's device: d_Xref (M x 4 float), d_knn (M x 4
 * int32 node ids) and d_skw (M x 4 float weights, >= 0) are device arrays,
 * copied (sorted by node tuple) -- the caller may free them afterwards;
 * node_pos (host, K x 3 double) and edges (host, E x 2 int32 directed
 * regulariser edges, no self-edges).  Synchronises the stream.  FR_EINVAL
 * for out-of-range ids, negative or non-finite weights, bad sizes. */
FR_API fr_status fr_nodegraph_create(fr_ctx *ctx, const float *d_Xref, const int32_t *d_knn,
                                     const float *d_skw, int64_t M, const double *node_pos, int K,
                                     const int32_t *edges, int E, fr_nodegraph **out);
/* Free the model (waits for the device; may follow fr_ctx_destroy). */
FR_API fr_status fr_nodegraph_destroy(fr_nodegraph *g);
/* opt->iters EM iterations (sigma schedule as fr_register_rigid; the lattice
 * is rebuilt when sigma changes) of the node-graph model against d_Y (N x 4)
 * (+ normals d_Yn for FR_PT2PL).  node_T (host, K x 16 row-major) carries
 * the initial poses in and the result out.  storage may be FR_FP32 or a
 * 16-bit mode (records converted after each build, read by the point
 * kernel); blur, kahan and stop_twist must be 0 (FR_ENOTSUPPORTED
 * otherwise); lambda >= 0;
 * 0 <= pcg_iters <= 10000.  rep (nullable): last iteration's inliers,
 * weight sum, cost (data + regulariser) and update norm. */
FR_API fr_status fr_register_nodegraph(fr_ctx *ctx, fr_nodegraph *g, const float *d_Y, const float *d_Yn,
                                       int64_t N, const fr_options *opt, double lambda, int pcg_iters,
                                       double *node_T, fr_report *rep);
/* One E step at sigma = opt->sigma_start and the Gauss-Newton system at the
 * node poses node_T: A_out (host, dense 6K x 6K, nullable) and g_out (host,
 * 6K, nullable), A dtheta = -g -- the assembly the registration runs,
 * exposed for checking. */
FR_API fr_status fr_nodegraph_system(fr_ctx *ctx, fr_nodegraph *g, const float *d_Y, const float *d_Yn,
                                     int64_t N, const fr_options *opt, double lambda,
                                     const double *node_T, double *A_out, double *g_out, fr_report *rep);
/* The model points warped by node_T (Eq. 21) into d_out (device, M x 4
 * float, the caller's point order). */
FR_API fr_status fr_nodegraph_warp(fr_ctx *ctx, fr_nodegraph *g, const double *node_T, float *d_out);

/* ---- serving: continuous batching -------------------------------------------
 * A server registers a stream of independent pairs (the rigid EM of
 * fr_register_rigid, Sections 3.1, 4, 5) with continuous batching: a worker
 * thread launches one batched EM kernel per tick over every live request,
 * each at its own iteration (a request's first tick builds its first
 * lattice; each later tick runs its next iteration; a last tick frees its
 * tables), admitting queued requests between ticks while their memory fits.
 * The paper has no counterpart; it runs one registration at a time.
 *
 * Memory: fr_server_create reserves `device_mem_budget` bytes on the
 * context's device once -- half for lattice tables (hash slots kept empty
 * between requests), half for per-request records and copied clouds -- and
 * admits a request only when its tables and records fit (first come, first
 * served).  A request that could never fit is refused at submission
 * (FR_ENOMEM).  At most `max_live` requests run at once (1..4096).
 *
 * The server has its own CUDA stream and thread; the context must outlive
 * it and may be used for other calls meanwhile.  Options (residual, iters,
 * kahan, renormalize_normals, storage) are fixed per server; with 16-bit
 * storage a build's records are converted in the tick after it (one more
 * tick per request); blur must be 0 (FR_ENOTSUPPORTED otherwise);
 * stop_twist is honoured. */
typedef struct fr_server fr_server;

/* One request.  Clouds are N x 4 / M x 4 float rows (16-byte aligned).
 * host == 0: device pointers, borrowed -- they must stay valid and unchanged
 * until the request completes.  host == 1: host pointers, copied to the
 * device when the request is admitted -- they too must stay valid until the
 * request completes (or until fr_server_destroy returns). */
typedef struct {
    const float *X;
    int64_t M;
    const float *Y;
    const float *Yn;            /* normals, FR_PT2PL only */
    int64_t N;
    float sigma_start, sigma_end, w;
    double T[16];               /* initial pose, row-major */
    int32_t host;
} fr_request;

/* What fr_server_poll reports for a completed request. */
typedef struct {
    fr_status status;           /* FR_OK, or the request's own error */
    double T[16];               /* final pose (initial pose on error) */
    fr_report report;
    int64_t submit_ns, admit_ns, complete_ns;  /* steady-clock timestamps */
} fr_result;

FR_API fr_status fr_server_create(fr_ctx *ctx, size_t device_mem_budget, int max_live,
                                  const fr_options *opt, fr_server **out);
/* Queue a request; *ticket identifies it.  FR_EINVAL for bad arguments,
 * FR_ENOMEM if it cannot fit the server's budget even alone. */
FR_API fr_status fr_server_submit(fr_server *srv, const fr_request *req, uint64_t *ticket);
/* *done = 1 and *out filled (nullable) once the request has completed;
 * *done = 0 otherwise.  A completed ticket stays readable until
 * fr_server_release.  FR_EINVAL for an unknown ticket. */
FR_API fr_status fr_server_poll(fr_server *srv, uint64_t ticket, int *done, fr_result *out);
/* Block until the request completes or timeout_ms passes (< 0: no limit);
 * FR_ETIMEOUT on timeout. */
FR_API fr_status fr_server_wait(fr_server *srv, uint64_t ticket, int64_t timeout_ms, fr_result *out);
/* Forget a completed ticket. */
FR_API fr_status fr_server_release(fr_server *srv, uint64_t ticket);
/* Counters: ticks launched, requests completed, kernels launched. */
FR_API fr_status fr_server_stats(const fr_server *srv, int64_t *ticks, int64_t *completed,
                                 int64_t *kernel_launches);
/* Finish every queued and live request, stop the worker, free the memory. */
FR_API fr_status fr_server_destroy(fr_server *srv);

/* ---- E step without allocation ---------------------------------------------
 * The paper has no counterpart to this entry point: it serves callers that
 * cannot call cudaMalloc -- a host framework whose allocator has reserved
 * the device's memory and forbids other allocations, or a real-time loop that
 * must not take the device-wide synchronisation cudaMalloc / cudaFree can
 * cause.
 *
 * fr_estep_noalloc: the E step of fr_estep without blur -- lattice over the
 * observation d_Y (N x 4) with values [1, y] (d_Yn == NULL) or [1, y, n_y]
 * (d_Yn, N x 4), sliced at the model points d_X (M x 4) moved by T (host
 * double[16]) -- written to d_out (float, M x 4 or M x 7) on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default) of the current device.  It needs no
 * context and allocates nothing: the hash table lives in a fixed scratch
 * array compiled into the library (about 4.5 MB on every device that loads
 * it, held until the process exits).  The first call on a device finds that
 * array's device address and empties it (synchronising the stream once); it
 * should come before any stream capture: made on a capturing stream it
 * returns FR_EINVAL and the set-up is tried again by the next call (a failed
 * set-up is never remembered).  Every call shares the array and
 * leaves it empty; calls that overlap on the GPU race and give wrong results.
 * Synchronises the stream.  FR_EINVAL for null or misaligned pointers,
 * M < 1, N < 1, N > FR_NOALLOC_MAX_OBS, sigma <= 0, a non-finite pose or
 * input; FR_ECAPACITY if the table fills; FR_ECUDA if a CUDA call fails. */
#define FR_NOALLOC_MAX_OBS 8192
FR_API fr_status fr_estep_noalloc(const float *d_X, int64_t M, const float *d_Y,
                                  const float *d_Yn, int64_t N, float sigma, const double T[16],
                                  float *d_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FILTERREG_H */
