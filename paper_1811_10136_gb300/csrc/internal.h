// Internal interfaces between the C-ABI host code (api.cu) and the kernels
// (kernels.cu).  Not installed, not part of the ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fr {

// Number of values each rigid reduction carries: the 21 upper-triangular
// entries of A = sum J^T J, the 6 of b = sum J^T r (Eq. 18), then
// sum of outlier weights, sum of squared residuals, the inlier count and --
// with the sigma update -- sum_i Q_i / (M0_i + c), Q_i = sum_j K_ij |x_i - y_j|^2.
constexpr int kRigidVals = 31;
// Points per thread of the step and build blocks of a batched launch: fewer,
// fuller blocks amortise each step block's 30-value reduction and each build
// block's list append, while the other registrations keep the GPU full.  (A
// single registration runs one point per thread: its blocks must fill the GPU
// by themselves; a serving tick, rarely a full GPU, runs two.)
constexpr int kMultiPointsPerThread = 8;
constexpr int kBlock = 256;

// Device flags (DeviceState::flags).
constexpr int kFlagRange = 1;     // non-finite or out-of-range coordinate
constexpr int kFlagCapacity = 2;  // hash table full

// Per-EM-iteration constants, computed on the host from the sigma schedule.
struct IterParams {
    float sigma;
    float s1, s2, s3;      // feature scales alpha / (sqrt(i (i+1)) sigma)
    float c_eff;           // outlier constant in the lattice kernel's units
    float inv_sigma2;      // Sigma^{-1} of Eq. 7
    int rebuild;           // lattice rebuilt at this iteration
    int nvert;             // vertices created by this iteration's build (device counter)
    float vscale;          // power of two applied to 16-bit records (keeps half below its range)
    float inv_vscale;
    float ws1, ws2, ws3;   // world units per key unit: 1/(2 s1), 1/(6 s2), 1/(12 s3)
    int pad[3];
};

// The per-call job: user buffers and sizes (copied to the device each call so
// that a captured graph can be replayed on new buffers).
struct RigidJob {
    const float4 *X;
    const float4 *Y;
    const float4 *Yn;
    int M, N;
    int renormalize;
    float stop_twist;
    double T0[16];         // initial pose
    // sigma as a decision variable (point-to-point): the constants the last
    // step block needs to set up the next iteration's parameters
    double sig_alpha[3];   // alpha / sqrt(i (i+1)), i = 1..3
    double sig_c;          // w / (1 - w) N / M
    double sig_G;          // kernel mass of the lattice
    double sig_floor;      // smallest sigma
    double sig_kappa;      // the lattice kernel's per-axis variance over sigma^2
};

// Device-resident state of one registration.
struct DeviceState {
    double T[16];          // current pose, row-major
    double sum_w, cost, twist_norm;
    long long inliers;
    int iters_run, degenerate;
    int done;              // stop_twist reached: later kernels return at once
    int ticket;            // last-block-done counter of the grid reduction
    int flags;
    int nvert;             // vertices created by the last build
    int builds;            // lattices built during this call
    long long nvert_total; // vertices summed over this call's builds
    // the last iteration's reduced Gauss-Newton values: A's upper triangle row
    // by row (21), b = sum J^T r (6), sum of weights, cost, inliers, sigma moment
    double sums[32];
};

// A lattice hash table: a power-of-two array of 64-byte slot records, two
// 32-byte sectors each --
//   sector 0: [key (8 B), unused (8 B), v0 = channels 0..3 (float4)]
//   sector 1: [v1 = channels 4..7 (float4), unused (16 B)]
// -- so that a lookup and its values, an insert's CAS and atomics touch one
// line, and a clear writes whole sectors.  With 16-bit storage the record
// [W, sum b (y - p_v), sum b n, 0] (16 B) is written over v0 once the build
// is complete (the convert role has read the float32 sums), so a 16-bit
// lookup reads one 16-byte record beside its key.  A free slot is all zero:
// kEmpty = 0 and every valid key has bit 63 set, so clearing a slot is
// zeroing its record.
constexpr int kRecWords = 8;  // 64-bit words per record
constexpr unsigned long long kEmpty = 0ull;

struct Table {
    unsigned long long *keys;  // slot s: keys + kRecWords * s
    uint32_t mask;             // capacity - 1 (capacity a power of two)
    uint32_t max_probe;        // an insert that probes this many taken slots reports overflow
    int vals;                  // value channels kept: 4 or 8
};

__host__ __device__ __forceinline__ unsigned long long *rec_key(unsigned long long *keys, uint32_t s) {
    return keys + (size_t)s * kRecWords;
}
// The 16-bit record (16-bit storage modes, after conversion): v0's place.
__host__ __device__ __forceinline__ uint4 *rec_cv(unsigned long long *keys, uint32_t s) {
    return reinterpret_cast<uint4 *>(keys + (size_t)s * kRecWords + 2);
}
__host__ __device__ __forceinline__ float4 *rec_v0(unsigned long long *keys, uint32_t s) {
    return reinterpret_cast<float4 *>(keys + (size_t)s * kRecWords + 2);
}
__host__ __device__ __forceinline__ float4 *rec_v1(unsigned long long *keys, uint32_t s) {
    return reinterpret_cast<float4 *>(keys + (size_t)s * kRecWords + 4);
}
// Bytes of a table of `slots` records.
inline size_t table_bytes(size_t slots) { return slots * kRecWords * sizeof(unsigned long long); }

// Lattice value storage of the slice (fr_storage): the float32 sums, or the
// 16-byte record [W, sum b (y - p_v) (3), sum b n (3), 0] in bfloat16 / half,
// made from them once a build completes (p_v: the vertex's position).
constexpr int kStoreF32 = 0, kStoreBF16 = 1, kStoreF16 = 2;

// Table sizing.  A point creates at most 4 vertices, so 6 N slots can never
// fill; but a lattice over a surface usually has far fewer vertices than 4 N
// (0.05 N to 0.5 N for dense depth frames, up to ~1.5 N for sparse ones at a
// small sigma), and a table sized to match keeps its working set small.  The
// compact size (3 N, so at most half full up to 1.5 N vertices) is tried
// first with inserts bounded to 128 probes -- which also bounds every lookup,
// present or absent; an overflow reruns the registration at the safe size.
inline uint32_t table_slots(long long n_points, bool safe) {
    const long long want = safe ? 6 * n_points : 3 * n_points;
    uint32_t c = 1024;
    while ((long long)c < want && c < (1u << 30)) c <<= 1;
    return c;
}
inline uint32_t table_probe_limit(uint32_t cap, bool safe) { return safe ? cap : (cap < 128 ? cap : 128); }

// One fused EM-iteration launch: blocks [0, gs) run the step of iteration
// `it` on table `step` (slice, residuals, reduction, last-block solve);
// blocks [gs, gs + gb) build the lattice of iteration `build_it` into table
// `build` (gb = 0: no build); blocks [gs + gb, gs + gb + gc) clear table
// `clear` (gc = 0: none).  Any role may be empty.
// Lattice tables in rotation: a build runs `lead` iterations ahead of the
// step that reads it (1 with float32 storage; 2 with 16-bit storage, whose
// records are converted one launch after the build completes), so up to
// lead + 2 tables are live (cleared, stepped, converted, built).
constexpr int kMaxTables = 4;

struct IterLaunch {
    const RigidJob *job;
    IterParams *ip;
    int it, build_it, clear_it;  // clear_it: the build whose table is cleared
    int conv_it;                 // the build whose table is converted
    Table step, build, clear, conv;
    int *build_list;       // slots claimed by the build (count: ip[build_it].nvert)
    const int *clear_list; // slots to free (count: ip[clear_it].nvert)
    const int *conv_list;  // slots to convert (count: ip[conv_it].nvert)
    float2 *partials;      // gs rows of kRigidVals (hi, lo) float pairs
    DeviceState *st;
    int gs, gv, gb, gc;    // blocks of the roles, in this order
    int check_done;        // roles return at once once st->done is set
    int sig_next;          // sigma update: the step sets up ip[it + 1] (it + 1 < iterations)
};

// ---- articulated model -------------------------------------------------------
constexpr int kMaxBodies = 32;
constexpr int kMaxJoints = 32;
constexpr int kMaxDof = 6 + kMaxJoints;
constexpr int kArtVals = 30;  // per body: 21 of J^T J, 6 of J^T r, weight sum, cost, count

// Kinematic tree (device copy).  Body 0 is the root; parent[b] < b.  Body b's
// frame is T_parent * offset_b * R(axis_j, q_j) ... over its joints
// [joint_begin[b], joint_begin[b+1]).
struct ArtTree {
    int nb, nj;
    int parent[kMaxBodies];
    unsigned sub[kMaxBodies];       // bit c set when body c is in the subtree of b (b included)
    int joint_begin[kMaxBodies + 1];
    int joint_body[kMaxJoints];
    float offset[kMaxBodies][12];   // row-major 3 x 4
    float axis[kMaxJoints][3];      // unit, in the frame the joint acts in
    double q_min[kMaxJoints], q_max[kMaxJoints];
};

struct ArtJob {
    RigidJob base;      // X = model points in body frames, Y, Yn, M, N, flags
    const int *body;    // body of each model point
    ArtTree tree;
};

struct ArtState {
    DeviceState ds;                         // ticket, flags, diagnostics, vertex counters
    double root_T[16];
    double q[kMaxJoints];
    float body_T[kMaxBodies][12];           // every body's pose at the current parameters
    float jaxis[kMaxJoints][3];             // world joint axes ...
    float jpoint[kMaxJoints][3];            // ... and a world point on each
    double acc[kMaxBodies][kArtVals];       // subtree sums of the running iteration (body b: the bodies under b)
};

struct ArtLaunch {
    const ArtJob *job;
    IterParams *ip;
    int it, build_it, clear_it, conv_it;
    Table step, build, clear, conv;
    int *build_list;
    const int *clear_list;
    const int *conv_list;
    ArtState *st;
    int gs, gv, gb, gc;
};

// One registration of a multi-registration launch (device-resident).
struct Slot {
    const RigidJob *job;
    DeviceState *st;
    IterParams *ip;        // [iters] of this registration
    float2 *partials;      // >= step blocks per launch rows of kRigidVals pairs
    Table tab[kMaxTables]; // rotating lattice tables
    int *list[kMaxTables]; // slots claimed by each table's last build
};

enum { kRoleNone = 0, kRoleStep = 1, kRoleBuild = 2, kRoleClear = 3, kRoleConvert = 4 };

// A run of nblk consecutive blocks (from blk0) doing one role for one slot:
// step of iteration `it` on table `tab`; build of iteration `it` into `tab`;
// clear of `tab`, whose claimed slots build `it` listed; or conversion of
// `tab` (build `it`) to 16-bit records.
struct Seg {
    int slot, role, it, tab;
    int blk0, nblk;
};

// ---- node-graph model (Section 5.2, Eq. 21) ----------------------------------
// Model points are stored sorted by their (node id sorted) 4-node tuple, so a
// run of points -- a segment -- shares its nodes and its 10 node-pair blocks
// (a <= b) of A.  Blocks are 6 x 6 float, row-major, rows of node a.
constexpr int kNgPairs = 10;  // tuple pairs (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),(2,2),(2,3),(3,3)

struct NgPoints {
    const float4 *X;        // model points (reference), segment-sorted
    const float4 *w;        // their skinning weights, in the tuple's order
    const int *perm;        // sorted position -> caller's index (warp output)
    const int *seg_start;   // S + 1
    const int4 *seg_nodes;  // S tuples (ascending node ids)
    const int *seg_blk;     // S x 10 block ids of the tuple pairs
    const float *seg_coef;  // S x 10: 2 for a repeated node off the diagonal, else 1
    int S;
    const float *node_dq;   // K x 8 dual quaternions of the node poses
    Table tab;              // the lattice over the observation
    const IterParams *ip;
    int renorm;
    float *blocks;          // nnzb x 36 accumulators
    float *g;               // 6 K accumulators
    double *stats;          // [sum of weights, cost]
    unsigned long long *inliers;
    int *flags;
    float4 *warp_out;       // warp only: warped points in the caller's order
};

struct NgEdges {
    const int2 *edges;      // E directed edges (j, k)
    const int *edge_blk;    // E x 3: blocks (j, j), (k, k), (min, max)
    int E;
    const double *node_T;   // K x 16
    const double *node_pos; // K x 3
    double lambda;
    const IterParams *ip;
    float *blocks, *g;
    double *stats;
};

// Block-Jacobi PCG over the node blocks, float64 vectors.
// The per-node PCG kernels give each node six consecutive lanes (one per
// component; lanes 30 and 31 of a warp idle) and run 64-thread blocks, so
// that their float64 work spreads over many SMs.
constexpr int kNgPcgBlock = 64;
constexpr int kNgNodesPerWarp = 5;
inline int ng_pcg_grid(int K) {
    const int per_block = kNgPcgBlock / 32 * kNgNodesPerWarp;
    return (K + per_block - 1) / per_block;
}
// The block-row product runs one warp per row.
inline int ng_spmv_grid(int K) { return (K + kNgPcgBlock / 32 - 1) / (kNgPcgBlock / 32); }

struct NgPcg {
    int K;
    int nnzb;
    const int *row_ptr;     // K + 1
    const int2 *ent;        // (block | transposed << 31, partner node)
    const int *diag_blk;    // K
    const float *blocks;
    double *blocks_d;       // float64 copy of the blocks, made by the set-up kernel
    const float *g;
    double *P;              // K x 36 preconditioner
    double *x, *r, *z, *Ap;
    const double *p_old;
    double *p_new;
    double *scal;           // [rz, alpha, beta, stop]
    double *partial;        // per-block partial sums
    int *ticket;
};

// ---- launchers (kernels.cu) -------------------------------------------------
void launch_em_multi(int pt2pl, int kahan, const Slot *slots, const Seg *segs,
                     const unsigned short *blockseg, int grid, int check_done, cudaStream_t s,
                     int storage);
void launch_art_iter(int pt2pl, const ArtLaunch &a, cudaStream_t s, int storage);
void launch_em_iter(int pt2pl, int kahan, const IterLaunch &a, cudaStream_t s, int storage);
// The same roles with sigma as a decision variable (point-to-point, float32):
// builds splat the extra moment, steps add Q_i / (M0_i + c) and the last step
// block writes the next iteration's parameters.
void launch_em_iter_sigma(int kahan, const IterLaunch &a, cudaStream_t s);
void launch_zero_values(Table t, int grid, cudaStream_t s);
void launch_ng_points(int pt2pl, const NgPoints &a, int warp_only, cudaStream_t s, int storage = kStoreF32);
void launch_ng_edges(const NgEdges &a, cudaStream_t s);
void launch_ng_pcg_init(const NgPcg &a, cudaStream_t s);
void launch_ng_pcg_spmv(const NgPcg &a, cudaStream_t s);
void launch_ng_pcg_update(const NgPcg &a, cudaStream_t s);
// T_k <- exp(dx_k) T_k (dx nullable: none) and the nodes' dual quaternions;
// |dx|^2 added to *twist2.
void launch_ng_update(int K, const double *dx, double *node_T, float *node_dq, double *twist2,
                      cudaStream_t s);
int em_iter_blocks_per_sm(int pt2pl, int kahan);
// Frees the slots listed by builds (list lists[i], count *counts[i]).
void launch_clear_lists(const Table *tabs, int *const *lists, const int *const *counts, int n,
                        int grid, cudaStream_t s);
void launch_blur_pass(Table in, Table out, int dir, int grid, const DeviceState *st, cudaStream_t s);
// A blur pass over the `*count` slots of `list` (a build's claimed slots).
void launch_blur_list(Table in, Table out, int dir, const int *list, const int *count, int grid,
                      const DeviceState *st, cudaStream_t s);
void launch_estep_out(int pt2pl, const RigidJob *job, const IterParams *ip, Table t, float *out,
                      DeviceState *st, int grid, cudaStream_t s, int storage);

// Lattice primitives.
void launch_embed(const float4 *P, int n, float s1, float s2, float s3, int *keys, float *bary,
                  int *flags, cudaStream_t s);
void launch_build_records(const float4 *P, int n, float s1, float s2, float s3, Table t,
                          int *rec_slot, float *rec_w, int *counters, cudaStream_t s);
void launch_splat_records(const float *vals, int vdim, int n, const int *rec_slot,
                          const float *rec_w, Table t, cudaStream_t s);
void launch_slice_out(const float4 *Q, int m, float s1, float s2, float s3, Table t, int vdim,
                      float *out, int *flags, cudaStream_t s);
void launch_vertices(Table t, int vdim, int *keys_out, float *vals_out, int *count,
                     cudaStream_t s);

int max_resident_blocks(const void *kernel_tag);

}  // namespace fr
