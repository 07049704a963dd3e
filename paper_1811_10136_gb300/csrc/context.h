// Internal host-side context of the C ABI, shared by the translation units
// that implement it (api.cu: context, lattice primitives, single
// registration; batch.cu: batched registration and the serving loop).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "filterreg.h"
#include "internal.h"

namespace fr {
struct BatchWorkspace;
struct ArtWorkspace;
struct ServerState;
struct FeatWorkspace;
}

namespace fr {

// Lattice scale alpha = sqrt(2/3) (d+1): splat-blur-slice then approximates a
// unit-std Gaussian in feature units (Section 4.2 / Adams et al. 2010).
inline const double kAlpha = std::sqrt(2.0 / 3.0) * 4.0;

// Integral of the unnormalised splat+slice kernel over feature space: the
// volume per lattice point of the remainder-class union in the hyperplane,
// (d+1)^(d - 1/2), divided by alpha^d; each blur pass doubles it.
inline double lattice_kernel_mass(int blur) {
    double g = std::pow(4.0, 2.5) / std::pow(kAlpha, 3.0);
    return blur ? g * 16.0 : g;
}

// Per-axis variance of the unblurred splat+slice kernel in units of sigma^2,
// averaged over positions: 2 M2 / (d covol), M2 the second moment of one
// vertex's hat.  The hat is linear on (d+1)! congruent simplices of volume
// covol / d! around its vertex, and the simplex moments give
// M2 = covol (|sum_k v_k|^2 + sum_k |v_k|^2) / ((d+2)(d+3)) over the
// canonical simplex's vertices v_1..v_d in feature units (1/4 for d = 3).
inline double lattice_kernel_variance() {
    constexpr int d = 3, D = 4;
    double colsum[D] = {0.0, 0.0, 0.0, 0.0}, norms = 0.0;
    for (int k = 1; k <= d; ++k)
        for (int j = 0; j < D; ++j) {
            const double c = j + k < D ? (double)k : (double)(k - D);  // canonical vertex k
            colsum[j] += c;
            norms += c * c;
        }
    double sumsq = 0.0;
    for (int j = 0; j < D; ++j) sumsq += colsum[j] * colsum[j];
    return 2.0 * (sumsq + norms) / (kAlpha * kAlpha) / (double)(d * (d + 2) * (d + 3));
}

inline void feature_scales(float sigma, float s[3]) {
    for (int i = 1; i <= 3; ++i)
        s[i - 1] = (float)(kAlpha / std::sqrt((double)(i * (i + 1))) / (double)sigma);
}

// Sigma of iteration k of the geometric schedule from sigma_start to
// sigma_end over o->iters iterations (Section 3.2's annealing), in float.
inline float schedule_sigma(const fr_options *o, int k) {
    const double s0 = o->sigma_start, s1 = o->sigma_end;
    if (o->iters <= 1 || s0 == s1) return (float)s0;
    return (float)(s0 * std::pow(s1 / s0, (double)k / (double)(o->iters - 1)));
}

inline uint32_t pow2_at_least(long long n) {
    uint32_t c = 1024;
    while ((long long)c < n && c < (1u << 30)) c <<= 1;
    return c;
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// A named NVTX range over one C-ABI call: what profilers show and filter on
// (ncu --nvtx --nvtx-include "<name>/"); without an attached tool a push and
// a pop are a few instructions.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Everything a captured graph bakes in besides the job descriptor.
struct GraphKey {
    int v[14];
    uint64_t ws_gen;
    bool operator==(const GraphKey &o) const {
        return ws_gen == o.ws_gen && std::memcmp(v, o.v, sizeof v) == 0;
    }
};

// Launch-shape tuning table: five size classes by observation count.
constexpr int kTuneClasses = 5;
inline int tune_class(long long n) {
    return n <= 4096 ? 0 : n <= 16384 ? 1 : n <= 65536 ? 2 : n <= 262144 ? 3 : 4;
}
inline fr_tune_params tune_default() { return fr_tune_params{8, 8, 6, 2}; }
inline bool tune_valid(const fr_tune_params &p) {
    auto ppt = [](int v) { return v >= 1 && v <= 64; };
    return ppt(p.step_points_per_thread) && ppt(p.build_points_per_thread) && ppt(p.serve_points_per_thread) &&
           p.table_slots_x2 >= 2 && p.table_slots_x2 <= 12;
}
// Compact table slots for N observation points: at least x2 / 2 per point.
inline uint32_t tuned_table_slots(long long n_points, int x2) {
    const long long want = (x2 * n_points + 1) / 2;
    uint32_t c = 1024;
    while ((long long)c < want && c < (1u << 30)) c <<= 1;
    return c;
}

struct CachedGraph {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    uint64_t last_use = 0;
};

// Host-side fault injection (fr_debug_fail_allocations): the library's next
// `skip` device allocations proceed, the `fail` after them fail as a full
// device's would.
std::atomic<int> &alloc_skip();   // api.cu
std::atomic<int> &alloc_fail();   // api.cu
inline bool take_one(std::atomic<int> &c) {
    int n = c.load();
    while (n > 0 && !c.compare_exchange_weak(n, n - 1)) {
    }
    return n > 0;
}
inline cudaError_t dev_malloc(void **p, size_t bytes) {
    if (!take_one(alloc_skip()) && take_one(alloc_fail())) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

template <typename T>
inline cudaError_t dev_alloc(T **p, size_t count) {
    return dev_malloc((void **)p, count * sizeof(T) + 16);
}

}  // namespace fr

struct fr_lattice {
    uint32_t cap = 0;
    int n = 0;
    int vdim = 0;
    float scale[3] = {0, 0, 0};
    unsigned long long *keys = nullptr;   // slot records (see Table)
    unsigned long long *tkeys = nullptr;  // blur ping-pong records
    int *rec_slot = nullptr;
    float *rec_w = nullptr;
    int *counters = nullptr;  // [0] vertices, [1] flags, [2] scratch count
    int64_t nvert = 0;
};

struct fr_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int num_sms = 0;
    size_t ws_limit = 0;  // largest lattice-table arena a batched call may hold (0: no limit)
    int64_t launches = 0;
    int64_t h2d_bytes = 0, d2h_bytes = 0;

    // workspace: three rotating lattice tables (the build of the next sigma
    // overlaps the slice of the current one), blur scratch planes, reduction
    // partials, device state, job descriptor and per-iteration constants.
    uint64_t ws_gen = 1;
    uint32_t table_cap = 0;
    fr::Table tables[fr::kMaxTables] = {};  // 3 with float32 storage, 4 with 16-bit storage
    int *lists[fr::kMaxTables] = {};        // slots claimed by each table's last build
    unsigned long long *blur = nullptr;   // blur ping-pong records (table_cap slots)
    float2 *partials = nullptr;
    int partial_rows = 0;
    fr::DeviceState *d_state = nullptr;
    fr::RigidJob *d_job = nullptr;
    fr::IterParams *d_ip = nullptr;
    int ip_cap = 0;
    float4 *stage = nullptr;  // host-call staging of X, Y, Yn
    size_t stage_cap = 0;     // in float4

    // pinned host mirrors
    fr::RigidJob *h_job = nullptr;
    fr::IterParams *h_ip = nullptr;
    fr::DeviceState *h_state = nullptr;

    std::vector<fr::CachedGraph> graphs;
    uint64_t use_clock = 0;
    int bpsm[2][2] = {{0, 0}, {0, 0}};  // resident fused-kernel blocks per SM

    fr_tune_params tune[fr::kTuneClasses] = {fr::tune_default(), fr::tune_default(), fr::tune_default(),
                                             fr::tune_default(), fr::tune_default()};
    fr::BatchWorkspace *batch = nullptr;  // batched-registration workspace (batch.cu)
    fr::ArtWorkspace *art = nullptr;      // articulated-registration workspace (articulated.cu)
    fr::FeatWorkspace *feat = nullptr;    // feature-space lattice table (features.cu)
    // Contexts of the concurrent registrations of a batched articulated call,
    // each with a stream of its own (made on first use, destroyed with this
    // context); own_stream marks a context that created its stream.
    std::vector<fr_ctx *> subs;
    bool own_stream = false;

    // per-kernel profiling: event pairs around each launch of a plan
    int profiling = 0;
    std::vector<cudaEvent_t> events;  // 2 per kernel, grown on demand, kept for the graphs
    std::vector<int> event_class;     // kernel class of each event pair of the last plan
    int64_t prof_launches[FR_K_CLASSES] = {};
    double prof_ms[FR_K_CLASSES] = {};

    fr_status fail(fr_status s, const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return s;
    }
    fr_status cuda(cudaError_t e, const char *what) {
        if (e == cudaSuccess) return FR_OK;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA, "%s: %s", what,
                    cudaGetErrorString(e));
    }
};

#define FR_TRY(expr)                         \
    do {                                     \
        fr_status _s = (expr);               \
        if (_s != FR_OK) return _s;          \
    } while (0)
#define FR_CUDA(ctx, call) FR_TRY((ctx)->cuda((call), #call))

// cudaMemcpyAsync on the context's stream, counting the bytes moved.
inline cudaError_t copy_async(fr_ctx *ctx, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
    if (kind == cudaMemcpyHostToDevice) ctx->h2d_bytes += (int64_t)bytes;
    if (kind == cudaMemcpyDeviceToHost) ctx->d2h_bytes += (int64_t)bytes;
    return cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream);
}


namespace fr {
// Helpers implemented in api.cu.
int blocks_for(const fr_ctx *ctx, long long n, int per_sm);
fr_status check_flags(fr_ctx *ctx, int flags);
fr_status validate_cloud(fr_ctx *ctx, const void *p, int64_t n, const char *name);
fr_status validate_options(fr_ctx *ctx, const fr_options *o);
bool fill_iter_params(const fr_options *o, int64_t M, int64_t N, IterParams *ip);
int fused_blocks_per_sm(fr_ctx *ctx, int pt2pl, int kahan);
void collect_profile(fr_ctx *ctx, int kernels);
void free_batch_workspace(fr_ctx *ctx);   // batch.cu
void free_art_workspace(fr_ctx *ctx);     // articulated.cu
void free_feat_workspace(fr_ctx *ctx);    // features.cu
fr_status ensure_tables(fr_ctx *ctx, uint32_t cap, bool blur, bool compact = false);
fr_status ensure_small(fr_ctx *ctx, int iters, int grid_rows);
}  // namespace fr
