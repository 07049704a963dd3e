// Host implementation of the C ABI declared in include/filterreg.h.
//
// A context owns a growable device workspace (one lattice hash table and its
// blur ping-pong planes, reduction partials, the device-resident pose state,
// the per-call job descriptor and per-iteration constants) plus pinned host
// mirrors of the small structures.  A registration copies its job descriptor
// to the device and replays a CUDA graph of the whole EM loop; graphs are
// cached per loop shape, so calls on new buffers of the same shape reuse them.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

using namespace fr;

namespace {

void drop_graphs(fr_ctx *ctx) {
    for (auto &g : ctx->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
}

void free_tables(fr_ctx *ctx) {
    for (int i = 0; i < kMaxTables; ++i) {
        Table &t = ctx->tables[i];
        cudaFree(t.keys);
        cudaFree(ctx->lists[i]);
        ctx->lists[i] = nullptr;
        t = Table{};
    }
    cudaFree(ctx->blur);
    ctx->blur = nullptr;
    ctx->table_cap = 0;
}

fr_status alloc_table(fr_ctx *ctx, int i, uint32_t cap) {
    Table &t = ctx->tables[i];
    cudaFree(ctx->lists[i]);  // left by an earlier attempt that failed part way
    ctx->lists[i] = nullptr;
    FR_CUDA(ctx, dev_alloc(&ctx->lists[i], cap));
    FR_CUDA(ctx, dev_alloc(&t.keys, (size_t)cap * kRecWords));
    FR_CUDA(ctx, cudaMemsetAsync(t.keys, 0, table_bytes(cap), ctx->stream));
    t.vals = 8;
    t.mask = cap - 1;
    t.max_probe = cap;
    return FR_OK;
}

// Three tables of at least `cap` slots, all empty; with `compact`, a fourth
// and the 16-bit record planes of all four; blur scratch if asked.
}  // namespace

namespace fr {
fr_status ensure_tables(fr_ctx *ctx, uint32_t cap, bool blur, bool compact) {
    if (cap > ctx->table_cap) {
        // Captured graphs go with the buffers they name, before any new
        // allocation can fail; a failed one leaves table_cap at 0, so the
        // next call allocates all again.
        cudaStreamSynchronize(ctx->stream);
        ctx->ws_gen++;
        drop_graphs(ctx);
        free_tables(ctx);
        for (int i = 0; i < 3; ++i) FR_TRY(alloc_table(ctx, i, cap));
        ctx->table_cap = cap;
    }
    if (compact && !ctx->tables[3].keys) {  // 16-bit storage: a fourth table in rotation
        ctx->ws_gen++;
        drop_graphs(ctx);
        FR_TRY(alloc_table(ctx, 3, ctx->table_cap));
    }
    if (blur && !ctx->blur) {
        ctx->ws_gen++;
        drop_graphs(ctx);
        FR_CUDA(ctx, dev_alloc(&ctx->blur, (size_t)ctx->table_cap * kRecWords));
        // Blur passes write only the slots their lattice holds and free them
        // afterwards: the scratch table starts empty and stays so.
        FR_CUDA(ctx, cudaMemsetAsync(ctx->blur, 0, table_bytes(ctx->table_cap), ctx->stream));
    }
    return FR_OK;
}
}  // namespace fr

namespace {

}  // namespace

namespace fr {
fr_status ensure_small(fr_ctx *ctx, int iters, int grid_rows) {
    // each buffer on its own test: an attempt that failed part way leaves
    // the ones it made, and the next call makes the rest
    if (!ctx->d_state) {
        FR_CUDA(ctx, dev_alloc(&ctx->d_state, 1));
        FR_CUDA(ctx, cudaMemsetAsync(ctx->d_state, 0, sizeof(DeviceState), ctx->stream));
    }
    if (!ctx->d_job) FR_CUDA(ctx, dev_alloc(&ctx->d_job, 1));
    if (!ctx->h_job) FR_CUDA(ctx, cudaMallocHost((void **)&ctx->h_job, sizeof(RigidJob)));
    if (!ctx->h_state) FR_CUDA(ctx, cudaMallocHost((void **)&ctx->h_state, sizeof(DeviceState)));
    int need = iters > 1 ? iters : 1;
    if (need > ctx->ip_cap) {
        cudaStreamSynchronize(ctx->stream);
        ctx->ws_gen++;
        drop_graphs(ctx);
        cudaFree(ctx->d_ip);
        cudaFreeHost(ctx->h_ip);
        ctx->d_ip = nullptr;
        ctx->h_ip = nullptr;
        ctx->ip_cap = 0;
        int cap = 64;
        while (cap < need) cap <<= 1;
        FR_CUDA(ctx, dev_alloc(&ctx->d_ip, cap));
        FR_CUDA(ctx, cudaMallocHost((void **)&ctx->h_ip, cap * sizeof(IterParams)));
        ctx->ip_cap = cap;
    }
    if (grid_rows > ctx->partial_rows) {
        cudaStreamSynchronize(ctx->stream);
        ctx->ws_gen++;
        drop_graphs(ctx);
        cudaFree(ctx->partials);
        ctx->partials = nullptr;
        ctx->partial_rows = 0;
        FR_CUDA(ctx, dev_alloc(&ctx->partials, (size_t)grid_rows * kRigidVals));
        ctx->partial_rows = grid_rows;
    }
    return FR_OK;
}
}  // namespace fr

namespace {

}  // namespace

namespace fr {
int blocks_for(const fr_ctx *ctx, long long n, int per_sm) {
    long long g = (n + kBlock - 1) / kBlock;
    long long cap = (long long)ctx->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}
fr_status check_flags(fr_ctx *ctx, int flags) {
    if (flags & kFlagCapacity)
        return ctx->fail(FR_ECAPACITY, "lattice hash table full");
    if (flags & kFlagRange)
        return ctx->fail(FR_EINVAL, "non-finite coordinate or elevated coordinate beyond +-1e6 "
                                    "(position / sigma too large)");
    return FR_OK;
}
}  // namespace fr

namespace {

// The registration as a sequence of launches (captured into a graph or
// issued directly).
//   fixed sigma:  build(0) -> step(0) .. step(iters-1) -> clear
//   annealed:     build(0) -> [step(k) | build(k+1) | clear(k-1)] for each k
//                 -> clear all three tables
// with 4 blur passes after every build when blur is on.
// Instantiated EM-loop graphs kept per context (least recently used out): one
// per distinct shape (sizes, sigma schedule kind, table size), enough for a
// stream of ragged requests to stop re-instantiating.
constexpr size_t kGraphCache = 64;

struct Plan {
    int iters, residual, blur, kahan, profile, annealed, storage;
    int sig;  // sigma as a decision variable: step and build launches alternate
    int gs, gv, gb, gc, g_blur, g_final;  // block counts of the roles
};

// Kernel launch wrapper: with profiling on, an event pair brackets each launch.
struct Issuer {
    fr_ctx *ctx;
    cudaStream_t s;
    int profile;
    int kernels = 0;
    // Inside stream capture an event record must be marked external to become
    // an event node of the graph; outside capture it is a plain record.
    void record(cudaEvent_t e) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &cs);
        if (cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else
            cudaEventRecord(e, s);
    }
    template <typename F>
    void operator()(int cls, F &&launch) {
        if (profile) {
            const size_t need = 2 * (size_t)(kernels + 1);
            while (ctx->events.size() < need) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ctx->events.push_back(e);
            }
            if (ctx->event_class.size() < (size_t)(kernels + 1)) ctx->event_class.resize(kernels + 1);
            ctx->event_class[kernels] = cls;
            record(ctx->events[2 * kernels]);
        }
        launch();
        if (profile) record(ctx->events[2 * kernels + 1]);
        ++kernels;
    }
};

// The four blur passes of the lattice a build left in table t (its claimed
// slots in `list`, their count at `count`), ping-ponging with the scratch
// table, which is emptied again afterwards.
void issue_blur(fr_ctx *ctx, Issuer &k, const Plan &p, const Table &t, const int *list, const int *count) {
    Table a = t, b = t;
    b.keys = ctx->blur;
    for (int dir = 0; dir < 4; ++dir)
        k(FR_K_BLUR, [&] {
            if (dir % 2 == 0)
                launch_blur_list(a, b, dir, list, count, p.g_blur, ctx->d_state, k.s);
            else
                launch_blur_list(b, a, dir, list, count, p.g_blur, ctx->d_state, k.s);
        });
    int *lists[1] = {const_cast<int *>(list)};
    const int *counts[1] = {count};
    k(FR_K_BLUR, [&] { launch_clear_lists(&b, lists, counts, 1, p.g_blur, k.s); });
}

// Builds run `lead` iterations ahead of the step that reads them: 1 with
// float32 storage; 2 with 16-bit storage, whose records are made by a
// convert role one launch after the build completed.
//   lead 1: build(0) -> [step k | build k+1 | clear k-1] ...
//   lead 2: build(0) -> [convert 0 | build 1] -> [step k | convert k+1 | build k+2 | clear k-1] ...
// A fixed sigma builds (and converts) table 0 only.  Then the tables left
// are cleared.
// Sigma as a decision variable: the next sigma is known once a step has
// finished, so each iteration is two launches on two alternating tables --
//   build(0) -> [step k | clear the other table (build k-1)] -> [build k+1] ...
// -> clear the last table.
int issue_plan_sigma(fr_ctx *ctx, const Plan &p, cudaStream_t s) {
    Issuer k{ctx, s, p.profile};
    Table *tab = ctx->tables;
    IterLaunch base{};
    base.job = ctx->d_job;
    base.ip = ctx->d_ip;
    base.partials = ctx->partials;
    base.st = ctx->d_state;
    base.check_done = 1;
    auto build = [&](int b) {
        IterLaunch L = base;
        L.check_done = b > 0;
        L.build = tab[b & 1];
        L.build_list = ctx->lists[b & 1];
        L.build_it = b;
        L.gb = p.gb + (b == 0 ? p.gs : 0);
        k(b == 0 ? FR_K_BUILD : FR_K_STEP, [&] { launch_em_iter_sigma(p.kahan, L, s); });
    };
    if (p.iters > 0) build(0);
    for (int it = 0; it < p.iters; ++it) {
        IterLaunch L = base;
        L.it = it;
        L.gs = p.gs;
        L.step = tab[it & 1];
        L.sig_next = it + 1 < p.iters;
        if (it >= 1) {
            L.clear = tab[(it - 1) & 1];
            L.clear_list = ctx->lists[(it - 1) & 1];
            L.clear_it = it - 1;
            L.gc = p.gc;
        }
        k(FR_K_STEP, [&] { launch_em_iter_sigma(p.kahan, L, s); });
        if (it + 1 < p.iters) build(it + 1);
    }
    if (p.iters > 0) {
        const int last = p.iters - 1;
        Table t[1] = {tab[last & 1]};
        int *lists[1] = {ctx->lists[last & 1]};
        const int *counts[1] = {&ctx->d_ip[last].nvert};
        k(FR_K_CLEAR, [&] { launch_clear_lists(t, lists, counts, 1, p.g_final, s); });
    }
    return k.kernels;
}

int issue_plan(fr_ctx *ctx, const Plan &p, cudaStream_t s) {
    if (p.sig) return issue_plan_sigma(ctx, p, s);
    Issuer k{ctx, s, p.profile};
    Table *tab = ctx->tables;
    const int lead = p.storage != FR_FP32 ? 2 : 1;
    const int ntab = lead + 2;
    IterLaunch base{};
    base.job = ctx->d_job;
    base.ip = ctx->d_ip;
    base.partials = ctx->partials;
    base.st = ctx->d_state;
    base.check_done = 1;
    auto which = [&](int build) { return p.annealed ? build % ntab : 0; };
    auto builds = [&](int b) { return b < p.iters && (p.annealed || b == 0); };
    auto add_build = [&](IterLaunch &L, int b, int blocks) {
        L.build = tab[which(b)];
        L.build_list = ctx->lists[which(b)];
        L.build_it = b;
        L.gb = blocks;
    };
    auto add_conv = [&](IterLaunch &L, int b) {
        L.conv = tab[which(b)];
        L.conv_list = ctx->lists[which(b)];
        L.conv_it = b;
        L.gv = p.gv;
    };
    // prologue: the first `lead` builds (and the conversion of build 0)
    for (int j = 0; j < lead && p.iters > 0; ++j) {
        IterLaunch L = base;
        L.check_done = 0;
        if (builds(j)) add_build(L, j, j == 0 ? p.gb + p.gs : p.gb);  // nothing else runs at first
        if (j >= 1) add_conv(L, j - 1);
        if (L.gb + L.gv == 0) continue;
        k(j == 0 ? FR_K_BUILD : FR_K_CONVERT, [&] { launch_em_iter(p.residual, p.kahan, L, s, p.storage); });
        if (p.blur && L.gb) issue_blur(ctx, k, p, L.build, L.build_list, &ctx->d_ip[L.build_it].nvert);
    }
    for (int it = 0; it < p.iters; ++it) {
        IterLaunch L = base;
        L.it = it;
        L.gs = p.gs;
        L.step = tab[which(it)];
        if (p.annealed && builds(it + lead)) add_build(L, it + lead, p.gb);
        if (lead == 2 && p.annealed && builds(it + 1)) add_conv(L, it + 1);
        if (p.annealed && it >= 1) {  // the table of build it-1, last read by step it-1
            L.clear = tab[which(it - 1)];
            L.clear_list = ctx->lists[which(it - 1)];
            L.clear_it = it - 1;
            L.gc = p.gc;
        }
        k(FR_K_STEP, [&] { launch_em_iter(p.residual, p.kahan, L, s, p.storage); });
        if (p.blur && L.gb) issue_blur(ctx, k, p, L.build, L.build_list, &ctx->d_ip[L.build_it].nvert);
    }
    if (p.iters > 0) {
        // Free what is left: the last build's table.  Every other table was
        // cleared by the launch after its step (clear roles run even after
        // the registration stopped).
        const int last = p.annealed ? p.iters - 1 : 0;
        Table t[1] = {tab[which(last)]};
        int *lists[1] = {ctx->lists[which(last)]};
        const int *counts[1] = {&ctx->d_ip[last].nvert};
        k(FR_K_CLEAR, [&] { launch_clear_lists(t, lists, counts, 1, p.g_final, s); });
    }
    return k.kernels;
}

// Kernels of a plan (all are profiled).
int plan_kernels(const Plan &p) {
    if (p.sig) return p.iters > 0 ? 2 * p.iters + 1 : 0;  // build 0, (step, build) ..., step, clear
    int n = 0;
    const int lead = p.storage != FR_FP32 ? 2 : 1;
    if (p.iters > 0) n += 2 + (p.blur ? 5 : 0) + (lead - 1);  // prologue (+ blur, scratch clear), final clear
    n += p.iters;
    if (p.annealed && p.blur && p.iters > 1) n += 5 * (p.iters - 1);
    return n;
}


fr_status run_plan(fr_ctx *ctx, const Plan &p, bool use_graph) {
    if (!use_graph) {
        ctx->launches += issue_plan(ctx, p, ctx->stream);
        return ctx->cuda(cudaGetLastError(), "kernel launch");
    }
    GraphKey key{{p.iters, p.residual, p.blur, p.kahan, p.profile, p.annealed, p.gs, p.gb, p.gc,
                  p.g_blur, p.g_final, (int)ctx->tables[0].mask, p.storage, p.sig},
                 ctx->ws_gen};
    CachedGraph *hit = nullptr;
    for (auto &g : ctx->graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        cudaStream_t cs;
        FR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int kernels = 0;
        if (e == cudaSuccess) {
            kernels = issue_plan(ctx, p, cs);
            e = cudaStreamEndCapture(cs, &graph);
        }
        cudaStreamDestroy(cs);
        FR_CUDA(ctx, e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        FR_CUDA(ctx, e);
        if (ctx->graphs.size() >= kGraphCache) {
            size_t old = 0;
            for (size_t i = 1; i < ctx->graphs.size(); ++i)
                if (ctx->graphs[i].last_use < ctx->graphs[old].last_use) old = i;
            cudaGraphExecDestroy(ctx->graphs[old].exec);
            ctx->graphs.erase(ctx->graphs.begin() + old);
        }
        ctx->graphs.push_back(CachedGraph{key, exec, kernels, 0});
        hit = &ctx->graphs.back();
    }
    hit->last_use = ++ctx->use_clock;
    FR_CUDA(ctx, cudaGraphLaunch(hit->exec, ctx->stream));
    ctx->launches += hit->kernels;
    return FR_OK;
}

}  // namespace

namespace fr {
fr_status validate_cloud(fr_ctx *ctx, const void *p, int64_t n, const char *name) {
    if (!p) return ctx->fail(FR_EINVAL, "%s is NULL", name);
    if (n < 1 || n > (1ll << 30)) return ctx->fail(FR_EINVAL, "%s: size %lld out of range", name, (long long)n);
    if (!aligned16(p)) return ctx->fail(FR_EINVAL, "%s must be 16-byte aligned (n x 4 floats)", name);
    return FR_OK;
}
fr_status validate_options(fr_ctx *ctx, const fr_options *o) {
    if (!o) return ctx->fail(FR_EINVAL, "options are NULL");
    if (o->residual != FR_PT2PT && o->residual != FR_PT2PL)
        return ctx->fail(FR_EINVAL, "residual must be FR_PT2PT or FR_PT2PL");
    if (o->iters < 0 || o->iters > 100000) return ctx->fail(FR_EINVAL, "iters out of range");
    if (!(o->sigma_start > 0.0f) || !(o->sigma_end > 0.0f) || !std::isfinite(o->sigma_start) ||
        !std::isfinite(o->sigma_end))
        return ctx->fail(FR_EINVAL, "sigma must be finite and > 0");
    if (!(o->w >= 0.0f && o->w < 1.0f)) return ctx->fail(FR_EINVAL, "w must lie in [0, 1)");
    if (o->storage != FR_FP32 && o->storage != FR_BF16 && o->storage != FR_FP16)
        return ctx->fail(FR_EINVAL, "storage must be FR_FP32, FR_BF16 or FR_FP16");
    if (o->storage != FR_FP32 && o->blur)
        return ctx->fail(FR_ENOTSUPPORTED, "16-bit lattice storage is implemented without blur");
    if (o->update_sigma && (o->residual != FR_PT2PT || o->storage != FR_FP32 || o->blur))
        return ctx->fail(FR_ENOTSUPPORTED, "the sigma update is point-to-point, float32 storage, no blur");
    if (o->update_sigma != 0 && o->update_sigma != 1) return ctx->fail(FR_EINVAL, "update_sigma must be 0 or 1");
    return FR_OK;
}
}  // namespace fr

namespace fr {

std::atomic<int> &alloc_skip() {
    static std::atomic<int> n{0};
    return n;
}
std::atomic<int> &alloc_fail() {
    static std::atomic<int> n{0};
    return n;
}

// After the stream is synchronised: add the event-pair durations of the last
// launches to the per-class totals.
void collect_profile(fr_ctx *ctx, int kernels) {
    for (int i = 0; i < kernels; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->events[2 * i], ctx->events[2 * i + 1]) == cudaSuccess) {
            ctx->prof_ms[ctx->event_class[i]] += ms;
            ctx->prof_launches[ctx->event_class[i]] += 1;
        }
    }
    cudaGetLastError();
}

// Host-side constants of every iteration: the sigma schedule (geometric
// between sigma_start and sigma_end), feature scales and outlier constant
// c = w/(1-w) N/M (Eq. 7) in the lattice kernel's units (times sigma^3 G).
// Returns true when sigma changes during the schedule (annealing).
bool fill_iter_params(const fr_options *o, int64_t M, int64_t N, IterParams *ip) {
    const double c = (double)o->w / (1.0 - (double)o->w) * ((double)N / (double)M);
    const double G = lattice_kernel_mass(o->blur);
    bool changes = false;
    for (int k = 0; k < o->iters; ++k) {
        const float sig = schedule_sigma(o, k);
        IterParams &p = ip[k];
        p.sigma = sig;
        float s[3];
        feature_scales(sig, s);
        p.s1 = s[0];
        p.s2 = s[1];
        p.s3 = s[2];
        const double sd = (double)sig;
        p.c_eff = (float)(c * sd * sd * sd * G);
        p.inv_sigma2 = (float)(1.0 / (sd * sd));
        p.rebuild = (k == 0 || sig != ip[k - 1].sigma) ? 1 : 0;
        p.nvert = 0;
        // A vertex's weight is at most N (every barycentric weight is <= 1):
        // half-precision records are scaled by 2^-e so that N 2^-e <= 2^14.
        int e = 0;
        while (o->storage == FR_FP16 && (double)N > std::ldexp(1.0, 14 + e)) ++e;
        p.vscale = (float)std::ldexp(1.0, -e);
        p.inv_vscale = (float)std::ldexp(1.0, e);
        p.ws1 = 1.0f / (2.0f * p.s1);
        p.ws2 = 1.0f / (6.0f * p.s2);
        p.ws3 = 1.0f / (12.0f * p.s3);
        p.pad[0] = p.pad[1] = p.pad[2] = 0;
        if (k > 0 && p.rebuild) changes = true;
    }
    return changes;
}
int fused_blocks_per_sm(fr_ctx *ctx, int pt2pl, int kahan) {
    int &bpsm = ctx->bpsm[pt2pl][kahan];
    if (!bpsm) bpsm = em_iter_blocks_per_sm(pt2pl, kahan);
    return bpsm;
}
}  // namespace fr

namespace {

// Splits the resident blocks of the fused kernel between its roles.
void plan_grids(fr_ctx *ctx, Plan &p, int64_t M, int64_t N, uint32_t cap) {
    const int bpsm = fused_blocks_per_sm(ctx, p.residual, p.kahan);
    const long long resident = (long long)bpsm * ctx->num_sms;
    long long gs = (M + kBlock - 1) / kBlock, gb = (N + kBlock - 1) / kBlock;
    long long gc = p.annealed ? std::max<long long>(8, std::min<long long>(64, cap / 16384)) : 0;
    const long long gv = p.storage != FR_FP32 ? std::max<long long>(8, std::min<long long>(128, cap / 4096)) : 0;
    if (!p.annealed) gb = std::max<long long>(1, std::min(gb, resident));
    const long long room = resident - gc - (p.annealed ? gv : 0);
    const long long want = gs + (p.annealed ? gb : 0);
    if (want > room) {
        const double f = (double)room / (double)want;
        gs = std::max<long long>(1, (long long)(gs * f));
        if (p.annealed) gb = std::max<long long>(1, (long long)(gb * f));
    }
    p.gs = (int)gs;
    p.gv = (int)gv;
    p.gb = (int)gb;
    p.gc = (int)gc;
    p.g_blur = blocks_for(ctx, 2 * N, 8);  // blur passes walk the build's vertex list (<= 4 N)
    p.g_final = (int)std::max<long long>(8, std::min<long long>(resident / 2, (N + kBlock - 1) / kBlock));
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

FR_API void fr_options_default(fr_options *o) {
    if (!o) return;
    o->residual = FR_PT2PT;
    o->blur = 0;
    o->iters = 30;
    o->sigma_start = 0.02f;
    o->sigma_end = 0.02f;
    o->w = 0.1f;
    o->storage = FR_FP32;
    o->kahan = 0;
    o->renormalize_normals = 0;
    o->stop_twist = 0.0f;
    o->use_graph = 1;
    o->update_sigma = 0;
}

FR_API const char *fr_status_string(fr_status s) {
    switch (s) {
    case FR_OK: return "ok";
    case FR_EINVAL: return "invalid argument";
    case FR_ENOMEM: return "out of memory";
    case FR_ECUDA: return "CUDA error";
    case FR_ECAPACITY: return "lattice capacity exceeded";
    case FR_ETIMEOUT: return "device wait timed out";
    case FR_ENOTSUPPORTED: return "not supported";
    }
    return "unknown status";
}

FR_API fr_status fr_ctx_create(int device, void *cuda_stream, fr_ctx **out) {
    if (!out) return FR_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return FR_ECUDA;
    fr_ctx *ctx = new fr_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (ctx->num_sms < 1) ctx->num_sms = 1;
    // A launch-shape table named by FR_TUNE_TABLE is loaded when it parses
    // (a missing or malformed one leaves the built-in defaults).
    if (const char *tt = std::getenv("FR_TUNE_TABLE"))
        if (*tt) fr_tune_load(ctx, tt);
    ctx->err.clear();
    *out = ctx;
    return FR_OK;
}

FR_API fr_status fr_ctx_destroy(fr_ctx *ctx) {
    if (!ctx) return FR_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    drop_graphs(ctx);
    free_batch_workspace(ctx);
    free_art_workspace(ctx);
    free_feat_workspace(ctx);
    for (cudaEvent_t e : ctx->events) cudaEventDestroy(e);
    free_tables(ctx);
    cudaFree(ctx->partials);
    cudaFree(ctx->d_state);
    cudaFree(ctx->d_job);
    cudaFree(ctx->d_ip);
    cudaFree(ctx->stage);
    cudaFreeHost(ctx->h_job);
    cudaFreeHost(ctx->h_ip);
    cudaFreeHost(ctx->h_state);
    for (fr_ctx *sub : ctx->subs) fr_ctx_destroy(sub);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return FR_OK;
}

FR_API fr_status fr_ctx_set_stream(fr_ctx *ctx, void *cuda_stream) {
    if (!ctx) return FR_EINVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return FR_OK;
}

FR_API fr_status fr_ctx_set_workspace_limit(fr_ctx *ctx, size_t bytes) {
    if (!ctx) return FR_EINVAL;
    ctx->ws_limit = bytes;
    return FR_OK;
}

FR_API fr_status fr_tune_get(const fr_ctx *ctx, int64_t n_points, fr_tune_params *out) {
    if (!ctx || !out || n_points < 1) return FR_EINVAL;
    *out = ctx->tune[tune_class(n_points)];
    return FR_OK;
}

FR_API fr_status fr_tune_set(fr_ctx *ctx, int64_t n_points, const fr_tune_params *p) {
    if (!ctx || !p || n_points < 1) return FR_EINVAL;
    if (!tune_valid(*p)) return ctx->fail(FR_EINVAL, "tuning parameters out of range");
    ctx->tune[tune_class(n_points)] = *p;
    return FR_OK;
}

// File format: one line per size class, "class step build table_x2 serve".
FR_API fr_status fr_tune_save(const fr_ctx *ctx, const char *path) {
    if (!ctx || !path) return FR_EINVAL;
    FILE *f = std::fopen(path, "w");
    if (!f) return FR_EINVAL;
    std::fprintf(f, "# filterreg launch tuning: class step_ppt build_ppt table_slots_x2 serve_ppt\n");
    for (int c = 0; c < kTuneClasses; ++c) {
        const fr_tune_params &p = ctx->tune[c];
        std::fprintf(f, "%d %d %d %d %d\n", c, p.step_points_per_thread, p.build_points_per_thread,
                     p.table_slots_x2, p.serve_points_per_thread);
    }
    return std::fclose(f) == 0 ? FR_OK : FR_EINVAL;
}

FR_API fr_status fr_tune_load(fr_ctx *ctx, const char *path) {
    if (!ctx || !path) return FR_EINVAL;
    FILE *f = std::fopen(path, "r");
    if (!f) return ctx->fail(FR_EINVAL, "cannot open tuning table %s", path);
    fr_tune_params t[kTuneClasses];
    for (int c = 0; c < kTuneClasses; ++c) t[c] = ctx->tune[c];
    char line[256];
    bool ok = true;
    while (ok && std::fgets(line, sizeof line, f)) {
        if (line[0] == '#' || line[0] == '\n') continue;
        int c, a, b, x, v;
        if (std::sscanf(line, "%d %d %d %d %d", &c, &a, &b, &x, &v) != 5 || c < 0 || c >= kTuneClasses) {
            ok = false;
            break;
        }
        t[c] = fr_tune_params{a, b, x, v};
        ok = tune_valid(t[c]);
    }
    std::fclose(f);
    if (!ok) return ctx->fail(FR_EINVAL, "malformed tuning table %s", path);
    for (int c = 0; c < kTuneClasses; ++c) ctx->tune[c] = t[c];
    return FR_OK;
}

FR_API const char *fr_ctx_last_error(const fr_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

FR_API int64_t fr_ctx_kernel_launches(const fr_ctx *ctx) { return ctx ? ctx->launches : 0; }

FR_API fr_status fr_ctx_transfer_bytes(const fr_ctx *ctx, int64_t *h2d, int64_t *d2h) {
    if (!ctx) return FR_EINVAL;
    if (h2d) *h2d = ctx->h2d_bytes;
    if (d2h) *d2h = ctx->d2h_bytes;
    return FR_OK;
}

FR_API fr_status fr_debug_fail_allocations(int32_t after, int32_t n) {
    if (after < 0 || n < 0) return FR_EINVAL;
    fr::alloc_fail().store(0);
    fr::alloc_skip().store(n > 0 ? after : 0);
    fr::alloc_fail().store(n);
    return FR_OK;
}

FR_API fr_status fr_ctx_set_profiling(fr_ctx *ctx, int on) {
    if (!ctx) return FR_EINVAL;
    ctx->profiling = on ? 1 : 0;
    return FR_OK;
}

FR_API fr_status fr_ctx_profile(fr_ctx *ctx, fr_profile *out, int reset) {
    if (!ctx) return FR_EINVAL;
    if (out)
        for (int c = 0; c < FR_K_CLASSES; ++c) {
            out->launches[c] = ctx->prof_launches[c];
            out->total_ms[c] = ctx->prof_ms[c];
        }
    if (reset)
        for (int c = 0; c < FR_K_CLASSES; ++c) {
            ctx->prof_launches[c] = 0;
            ctx->prof_ms[c] = 0.0;
        }
    return FR_OK;
}

// ---- lattice primitives -----------------------------------------------------

FR_API fr_status fr_lattice_embed(fr_ctx *ctx, const float *d_pos, int64_t n, float sigma,
                                  int32_t *d_keys, float *d_bary) {
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_cloud(ctx, d_pos, n, "d_pos"));
    if (!(sigma > 0.0f)) return ctx->fail(FR_EINVAL, "sigma must be > 0");
    if (d_keys && !aligned16(d_keys)) return ctx->fail(FR_EINVAL, "d_keys must be 16-byte aligned");
    cudaSetDevice(ctx->device);
    FR_TRY(ensure_small(ctx, 1, 1));
    float s[3];
    feature_scales(sigma, s);
    int *flags = &ctx->d_state->flags;
    FR_CUDA(ctx, cudaMemsetAsync(flags, 0, sizeof(int), ctx->stream));
    launch_embed((const float4 *)d_pos, (int)n, s[0], s[1], s[2], d_keys, d_bary, flags, ctx->stream);
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    int h = 0;
    FR_CUDA(ctx, copy_async(ctx, &h, flags, sizeof(int), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx, h);
}

FR_API fr_status fr_lattice_build(fr_ctx *ctx, const float *d_pos, int64_t n, float sigma,
                                  int64_t capacity_hint, fr_lattice **out) {
    if (!ctx || !out) return FR_EINVAL;
    *out = nullptr;
    FR_TRY(validate_cloud(ctx, d_pos, n, "d_pos"));
    if (!(sigma > 0.0f) || !std::isfinite(sigma)) return ctx->fail(FR_EINVAL, "sigma must be > 0");
    cudaSetDevice(ctx->device);
    fr_lattice *lat = new fr_lattice();
    long long want = capacity_hint > 8 * n ? capacity_hint : 8 * n;
    lat->cap = pow2_at_least(want);
    lat->n = (int)n;
    feature_scales(sigma, lat->scale);
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc(&lat->keys, (size_t)lat->cap * kRecWords);
    if (e == cudaSuccess) e = dev_alloc(&lat->rec_slot, (size_t)n * 4);
    if (e == cudaSuccess) e = dev_alloc(&lat->rec_w, (size_t)n * 4);
    if (e == cudaSuccess) e = dev_alloc(&lat->counters, 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(lat->keys, 0, table_bytes(lat->cap), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lat->counters, 0, 4 * sizeof(int), ctx->stream);
    if (e != cudaSuccess) {
        fr_lattice_destroy(ctx, lat);
        return ctx->cuda(e, "fr_lattice_build allocation");
    }
    Table t{lat->keys, lat->cap - 1, lat->cap, lat->vdim > 4 ? 8 : 4};
    launch_build_records((const float4 *)d_pos, (int)n, lat->scale[0], lat->scale[1], lat->scale[2], t,
                         lat->rec_slot, lat->rec_w, lat->counters, ctx->stream);
    ctx->launches += 1;
    int h[2] = {0, 0};
    e = cudaGetLastError();
    if (e == cudaSuccess) e = copy_async(ctx, h, lat->counters, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        fr_lattice_destroy(ctx, lat);
        return ctx->cuda(e, "fr_lattice_build");
    }
    lat->nvert = h[0];
    fr_status st = check_flags(ctx, h[1]);
    if (st != FR_OK) {
        fr_lattice_destroy(ctx, lat);
        return st;
    }
    *out = lat;
    return FR_OK;
}

FR_API fr_status fr_lattice_splat(fr_ctx *ctx, fr_lattice *lat, const float *d_vals, int val_dim) {
    if (!ctx || !lat) return FR_EINVAL;
    if (!d_vals) return ctx->fail(FR_EINVAL, "d_vals is NULL");
    if (val_dim < 1 || val_dim > 8) return ctx->fail(FR_EINVAL, "val_dim must be 1..8");
    cudaSetDevice(ctx->device);
    lat->vdim = val_dim;
    Table t{lat->keys, lat->cap - 1, lat->cap, 8};
    launch_zero_values(t, blocks_for(ctx, lat->cap, 16), ctx->stream);
    launch_splat_records(d_vals, val_dim, lat->n, lat->rec_slot, lat->rec_w, t, ctx->stream);
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}

FR_API fr_status fr_lattice_blur(fr_ctx *ctx, fr_lattice *lat) {
    if (!ctx || !lat) return FR_EINVAL;
    cudaSetDevice(ctx->device);
    if (!lat->tkeys) FR_CUDA(ctx, dev_alloc(&lat->tkeys, (size_t)lat->cap * kRecWords));
    Table a{lat->keys, lat->cap - 1, lat->cap, lat->vdim > 4 ? 8 : 4};
    Table b{lat->tkeys, lat->cap - 1, lat->cap, lat->vdim > 4 ? 8 : 4};
    int grid = blocks_for(ctx, lat->cap, 16);
    for (int dir = 0; dir < 4; ++dir) {
        if (dir % 2 == 0)
            launch_blur_pass(a, b, dir, grid, nullptr, ctx->stream);
        else
            launch_blur_pass(b, a, dir, grid, nullptr, ctx->stream);
    }
    ctx->launches += 4;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}

FR_API fr_status fr_lattice_slice(fr_ctx *ctx, const fr_lattice *lat, const float *d_query,
                                  int64_t m, float *d_out) {
    if (!ctx || !lat) return FR_EINVAL;
    FR_TRY(validate_cloud(ctx, d_query, m, "d_query"));
    if (!d_out) return ctx->fail(FR_EINVAL, "d_out is NULL");
    if (lat->vdim < 1) return ctx->fail(FR_EINVAL, "lattice has no values (call fr_lattice_splat)");
    cudaSetDevice(ctx->device);
    Table t{lat->keys, lat->cap - 1, lat->cap, lat->vdim > 4 ? 8 : 4};
    FR_CUDA(ctx, cudaMemsetAsync(lat->counters + 1, 0, sizeof(int), ctx->stream));
    launch_slice_out((const float4 *)d_query, (int)m, lat->scale[0], lat->scale[1], lat->scale[2], t,
                     lat->vdim, d_out, lat->counters + 1, ctx->stream);
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    int h = 0;
    FR_CUDA(ctx, copy_async(ctx, &h, lat->counters + 1, sizeof(int), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx, h);
}

FR_API fr_status fr_lattice_vertices(fr_ctx *ctx, const fr_lattice *lat, int32_t *d_keys,
                                     float *d_vals, int64_t *n_vertices) {
    if (!ctx || !lat) return FR_EINVAL;
    if (!d_keys || !aligned16(d_keys)) return ctx->fail(FR_EINVAL, "d_keys must be a 16-byte aligned buffer");
    cudaSetDevice(ctx->device);
    Table t{lat->keys, lat->cap - 1, lat->cap, lat->vdim > 4 ? 8 : 4};
    FR_CUDA(ctx, cudaMemsetAsync(lat->counters + 2, 0, sizeof(int), ctx->stream));
    launch_vertices(t, lat->vdim > 0 ? lat->vdim : 1, d_keys, lat->vdim > 0 ? d_vals : nullptr,
                    lat->counters + 2, ctx->stream);
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    int h = 0;
    FR_CUDA(ctx, copy_async(ctx, &h, lat->counters + 2, sizeof(int), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (n_vertices) *n_vertices = h;
    return FR_OK;
}

FR_API fr_status fr_lattice_info(fr_ctx *ctx, const fr_lattice *lat, int64_t *n_vertices,
                                 int64_t *capacity, int32_t *val_dim) {
    if (!ctx || !lat) return FR_EINVAL;
    if (n_vertices) *n_vertices = lat->nvert;
    if (capacity) *capacity = lat->cap;
    if (val_dim) *val_dim = lat->vdim;
    return FR_OK;
}

FR_API fr_status fr_lattice_destroy(fr_ctx *ctx, fr_lattice *lat) {
    if (!lat) return FR_OK;
    if (ctx) {
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize(ctx->stream);
    }
    cudaFree(lat->keys);
    cudaFree(lat->tkeys);
    cudaFree(lat->rec_slot);
    cudaFree(lat->rec_w);
    cudaFree(lat->counters);
    delete lat;
    return FR_OK;
}

// ---- E step -----------------------------------------------------------------

static fr_status estep_impl(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                            const float *d_Yn, int64_t N, float sigma, int blur, int storage,
                            const double T[16], float *d_out) {
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_cloud(ctx, d_X, M, "d_X"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (d_Yn) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn"));
    if (!d_out || !T) return ctx->fail(FR_EINVAL, "d_out and T must not be NULL");
    if (!(sigma > 0.0f) || !std::isfinite(sigma)) return ctx->fail(FR_EINVAL, "sigma must be > 0");
    cudaSetDevice(ctx->device);
    const int pt2pl = d_Yn ? 1 : 0;
    const uint32_t cap = table_slots(N, true);
    if (storage != FR_FP32 && storage != FR_BF16 && storage != FR_FP16)
        return ctx->fail(FR_EINVAL, "storage must be FR_FP32, FR_BF16 or FR_FP16");
    FR_TRY(ensure_small(ctx, 1, 1));
    FR_TRY(ensure_tables(ctx, cap, blur != 0, storage != FR_FP32));
    Table t = ctx->tables[0];
    t.mask = cap - 1;
    t.max_probe = table_probe_limit(cap, true);
    fr_options o;
    fr_options_default(&o);
    o.iters = 1;
    o.sigma_start = o.sigma_end = sigma;
    o.blur = blur;
    o.storage = storage;
    fill_iter_params(&o, M, N, ctx->h_ip);
    RigidJob *j = ctx->h_job;
    *j = RigidJob{};
    j->X = (const float4 *)d_X;
    j->Y = (const float4 *)d_Y;
    j->Yn = (const float4 *)d_Yn;
    j->M = (int)M;
    j->N = (int)N;
    DeviceState *hs = ctx->h_state;
    *hs = DeviceState{};
    for (int i = 0; i < 16; ++i) hs->T[i] = T[i];
    FR_CUDA(ctx, copy_async(ctx, ctx->d_job, j, sizeof(RigidJob), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, ctx->d_ip, ctx->h_ip, sizeof(IterParams), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, ctx->d_state, hs, sizeof(DeviceState), cudaMemcpyHostToDevice));
    IterLaunch b{};
    b.job = ctx->d_job;
    b.ip = ctx->d_ip;
    b.st = ctx->d_state;
    b.build = t;
    b.build_list = ctx->lists[0];
    b.build_it = 0;
    b.gb = blocks_for(ctx, N, 8);
    launch_em_iter(pt2pl, 0, b, ctx->stream, storage);
    ctx->launches += 1;
    if (storage != FR_FP32) {  // 16-bit records of the completed build
        IterLaunch c{};
        c.job = ctx->d_job;
        c.ip = ctx->d_ip;
        c.st = ctx->d_state;
        c.conv = t;
        c.conv_list = ctx->lists[0];
        c.conv_it = 0;
        c.gv = blocks_for(ctx, cap, 4);
        launch_em_iter(pt2pl, 0, c, ctx->stream, storage);
        ctx->launches += 1;
    }
    if (blur) {
        Table a = t, c = t;
        c.keys = ctx->blur;
        const int gb = blocks_for(ctx, N, 8);
        const int *cnt = &ctx->d_ip[0].nvert;
        for (int dir = 0; dir < 4; ++dir) {
            if (dir % 2 == 0)
                launch_blur_list(a, c, dir, ctx->lists[0], cnt, gb, ctx->d_state, ctx->stream);
            else
                launch_blur_list(c, a, dir, ctx->lists[0], cnt, gb, ctx->d_state, ctx->stream);
        }
        int *lc = ctx->lists[0];
        launch_clear_lists(&c, &lc, &cnt, 1, gb, ctx->stream);
        ctx->launches += 5;
    }
    launch_estep_out(pt2pl, ctx->d_job, ctx->d_ip, t, d_out, ctx->d_state, blocks_for(ctx, M, 8),
                     ctx->stream, storage);
    int *l0 = ctx->lists[0];
    const int *c0 = &ctx->d_ip[0].nvert;
    launch_clear_lists(&t, &l0, &c0, 1, blocks_for(ctx, N, 4), ctx->stream);
    ctx->launches += 2;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, copy_async(ctx, hs, ctx->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx, hs->flags);
}

FR_API fr_status fr_estep(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                          const float *d_Yn, int64_t N, float sigma, int blur, const double T[16],
                          float *d_out) {
    fr::NvtxRange nvtx_("fr_estep");
    return estep_impl(ctx, d_X, M, d_Y, d_Yn, N, sigma, blur, FR_FP32, T, d_out);
}

FR_API fr_status fr_estep_storage(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                  const float *d_Yn, int64_t N, float sigma, int32_t storage,
                                  const double T[16], float *d_out) {
    fr::NvtxRange nvtx_("fr_estep_storage");
    return estep_impl(ctx, d_X, M, d_Y, d_Yn, N, sigma, 0, storage, T, d_out);
}

// ---- rigid registration -----------------------------------------------------

// m_outlier: the model point count in Eq. 7's outlier constant (the whole
// model's when X is one shard of it; 0 = M).
static fr_status register_rigid_once(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                     const float *d_Yn, int64_t N, const fr_options *opt,
                                     double T_inout[16], fr_report *rep, bool safe, int64_t m_outlier = 0) {
    const int64_t Mo = m_outlier > 0 ? m_outlier : M;
    const int pt2pl = opt->residual == FR_PT2PL;
    const uint32_t cap = table_slots(N, safe);
    FR_TRY(ensure_small(ctx, opt->iters, 1));
    Plan p{};
    p.iters = opt->iters;
    p.residual = pt2pl;
    p.blur = opt->blur ? 1 : 0;
    p.kahan = opt->kahan ? 1 : 0;
    p.storage = opt->storage;
    p.profile = ctx->profiling;
    p.sig = opt->update_sigma ? 1 : 0;
    if (p.sig) {
        // iteration 0 at sigma_start; the steps set up the later ones
        fr_options o0 = *opt;
        o0.sigma_end = opt->sigma_start;
        fill_iter_params(&o0, Mo, N, ctx->h_ip);
        p.annealed = 1;
    } else {
        p.annealed = fill_iter_params(opt, Mo, N, ctx->h_ip) ? 1 : 0;
    }
    plan_grids(ctx, p, M, N, cap);
    FR_TRY(ensure_small(ctx, opt->iters, p.gs));
    FR_TRY(ensure_tables(ctx, cap, p.blur != 0, p.storage != FR_FP32));
    for (Table &t : ctx->tables) {
        t.mask = cap - 1;
        t.max_probe = table_probe_limit(cap, safe);
    }

    RigidJob *j = ctx->h_job;
    *j = RigidJob{};
    j->X = (const float4 *)d_X;
    j->Y = (const float4 *)d_Y;
    j->Yn = (const float4 *)d_Yn;
    j->M = (int)M;
    j->N = (int)N;
    j->renormalize = opt->renormalize_normals ? 1 : 0;
    j->stop_twist = opt->stop_twist;
    for (int i = 0; i < 16; ++i) j->T0[i] = T_inout[i];
    for (int i = 1; i <= 3; ++i) j->sig_alpha[i - 1] = kAlpha / std::sqrt((double)(i * (i + 1)));
    j->sig_c = (double)opt->w / (1.0 - (double)opt->w) * ((double)N / (double)Mo);
    j->sig_G = lattice_kernel_mass(0);
    j->sig_floor = (double)opt->sigma_end;
    j->sig_kappa = lattice_kernel_variance();
    DeviceState *hs = ctx->h_state;
    *hs = DeviceState{};
    for (int i = 0; i < 16; ++i) hs->T[i] = T_inout[i];
    FR_CUDA(ctx, copy_async(ctx, ctx->d_job, j, sizeof(RigidJob), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, ctx->d_state, hs, sizeof(DeviceState), cudaMemcpyHostToDevice));
    if (opt->iters > 0)
        FR_CUDA(ctx, copy_async(ctx, ctx->d_ip, ctx->h_ip, opt->iters * sizeof(IterParams),
                                cudaMemcpyHostToDevice));
    FR_TRY(run_plan(ctx, p, opt->use_graph != 0));
    FR_CUDA(ctx, copy_async(ctx, hs, ctx->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost));
    if (opt->iters > 0)
        FR_CUDA(ctx, copy_async(ctx, ctx->h_ip, ctx->d_ip, opt->iters * sizeof(IterParams),
                                cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (p.profile) collect_profile(ctx, plan_kernels(p));
    const DeviceState &s = *hs;
    FR_TRY(check_flags(ctx, s.flags));
    for (int i = 0; i < 16; ++i) T_inout[i] = s.T[i];
    if (rep) {
        rep->iters_run = s.iters_run;
        rep->degenerate_iters = s.degenerate;
        rep->last_inliers = s.inliers;
        rep->last_sum_w = s.sum_w;
        rep->last_cost = s.cost;
        rep->last_twist_norm = s.twist_norm;
        const int last_build = (p.annealed && s.iters_run > 0) ? s.iters_run - 1 : 0;
        rep->lattice_vertices = opt->iters > 0 ? ctx->h_ip[last_build].nvert : 0;
        rep->lattice_builds = s.builds;
        rep->lattice_vertices_sum = s.nvert_total;
        rep->last_sigma = (opt->iters > 0 && s.iters_run > 0) ? ctx->h_ip[s.iters_run - 1].sigma : 0.0;
    }
    return FR_OK;
}

// Compact tables first; if one overflows, the registration is rerun from its
// initial pose at the size that cannot overflow.
static fr_status register_rigid_impl(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                     const float *d_Yn, int64_t N, const fr_options *opt,
                                     double T_inout[16], fr_report *rep) {
    const fr_status s = register_rigid_once(ctx, d_X, M, d_Y, d_Yn, N, opt, T_inout, rep, false);
    if (s != FR_ECAPACITY) return s;
    return register_rigid_once(ctx, d_X, M, d_Y, d_Yn, N, opt, T_inout, rep, true);
}

FR_API fr_status fr_rigid_normal_equations(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                           const float *d_Yn, int64_t N, const fr_options *opt, int64_t M_total,
                                           const double T[16], double ne[FR_NE_VALS]) {
    fr::NvtxRange nvtx_("fr_rigid_normal_equations");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_options(ctx, opt));
    FR_TRY(validate_cloud(ctx, d_X, M, "d_X"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (opt->residual == FR_PT2PL) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn (normals, required for FR_PT2PL)"));
    if (opt->update_sigma) return ctx->fail(FR_ENOTSUPPORTED, "normal equations are taken at a given sigma");
    if (M_total < M || M_total > (1ll << 40)) return ctx->fail(FR_EINVAL, "M_total must be >= M");
    if (!T || !ne) return ctx->fail(FR_EINVAL, "T and ne must not be NULL");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T[i])) return ctx->fail(FR_EINVAL, "T is not finite");
    cudaSetDevice(ctx->device);
    // one EM iteration at sigma_start: its E step and reduced sums (the pose
    // update it also makes is discarded)
    fr_options o = *opt;
    o.iters = 1;
    o.sigma_end = o.sigma_start;
    o.stop_twist = 0.0f;
    double Tw[16];
    for (int i = 0; i < 16; ++i) Tw[i] = T[i];
    const float *yn = opt->residual == FR_PT2PL ? d_Yn : nullptr;
    fr_status st = register_rigid_once(ctx, d_X, M, d_Y, yn, N, &o, Tw, nullptr, false, M_total);
    if (st == FR_ECAPACITY) {
        for (int i = 0; i < 16; ++i) Tw[i] = T[i];
        st = register_rigid_once(ctx, d_X, M, d_Y, yn, N, &o, Tw, nullptr, true, M_total);
    }
    if (st != FR_OK) return st;
    const double *v = ctx->h_state->sums;
    for (int i = 0; i < FR_NE_VALS; ++i) ne[i] = v[i];
    return FR_OK;
}

FR_API fr_status fr_register_rigid(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                   const float *d_Yn, int64_t N, const fr_options *opt,
                                   double T_inout[16], fr_report *report) {
    fr::NvtxRange nvtx_("fr_register_rigid");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_options(ctx, opt));
    FR_TRY(validate_cloud(ctx, d_X, M, "d_X"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (opt->residual == FR_PT2PL) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn (normals, required for FR_PT2PL)"));
    if (!T_inout) return ctx->fail(FR_EINVAL, "T_inout is NULL");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T_inout[i])) return ctx->fail(FR_EINVAL, "T_inout is not finite");
    cudaSetDevice(ctx->device);
    return register_rigid_impl(ctx, d_X, M, d_Y, opt->residual == FR_PT2PL ? d_Yn : nullptr, N, opt,
                               T_inout, report);
}

FR_API fr_status fr_register_rigid_host(fr_ctx *ctx, const float *h_X, int64_t M,
                                        const float *h_Y, const float *h_Yn, int64_t N,
                                        const fr_options *opt, double T_inout[16],
                                        fr_report *report) {
    fr::NvtxRange nvtx_("fr_register_rigid_host");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_options(ctx, opt));
    if (!h_X || !h_Y || M < 1 || N < 1 || M > (1ll << 30) || N > (1ll << 30))
        return ctx->fail(FR_EINVAL, "host clouds must be non-NULL with 1 <= size <= 2^30");
    const int pt2pl = opt->residual == FR_PT2PL;
    if (pt2pl && !h_Yn) return ctx->fail(FR_EINVAL, "h_Yn (normals) is required for FR_PT2PL");
    if (!T_inout) return ctx->fail(FR_EINVAL, "T_inout is NULL");
    cudaSetDevice(ctx->device);
    const size_t need = (size_t)M + (size_t)N * (pt2pl ? 2 : 1);
    if (need > ctx->stage_cap) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->stage);
        ctx->stage = nullptr;
        ctx->stage_cap = 0;
        FR_CUDA(ctx, dev_alloc(&ctx->stage, need));
        ctx->stage_cap = need;
    }
    float4 *dX = ctx->stage, *dY = dX + M, *dN = pt2pl ? dY + N : nullptr;
    FR_CUDA(ctx, copy_async(ctx, dX, h_X, M * sizeof(float4), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, dY, h_Y, N * sizeof(float4), cudaMemcpyHostToDevice));
    if (pt2pl)
        FR_CUDA(ctx, copy_async(ctx, dN, h_Yn, N * sizeof(float4), cudaMemcpyHostToDevice));
    return register_rigid_impl(ctx, (const float *)dX, M, (const float *)dY, (const float *)dN, N,
                               opt, T_inout, report);
}

}  // extern "C"
