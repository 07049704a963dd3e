// Batched rigid registration: many registrations advanced together, one
// launch of k_em_multi per EM iteration for the whole batch.
//
// Each registration ("slot") gets its own rotating lattice tables, its own
// reduction partials, pose state and per-iteration constants; one launch
// runs, for every slot, the step of iteration k (slice + reduction, the last
// block of the slot solving its 6x6 system), the build of iteration k+1 when
// the slot's sigma is annealed, and the clear of the table of build k-1.
// While one slot's last block runs its float64 solve, the other slots'
// blocks keep the SMs busy -- the latency tail of a single registration is
// hidden by the batch.
//
// Launch shapes (points per thread of step and build blocks, compact table
// size) come from the context's tuning table, per size class; a call's
// launch sequence is captured once per shape into a CUDA graph and replayed
// by later calls of the same shape, only the descriptors being uploaded.
//
// Memory: the key and value arenas hold every slot's tables.  They are empty
// (keys all-ones, values zero) between calls -- every call frees what it
// claimed -- so a call may carve them differently from the last one.  The
// misc arena (descriptors, slot lists, partials) needs no initial state.
#include "context.h"

#include <algorithm>

using namespace fr;

namespace fr {

// A captured batched launch sequence and the shape it was captured for.
struct BatchGraph {
    std::vector<long long> key;
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    uint64_t last_use = 0;
};

struct BatchWorkspace {
    unsigned long long *keys = nullptr;  // slot-record arena, all free (zero) between calls
    size_t slots_cap = 0;                // table slots in the arena
    unsigned char *misc = nullptr;       // descriptors, lists, partials
    size_t misc_cap = 0;
    unsigned char *h_up = nullptr;       // pinned staging of the uploaded descriptors
    size_t h_up_cap = 0;
    unsigned char *h_down = nullptr;     // pinned staging of the results
    size_t h_down_cap = 0;
    float4 *stage = nullptr;             // inputs of the host-buffer variant
    size_t stage_cap = 0;
    void *d_chunks = nullptr;            // gather chunk table (device) ...
    void *h_chunks = nullptr;            // ... and its pinned staging
    size_t chunks_cap = 0;               // bytes of each
    std::vector<BatchGraph> graphs;      // least recently used out
    uint64_t use_clock = 0;
};

void drop_batch_graphs(BatchWorkspace *w) {
    for (auto &g : w->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    w->graphs.clear();
}

void free_batch_workspace(fr_ctx *ctx) {
    BatchWorkspace *w = ctx->batch;
    if (!w) return;
    drop_batch_graphs(w);
    cudaFree(w->d_chunks);
    cudaFreeHost(w->h_chunks);
    cudaFree(w->keys);
    cudaFree(w->misc);
    cudaFree(w->stage);
    cudaFreeHost(w->h_up);
    cudaFreeHost(w->h_down);
    delete w;
    ctx->batch = nullptr;
}

}  // namespace fr

namespace {


size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

fr_status ensure_arenas(fr_ctx *ctx, size_t slots, size_t misc, size_t up, size_t down,
                        bool compact) {
    if (!ctx->batch) ctx->batch = new BatchWorkspace();
    BatchWorkspace *w = ctx->batch;
    if (slots > w->slots_cap) {
        if (ctx->ws_limit && table_bytes(slots) > ctx->ws_limit)
            return ctx->fail(FR_ENOMEM, "batch tables need %zu bytes, above the context's workspace limit %zu",
                             table_bytes(slots), ctx->ws_limit);
        size_t cap = std::max(slots, w->slots_cap * 3 / 2);
        if (ctx->ws_limit) cap = std::min(cap, ctx->ws_limit / table_bytes(1));
        cudaStreamSynchronize(ctx->stream);
        cudaFree(w->keys);
        w->keys = nullptr;
        w->slots_cap = 0;
        FR_CUDA(ctx, dev_alloc(&w->keys, cap * kRecWords));
        FR_CUDA(ctx, cudaMemsetAsync(w->keys, 0, table_bytes(cap), ctx->stream));
        w->slots_cap = cap;
    }

    if (misc > w->misc_cap) {
        const size_t cap = std::max(misc, w->misc_cap * 3 / 2);
        cudaStreamSynchronize(ctx->stream);
        drop_batch_graphs(w);
        cudaFree(w->misc);
        w->misc = nullptr;
        w->misc_cap = 0;
        FR_CUDA(ctx, dev_alloc(&w->misc, cap));
        w->misc_cap = cap;
    }
    if (up > w->h_up_cap) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeHost(w->h_up);
        w->h_up = nullptr;
        w->h_up_cap = 0;
        FR_CUDA(ctx, cudaMallocHost((void **)&w->h_up, up));
        w->h_up_cap = up;
    }
    if (down > w->h_down_cap) {
        cudaStreamSynchronize(ctx->stream);
        cudaFreeHost(w->h_down);
        w->h_down = nullptr;
        w->h_down_cap = 0;
        FR_CUDA(ctx, cudaMallocHost((void **)&w->h_down, down));
        w->h_down_cap = down;
    }
    return FR_OK;
}

int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

struct ItemPlan {
    uint32_t cap;
    int annealed;
    int gs, gb, gc, gp, gv;    // step, build, clear blocks per launch; first-build blocks; convert
    int gf;                    // blocks of the final clear
    size_t tab_off;            // first slot of its tables in the arenas
    size_t list_off, part_off; // in misc (bytes)
};

constexpr size_t kBatchGraphCache = 16;

// One launch of the batched sequence: its segment table, block -> segment
// map, grid and profile class.
struct BatchLaunch {
    size_t segs_off, map_off;  // in the misc arena
    int grid, check_done, cls;
};

// Issues the launch sequence on `s` (plain, or inside a stream capture);
// with profiling on, an event pair brackets each launch (an external record
// inside a capture, so that the graph keeps it).
void issue_batch(fr_ctx *ctx, const std::vector<BatchLaunch> &L, const Slot *dslots, unsigned char *D,
                 int pt2pl, int kahan, int storage, cudaStream_t s, bool capturing) {
    for (size_t i = 0; i < L.size(); ++i) {
        if (ctx->profiling) {
            while (ctx->events.size() < 2 * (i + 1)) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ctx->events.push_back(e);
            }
            if (ctx->event_class.size() < i + 1) ctx->event_class.resize(i + 1);
            ctx->event_class[i] = L[i].cls;
            if (capturing) cudaEventRecordWithFlags(ctx->events[2 * i], s, cudaEventRecordExternal);
            else cudaEventRecord(ctx->events[2 * i], s);
        }
        launch_em_multi(pt2pl, kahan, dslots, (const Seg *)(D + L[i].segs_off),
                        (const unsigned short *)(D + L[i].map_off), L[i].grid, L[i].check_done, s, storage);
        if (ctx->profiling) {
            if (capturing) cudaEventRecordWithFlags(ctx->events[2 * i + 1], s, cudaEventRecordExternal);
            else cudaEventRecord(ctx->events[2 * i + 1], s);
        }
    }
}

// Replays the cached graph of this launch shape, capturing it first when
// new; without a graph (capture refused) the launches are issued directly.
fr_status run_launches(fr_ctx *ctx, const std::vector<long long> &key, const std::vector<BatchLaunch> &L,
                       const Slot *dslots, unsigned char *D, int pt2pl, int kahan, int storage) {
    BatchWorkspace *w = ctx->batch;
    BatchGraph *hit = nullptr;
    for (auto &g : w->graphs)
        if (g.key == key) hit = &g;
    if (!hit) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            issue_batch(ctx, L, dslots, D, pt2pl, kahan, storage, ctx->stream, true);
            const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
            if (e == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();
        if (!exec) {  // direct launches
            issue_batch(ctx, L, dslots, D, pt2pl, kahan, storage, ctx->stream, false);
            ctx->launches += (int64_t)L.size();
            return ctx->cuda(cudaGetLastError(), "batched launch");
        }
        if (w->graphs.size() >= kBatchGraphCache) {
            auto lru = std::min_element(w->graphs.begin(), w->graphs.end(),
                                        [](const BatchGraph &a, const BatchGraph &b) { return a.last_use < b.last_use; });
            cudaGraphExecDestroy(lru->exec);
            w->graphs.erase(lru);
        }
        w->graphs.push_back(BatchGraph{key, exec, (int)L.size(), 0});
        hit = &w->graphs.back();
    }
    hit->last_use = ++w->use_clock;
    FR_CUDA(ctx, cudaGraphLaunch(hit->exec, ctx->stream));
    ctx->launches += hit->kernels;
    return FR_OK;
}

// `force` (nullable) gives every item the same launch shape (the autotuner);
// otherwise each item takes its size class's entry of the tuning table.
fr_status run_batch(fr_ctx *ctx, fr_batch_item *items, int n, const fr_options *opt,
                    fr_report *reports, bool safe, const fr_tune_params *force = nullptr) {
    const int pt2pl = opt->residual == FR_PT2PL;
    const int kahan = opt->kahan ? 1 : 0;
    const int iters = opt->iters;
    const int iters1 = iters > 0 ? iters : 1;
    // Builds run `lead` iterations ahead of their step (2 with 16-bit storage:
    // a build's records are converted in the launch after it), so
    // lead + 2 tables rotate per item.
    const int lead = opt->storage != FR_FP32 ? 2 : 1;
    const int ntab = lead + 2;

    // ---- per-item plans and the arena layout --------------------------------
    std::vector<ItemPlan> ip(n);
    size_t slots = 0;
    int seg_per_iter = 0, grid_iter = 0, grid_pro = 0, grid_pro2 = 0, grid_epi = 0;
    for (int b = 0; b < n; ++b) {
        const fr_batch_item &it = items[b];
        ItemPlan &p = ip[b];
        const fr_tune_params &tp = force ? *force : ctx->tune[tune_class(it.N)];
        p.cap = safe ? table_slots(it.N, true) : tuned_table_slots(it.N, tp.table_slots_x2);
        p.tab_off = slots;
        slots += ntab * (size_t)p.cap;
        p.gs = div_up(it.M, (long long)kBlock * tp.step_points_per_thread);
        p.gp = div_up(it.N, (long long)kBlock * tp.build_points_per_thread);
        p.annealed = (it.sigma_start != it.sigma_end && iters > 1) ? 1 : 0;
        p.gb = p.annealed ? p.gp : 0;
        p.gc = p.annealed ? std::max(1, div_up(it.N, 4096)) : 0;
        p.gv = lead == 2 ? std::max(1, div_up(it.N, 2048)) : 0;
        p.gf = std::max(1, div_up(it.N, 1024));
        seg_per_iter += 1 + (p.annealed ? 2 + (lead - 1) : 0);
        grid_iter += p.gs + p.gb + p.gc + (p.annealed ? p.gv : 0);
        grid_pro += p.gp;
        grid_pro2 += p.gv + (p.annealed ? p.gb : 0);
        grid_epi += p.gf;
    }
    if (lead == 1) grid_pro2 = 0;
    const int seg_pro = n, seg_pro2 = 2 * n, seg_epi_max = n;
    // upload region (also the device layout of the misc arena's head)
    size_t off = 0;
    const size_t o_jobs = off; off = align256(off + n * sizeof(RigidJob));
    const size_t o_states = off; off = align256(off + n * sizeof(DeviceState));
    const size_t o_ips = off; off = align256(off + (size_t)n * iters1 * sizeof(IterParams));
    const size_t o_slots = off; off = align256(off + n * sizeof(Slot));
    const size_t o_segs = off;
    off = align256(off + (size_t)(iters1 * seg_per_iter + seg_pro + seg_pro2 + seg_epi_max) * sizeof(Seg));
    const size_t o_bs_iter = off; off = align256(off + grid_iter * sizeof(unsigned short));
    const size_t o_bs_pro = off; off = align256(off + grid_pro * sizeof(unsigned short));
    const size_t o_bs_pro2 = off; off = align256(off + grid_pro2 * sizeof(unsigned short));
    const size_t o_bs_epi = off; off = align256(off + grid_epi * sizeof(unsigned short));
    const size_t up_bytes = off;
    for (int b = 0; b < n; ++b) {
        ip[b].list_off = off;
        off = align256(off + ntab * (size_t)ip[b].cap * sizeof(int));
    }
    for (int b = 0; b < n; ++b) {
        ip[b].part_off = off;
        off = align256(off + (size_t)ip[b].gs * kRigidVals * sizeof(float2));
    }
    const size_t misc_bytes = off;
    const size_t down_bytes = align256(n * sizeof(DeviceState)) + (size_t)n * iters1 * sizeof(IterParams);
    FR_TRY(ensure_arenas(ctx, slots, misc_bytes, up_bytes, down_bytes, opt->storage != FR_FP32));
    BatchWorkspace *w = ctx->batch;
    unsigned char *U = w->h_up, *D = w->misc;

    // ---- descriptors ----------------------------------------------------------
    RigidJob *jobs = (RigidJob *)(U + o_jobs);
    DeviceState *states = (DeviceState *)(U + o_states);
    IterParams *ips = (IterParams *)(U + o_ips);
    Slot *sl = (Slot *)(U + o_slots);
    for (int b = 0; b < n; ++b) {
        const fr_batch_item &it = items[b];
        RigidJob &j = jobs[b];
        j = RigidJob{};
        j.X = (const float4 *)it.d_X;
        j.Y = (const float4 *)it.d_Y;
        j.Yn = pt2pl ? (const float4 *)it.d_Yn : nullptr;
        j.M = (int)it.M;
        j.N = (int)it.N;
        j.renormalize = opt->renormalize_normals ? 1 : 0;
        j.stop_twist = opt->stop_twist;
        for (int i = 0; i < 16; ++i) j.T0[i] = it.T[i];
        states[b] = DeviceState{};
        for (int i = 0; i < 16; ++i) states[b].T[i] = it.T[i];
        fr_options o = *opt;
        o.sigma_start = it.sigma_start;
        o.sigma_end = it.sigma_end;
        o.w = it.w;
        o.blur = 0;
        fill_iter_params(&o, it.M, it.N, ips + (size_t)b * iters1);
        Slot &s = sl[b];
        s.job = (const RigidJob *)(D + o_jobs) + b;
        s.st = (DeviceState *)(D + o_states) + b;
        s.ip = (IterParams *)(D + o_ips) + (size_t)b * iters1;
        s.partials = (float2 *)(D + ip[b].part_off);
        for (int t = 0; t < ntab; ++t) {
            const size_t base = ip[b].tab_off + (size_t)t * ip[b].cap;
            s.tab[t] = Table{w->keys + base * kRecWords, ip[b].cap - 1, table_probe_limit(ip[b].cap, safe),
                             pt2pl ? 8 : 4};
            s.list[t] = (int *)(D + ip[b].list_off) + (size_t)t * ip[b].cap;
        }
    }
    // segment tables: iterations (same block map for all), first build, final clear
    Seg *segs = (Seg *)(U + o_segs);
    unsigned short *bs_iter = (unsigned short *)(U + o_bs_iter);
    unsigned short *bs_pro = (unsigned short *)(U + o_bs_pro);
    unsigned short *bs_pro2 = (unsigned short *)(U + o_bs_pro2);
    unsigned short *bs_epi = (unsigned short *)(U + o_bs_epi);
    auto tab_of = [&](int b, int build) { return ip[b].annealed ? build % ntab : 0; };
    // iteration k: every item's step k first, then the clears k-1 and the
    // builds k+lead (annealed items) and conversions k+1 (lead 2): blocks are
    // dispatched in index order, so the steps -- and their float64 tails --
    // start before the builds rather than the last items' steps ending the
    // launch.
    // Phase q: 0 step, 1 build, 2 convert, 3 clear.
    auto seg_blocks = [&](int b, int q) {
        if (q == 0) return ip[b].gs;
        if (!ip[b].annealed) return -1;  // no segment
        if (q == 1) return ip[b].gb;
        if (q == 2) return lead == 2 ? ip[b].gv : -1;
        return ip[b].gc;
    };
    // Dispatch order of the phases, measured on the batched depth-frame step:
    // steps, clears, builds, conversions 98.0 us per launch; steps, builds,
    // conversions, clears 99.8; builds first 103.9.
    const int qord[4] = {0, 3, 1, 2};
    for (int k = 0; k < iters; ++k) {
        Seg *S = segs + (size_t)k * seg_per_iter;
        int si = 0, blk = 0;
        for (int qi = 0; qi < 4; ++qi)
            for (int b = 0, q = qord[qi]; b < n; ++b) {
                const int nb = seg_blocks(b, q);
                if (nb < 0) continue;
                Seg sg{b, kRoleNone, 0, 0, blk, nb};
                if (q == 0) {
                    sg.role = kRoleStep;
                    sg.it = k;
                    sg.tab = tab_of(b, k);
                } else if (q == 1 && k + lead < iters) {
                    sg.role = kRoleBuild;
                    sg.it = k + lead;
                    sg.tab = tab_of(b, k + lead);
                } else if (q == 2 && k + 1 < iters) {
                    sg.role = kRoleConvert;
                    sg.it = k + 1;
                    sg.tab = tab_of(b, k + 1);
                } else if (q == 3 && k >= 1) {
                    sg.role = kRoleClear;
                    sg.it = k - 1;
                    sg.tab = tab_of(b, k - 1);
                }
                S[si++] = sg;
                blk += nb;
            }
    }
    {
        int si = 0, blk = 0;
        for (int qi = 0; qi < 4; ++qi)
            for (int b = 0, q = qord[qi]; b < n; ++b) {
                const int nb = seg_blocks(b, q);
                if (nb < 0) continue;
                for (int r = 0; r < nb; ++r) bs_iter[blk++] = (unsigned short)si;
                ++si;
            }
        if (blk != grid_iter) return ctx->fail(FR_EINVAL, "internal: iteration block map");
    }
    // prologue: build 0; with lead 2 a second launch converts 0 and builds 1
    Seg *Spro = segs + (size_t)iters1 * seg_per_iter;
    {
        int blk = 0;
        for (int b = 0; b < n; ++b) {
            Spro[b] = Seg{b, kRoleBuild, 0, 0, blk, ip[b].gp};
            for (int q = 0; q < ip[b].gp; ++q) bs_pro[blk++] = (unsigned short)b;
        }
        if (blk != grid_pro) return ctx->fail(FR_EINVAL, "internal: first build block map");
    }
    Seg *Spro2 = Spro + seg_pro;
    if (lead == 2) {
        int blk = 0, si = 0;
        for (int b = 0; b < n; ++b) {
            Spro2[si] = Seg{b, kRoleConvert, 0, 0, blk, ip[b].gv};
            for (int q = 0; q < ip[b].gv; ++q) bs_pro2[blk++] = (unsigned short)si;
            ++si;
            if (ip[b].annealed) {
                Spro2[si] = Seg{b, iters > 1 ? kRoleBuild : kRoleNone, 1, tab_of(b, 1), blk, ip[b].gb};
                for (int q = 0; q < ip[b].gb; ++q) bs_pro2[blk++] = (unsigned short)si;
                ++si;
            }
        }
        if (blk != grid_pro2) return ctx->fail(FR_EINVAL, "internal: second prologue block map");
    }
    Seg *Sepi = Spro2 + seg_pro2;
    int n_epi = 0;
    {
        int blk = 0;
        for (int b = 0; b < n; ++b) {
            // Every other table was cleared by the launch after its step
            // (clears run even after a registration stopped).
            const int last = ip[b].annealed ? iters - 1 : 0;
            Sepi[n_epi] = Seg{b, kRoleClear, last, tab_of(b, last), blk, ip[b].gf};
            for (int q = 0; q < ip[b].gf; ++q) bs_epi[blk++] = (unsigned short)n_epi;
            ++n_epi;
        }
        if (blk != grid_epi) return ctx->fail(FR_EINVAL, "internal: final clear block map");
    }

    // ---- upload, launch (a cached graph per launch shape), read back -------------
    FR_CUDA(ctx, copy_async(ctx, D, U, up_bytes, cudaMemcpyHostToDevice));
    const Slot *dslots = (const Slot *)(D + o_slots);
    // Profile classes: first build, EM iteration, final clear.
    std::vector<BatchLaunch> launches;
    if (iters > 0) {
        const size_t seg0 = o_segs + (size_t)iters1 * seg_per_iter * sizeof(Seg);
        launches.push_back(BatchLaunch{seg0, o_bs_pro, grid_pro, 0, FR_K_BUILD});
        if (lead == 2)
            launches.push_back(BatchLaunch{seg0 + seg_pro * sizeof(Seg), o_bs_pro2, grid_pro2, 0, FR_K_CONVERT});
        for (int k = 0; k < iters; ++k)
            launches.push_back(BatchLaunch{o_segs + (size_t)k * seg_per_iter * sizeof(Seg), o_bs_iter, grid_iter, 1,
                                           FR_K_STEP});
        launches.push_back(BatchLaunch{seg0 + (size_t)(seg_pro + seg_pro2) * sizeof(Seg), o_bs_epi, grid_epi, 0,
                                       FR_K_CLEAR});
    }
    if (!launches.empty()) {
        std::vector<long long> key = {n, iters, lead, pt2pl, kahan, (long long)opt->storage, ctx->profiling,
                                      (long long)(uintptr_t)D, (long long)up_bytes};
        for (const BatchLaunch &l : launches) {
            key.push_back((long long)l.segs_off);
            key.push_back((long long)l.map_off);
            key.push_back(l.grid);
        }
        FR_TRY(run_launches(ctx, key, launches, dslots, D, pt2pl, kahan, opt->storage));
    }
    const int nprof = (int)launches.size();
    FR_CUDA(ctx, cudaGetLastError());
    unsigned char *H = w->h_down;
    FR_CUDA(ctx, copy_async(ctx, H, D + o_states, n * sizeof(DeviceState), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, copy_async(ctx, H + align256(n * sizeof(DeviceState)), D + o_ips,
                            (size_t)n * iters1 * sizeof(IterParams), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->profiling) collect_profile(ctx, nprof);
    const DeviceState *rs = (const DeviceState *)H;
    const IterParams *rip = (const IterParams *)(H + align256(n * sizeof(DeviceState)));
    fr_status first_bad = FR_OK;
    for (int b = 0; b < n; ++b) {
        const DeviceState &s = rs[b];
        fr_status st = FR_OK;
        if (s.flags & kFlagCapacity) st = FR_ECAPACITY;
        else if (s.flags & kFlagRange) st = FR_EINVAL;
        items[b].status = st;
        if (st != FR_OK && first_bad == FR_OK) {
            first_bad = st;
            ctx->fail(st, "batch item %d: %s", b, st == FR_ECAPACITY ? "lattice hash table full"
                                                                   : "non-finite or out-of-range coordinate");
        }
        if (st == FR_OK)
            for (int i = 0; i < 16; ++i) items[b].T[i] = s.T[i];
        if (reports) {
            fr_report &r = reports[b];
            r.iters_run = s.iters_run;
            r.degenerate_iters = s.degenerate;
            r.last_inliers = s.inliers;
            r.last_sum_w = s.sum_w;
            r.last_cost = s.cost;
            r.last_twist_norm = s.twist_norm;
            const int last_build = (ip[b].annealed && s.iters_run > 0) ? s.iters_run - 1 : 0;
            r.lattice_vertices = iters > 0 ? rip[(size_t)b * iters1 + last_build].nvert : 0;
            r.lattice_builds = s.builds;
            r.lattice_vertices_sum = s.nvert_total;
        }
    }
    return first_bad;
}

// One chunk of a host -> device gather: `count` float4 from src to dst.
struct GatherChunk {
    const float4 *src;
    float4 *dst;
    long long count;
};
constexpr long long kGatherChunk = 16384;  // float4 per block (256 KiB)

// Copies every chunk (block c takes chunk c) with eight 16-byte loads in
// flight per thread: reading page-locked host memory across the host link in
// one launch instead of one copy per cloud.
__global__ void __launch_bounds__(256) k_gather(const GatherChunk *chunks) {
    const GatherChunk g = chunks[blockIdx.x];
    constexpr int kU = 8;
    for (long long e0 = (long long)threadIdx.x; e0 < g.count; e0 += 256LL * kU) {
        float4 v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const long long e = e0 + 256LL * u;
            if (e < g.count) v[u] = g.src[e];
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const long long e = e0 + 256LL * u;
            if (e < g.count) g.dst[e] = v[u];
        }
    }
}

// Device address of page-locked host memory at p (nullptr when p is
// pageable, device or misaligned memory: copy it instead).
const void *mapped_host(const void *p) {
    if (!p || ((uintptr_t)p & 15u)) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Status of an item that run_batch has not reached yet: a call that fails
// before its per-item results (an allocation, a CUDA error) leaves it set.
constexpr fr_status kUnset = (fr_status)-1;

// Compact tables first; items whose table overflowed are rerun (from their
// initial poses) at the size that cannot overflow.  Every item leaves with
// its own outcome: an item the call never reached takes the call's status,
// and a rerun that fails takes the rerun's status, not its earlier one.
fr_status run_batch_sized(fr_ctx *ctx, fr_batch_item *items, int n, const fr_options *opt,
                          fr_report *reports, const fr_tune_params *force = nullptr) {
    std::vector<fr_batch_item> init(items, items + n);
    for (int b = 0; b < n; ++b) items[b].status = kUnset;
    fr_status st = run_batch(ctx, items, n, opt, reports, false, force);
    bool reached = true;
    for (int b = 0; b < n; ++b)
        if (items[b].status == kUnset) {
            items[b] = init[b];
            items[b].status = st != FR_OK ? st : FR_ECUDA;
            reached = false;
        }
    if (!reached) return st != FR_OK ? st : FR_ECUDA;
    std::vector<int> redo;
    for (int b = 0; b < n; ++b)
        if (items[b].status == FR_ECAPACITY) redo.push_back(b);
    if (redo.empty()) return st;
    std::vector<fr_batch_item> sub;
    std::vector<fr_report> subrep(redo.size());
    for (int b : redo) {
        sub.push_back(init[b]);
        sub.back().status = kUnset;
    }
    const fr_status rs = run_batch(ctx, sub.data(), (int)sub.size(), opt, reports ? subrep.data() : nullptr, true, force);
    for (size_t q = 0; q < redo.size(); ++q) {
        if (sub[q].status == kUnset) {
            sub[q] = init[redo[q]];
            sub[q].status = rs != FR_OK ? rs : FR_ECUDA;
        }
        items[redo[q]] = sub[q];
        if (reports) reports[redo[q]] = subrep[q];
    }
    st = FR_OK;
    for (int b = 0; b < n; ++b)
        if (items[b].status != FR_OK && st == FR_OK) st = items[b].status;
    return st;
}

fr_status validate_batch(fr_ctx *ctx, const fr_batch_item *items, int n, const fr_options *opt,
                         bool on_host) {
    FR_TRY(validate_options(ctx, opt));
    if (opt->blur) return ctx->fail(FR_ENOTSUPPORTED, "batched registration does not blur");
    if (opt->update_sigma) return ctx->fail(FR_ENOTSUPPORTED, "batched registration runs a sigma schedule");
    // block -> segment maps hold 16-bit segment indices: at most 65536
    // segments per launch, 4 per item (5 with 16-bit storage)
    const int max_items = opt->storage != FR_FP32 ? 65536 / 5 : 65536 / 4;
    if (!items || n < 1 || n > max_items) return ctx->fail(FR_EINVAL, "need 1..%d batch items", max_items);
    for (int b = 0; b < n; ++b) {
        const fr_batch_item &it = items[b];
        if (!it.d_X || !it.d_Y || it.M < 1 || it.N < 1 || it.M > (1ll << 30) || it.N > (1ll << 30))
            return ctx->fail(FR_EINVAL, "batch item %d: clouds must be non-NULL, 1 <= size <= 2^30", b);
        if (opt->residual == FR_PT2PL && !it.d_Yn)
            return ctx->fail(FR_EINVAL, "batch item %d: normals required for FR_PT2PL", b);
        if (!on_host && (!aligned16(it.d_X) || !aligned16(it.d_Y) || (it.d_Yn && !aligned16(it.d_Yn))))
            return ctx->fail(FR_EINVAL, "batch item %d: clouds must be 16-byte aligned", b);
        if (!(it.sigma_start > 0.0f) || !(it.sigma_end > 0.0f) || !std::isfinite(it.sigma_start) ||
            !std::isfinite(it.sigma_end))
            return ctx->fail(FR_EINVAL, "batch item %d: sigma must be finite and > 0", b);
        if (!(it.w >= 0.0f && it.w < 1.0f)) return ctx->fail(FR_EINVAL, "batch item %d: w outside [0,1)", b);
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(it.T[i])) return ctx->fail(FR_EINVAL, "batch item %d: pose not finite", b);
    }
    return FR_OK;
}

}  // namespace

extern "C" {

FR_API fr_status fr_register_rigid_batch(fr_ctx *ctx, fr_batch_item *items, int n_items,
                                         const fr_options *opt, fr_report *reports) {
    fr::NvtxRange nvtx_("fr_register_rigid_batch");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_batch(ctx, items, n_items, opt, false));
    cudaSetDevice(ctx->device);
    return run_batch_sized(ctx, items, n_items, opt, reports);
}

FR_API fr_status fr_register_rigid_batch_host(fr_ctx *ctx, fr_batch_item *items, int n_items,
                                              const fr_options *opt, fr_report *reports) {
    fr::NvtxRange nvtx_("fr_register_rigid_batch_host");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_batch(ctx, items, n_items, opt, true));
    cudaSetDevice(ctx->device);
    const int pt2pl = opt->residual == FR_PT2PL;
    size_t need = 0;
    for (int b = 0; b < n_items; ++b) need += items[b].M + items[b].N * (pt2pl ? 2 : 1);
    if (!ctx->batch) ctx->batch = new BatchWorkspace();
    BatchWorkspace *w = ctx->batch;
    if (need > w->stage_cap) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(w->stage);
        w->stage = nullptr;
        w->stage_cap = 0;
        FR_CUDA(ctx, dev_alloc(&w->stage, need));
        w->stage_cap = need;
    }
    // The clouds go to the staging area: one gather launch when every cloud
    // is page-locked host memory, else one copy per cloud.
    struct Src { const void *h, *d; size_t n; float4 *dst; };
    std::vector<Src> src;
    std::vector<fr_batch_item> dev(items, items + n_items);
    float4 *p = w->stage;
    bool mapped = true;
    auto add = [&](const float *h, size_t n) {
        const void *d = mapped_host(h);
        mapped = mapped && d;
        src.push_back(Src{h, d, n, p});
        p += n;
        return (const float *)src.back().dst;
    };
    for (int b = 0; b < n_items; ++b) {
        const fr_batch_item &h = items[b];
        dev[b].d_X = add(h.d_X, (size_t)h.M);
        dev[b].d_Y = add(h.d_Y, (size_t)h.N);
        dev[b].d_Yn = pt2pl ? add(h.d_Yn, (size_t)h.N) : nullptr;
    }
    if (mapped) {
        std::vector<GatherChunk> chunks;
        for (const Src &c : src)
            for (size_t o = 0; o < c.n; o += kGatherChunk)
                chunks.push_back(GatherChunk{(const float4 *)c.d + o, c.dst + o,
                                             (long long)std::min<size_t>(kGatherChunk, c.n - o)});
        const size_t bytes = chunks.size() * sizeof(GatherChunk);
        if (bytes > w->chunks_cap) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(w->d_chunks);
            cudaFreeHost(w->h_chunks);
            w->d_chunks = w->h_chunks = nullptr;
            w->chunks_cap = 0;
            const size_t cap = std::max(bytes * 2, (size_t)4096);
            FR_CUDA(ctx, fr::dev_malloc(&w->d_chunks, cap));
            FR_CUDA(ctx, cudaMallocHost(&w->h_chunks, cap));
            w->chunks_cap = cap;
        }
        // (every call ends synchronised, so the pinned table is free to rewrite)
        std::memcpy(w->h_chunks, chunks.data(), bytes);
        FR_CUDA(ctx, cudaMemcpyAsync(w->d_chunks, w->h_chunks, bytes, cudaMemcpyHostToDevice, ctx->stream));
        k_gather<<<(int)chunks.size(), 256, 0, ctx->stream>>>((const GatherChunk *)w->d_chunks);
        FR_CUDA(ctx, cudaGetLastError());
        ctx->launches += 1;
        for (const Src &c : src) ctx->h2d_bytes += (int64_t)(c.n * sizeof(float4));
    } else {
        for (const Src &c : src) FR_CUDA(ctx, copy_async(ctx, c.dst, c.h, c.n * sizeof(float4), cudaMemcpyHostToDevice));
    }
    const fr_status st = run_batch_sized(ctx, dev.data(), n_items, opt, reports);
    for (int b = 0; b < n_items; ++b) {
        items[b].status = dev[b].status;
        for (int i = 0; i < 16; ++i) items[b].T[i] = dev[b].T[i];
    }
    return st;
}

FR_API fr_status fr_autotune_batch(fr_ctx *ctx, const fr_batch_item *items, int n_items, const fr_options *opt,
                                   int objective, int reps, fr_tune_params *best, double *best_ms,
                                   double *default_ms) {
    fr::NvtxRange nvtx_("fr_autotune_batch");
    if (!ctx || !best) return FR_EINVAL;
    if (objective != FR_TUNE_THROUGHPUT && objective != FR_TUNE_LATENCY)
        return ctx->fail(FR_EINVAL, "objective must be FR_TUNE_THROUGHPUT or FR_TUNE_LATENCY");
    if (reps < 1 || reps > 50) return ctx->fail(FR_EINVAL, "reps must be in 1..50");
    FR_TRY(validate_batch(ctx, items, n_items, opt, false));
    cudaSetDevice(ctx->device);
    long long nsum = 0;
    for (int b = 0; b < n_items; ++b) nsum += items[b].N;
    const int cls = tune_class(nsum / n_items);
    const fr_tune_params cur = ctx->tune[cls];
    std::vector<fr_tune_params> cand;
    if (objective == FR_TUNE_THROUGHPUT) {
        for (int sp : {2, 4, 8, 16})
            for (int bp : {4, 8, 16})
                for (int x2 : {3, 6}) cand.push_back(fr_tune_params{sp, bp, x2, cur.serve_points_per_thread});
    } else {
        for (int pp : {1, 2, 4, 8}) cand.push_back(fr_tune_params{pp, pp, cur.table_slots_x2, pp});
    }
    cudaEvent_t e0, e1;
    FR_CUDA(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ctx->cuda(cudaGetLastError(), "cudaEventCreate");
    }
    std::vector<fr_batch_item> work(items, items + n_items);
    // Median time of `reps` calls (after one untimed call that captures the graph).
    auto measure = [&](const fr_tune_params &tp, double &ms) -> fr_status {
        std::vector<double> t;
        for (int r = 0; r <= reps; ++r) {
            std::copy(items, items + n_items, work.begin());
            cudaEventRecord(e0, ctx->stream);
            const fr_status st = run_batch_sized(ctx, work.data(), n_items, opt, nullptr, &tp);
            cudaEventRecord(e1, ctx->stream);
            if (st != FR_OK) return st;
            FR_CUDA(ctx, cudaEventSynchronize(e1));
            float f = 0.0f;
            cudaEventElapsedTime(&f, e0, e1);
            if (r > 0) t.push_back(f);
        }
        std::sort(t.begin(), t.end());
        ms = t[t.size() / 2];
        return FR_OK;
    };
    fr_status st = FR_OK;
    fr_tune_params dflt = tune_default();
    if (objective == FR_TUNE_LATENCY)
        dflt = fr_tune_params{dflt.serve_points_per_thread, dflt.serve_points_per_thread, cur.table_slots_x2,
                              dflt.serve_points_per_thread};
    double d_ms = 0.0, b_ms = 1e300;
    fr_tune_params win = dflt;
    st = measure(dflt, d_ms);
    if (st == FR_OK) {
        b_ms = d_ms;
        for (const fr_tune_params &c : cand) {
            double ms = 0.0;
            st = measure(c, ms);
            if (st != FR_OK) break;
            if (ms < b_ms) {
                b_ms = ms;
                win = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FR_OK) return st;
    fr_tune_params inst = cur;
    if (objective == FR_TUNE_THROUGHPUT) {
        inst.step_points_per_thread = win.step_points_per_thread;
        inst.build_points_per_thread = win.build_points_per_thread;
        inst.table_slots_x2 = win.table_slots_x2;
    } else {
        inst.serve_points_per_thread = win.serve_points_per_thread;
    }
    ctx->tune[cls] = inst;
    *best = inst;
    if (best_ms) *best_ms = b_ms;
    if (default_ms) *default_ms = d_ms;
    return FR_OK;
}

}  // extern "C"
