// Batched rigid registration: many registrations advanced together, one
// launch of k_em_multi per EM iteration for the whole batch.
//
// Each registration ("slot") gets its own three rotating lattice tables, its
// own reduction partials, pose state and per-iteration constants; one launch
// runs, for every slot, the step of iteration k (slice + reduction, the last
// block of the slot solving its 6x6 system), the build of iteration k+1 when
// the slot's sigma is annealed, and the clear of the table of build k-1.
// While one slot's last block runs its float64 solve, the other slots'
// blocks keep the SMs busy -- the latency tail of a single registration is
// hidden by the batch.
//
// Memory: the key and value arenas hold every slot's tables.  They are empty
// (keys all-ones, values zero) between calls -- every call frees what it
// claimed -- so a call may carve them differently from the last one.  The
// misc arena (descriptors, slot lists, partials) needs no initial state.
#include "context.h"

#include <algorithm>

using namespace fr;

namespace fr {

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
};

void free_batch_workspace(fr_ctx *ctx) {
    BatchWorkspace *w = ctx->batch;
    if (!w) return;
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

fr_status run_batch(fr_ctx *ctx, fr_batch_item *items, int n, const fr_options *opt,
                    fr_report *reports, bool safe) {
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
        p.cap = table_slots(it.N, safe);
        p.tab_off = slots;
        slots += ntab * (size_t)p.cap;
        p.gs = div_up(it.M, (long long)kBlock * kMultiPointsPerThread);
        p.gp = div_up(it.N, (long long)kBlock * kMultiPointsPerThread);
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
    // iteration k: every item's step k first, then the builds k+lead (annealed
    // items), conversions k+1 (lead 2) and clears k-1: blocks are dispatched in
    // index order, so the steps -- and their float64 tails -- start before the
    // builds rather than the last items' steps ending the launch.
    // Phase q: 0 step, 1 build, 2 convert, 3 clear.
    auto seg_blocks = [&](int b, int q) {
        if (q == 0) return ip[b].gs;
        if (!ip[b].annealed) return -1;  // no segment
        if (q == 1) return ip[b].gb;
        if (q == 2) return lead == 2 ? ip[b].gv : -1;
        return ip[b].gc;
    };
    for (int k = 0; k < iters; ++k) {
        Seg *S = segs + (size_t)k * seg_per_iter;
        int si = 0, blk = 0;
        for (int q = 0; q < 4; ++q)
            for (int b = 0; b < n; ++b) {
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
        for (int q = 0; q < 4; ++q)
            for (int b = 0; b < n; ++b) {
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

    // ---- upload, launch, read back ---------------------------------------------
    FR_CUDA(ctx, copy_async(ctx, D, U, up_bytes, cudaMemcpyHostToDevice));
    const Slot *dslots = (const Slot *)(D + o_slots);
    const Seg *dsegs = (const Seg *)(D + o_segs);
    // With profiling on, an event pair brackets each launch (classes: first
    // build, EM iteration, final clear).
    int nprof = 0;
    auto timed = [&](int cls, auto &&launch) {
        if (ctx->profiling) {
            while (ctx->events.size() < 2 * (size_t)(nprof + 1)) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                ctx->events.push_back(e);
            }
            if (ctx->event_class.size() < (size_t)(nprof + 1)) ctx->event_class.resize(nprof + 1);
            ctx->event_class[nprof] = cls;
            cudaEventRecord(ctx->events[2 * nprof], ctx->stream);
        }
        launch();
        if (ctx->profiling) cudaEventRecord(ctx->events[2 * nprof + 1], ctx->stream);
        ++nprof;
    };
    if (iters > 0) {
        timed(FR_K_BUILD, [&] {
            launch_em_multi(pt2pl, kahan, dslots, dsegs + (size_t)iters1 * seg_per_iter,
                            (const unsigned short *)(D + o_bs_pro), grid_pro, 0, ctx->stream, opt->storage);
        });
        if (lead == 2)
            timed(FR_K_CONVERT, [&] {
                launch_em_multi(pt2pl, kahan, dslots, dsegs + (size_t)iters1 * seg_per_iter + seg_pro,
                                (const unsigned short *)(D + o_bs_pro2), grid_pro2, 0, ctx->stream,
                                opt->storage);
            });
        for (int k = 0; k < iters; ++k)
            timed(FR_K_STEP, [&] {
                launch_em_multi(pt2pl, kahan, dslots, dsegs + (size_t)k * seg_per_iter,
                                (const unsigned short *)(D + o_bs_iter), grid_iter, 1, ctx->stream,
                                opt->storage);
            });
        timed(FR_K_CLEAR, [&] {
            launch_em_multi(pt2pl, kahan, dslots, dsegs + (size_t)iters1 * seg_per_iter + seg_pro + seg_pro2,
                            (const unsigned short *)(D + o_bs_epi), grid_epi, 0, ctx->stream, opt->storage);
        });
        ctx->launches += iters + 2 + (lead - 1);
    }
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

// Status of an item that run_batch has not reached yet: a call that fails
// before its per-item results (an allocation, a CUDA error) leaves it set.
constexpr fr_status kUnset = (fr_status)-1;

// Compact tables first; items whose table overflowed are rerun (from their
// initial poses) at the size that cannot overflow.  Every item leaves with
// its own outcome: an item the call never reached takes the call's status,
// and a rerun that fails takes the rerun's status, not its earlier one.
fr_status run_batch_sized(fr_ctx *ctx, fr_batch_item *items, int n, const fr_options *opt,
                          fr_report *reports) {
    std::vector<fr_batch_item> init(items, items + n);
    for (int b = 0; b < n; ++b) items[b].status = kUnset;
    fr_status st = run_batch(ctx, items, n, opt, reports, false);
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
    const fr_status rs = run_batch(ctx, sub.data(), (int)sub.size(), opt, reports ? subrep.data() : nullptr, true);
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
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_batch(ctx, items, n_items, opt, false));
    cudaSetDevice(ctx->device);
    return run_batch_sized(ctx, items, n_items, opt, reports);
}

FR_API fr_status fr_register_rigid_batch_host(fr_ctx *ctx, fr_batch_item *items, int n_items,
                                              const fr_options *opt, fr_report *reports) {
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
    std::vector<fr_batch_item> dev(items, items + n_items);
    float4 *p = w->stage;
    for (int b = 0; b < n_items; ++b) {
        const fr_batch_item &h = items[b];
        FR_CUDA(ctx, copy_async(ctx, p, h.d_X, h.M * sizeof(float4), cudaMemcpyHostToDevice));
        dev[b].d_X = (const float *)p;
        p += h.M;
        FR_CUDA(ctx, copy_async(ctx, p, h.d_Y, h.N * sizeof(float4), cudaMemcpyHostToDevice));
        dev[b].d_Y = (const float *)p;
        p += h.N;
        if (pt2pl) {
            FR_CUDA(ctx, copy_async(ctx, p, h.d_Yn, h.N * sizeof(float4), cudaMemcpyHostToDevice));
            dev[b].d_Yn = (const float *)p;
            p += h.N;
        } else {
            dev[b].d_Yn = nullptr;
        }
    }
    const fr_status st = run_batch_sized(ctx, dev.data(), n_items, opt, reports);
    for (int b = 0; b < n_items; ++b) {
        items[b].status = dev[b].status;
        for (int i = 0; i < 16; ++i) items[b].T[i] = dev[b].T[i];
    }
    return st;
}

}  // extern "C"
