// Serving: continuous batching of independent rigid registrations.
//
// A worker thread launches one k_em_multi per tick over every live request,
// each at its own stage.  With float32 storage (lead L = 1): stage 0 builds
// its first lattice; stage 1 + k runs EM iteration k (step k, build k+1 and
// clear k-1 when sigma is annealed, Section 3.2).  With 16-bit storage
// (L = 2) a build's records are converted in the tick after it: stages 0 and
// 1 build 0 and 1 (and convert 0), stage 2 + k runs step k, converts k+1,
// builds k+2 and clears k-1.  The stage after the last iteration clears the
// remaining table.  The result is read back after the tick of the last iteration and
// the memory is reclaimed after the clearing tick.  Requests are admitted
// between ticks, first come first served, when their tables and records fit
// the server's arenas:
//   - a table arena of hash-slot records that every request
//     leaves empty again, so admission needs no clearing;
//   - a byte arena for each request's descriptors, reduction partials, slot
//     lists and (host requests) its copied clouds.
// Both are managed by buddy allocators on the host.  The paper registers one
// pair at a time; this loop is a systems addition around its EM.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>

#include "context.h"

using namespace fr;

namespace {

int64_t steady_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

constexpr int kMaxAhead = 2;         // ticks queued on the GPU before the worker waits
// Points per thread of a request's step and build blocks come from the
// context's tuning table (serve_points_per_thread, default 2): a serving tick
// is rarely a full GPU, so its duration is the longest per-thread chain, and
// short chains (more, smaller blocks) keep the latency down.
constexpr size_t kByteUnit = 256;    // byte-arena granularity
constexpr int kMinTableOrder = 10;   // smallest table: 1024 slots

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }
int order_of(size_t units) {
    int o = 0;
    while (((size_t)1 << o) < units) ++o;
    return o;
}

// Power-of-two buddy allocator over [0, 2^top) units.
struct Buddy {
    int top = -1;
    std::vector<std::set<size_t>> free_;
    void init(int top_order) {
        top = top_order;
        free_.assign(top + 1, {});
        free_[top].insert(0);
    }
    bool alloc(int order, size_t &off) {
        int o = order;
        while (o <= top && free_[o].empty()) ++o;
        if (o > top) return false;
        off = *free_[o].begin();
        free_[o].erase(free_[o].begin());
        while (o > order) {
            --o;
            free_[o].insert(off + ((size_t)1 << o));
        }
        return true;
    }
    void release(size_t off, int order) {
        while (order < top) {
            const size_t buddy = off ^ ((size_t)1 << order);
            auto it = free_[order].find(buddy);
            if (it == free_[order].end()) break;
            free_[order].erase(it);
            off = std::min(off, buddy);
            ++order;
        }
        free_[order].insert(off);
    }
};

enum class RState { Queued, Live, Done };

struct Request {
    uint64_t ticket = 0;
    fr_request req{};
    RState state = RState::Queued;
    bool safe = false;       // table sized so that it cannot overflow (after an overflow)
    int annealed = 0, ntab = 1;
    uint32_t cap = 0;
    int gs = 0, gp = 0, gb = 0, gc = 0, gf = 0, gv = 0;
    int slot = -1, stage = 0;
    size_t tab_off[kMaxTables] = {0, 0, 0, 0};
    size_t byte_off = 0;
    int byte_order = -1;
    size_t byte_need = 0;
    size_t o_job = 0, o_state = 0, o_ip = 0, o_part = 0, o_list = 0, o_X = 0, o_Y = 0, o_Yn = 0;
    fr_result res{};
    bool released = false;   // the client forgot the ticket: delete once retired
    bool retired = false;    // memory back in the arenas (or never taken)
};

struct Tick {
    cudaEvent_t ev;
    std::vector<Request *> results;  // last iteration ran in this tick: read the result
    std::vector<Request *> retire;   // tables cleared in this tick: free the memory
};

// Per-slot pinned staging: upload [job | state | ip[iters]] and the Slot
// record; download [state | ip[iters]].
struct SlotStage {
    unsigned char *up = nullptr;
    unsigned char *down = nullptr;
};

}  // namespace

struct fr_server {
    fr_ctx *ctx = nullptr;
    fr_options opt{};
    int pt2pl = 0, kahan = 0, iters1 = 1;
    int lead = 1;  // builds run this many ticks ahead of their step (2 with 16-bit storage)
    int max_live = 0;
    cudaStream_t stream = nullptr;

    // arenas
    unsigned long long *keys = nullptr;  // slot records, all free (zero) between requests
    size_t table_slots_total = 0;
    unsigned char *bytes = nullptr;
    size_t bytes_total = 0;
    Buddy tab_buddy, byte_buddy;

    // descriptors
    Slot *d_slots = nullptr;
    Seg *d_segs = nullptr;
    unsigned short *d_map = nullptr;
    size_t map_cap = 0;
    unsigned char *h_tick[2] = {nullptr, nullptr};  // pinned [segs | map] per tick parity
    size_t h_tick_cap = 0;
    size_t stage_up = 0, stage_down = 0;
    std::vector<SlotStage> stages;
    unsigned char *h_stage_block = nullptr;
    std::vector<int> free_slots;
    std::vector<cudaEvent_t> event_pool;

    // requests
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::vector<Request *> live;
    std::deque<Tick> inflight;
    std::unordered_map<uint64_t, Request *> table;
    uint64_t next_ticket = 1;
    bool stop = false;
    fr_status failed = FR_OK;
    std::string failed_msg;
    std::thread worker;
    std::atomic<int64_t> ticks{0}, completed{0}, launches{0};
    uint64_t tick_parity = 0;

    // ---- sizing --------------------------------------------------------------
    void plan(Request &r) const {
        const fr_request &q = r.req;
        r.annealed = (q.sigma_start != q.sigma_end && opt.iters > 1) ? 1 : 0;
        r.ntab = r.annealed ? lead + 2 : 1;
        const fr_tune_params &tp = ctx->tune[tune_class(q.N)];
        r.cap = r.safe ? table_slots(q.N, true) : tuned_table_slots(q.N, tp.table_slots_x2);
        r.gs = div_up(q.M, (long long)kBlock * tp.serve_points_per_thread);
        r.gp = div_up(q.N, (long long)kBlock * tp.serve_points_per_thread);
        r.gb = r.annealed ? r.gp : 0;
        r.gc = r.annealed ? std::max(1, div_up(q.N, 4096)) : 0;
        r.gf = std::max(1, div_up(q.N, 4096));
        r.gv = lead == 2 ? std::max(1, div_up(q.N, 2048)) : 0;
        size_t off = 0;
        r.o_job = off; off = align256(off + sizeof(RigidJob));
        r.o_state = off; off = align256(off + sizeof(DeviceState));
        r.o_ip = off; off = align256(off + (size_t)iters1 * sizeof(IterParams));
        r.o_part = off; off = align256(off + (size_t)r.gs * kRigidVals * sizeof(float2));
        r.o_list = off; off = align256(off + (size_t)r.ntab * r.cap * sizeof(int));
        if (q.host) {
            r.o_X = off; off = align256(off + (size_t)q.M * sizeof(float4));
            r.o_Y = off; off = align256(off + (size_t)q.N * sizeof(float4));
            if (pt2pl) { r.o_Yn = off; off = align256(off + (size_t)q.N * sizeof(float4)); }
        }
        r.byte_need = off;
    }
    bool fits_alone(const Request &r) const {
        return order_of((r.byte_need + kByteUnit - 1) / kByteUnit) <= byte_buddy.top &&
               order_of(r.cap) <= tab_buddy.top && (size_t)r.ntab * r.cap <= table_slots_total;
    }

    // ---- admission (lock held) -----------------------------------------------
    bool try_admit(Request &r) {
        if (free_slots.empty()) return false;
        const int bo = order_of((r.byte_need + kByteUnit - 1) / kByteUnit);
        size_t boff;
        if (!byte_buddy.alloc(bo, boff)) return false;
        const int to = order_of(r.cap);
        int got = 0;
        for (; got < r.ntab; ++got)
            if (!tab_buddy.alloc(to, r.tab_off[got])) break;
        if (got < r.ntab) {
            for (int t = 0; t < got; ++t) tab_buddy.release(r.tab_off[t], to);
            byte_buddy.release(boff, bo);
            return false;
        }
        r.byte_off = boff * kByteUnit;
        r.byte_order = bo;
        r.slot = free_slots.back();
        free_slots.pop_back();
        r.retired = false;
        r.stage = 0;
        r.state = RState::Live;
        r.res.admit_ns = steady_ns();
        upload(r);
        return true;
    }
    void release_memory(Request &r) {
        const int to = order_of(r.cap);
        for (int t = 0; t < r.ntab; ++t) tab_buddy.release(r.tab_off[t], to);
        byte_buddy.release(r.byte_off / kByteUnit, r.byte_order);
        free_slots.push_back(r.slot);
        r.slot = -1;
        r.byte_order = -1;
        r.retired = true;
    }
    // Descriptors of a newly admitted request, and its copied clouds.
    void upload(Request &r) {
        const fr_request &q = r.req;
        unsigned char *D = bytes + r.byte_off;
        const SlotStage &sg = stages[r.slot];
        RigidJob *j = (RigidJob *)sg.up;
        *j = RigidJob{};
        j->X = (const float4 *)(q.host ? D + r.o_X : (const unsigned char *)q.X);
        j->Y = (const float4 *)(q.host ? D + r.o_Y : (const unsigned char *)q.Y);
        j->Yn = pt2pl ? (const float4 *)(q.host ? D + r.o_Yn : (const unsigned char *)q.Yn) : nullptr;
        j->M = (int)q.M;
        j->N = (int)q.N;
        j->renormalize = opt.renormalize_normals ? 1 : 0;
        j->stop_twist = opt.stop_twist;
        for (int i = 0; i < 16; ++i) j->T0[i] = q.T[i];
        DeviceState *s = (DeviceState *)(sg.up + align256(sizeof(RigidJob)));
        *s = DeviceState{};
        for (int i = 0; i < 16; ++i) s->T[i] = q.T[i];
        IterParams *ip = (IterParams *)(sg.up + align256(sizeof(RigidJob)) + align256(sizeof(DeviceState)));
        fr_options o = opt;
        o.sigma_start = q.sigma_start;
        o.sigma_end = q.sigma_end;
        o.w = q.w;
        fill_iter_params(&o, q.M, q.N, ip);
        Slot *sl = (Slot *)(sg.up + stage_up - align256(sizeof(Slot)));
        *sl = Slot{};
        sl->job = (const RigidJob *)(D + r.o_job);
        sl->st = (DeviceState *)(D + r.o_state);
        sl->ip = (IterParams *)(D + r.o_ip);
        sl->partials = (float2 *)(D + r.o_part);
        for (int t = 0; t < r.ntab; ++t) {
            const size_t b = r.tab_off[t];  // table arena offsets are in slots
            sl->tab[t] = Table{keys + b * kRecWords, r.cap - 1, table_probe_limit(r.cap, r.safe),
                               pt2pl ? 8 : 4};
            sl->list[t] = (int *)(D + r.o_list) + (size_t)t * r.cap;
        }
        // job, state and iteration parameters sit at the same offsets in the byte block
        const size_t head = align256(sizeof(RigidJob)) + align256(sizeof(DeviceState)) +
                            (size_t)iters1 * sizeof(IterParams);
        cudaMemcpyAsync(D + r.o_job, sg.up, head, cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(d_slots + r.slot, sl, sizeof(Slot), cudaMemcpyHostToDevice, stream);
        if (q.host) {
            cudaMemcpyAsync(D + r.o_X, q.X, (size_t)q.M * sizeof(float4), cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(D + r.o_Y, q.Y, (size_t)q.N * sizeof(float4), cudaMemcpyHostToDevice, stream);
            if (pt2pl)
                cudaMemcpyAsync(D + r.o_Yn, q.Yn, (size_t)q.N * sizeof(float4), cudaMemcpyHostToDevice, stream);
        }
    }

    // ---- one tick (lock held) ------------------------------------------------
    int tab_of(const Request &r, int build) const { return r.annealed ? build % r.ntab : 0; }

    fr_status launch_tick() {
        NvtxRange nvtx_("fr_server_tick");
        std::vector<Seg> segs;
        segs.reserve(live.size() * 3);
        int blk = 0;
        Tick tk{};
        auto add = [&](const Request &r, int role, int it, int tab, int n) {
            if (n <= 0) return;
            segs.push_back(Seg{r.slot, role, it, tab, blk, n});
            blk += n;
        };
        const int last_it = opt.iters - 1;
        for (Request *rp : live) {
            Request &r = *rp;
            if (r.stage < lead) {
                // prologue: build j (fixed sigma builds only 0), convert j - 1
                const int j = r.stage;
                if (j == 0 || (r.annealed && j < opt.iters)) add(r, kRoleBuild, j, tab_of(r, j), r.gp);
                if (j >= 1) add(r, kRoleConvert, j - 1, tab_of(r, j - 1), r.gv);
            } else if (r.stage < lead + opt.iters) {
                const int k = r.stage - lead;
                add(r, kRoleStep, k, tab_of(r, k), r.gs);
                if (r.annealed && k + lead < opt.iters) add(r, kRoleBuild, k + lead, tab_of(r, k + lead), r.gb);
                if (r.annealed && lead == 2 && k + 1 < opt.iters) add(r, kRoleConvert, k + 1, tab_of(r, k + 1), r.gv);
                if (r.annealed && k >= 1) add(r, kRoleClear, k - 1, tab_of(r, k - 1), r.gc);
                if (k == last_it) tk.results.push_back(rp);
            } else {
                // the last build's table; every other one was cleared by the
                // tick after its step (clears run even after a stop)
                const int last = r.annealed ? last_it : 0;
                add(r, kRoleClear, last, tab_of(r, last), r.gf);
                tk.retire.push_back(rp);
            }
            ++r.stage;
        }
        const int grid = blk;
        // upload [segs | block -> segment map] through this tick's pinned buffer
        const size_t seg_bytes = align256(segs.size() * sizeof(Seg));
        const size_t need = seg_bytes + (size_t)grid * sizeof(unsigned short);
        if (need > h_tick_cap || segs.size() > map_cap || (size_t)grid > map_cap) {
            cudaStreamSynchronize(stream);
            cudaFreeHost(h_tick[0]);
            cudaFreeHost(h_tick[1]);
            cudaFree(d_segs);
            cudaFree(d_map);
            h_tick[0] = h_tick[1] = nullptr;
            d_segs = nullptr;
            d_map = nullptr;
            const size_t cap = std::max(need * 2, (size_t)1 << 16);
            map_cap = cap / sizeof(unsigned short);
            if (cudaMallocHost((void **)&h_tick[0], cap) != cudaSuccess ||
                cudaMallocHost((void **)&h_tick[1], cap) != cudaSuccess ||
                fr::dev_malloc((void **)&d_segs, map_cap * sizeof(Seg)) != cudaSuccess ||
                fr::dev_malloc((void **)&d_map, cap) != cudaSuccess) {
                map_cap = 0;
                h_tick_cap = 0;
                return FR_ENOMEM;
            }
            h_tick_cap = cap;
        }
        unsigned char *H = h_tick[tick_parity & 1];
        std::memcpy(H, segs.data(), segs.size() * sizeof(Seg));
        unsigned short *map = (unsigned short *)(H + seg_bytes);
        for (size_t si = 0; si < segs.size(); ++si)
            for (int q = 0; q < segs[si].nblk; ++q) map[segs[si].blk0 + q] = (unsigned short)si;
        cudaMemcpyAsync(d_segs, H, segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, stream);
        cudaMemcpyAsync(d_map, map, (size_t)grid * sizeof(unsigned short), cudaMemcpyHostToDevice, stream);
        launch_em_multi(pt2pl, kahan, d_slots, d_segs, d_map, grid, 1, stream, opt.storage);
        launches.fetch_add(1);
        for (Request *rp : tk.results) {
            unsigned char *D = bytes + rp->byte_off;
            const SlotStage &sg = stages[rp->slot];
            cudaMemcpyAsync(sg.down, D + rp->o_state, sizeof(DeviceState), cudaMemcpyDeviceToHost, stream);
            cudaMemcpyAsync(sg.down + align256(sizeof(DeviceState)), D + rp->o_ip,
                            (size_t)iters1 * sizeof(IterParams), cudaMemcpyDeviceToHost, stream);
        }
        if (event_pool.empty()) {
            cudaEvent_t e;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return FR_ECUDA;
            event_pool.push_back(e);
        }
        tk.ev = event_pool.back();
        event_pool.pop_back();
        cudaEventRecord(tk.ev, stream);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            failed_msg = cudaGetErrorString(e);
            return FR_ECUDA;
        }
        ++tick_parity;
        ticks.fetch_add(1);
        inflight.push_back(std::move(tk));
        // requests whose tables are being cleared leave the live set now
        live.erase(std::remove_if(live.begin(), live.end(),
                                  [&](Request *r) { return r->stage > opt.iters + lead; }),
                   live.end());
        return FR_OK;
    }

    // A tick has completed on the GPU (lock held).
    void finish_tick(Tick &tk) {
        const int64_t now = steady_ns();
        for (Request *rp : tk.results) {
            Request &r = *rp;
            const SlotStage &sg = stages[r.slot];
            const DeviceState &s = *(const DeviceState *)sg.down;
            const IterParams *ip = (const IterParams *)(sg.down + align256(sizeof(DeviceState)));
            if ((s.flags & kFlagCapacity) && !r.safe) {
                r.res.status = FR_ECAPACITY;  // rerun at the size that cannot overflow (below)
                continue;
            }
            r.res.status = (s.flags & kFlagRange) ? FR_EINVAL : (s.flags & kFlagCapacity) ? FR_ECAPACITY : FR_OK;
            for (int i = 0; i < 16; ++i) r.res.T[i] = r.res.status == FR_OK ? s.T[i] : r.req.T[i];
            fr_report &rep = r.res.report;
            rep.iters_run = s.iters_run;
            rep.degenerate_iters = s.degenerate;
            rep.last_inliers = s.inliers;
            rep.last_sum_w = s.sum_w;
            rep.last_cost = s.cost;
            rep.last_twist_norm = s.twist_norm;
            const int last_build = (r.annealed && s.iters_run > 0) ? s.iters_run - 1 : 0;
            rep.lattice_vertices = ip[last_build].nvert;
            rep.lattice_builds = s.builds;
            rep.lattice_vertices_sum = s.nvert_total;
            r.res.complete_ns = now;
            r.state = RState::Done;
            completed.fetch_add(1);
        }
        for (Request *rp : tk.retire) {
            Request &r = *rp;
            release_memory(r);
            if (r.released) {  // result already taken and the ticket forgotten
                delete rp;
                continue;
            }
            if (r.res.status == FR_ECAPACITY && !r.safe && r.state != RState::Done) {
                // the compact table overflowed: rerun from the initial pose at the safe size
                r.safe = true;
                plan(r);
                if (fits_alone(r)) {
                    r.res.status = FR_OK;
                    r.state = RState::Queued;
                    pending.push_front(rp);
                } else {
                    for (int i = 0; i < 16; ++i) r.res.T[i] = r.req.T[i];
                    r.res.complete_ns = steady_ns();
                    r.state = RState::Done;
                    completed.fetch_add(1);
                    cv_done.notify_all();
                }
            }
        }
        event_pool.push_back(tk.ev);
        if (!tk.results.empty()) cv_done.notify_all();
    }

    // A CUDA error: the server stops serving.  Every unfinished request
    // completes with the error; memory is not reused again.
    void fail_all(fr_status st) {
        failed = st;
        cudaStreamSynchronize(stream);
        cudaGetLastError();
        std::set<Request *> all(pending.begin(), pending.end());
        all.insert(live.begin(), live.end());
        for (Tick &t : inflight) {
            all.insert(t.results.begin(), t.results.end());
            all.insert(t.retire.begin(), t.retire.end());
            event_pool.push_back(t.ev);
        }
        inflight.clear();
        pending.clear();
        live.clear();
        for (Request *r : all) {
            if (r->state != RState::Done) {
                r->res.status = st;
                for (int i = 0; i < 16; ++i) r->res.T[i] = r->req.T[i];
                r->res.complete_ns = steady_ns();
                r->state = RState::Done;
            }
            r->retired = true;
            if (r->released) delete r;
        }
        cv_done.notify_all();
    }

    void run() {
        cudaSetDevice(ctx->device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            // completed ticks, waiting for the oldest when too many are queued
            while (!inflight.empty()) {
                cudaEvent_t ev = inflight.front().ev;
                cudaError_t q;
                if (inflight.size() >= (size_t)kMaxAhead) {
                    lk.unlock();
                    q = cudaEventSynchronize(ev);
                    lk.lock();
                } else {
                    q = cudaEventQuery(ev);
                    if (q == cudaErrorNotReady) break;
                }
                if (q != cudaSuccess) {
                    failed_msg = cudaGetErrorString(q);
                    fail_all(FR_ECUDA);
                    break;
                }
                finish_tick(inflight.front());
                inflight.pop_front();
            }
            if (failed == FR_OK)
                while (!pending.empty() && try_admit(*pending.front())) {
                    live.push_back(pending.front());
                    pending.pop_front();
                }
            if (live.empty() || failed != FR_OK) {
                if (!inflight.empty()) {
                    cudaEvent_t ev = inflight.front().ev;
                    lk.unlock();
                    cudaEventSynchronize(ev);
                    lk.lock();
                    continue;
                }
                if (stop && (pending.empty() || failed != FR_OK)) break;
                cv_work.wait(lk, [&] { return stop || (!pending.empty() && failed == FR_OK); });
                continue;
            }
            const fr_status st = launch_tick();
            if (st != FR_OK) fail_all(st);
        }
    }
};

namespace {

fr_status validate_request(fr_server *s, const fr_request *q) {
    fr_ctx *ctx = s->ctx;
    if (!q) return ctx->fail(FR_EINVAL, "request is NULL");
    if (!q->X || !q->Y || q->M < 1 || q->N < 1 || q->M > (1ll << 30) || q->N > (1ll << 30))
        return ctx->fail(FR_EINVAL, "request clouds must be non-NULL, 1 <= size <= 2^30");
    if (s->pt2pl && !q->Yn) return ctx->fail(FR_EINVAL, "point-to-plane request without normals");
    if (!aligned16(q->X) || !aligned16(q->Y) || (s->pt2pl && !aligned16(q->Yn)))
        return ctx->fail(FR_EINVAL, "request clouds must be 16-byte aligned");
    if (!(q->sigma_start > 0.0f) || !(q->sigma_end > 0.0f) || !std::isfinite(q->sigma_start) ||
        !std::isfinite(q->sigma_end))
        return ctx->fail(FR_EINVAL, "request sigmas must be finite and > 0");
    if (!(q->w >= 0.0f && q->w < 1.0f)) return ctx->fail(FR_EINVAL, "request w must be in [0, 1)");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(q->T[i])) return ctx->fail(FR_EINVAL, "request pose is not finite");
    return FR_OK;
}

}  // namespace

FR_API fr_status fr_server_create(fr_ctx *ctx, size_t budget, int max_live, const fr_options *opt,
                                  fr_server **out) {
    if (!ctx || !out) return FR_EINVAL;
    *out = nullptr;
    FR_TRY(validate_options(ctx, opt));
    if (opt->update_sigma) return ctx->fail(FR_ENOTSUPPORTED, "the sigma update is implemented for rigid registration");
    if (opt->blur) return ctx->fail(FR_ENOTSUPPORTED, "the server runs without blur");
    if (opt->iters < 1) return ctx->fail(FR_EINVAL, "the server needs iters >= 1");
    if (max_live < 1 || max_live > 4096) return ctx->fail(FR_EINVAL, "max_live must be in 1..4096");
    if (budget < ((size_t)1 << 24)) return ctx->fail(FR_EINVAL, "device_mem_budget must be >= 16 MiB");
    cudaSetDevice(ctx->device);
    fr_server *s = new fr_server();
    s->ctx = ctx;
    s->opt = *opt;
    s->pt2pl = opt->residual == FR_PT2PL;
    s->kahan = opt->kahan ? 1 : 0;
    s->iters1 = opt->iters > 0 ? opt->iters : 1;
    s->lead = opt->storage != FR_FP32 ? 2 : 1;
    s->max_live = max_live;
    auto bail = [&](fr_status st, const char *what) {
        fr_server_destroy(s);
        return ctx->fail(st, "fr_server_create: %s", what);
    };
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(FR_ECUDA, "stream");
    // table arena: the largest power of two of slots within half the budget
    const size_t per_slot = table_bytes(1);
    int top = kMinTableOrder;
    while (((size_t)2 << top) * per_slot <= budget / 2 && top < 31) ++top;
    s->table_slots_total = (size_t)1 << top;
    s->tab_buddy.init(top);
    const size_t S = s->table_slots_total;
    if (fr::dev_malloc((void **)&s->keys, table_bytes(S)) != cudaSuccess)
        return bail(FR_ENOMEM, "table arena");
    cudaMemsetAsync(s->keys, 0, table_bytes(S), s->stream);
    // byte arena
    int btop = 0;
    while (((size_t)2 << btop) * kByteUnit <= budget - S * per_slot && btop < 40) ++btop;
    s->bytes_total = ((size_t)1 << btop) * kByteUnit;
    s->byte_buddy.init(btop);
    if (fr::dev_malloc((void **)&s->bytes, s->bytes_total) != cudaSuccess) return bail(FR_ENOMEM, "byte arena");
    if (fr::dev_malloc((void **)&s->d_slots, (size_t)max_live * sizeof(Slot)) != cudaSuccess)
        return bail(FR_ENOMEM, "slot table");
    // pinned per-slot staging
    s->stage_up = align256(sizeof(RigidJob)) + align256(sizeof(DeviceState)) +
                  align256((size_t)s->iters1 * sizeof(IterParams)) + align256(sizeof(Slot));
    s->stage_down = align256(sizeof(DeviceState)) + align256((size_t)s->iters1 * sizeof(IterParams));
    if (cudaMallocHost((void **)&s->h_stage_block, (size_t)max_live * (s->stage_up + s->stage_down)) != cudaSuccess)
        return bail(FR_ENOMEM, "pinned staging");
    s->stages.resize(max_live);
    for (int i = 0; i < max_live; ++i) {
        s->stages[i].up = s->h_stage_block + (size_t)i * (s->stage_up + s->stage_down);
        s->stages[i].down = s->stages[i].up + s->stage_up;
    }
    for (int i = max_live - 1; i >= 0; --i) s->free_slots.push_back(i);
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bail(FR_ECUDA, "arena clearing");
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FR_OK;
}

FR_API fr_status fr_server_submit(fr_server *s, const fr_request *q, uint64_t *ticket) {
    if (!s || !ticket) return FR_EINVAL;
    FR_TRY(validate_request(s, q));
    Request *r = new Request();
    r->req = *q;
    r->res.submit_ns = steady_ns();
    s->plan(*r);
    if (!s->fits_alone(*r)) {
        delete r;
        return s->ctx->fail(FR_ENOMEM, "request (M %lld, N %lld) exceeds the server's memory budget",
                            (long long)q->M, (long long)q->N);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return s->ctx->fail(FR_EINVAL, "server is stopping");
        }
        if (s->failed != FR_OK) {
            delete r;
            return s->ctx->fail(s->failed, "server failed: %s", s->failed_msg.c_str());
        }
        r->ticket = s->next_ticket++;
        s->table[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return FR_OK;
}

FR_API fr_status fr_server_poll(fr_server *s, uint64_t ticket, int *done, fr_result *out) {
    if (!s || !done) return FR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return s->ctx->fail(FR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->state == RState::Done ? 1 : 0;
    if (*done && out) *out = it->second->res;
    return FR_OK;
}

FR_API fr_status fr_server_wait(fr_server *s, uint64_t ticket, int64_t timeout_ms, fr_result *out) {
    if (!s) return FR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return s->ctx->fail(FR_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    Request *r = it->second;
    auto ready = [&] { return r->state == RState::Done; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return FR_ETIMEOUT;
    if (out) *out = r->res;
    return FR_OK;
}

FR_API fr_status fr_server_release(fr_server *s, uint64_t ticket) {
    if (!s) return FR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end() || it->second->state != RState::Done)
        return s->ctx->fail(FR_EINVAL, "ticket %llu is unknown or not complete", (unsigned long long)ticket);
    Request *r = it->second;
    s->table.erase(it);
    if (r->retired)
        delete r;
    else
        r->released = true;  // still clearing its tables: the worker deletes it when retired
    return FR_OK;
}

FR_API fr_status fr_server_stats(const fr_server *s, int64_t *ticks, int64_t *completed, int64_t *launches) {
    if (!s) return FR_EINVAL;
    if (ticks) *ticks = s->ticks.load();
    if (completed) *completed = s->completed.load();
    if (launches) *launches = s->launches.load();
    return FR_OK;
}

FR_API fr_status fr_server_destroy(fr_server *s) {
    if (!s) return FR_EINVAL;
    if (s->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->stop = true;
        }
        s->cv_work.notify_all();
        s->worker.join();
    }
    if (s->stream) cudaStreamSynchronize(s->stream);
    for (auto &kv : s->table) delete kv.second;
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    cudaFree(s->keys);
    cudaFree(s->bytes);
    cudaFree(s->d_slots);
    cudaFree(s->d_segs);
    cudaFree(s->d_map);
    cudaFreeHost(s->h_tick[0]);
    cudaFreeHost(s->h_tick[1]);
    cudaFreeHost(s->h_stage_block);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return FR_OK;
}
