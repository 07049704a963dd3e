// Host side of articulated registration (Section 5.1, Eq. 20, Algorithm 1).
//
// Per EM iteration one k_art_iter launch: step blocks slice the lattice at
// the posed model points and sum J^T J / J^T r per body; the last step block
// assembles and solves the normal equations in float64, updates the root
// pose and the joint angles and runs the kinematics of the new pose; when
// sigma is annealed, build blocks splat the next sigma's lattice and clear
// blocks free the table of two iterations back (three rotating tables, as in
// the rigid path).  The first build and the final clear are their own
// launches.
#include "context.h"

#include <algorithm>

using namespace fr;

namespace fr {

struct ArtWorkspace {
    ArtJob *d_job = nullptr;
    ArtState *d_state = nullptr;
    ArtJob *h_job = nullptr;
    ArtState *h_state = nullptr;
    bool annealed = false;  // of the registration last enqueued
};

void free_art_workspace(fr_ctx *ctx) {
    ArtWorkspace *w = ctx->art;
    if (!w) return;
    cudaFree(w->d_job);
    cudaFree(w->d_state);
    cudaFreeHost(w->h_job);
    cudaFreeHost(w->h_state);
    delete w;
    ctx->art = nullptr;
}

}  // namespace fr

namespace {

fr_status validate_tree(fr_ctx *ctx, const fr_kintree *t) {
    if (!t) return ctx->fail(FR_EINVAL, "kinematic tree is NULL");
    if (t->n_bodies < 1 || t->n_bodies > kMaxBodies)
        return ctx->fail(FR_EINVAL, "n_bodies must be 1..%d", kMaxBodies);
    if (t->n_joints < 0 || t->n_joints > kMaxJoints)
        return ctx->fail(FR_EINVAL, "n_joints must be 0..%d", kMaxJoints);
    if (!t->parent || !t->offset || (t->n_joints && (!t->joint_body || !t->joint_axis || !t->q_min || !t->q_max)))
        return ctx->fail(FR_EINVAL, "kinematic tree arrays must not be NULL");
    for (int b = 1; b < t->n_bodies; ++b)
        if (t->parent[b] < 0 || t->parent[b] >= b)
            return ctx->fail(FR_EINVAL, "parent[%d] must lie in [0, %d)", b, b);
    for (int j = 0; j < t->n_joints; ++j) {
        if (t->joint_body[j] < 0 || t->joint_body[j] >= t->n_bodies || (j && t->joint_body[j] < t->joint_body[j - 1]))
            return ctx->fail(FR_EINVAL, "joint_body must be non-decreasing body indices");
        const double *a = t->joint_axis + 3 * j;
        const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        if (!(n > 0.5 && n < 2.0)) return ctx->fail(FR_EINVAL, "joint_axis[%d] is not a unit vector", j);
        if (!(t->q_min[j] <= t->q_max[j])) return ctx->fail(FR_EINVAL, "q_min[%d] > q_max[%d]", j, j);
    }
    for (int k = 0; k < 16 * t->n_bodies; ++k)
        if (!std::isfinite(t->offset[k])) return ctx->fail(FR_EINVAL, "offset is not finite");
    return FR_OK;
}

void mul44(const double *a, const double *b, double *c) {
    double t[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += a[4 * i + k] * b[4 * k + j];
            t[4 * i + j] = s;
        }
    std::memcpy(c, t, sizeof t);
}

// Kinematics of the initial parameters (host, float64), giving the device
// state its first body poses and joint axes.
void host_fk(const ArtTree &t, const double *root_T, const double *q, ArtState &st,
             const double *offsets) {
    std::vector<double> T((size_t)t.nb * 16);
    for (int b = 0; b < t.nb; ++b) {
        double F[16];
        std::memcpy(F, b == 0 ? root_T : &T[16 * (size_t)t.parent[b]], sizeof F);
        mul44(F, offsets + 16 * b, F);
        for (int j = t.joint_begin[b]; j < t.joint_begin[b + 1]; ++j) {
            const double u[3] = {t.axis[j][0], t.axis[j][1], t.axis[j][2]};
            for (int r = 0; r < 3; ++r) {
                st.jaxis[j][r] = (float)(F[4 * r] * u[0] + F[4 * r + 1] * u[1] + F[4 * r + 2] * u[2]);
                st.jpoint[j][r] = (float)F[4 * r + 3];
            }
            const double c = std::cos(q[j]), s = std::sin(q[j]), v = 1.0 - c;
            const double R[16] = {c + u[0] * u[0] * v, u[0] * u[1] * v - u[2] * s, u[0] * u[2] * v + u[1] * s, 0,
                                  u[1] * u[0] * v + u[2] * s, c + u[1] * u[1] * v, u[1] * u[2] * v - u[0] * s, 0,
                                  u[2] * u[0] * v - u[1] * s, u[2] * u[1] * v + u[0] * s, c + u[2] * u[2] * v, 0,
                                  0, 0, 0, 1};
            mul44(F, R, F);
        }
        std::memcpy(&T[16 * (size_t)b], F, sizeof F);
        for (int k = 0; k < 12; ++k) st.body_T[b][k] = (float)F[k];
    }
}

// Everything of one registration on ctx's stream up to the final wait: the
// job, the launches and the copies of the result to the pinned mirrors.
// art_finish waits for them and hands the result out.
fr_status art_enqueue(fr_ctx *ctx, const float *d_Xref, const int32_t *d_body, int64_t M,
                      const fr_kintree *tree, const float *d_Y, const float *d_Yn, int64_t N,
                      const fr_options *opt, const double root_T[16], const double *q, bool safe) {
    const int pt2pl = opt->residual == FR_PT2PL;
    if (!ctx->art) ctx->art = new ArtWorkspace();
    ArtWorkspace *w = ctx->art;
    // each on its own test: a failed attempt may have made some of them
    if (!w->d_job) FR_CUDA(ctx, dev_alloc(&w->d_job, 1));
    if (!w->d_state) FR_CUDA(ctx, dev_alloc(&w->d_state, 1));
    if (!w->h_job) FR_CUDA(ctx, cudaMallocHost((void **)&w->h_job, sizeof(ArtJob)));
    if (!w->h_state) FR_CUDA(ctx, cudaMallocHost((void **)&w->h_state, sizeof(ArtState)));
    const uint32_t cap = table_slots(N, safe);
    FR_TRY(ensure_small(ctx, opt->iters, 1));
    FR_TRY(ensure_tables(ctx, cap, false, opt->storage != FR_FP32));
    Table tab[kMaxTables];
    for (int i = 0; i < kMaxTables; ++i) {
        tab[i] = ctx->tables[i];
        tab[i].mask = cap - 1;
        tab[i].max_probe = table_probe_limit(cap, safe);
    }
    const bool annealed = fill_iter_params(opt, M, N, ctx->h_ip);
    w->annealed = annealed;

    // ---- job and initial state ---------------------------------------------
    ArtJob &J = *w->h_job;
    J = ArtJob{};
    J.base.X = (const float4 *)d_Xref;
    J.base.Y = (const float4 *)d_Y;
    J.base.Yn = pt2pl ? (const float4 *)d_Yn : nullptr;
    J.base.M = (int)M;
    J.base.N = (int)N;
    J.base.renormalize = opt->renormalize_normals ? 1 : 0;
    J.base.stop_twist = opt->stop_twist;
    J.body = d_body;
    ArtTree &T = J.tree;
    T.nb = tree->n_bodies;
    T.nj = tree->n_joints;
    for (int b = 0; b < T.nb; ++b) {
        T.parent[b] = b == 0 ? -1 : tree->parent[b];
        for (int k = 0; k < 12; ++k) T.offset[b][k] = (float)tree->offset[16 * b + k];
    }
    for (int b = T.nb - 1; b >= 0; --b) {  // parent[b] < b: children are complete first
        T.sub[b] |= 1u << b;
        if (b > 0) T.sub[T.parent[b]] |= T.sub[b];
    }
    for (int b = 0, j = 0; b <= T.nb; ++b) {
        while (j < T.nj && tree->joint_body[j] < b) ++j;
        T.joint_begin[b] = (b == T.nb) ? T.nj : j;
    }
    for (int j = 0; j < T.nj; ++j) {
        T.joint_body[j] = tree->joint_body[j];
        const double *a = tree->joint_axis + 3 * j;
        const double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int r = 0; r < 3; ++r) T.axis[j][r] = (float)(a[r] / n);
        T.q_min[j] = tree->q_min[j];
        T.q_max[j] = tree->q_max[j];
    }
    ArtState &S = *w->h_state;
    S = ArtState{};
    for (int k = 0; k < 16; ++k) S.root_T[k] = root_T[k];
    for (int j = 0; j < T.nj; ++j) S.q[j] = std::min(std::max(q[j], T.q_min[j]), T.q_max[j]);
    host_fk(T, S.root_T, S.q, S, tree->offset);
    FR_CUDA(ctx, copy_async(ctx, w->d_job, w->h_job, sizeof(ArtJob), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, w->d_state, w->h_state, sizeof(ArtState), cudaMemcpyHostToDevice));
    if (opt->iters > 0)
        FR_CUDA(ctx, copy_async(ctx, ctx->d_ip, ctx->h_ip, opt->iters * sizeof(IterParams),
                                cudaMemcpyHostToDevice));

    // ---- launches ----------------------------------------------------------
    const int gs = blocks_for(ctx, M, 4), gb = blocks_for(ctx, N, 4);
    const int gc = annealed ? std::max(8, std::min(64, (int)(N / 4096) + 1)) : 0;
    // Builds run `lead` iterations ahead of their step: 2 with 16-bit storage,
    // whose records are converted in the launch after the build.
    const int lead = opt->storage != FR_FP32 ? 2 : 1;
    const int gv = lead == 2 ? blocks_for(ctx, cap, 1) : 0;
    auto tab_of = [&](int build) { return annealed ? build % (lead + 2) : 0; };
    auto builds = [&](int b) { return b < opt->iters && (annealed || b == 0); };
    for (int j = 0; j < lead && opt->iters > 0; ++j) {  // prologue: builds 0..lead-1, convert 0
        IterLaunch b0{};
        b0.job = &w->d_job->base;
        b0.ip = ctx->d_ip;
        b0.st = &w->d_state->ds;
        if (builds(j)) {
            b0.build = tab[tab_of(j)];
            b0.build_list = ctx->lists[tab_of(j)];
            b0.build_it = j;
            b0.gb = blocks_for(ctx, N, 8);
        }
        if (j >= 1) {
            b0.conv = tab[tab_of(j - 1)];
            b0.conv_list = ctx->lists[tab_of(j - 1)];
            b0.conv_it = j - 1;
            b0.gv = gv;
        }
        launch_em_iter(pt2pl, 0, b0, ctx->stream, opt->storage);
        ctx->launches += 1;
    }
    for (int it = 0; it < opt->iters; ++it) {
        ArtLaunch L{};
        L.job = w->d_job;
        L.ip = ctx->d_ip;
        L.st = w->d_state;
        L.it = it;
        L.step = tab[tab_of(it)];
        L.gs = gs;
        if (annealed && builds(it + lead)) {
            L.build = tab[tab_of(it + lead)];
            L.build_list = ctx->lists[tab_of(it + lead)];
            L.build_it = it + lead;
            L.gb = gb;
        }
        if (lead == 2 && annealed && builds(it + 1)) {
            L.conv = tab[tab_of(it + 1)];
            L.conv_list = ctx->lists[tab_of(it + 1)];
            L.conv_it = it + 1;
            L.gv = gv;
        }
        if (annealed && it >= 1) {
            L.clear = tab[tab_of(it - 1)];
            L.clear_list = ctx->lists[tab_of(it - 1)];
            L.clear_it = it - 1;
            L.gc = gc;
        }
        launch_art_iter(pt2pl, L, ctx->stream, opt->storage);
        ctx->launches += 1;
    }
    if (opt->iters > 0) {
        // the last build's table (the launch after each step cleared the others)
        const int last = annealed ? opt->iters - 1 : 0;
        Table t[1] = {tab[tab_of(last)]};
        int *lists[1] = {ctx->lists[tab_of(last)]};
        const int *counts[1] = {&ctx->d_ip[last].nvert};
        launch_clear_lists(t, lists, counts, 1, blocks_for(ctx, N, 2), ctx->stream);
        ctx->launches += 1;
    }
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, copy_async(ctx, w->h_state, w->d_state, sizeof(ArtState), cudaMemcpyDeviceToHost));
    if (opt->iters > 0)
        FR_CUDA(ctx, copy_async(ctx, ctx->h_ip, ctx->d_ip, opt->iters * sizeof(IterParams),
                                cudaMemcpyDeviceToHost));
    return FR_OK;
}

fr_status art_finish(fr_ctx *ctx, const fr_options *opt, double root_T[16], double *q, fr_report *rep) {
    ArtWorkspace *w = ctx->art;
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const ArtState &S = *w->h_state;
    const ArtTree &T = w->h_job->tree;
    const bool annealed = w->annealed;
    const DeviceState &ds = S.ds;
    FR_TRY(check_flags(ctx, ds.flags));
    for (int k = 0; k < 16; ++k) root_T[k] = S.root_T[k];
    for (int j = 0; j < T.nj; ++j) q[j] = S.q[j];
    if (rep) {
        rep->iters_run = ds.iters_run;
        rep->degenerate_iters = ds.degenerate;
        rep->last_inliers = ds.inliers;
        rep->last_sum_w = ds.sum_w;
        rep->last_cost = ds.cost;
        rep->last_twist_norm = ds.twist_norm;
        const int last_build = (annealed && ds.iters_run > 0) ? ds.iters_run - 1 : 0;
        rep->lattice_vertices = opt->iters > 0 ? ctx->h_ip[last_build].nvert : 0;
        rep->lattice_builds = ds.builds;
        rep->lattice_vertices_sum = ds.nvert_total;
    }
    return FR_OK;
}

fr_status run_articulated(fr_ctx *ctx, const float *d_Xref, const int32_t *d_body, int64_t M,
                          const fr_kintree *tree, const float *d_Y, const float *d_Yn, int64_t N,
                          const fr_options *opt, double root_T[16], double *q, fr_report *rep,
                          bool safe) {
    FR_TRY(art_enqueue(ctx, d_Xref, d_body, M, tree, d_Y, d_Yn, N, opt, root_T, q, safe));
    return art_finish(ctx, opt, root_T, q, rep);
}

fr_status validate_articulated(fr_ctx *ctx, const fr_options *opt, const fr_kintree *tree) {
    FR_TRY(validate_options(ctx, opt));
    if (opt->update_sigma) return ctx->fail(FR_ENOTSUPPORTED, "the sigma update is implemented for rigid registration");
    if (opt->blur || opt->kahan)
        return ctx->fail(FR_ENOTSUPPORTED, "articulated registration supports neither blur nor Kahan sums");
    return validate_tree(ctx, tree);
}

fr_status validate_articulated_clouds(fr_ctx *ctx, const fr_options *opt, const float *d_Xref,
                                      const int32_t *d_body, int64_t M, const float *d_Y, const float *d_Yn,
                                      int64_t N) {
    FR_TRY(validate_cloud(ctx, d_Xref, M, "d_Xref"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (!d_body) return ctx->fail(FR_EINVAL, "d_body is NULL");
    if (opt->residual == FR_PT2PL) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn (normals, required for FR_PT2PL)"));
    return FR_OK;
}

// A context of ctx's device with a non-blocking stream of its own, sharing
// ctx's launch-shape table and workspace limit.
fr_status make_sub(fr_ctx *ctx, fr_ctx **out) {
    fr_ctx *sub = new fr_ctx();
    sub->device = ctx->device;
    sub->num_sms = ctx->num_sms;
    sub->ws_limit = ctx->ws_limit;
    for (int c = 0; c < kTuneClasses; ++c) sub->tune[c] = ctx->tune[c];
    if (cudaStreamCreateWithFlags(&sub->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sub;
        return ctx->cuda(cudaGetLastError(), "stream of a concurrent registration");
    }
    sub->own_stream = true;
    *out = sub;
    return FR_OK;
}

}  // namespace

extern "C" FR_API fr_status fr_register_articulated(fr_ctx *ctx, const float *d_Xref,
                                                    const int32_t *d_body, int64_t M,
                                                    const fr_kintree *tree, const float *d_Y,
                                                    const float *d_Yn, int64_t N,
                                                    const fr_options *opt, double root_T_inout[16],
                                                    double *q_inout, fr_report *report) {
    fr::NvtxRange nvtx_("fr_register_articulated");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_articulated(ctx, opt, tree));
    FR_TRY(validate_articulated_clouds(ctx, opt, d_Xref, d_body, M, d_Y, d_Yn, N));
    if (!root_T_inout || (tree->n_joints && !q_inout)) return ctx->fail(FR_EINVAL, "pose outputs are NULL");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(root_T_inout[k])) return ctx->fail(FR_EINVAL, "root pose is not finite");
    cudaSetDevice(ctx->device);
    double R0[16];
    std::vector<double> q0(q_inout, q_inout + tree->n_joints);
    std::memcpy(R0, root_T_inout, sizeof R0);
    fr_status s = run_articulated(ctx, d_Xref, d_body, M, tree, d_Y, d_Yn, N, opt, root_T_inout,
                                  q_inout, report, false);
    if (s != FR_ECAPACITY) return s;
    std::memcpy(root_T_inout, R0, sizeof R0);
    std::copy(q0.begin(), q0.end(), q_inout);
    return run_articulated(ctx, d_Xref, d_body, M, tree, d_Y, d_Yn, N, opt, root_T_inout, q_inout,
                           report, true);
}

extern "C" FR_API fr_status fr_register_articulated_batch(fr_ctx *ctx, const fr_kintree *tree,
                                                          fr_articulated_item *items, int32_t n_items,
                                                          const fr_options *opt, fr_report *reports) {
    fr::NvtxRange nvtx_("fr_register_articulated_batch");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_articulated(ctx, opt, tree));
    if (!items || n_items < 1 || n_items > FR_ART_BATCH_MAX)
        return ctx->fail(FR_EINVAL, "need 1..%d items", FR_ART_BATCH_MAX);
    for (int b = 0; b < n_items; ++b) {
        const fr_articulated_item &it = items[b];
        FR_TRY(validate_articulated_clouds(ctx, opt, it.d_Xref, it.d_body, it.M, it.d_Y, it.d_Yn, it.N));
        if (tree->n_joints && !it.q) return ctx->fail(FR_EINVAL, "item %d: q is NULL", b);
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(it.root_T[k])) return ctx->fail(FR_EINVAL, "item %d: root pose is not finite", b);
    }
    cudaSetDevice(ctx->device);
    while ((int)ctx->subs.size() < std::min<int>(n_items, FR_ART_CONCURRENT)) {
        fr_ctx *sub = nullptr;
        FR_TRY(make_sub(ctx, &sub));
        ctx->subs.push_back(sub);
    }
    for (fr_ctx *sub : ctx->subs) {  // the context's current shapes and limit
        sub->ws_limit = ctx->ws_limit;
        for (int c = 0; c < kTuneClasses; ++c) sub->tune[c] = ctx->tune[c];
    }
    // the items' clouds were written in ctx's stream order: every item's
    // stream starts after what ctx's stream holds now
    cudaEvent_t ready;
    FR_CUDA(ctx, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ready, ctx->stream);
    fr_status first = FR_OK;
    const int nj = tree->n_joints;
    for (int w0 = 0; w0 < n_items && e == cudaSuccess; w0 += FR_ART_CONCURRENT) {
        const int w1 = std::min(n_items, w0 + FR_ART_CONCURRENT);
        std::vector<fr_status> st(w1 - w0, FR_OK);
        std::vector<int64_t> l0(w1 - w0), h0(w1 - w0), d0(w1 - w0);
        for (int b = w0; b < w1; ++b) {
            fr_ctx *sub = ctx->subs[b - w0];
            l0[b - w0] = sub->launches;
            h0[b - w0] = sub->h2d_bytes;
            d0[b - w0] = sub->d2h_bytes;
            if (cudaStreamWaitEvent(sub->stream, ready, 0) != cudaSuccess) {
                st[b - w0] = sub->cuda(cudaGetLastError(), "stream wait");
                continue;
            }
            const fr_articulated_item &it = items[b];
            st[b - w0] = art_enqueue(sub, it.d_Xref, it.d_body, it.M, tree, it.d_Y, it.d_Yn, it.N, opt,
                                     it.root_T, it.q, false);
        }
        for (int b = w0; b < w1; ++b) {
            fr_ctx *sub = ctx->subs[b - w0];
            fr_articulated_item &it = items[b];
            fr_report *rep = reports ? reports + b : nullptr;
            double R0[16];
            std::vector<double> q0(it.q, it.q + nj);
            std::memcpy(R0, it.root_T, sizeof R0);
            fr_status s = st[b - w0];
            if (s == FR_OK) s = art_finish(sub, opt, it.root_T, it.q, rep);
            if (s == FR_ECAPACITY) {  // this item alone again, at the safe table size
                std::memcpy(it.root_T, R0, sizeof R0);
                std::copy(q0.begin(), q0.end(), it.q);
                s = run_articulated(sub, it.d_Xref, it.d_body, it.M, tree, it.d_Y, it.d_Yn, it.N, opt,
                                    it.root_T, it.q, rep, true);
            }
            if (s != FR_OK) {
                cudaStreamSynchronize(sub->stream);
                std::memcpy(it.root_T, R0, sizeof R0);
                std::copy(q0.begin(), q0.end(), it.q);
                if (first == FR_OK) {
                    first = s;
                    ctx->err = "item " + std::to_string(b) + ": " + sub->err;
                }
            }
            it.status = s;
            ctx->launches += sub->launches - l0[b - w0];
            ctx->h2d_bytes += sub->h2d_bytes - h0[b - w0];
            ctx->d2h_bytes += sub->d2h_bytes - d0[b - w0];
        }
    }
    cudaEventDestroy(ready);
    if (e != cudaSuccess) {
        for (int b = 0; b < n_items; ++b) items[b].status = FR_ECUDA;
        return ctx->cuda(e, "event record");
    }
    return first;
}
