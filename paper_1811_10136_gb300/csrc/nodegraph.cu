// Node-graph deformable registration (Section 5.2, Eq. 21): model handle,
// EM driver and the checking entry points.
//
// fr_nodegraph_create sorts the model points by their (ascending) 4-node
// tuple, so that runs of points -- segments -- share their nodes; it lists
// the node-pair blocks of A that any segment or regulariser edge touches
// (a <= b, 6 x 6 each), the block of every tuple pair of every segment, the
// blocks of every edge, and a block-row index (each block once per row it
// appears in, transposed for the lower triangle) for the PCG products.
//
// One EM iteration on the device: the point kernel (warp, slice, rigid
// terms, pair-block sums), the edge kernel (regulariser), block-Jacobi PCG
// (set-up, then per iteration a product kernel and an update kernel), and
// the node update T_k <- exp(dzeta_k^) T_k.  The lattice is built once per
// sigma (rebuilt when the schedule changes it).
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <vector>

#include "context.h"

using namespace fr;

namespace {
struct NgGraph {
    long long key[10];
    cudaGraphExec_t exec;
    int kernels;
};
}  // namespace

struct fr_nodegraph {
    fr_ctx *ctx = nullptr;   // the creating context (not used by fr_nodegraph_destroy)
    int device = 0;
    int64_t M = 0;
    int K = 0, E = 0, S = 0, nnzb = 0, grid_max = 1;
    // model (device)
    float4 *X = nullptr, *w = nullptr;
    int *perm = nullptr, *seg_start = nullptr, *seg_blk = nullptr;
    int4 *seg_nodes = nullptr;
    float *seg_coef = nullptr;
    int2 *edges = nullptr;
    int *edge_blk = nullptr;
    double *node_pos = nullptr;
    int *row_ptr = nullptr, *diag_blk = nullptr;
    int2 *ent = nullptr;
    // workspace (device)
    float *blocks = nullptr, *g = nullptr, *node_dq = nullptr;
    double *blocks_d = nullptr;   // float64 copy for the PCG
    double *stats = nullptr;  // [sum_w, cost, twist^2, pad]
    unsigned long long *inliers = nullptr;
    double *node_T = nullptr, *P = nullptr, *x = nullptr, *r = nullptr, *z = nullptr, *Ap = nullptr;
    double *p[2] = {nullptr, nullptr};
    double *scal = nullptr, *partial = nullptr;
    int *ticket = nullptr;
    // host staging
    std::vector<int> h_blocks_a, h_blocks_b;  // the pair of every block
    // captured registrations, by shape
    std::vector<NgGraph> graphs;
};

namespace {

template <typename T>
cudaError_t up(T **d, const std::vector<T> &h) {
    cudaError_t e = fr::dev_malloc((void **)d, std::max<size_t>(1, h.size()) * sizeof(T));
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_model(fr_nodegraph *g) {
    void *ptrs[] = {g->X, g->w, g->perm, g->seg_start, g->seg_blk, g->seg_nodes, g->seg_coef, g->edges,
                    g->edge_blk, g->node_pos, g->row_ptr, g->diag_blk, g->ent, g->blocks, g->blocks_d, g->g,
                    g->node_dq, g->stats, g->inliers, g->node_T, g->P, g->x, g->r, g->z, g->Ap,
                    g->p[0], g->p[1], g->scal, g->partial, g->ticket};
    for (void *q : ptrs) cudaFree(q);
    for (auto &e : g->graphs) cudaGraphExecDestroy(e.exec);
    g->graphs.clear();
}

constexpr int kPairI[kNgPairs] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
constexpr int kPairJ[kNgPairs] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};

}  // namespace

FR_API fr_status fr_nodegraph_create(fr_ctx *ctx, const float *d_Xref, const int32_t *d_knn,
                                     const float *d_skw, int64_t M, const double *node_pos, int K,
                                     const int32_t *edges, int E, fr_nodegraph **out) {
    fr::NvtxRange nvtx_("fr_nodegraph_create");
    if (!ctx || !out) return FR_EINVAL;
    *out = nullptr;
    FR_TRY(validate_cloud(ctx, d_Xref, M, "d_Xref"));
    if (!d_knn || !d_skw || !aligned16(d_knn) || !aligned16(d_skw))
        return ctx->fail(FR_EINVAL, "d_knn and d_skw must be non-NULL, 16-byte aligned M x 4 arrays");
    if (K < 1 || K > (1 << 24) || !node_pos) return ctx->fail(FR_EINVAL, "need 1 <= K <= 2^24 node positions");
    if (E < 0 || (E > 0 && !edges)) return ctx->fail(FR_EINVAL, "edges: E >= 0 pairs");
    for (int e = 0; e < E; ++e) {
        const int j = edges[2 * e], k = edges[2 * e + 1];
        if (j < 0 || j >= K || k < 0 || k >= K || j == k)
            return ctx->fail(FR_EINVAL, "edge %d (%d, %d): nodes out of range or equal", e, j, k);
    }
    for (int k = 0; k < 3 * K; ++k)
        if (!std::isfinite(node_pos[k])) return ctx->fail(FR_EINVAL, "node positions must be finite");
    cudaSetDevice(ctx->device);
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<float> hX((size_t)M * 4), hw((size_t)M * 4);
    std::vector<int32_t> hk((size_t)M * 4);
    FR_CUDA(ctx, cudaMemcpy(hX.data(), d_Xref, hX.size() * sizeof(float), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaMemcpy(hw.data(), d_skw, hw.size() * sizeof(float), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaMemcpy(hk.data(), d_knn, hk.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < 4 * M; ++i) {
        if (hk[i] < 0 || hk[i] >= K) return ctx->fail(FR_EINVAL, "knn entry %lld out of range", (long long)i);
        if (!std::isfinite(hw[i]) || hw[i] < 0.0f)
            return ctx->fail(FR_EINVAL, "skinning weights must be finite and >= 0");
    }
    for (int64_t i = 0; i < M; ++i)
        if (!(hw[4 * i] + hw[4 * i + 1] + hw[4 * i + 2] + hw[4 * i + 3] > 0.0f))
            return ctx->fail(FR_EINVAL, "point %lld has no positive skinning weight", (long long)i);
    // each point's (node, weight) pairs by ascending node (stable)
    for (int64_t i = 0; i < M; ++i) {
        int o[4] = {0, 1, 2, 3};
        std::stable_sort(o, o + 4, [&](int a, int b) { return hk[4 * i + a] < hk[4 * i + b]; });
        int32_t kk[4];
        float ww[4];
        for (int a = 0; a < 4; ++a) {
            kk[a] = hk[4 * i + o[a]];
            ww[a] = hw[4 * i + o[a]];
        }
        for (int a = 0; a < 4; ++a) {
            hk[4 * i + a] = kk[a];
            hw[4 * i + a] = ww[a];
        }
    }
    // points by tuple
    std::vector<int> order(M);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return std::lexicographical_compare(&hk[4 * (size_t)a], &hk[4 * (size_t)a] + 4, &hk[4 * (size_t)b],
                                            &hk[4 * (size_t)b] + 4);
    });
    std::vector<float4> sX(M), sw(M);
    std::vector<int> seg_start;
    std::vector<int4> seg_nodes;
    for (int64_t q = 0; q < M; ++q) {
        const size_t i = (size_t)order[q];
        sX[q] = make_float4(hX[4 * i], hX[4 * i + 1], hX[4 * i + 2], 0.0f);
        sw[q] = make_float4(hw[4 * i], hw[4 * i + 1], hw[4 * i + 2], hw[4 * i + 3]);
        if (q == 0 || !std::equal(&hk[4 * i], &hk[4 * i] + 4, &hk[4 * (size_t)order[q - 1]])) {
            seg_start.push_back((int)q);
            seg_nodes.push_back(make_int4(hk[4 * i], hk[4 * i + 1], hk[4 * i + 2], hk[4 * i + 3]));
        }
    }
    seg_start.push_back((int)M);
    const int S = (int)seg_nodes.size();
    // the blocks: every tuple pair, every edge's three, every diagonal
    auto key = [&](int a, int b) { return (uint64_t)std::min(a, b) * (uint64_t)K + (uint64_t)std::max(a, b); };
    std::vector<uint64_t> keys;
    keys.reserve((size_t)S * kNgPairs + 3 * (size_t)E + K);
    for (int sgi = 0; sgi < S; ++sgi) {
        const int n[4] = {seg_nodes[sgi].x, seg_nodes[sgi].y, seg_nodes[sgi].z, seg_nodes[sgi].w};
        for (int pr = 0; pr < kNgPairs; ++pr) keys.push_back(key(n[kPairI[pr]], n[kPairJ[pr]]));
    }
    for (int e = 0; e < E; ++e) keys.push_back(key(edges[2 * e], edges[2 * e + 1]));
    for (int k = 0; k < K; ++k) keys.push_back(key(k, k));
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    const int nnzb = (int)keys.size();
    auto blk = [&](int a, int b) {
        return (int)(std::lower_bound(keys.begin(), keys.end(), key(a, b)) - keys.begin());
    };
    std::vector<int> seg_blk((size_t)S * kNgPairs);
    std::vector<float> seg_coef((size_t)S * kNgPairs);
    for (int sgi = 0; sgi < S; ++sgi) {
        const int n[4] = {seg_nodes[sgi].x, seg_nodes[sgi].y, seg_nodes[sgi].z, seg_nodes[sgi].w};
        for (int pr = 0; pr < kNgPairs; ++pr) {
            const int a = n[kPairI[pr]], b = n[kPairJ[pr]];
            seg_blk[(size_t)sgi * kNgPairs + pr] = blk(a, b);
            // a repeated node off the diagonal stands for both orders (i, j) and (j, i)
            seg_coef[(size_t)sgi * kNgPairs + pr] = (kPairI[pr] != kPairJ[pr] && a == b) ? 2.0f : 1.0f;
        }
    }
    std::vector<int2> hedges(E);
    std::vector<int> edge_blk(3 * (size_t)E);
    for (int e = 0; e < E; ++e) {
        const int j = edges[2 * e], k = edges[2 * e + 1];
        hedges[e] = make_int2(j, k);
        edge_blk[3 * (size_t)e] = blk(j, j);
        edge_blk[3 * (size_t)e + 1] = blk(k, k);
        edge_blk[3 * (size_t)e + 2] = blk(j, k);
    }
    // block rows: block (a, b) in row a as is, in row b transposed
    std::vector<int> row_cnt(K + 1, 0), diag(K);
    std::vector<int> ba(nnzb), bb(nnzb);
    for (int q = 0; q < nnzb; ++q) {
        ba[q] = (int)(keys[q] / (uint64_t)K);
        bb[q] = (int)(keys[q] % (uint64_t)K);
        ++row_cnt[ba[q] + 1];
        if (ba[q] != bb[q]) ++row_cnt[bb[q] + 1];
        else diag[ba[q]] = q;
    }
    for (int k = 0; k < K; ++k) row_cnt[k + 1] += row_cnt[k];
    std::vector<int2> ent(row_cnt[K]);
    std::vector<int> fill(row_cnt.begin(), row_cnt.end() - 1);
    for (int q = 0; q < nnzb; ++q) {
        ent[fill[ba[q]]++] = make_int2(q, bb[q]);
        if (ba[q] != bb[q]) ent[fill[bb[q]]++] = make_int2((int)(q | 0x80000000u), ba[q]);
    }
    std::vector<double> npos(node_pos, node_pos + 3 * (size_t)K);

    fr_nodegraph *g = new fr_nodegraph();
    g->ctx = ctx;
    g->device = ctx->device;
    g->M = M;
    g->K = K;
    g->E = E;
    g->S = S;
    g->nnzb = nnzb;
    g->grid_max = std::max(ng_pcg_grid(K), ng_spmv_grid(K));  // the grid-sum kernels
    g->h_blocks_a = ba;
    g->h_blocks_b = bb;
    std::vector<int> perm(order.begin(), order.end());
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t c) {
        if (e == cudaSuccess) e = c;
    };
    chk(up(&g->X, sX));
    chk(up(&g->w, sw));
    chk(up(&g->perm, perm));
    chk(up(&g->seg_start, seg_start));
    chk(up(&g->seg_nodes, seg_nodes));
    chk(up(&g->seg_blk, seg_blk));
    chk(up(&g->seg_coef, seg_coef));
    chk(up(&g->edges, hedges));
    chk(up(&g->edge_blk, edge_blk));
    chk(up(&g->node_pos, npos));
    chk(up(&g->row_ptr, row_cnt));
    chk(up(&g->diag_blk, diag));
    chk(up(&g->ent, ent));
    const size_t n6 = 6 * (size_t)K;
    chk(fr::dev_malloc((void **)&g->blocks, (size_t)nnzb * 36 * sizeof(float)));
    chk(fr::dev_malloc((void **)&g->blocks_d, (size_t)nnzb * 36 * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->g, n6 * sizeof(float)));
    chk(fr::dev_malloc((void **)&g->node_dq, (size_t)K * 8 * sizeof(float)));
    chk(fr::dev_malloc((void **)&g->stats, 4 * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->inliers, sizeof(unsigned long long)));
    chk(fr::dev_malloc((void **)&g->node_T, (size_t)K * 16 * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->P, (size_t)K * 36 * sizeof(double)));
    for (double **v : {&g->x, &g->r, &g->z, &g->Ap, &g->p[0], &g->p[1]})
        chk(fr::dev_malloc((void **)v, n6 * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->scal, 4 * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->partial, (size_t)g->grid_max * sizeof(double)));
    chk(fr::dev_malloc((void **)&g->ticket, sizeof(int)));
    if (e == cudaSuccess) e = cudaMemset(g->ticket, 0, sizeof(int));
    if (e != cudaSuccess) {
        free_model(g);
        delete g;
        return ctx->cuda(e, "fr_nodegraph_create");
    }
    *out = g;
    return FR_OK;
}

FR_API fr_status fr_nodegraph_destroy(fr_nodegraph *g) {
    if (!g) return FR_EINVAL;
    // cudaFree waits for the device: no use of the (possibly destroyed) context
    cudaSetDevice(g->device);
    free_model(g);
    delete g;
    return FR_OK;
}

namespace {

// With profiling on, event pairs bracket spans of launches (one class each).
struct Spans {
    fr_ctx *ctx;
    cudaStream_t s;
    int n = 0;
    void begin(int cls) {
        if (!ctx->profiling) return;
        while (ctx->events.size() < 2 * (size_t)(n + 1)) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            ctx->events.push_back(e);
        }
        if (ctx->event_class.size() < (size_t)(n + 1)) ctx->event_class.resize(n + 1);
        ctx->event_class[n] = cls;
        cudaEventRecord(ctx->events[2 * n], s);
    }
    void end() {
        if (!ctx->profiling) return;
        cudaEventRecord(ctx->events[2 * n + 1], s);
        ++n;
    }
};

struct NgRun {
    int pt2pl = 0, iters = 0, pcg_iters = 0;
    int storage = FR_FP32;  // lattice values the point kernel reads (16-bit: converted after each build)
    double lambda = 0.0;
    bool solve = true;  // false: assemble A, g once (fr_nodegraph_system)
};

fr_status ng_validate(fr_ctx *ctx, const fr_nodegraph *g, const float *d_Y, const float *d_Yn, int64_t N,
                      const fr_options *opt, double lambda, int pcg_iters) {
    if (!ctx || !g) return FR_EINVAL;
    if (g->ctx != ctx) return ctx->fail(FR_EINVAL, "the node graph belongs to another context");
    FR_TRY(validate_options(ctx, opt));
    if (opt->update_sigma) return ctx->fail(FR_ENOTSUPPORTED, "the sigma update is implemented for rigid registration");
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (opt->residual == FR_PT2PL) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn"));
    if (opt->blur || opt->kahan || opt->stop_twist > 0.0f)
        return ctx->fail(FR_ENOTSUPPORTED, "node graphs run without blur, Kahan sums or stop_twist");
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return ctx->fail(FR_EINVAL, "lambda must be >= 0");
    if (pcg_iters < 0 || pcg_iters > 10000) return ctx->fail(FR_EINVAL, "pcg_iters out of range");
    return FR_OK;
}

// The E step and assembly of iteration `it` at the current node poses.
void ng_assemble(fr_ctx *ctx, fr_nodegraph *g, const NgRun &run, Table t, int it, Spans &sp,
                 cudaStream_t s) {
    sp.begin(FR_K_NG_ASSEMBLE);
    cudaMemsetAsync(g->blocks, 0, (size_t)g->nnzb * 36 * sizeof(float), s);
    cudaMemsetAsync(g->g, 0, 6 * (size_t)g->K * sizeof(float), s);
    cudaMemsetAsync(g->stats, 0, 4 * sizeof(double), s);
    cudaMemsetAsync(g->inliers, 0, sizeof(unsigned long long), s);
    NgPoints P{};
    P.X = g->X;
    P.w = g->w;
    P.perm = g->perm;
    P.seg_start = g->seg_start;
    P.seg_nodes = g->seg_nodes;
    P.seg_blk = g->seg_blk;
    P.seg_coef = g->seg_coef;
    P.S = g->S;
    P.node_dq = g->node_dq;
    P.tab = t;
    P.ip = ctx->d_ip + it;
    P.renorm = 0;
    P.blocks = g->blocks;
    P.g = g->g;
    P.stats = g->stats;
    P.inliers = g->inliers;
    P.flags = &ctx->d_state->flags;
    launch_ng_points(run.pt2pl, P, 0, s, run.storage);
    NgEdges Ed{};
    Ed.edges = g->edges;
    Ed.edge_blk = g->edge_blk;
    Ed.E = g->E;
    Ed.node_T = g->node_T;
    Ed.node_pos = g->node_pos;
    Ed.lambda = run.lambda;
    Ed.ip = ctx->d_ip + it;
    Ed.blocks = g->blocks;
    Ed.g = g->g;
    Ed.stats = g->stats;
    launch_ng_edges(Ed, s);
    sp.end();
}

void ng_solve_update(fr_ctx *ctx, fr_nodegraph *g, const NgRun &run, Spans &sp, cudaStream_t s) {
    sp.begin(FR_K_NG_SOLVE);
    NgPcg L{};
    L.K = g->K;
    L.row_ptr = g->row_ptr;
    L.ent = g->ent;
    L.diag_blk = g->diag_blk;
    L.nnzb = g->nnzb;
    L.blocks = g->blocks;
    L.blocks_d = g->blocks_d;
    L.g = g->g;
    L.P = g->P;
    L.x = g->x;
    L.r = g->r;
    L.z = g->z;
    L.Ap = g->Ap;
    L.scal = g->scal;
    L.partial = g->partial;
    L.ticket = g->ticket;
    cudaMemsetAsync(g->p[0], 0, 6 * (size_t)g->K * sizeof(double), s);
    launch_ng_pcg_init(L, s);
    for (int k = 0; k < run.pcg_iters; ++k) {
        L.p_old = g->p[k & 1];
        L.p_new = g->p[(k + 1) & 1];
        launch_ng_pcg_spmv(L, s);
        launch_ng_pcg_update(L, s);
    }
    launch_ng_update(g->K, g->x, g->node_T, g->node_dq, g->stats + 2, s);
    sp.end();
}

// The registration's kernels after the uploads, on stream s: node dual
// quaternions, the first lattice, then per iteration (a rebuild when sigma
// changes,) the assembly and the solve with the node update; finally the
// last table is freed.  Returns the number of kernels (the callers count
// them: directly issued, or once per graph replay).
int ng_issue(fr_ctx *ctx, fr_nodegraph *g, const NgRun &run, const Table tab[2], int iters, int64_t N,
             cudaStream_t s, Spans &sp) {
    int launches = 1;
    launch_ng_update(g->K, nullptr, g->node_T, g->node_dq, nullptr, s);
    int cur = 0, cur_build = 0;
    auto build = [&](int t, int it) {
        IterLaunch b{};
        b.job = ctx->d_job;
        b.ip = ctx->d_ip;
        b.st = ctx->d_state;
        b.build = tab[t];
        b.build_list = ctx->lists[t];
        b.build_it = it;
        b.gb = blocks_for(ctx, N, 8);
        sp.begin(FR_K_BUILD);
        launch_em_iter(run.pt2pl, 0, b, s, run.storage);
        sp.end();
        ++launches;
        if (run.storage != FR_FP32) {  // 16-bit records of the completed build
            IterLaunch c{};
            c.job = ctx->d_job;
            c.ip = ctx->d_ip;
            c.st = ctx->d_state;
            c.conv = tab[t];
            c.conv_list = ctx->lists[t];
            c.conv_it = it;
            c.gv = blocks_for(ctx, N, 4);
            sp.begin(FR_K_CONVERT);
            launch_em_iter(run.pt2pl, 0, c, s, run.storage);
            sp.end();
            ++launches;
        }
    };
    auto clear = [&](int t, int it) {
        Table tc = tab[t];
        int *l = ctx->lists[t];
        const int *c = &ctx->d_ip[it].nvert;
        launch_clear_lists(&tc, &l, &c, 1, blocks_for(ctx, N, 4), s);
        ++launches;
    };
    build(0, 0);
    for (int it = 0; it < iters; ++it) {
        if (it > 0 && ctx->h_ip[it].rebuild) {
            clear(cur, cur_build);
            cur ^= 1;
            cur_build = it;
            build(cur, it);
        }
        ng_assemble(ctx, g, run, tab[cur], it, sp, s);
        launches += 2;
        if (run.solve) {
            ng_solve_update(ctx, g, run, sp, s);
            launches += 2 + 2 * run.pcg_iters;
        }
    }
    clear(cur, cur_build);
    return launches;
}

// The same captured once per shape as a CUDA graph and replayed: the
// per-call data (poses, sigma schedule, observation pointers and size) is
// read from device descriptors uploaded before the launch.
fr_status ng_graph_launch(fr_ctx *ctx, fr_nodegraph *g, const NgRun &run, const Table tab[2], int iters,
                          int64_t N, uint32_t cap, unsigned long long rebuilds) {
    long long lam_bits;
    std::memcpy(&lam_bits, &run.lambda, sizeof lam_bits);  // lambda is a kernel argument of the graph
    const long long key[10] = {N, iters, run.pcg_iters, run.pt2pl, (long long)cap, run.solve ? 1 : 0,
                               (long long)rebuilds, (long long)ctx->ws_gen, lam_bits, run.storage};
    NgGraph *hit = nullptr;
    for (auto &e : g->graphs)
        if (std::equal(key, key + 10, e.key)) hit = &e;
    if (!hit) {
        cudaStream_t cs;
        FR_CUDA(ctx, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        Spans none{ctx, cs};
        int kernels = 0;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            kernels = ng_issue(ctx, g, run, tab, iters, N, cs, none);
            e = cudaStreamEndCapture(cs, &graph);
        }
        cudaStreamDestroy(cs);
        FR_CUDA(ctx, e);
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        FR_CUDA(ctx, e);
        if (g->graphs.size() >= 8) {
            cudaGraphExecDestroy(g->graphs.front().exec);
            g->graphs.erase(g->graphs.begin());
        }
        NgGraph ng{};
        std::copy(key, key + 10, ng.key);
        ng.exec = exec;
        ng.kernels = kernels;
        g->graphs.push_back(ng);
        hit = &g->graphs.back();
    }
    FR_CUDA(ctx, cudaGraphLaunch(hit->exec, ctx->stream));
    ctx->launches += hit->kernels;
    return FR_OK;
}

fr_status ng_run(fr_ctx *ctx, fr_nodegraph *g, const float *d_Y, const float *d_Yn, int64_t N,
                 const fr_options *opt, const NgRun &run, double *node_T, fr_report *rep, bool safe,
                 double *A_out, double *g_out) {
    const int iters = run.solve ? opt->iters : 1;
    const uint32_t cap = table_slots(N, safe);
    FR_TRY(ensure_small(ctx, std::max(iters, 1), 1));
    FR_TRY(ensure_tables(ctx, cap, false));
    Table tab[2];
    for (int i = 0; i < 2; ++i) {
        tab[i] = ctx->tables[i];
        tab[i].mask = cap - 1;
        tab[i].max_probe = table_probe_limit(cap, safe);
    }
    fr_options o = *opt;
    o.iters = std::max(iters, 1);
    fill_iter_params(&o, g->M, N, ctx->h_ip);
    RigidJob *j = ctx->h_job;
    *j = RigidJob{};
    j->Y = (const float4 *)d_Y;
    j->Yn = run.pt2pl ? (const float4 *)d_Yn : nullptr;
    j->M = (int)std::min<int64_t>(g->M, INT32_MAX);
    j->N = (int)N;
    DeviceState *hs = ctx->h_state;
    *hs = DeviceState{};
    cudaStream_t s = ctx->stream;
    FR_CUDA(ctx, copy_async(ctx, ctx->d_job, j, sizeof(RigidJob), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, ctx->d_ip, ctx->h_ip, o.iters * sizeof(IterParams), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, ctx->d_state, hs, sizeof(DeviceState), cudaMemcpyHostToDevice));
    FR_CUDA(ctx, copy_async(ctx, g->node_T, node_T, (size_t)g->K * 16 * sizeof(double), cudaMemcpyHostToDevice));
    Spans sp{ctx, s};
    // the rebuild pattern (which iterations rebuild the lattice) shapes the graph
    unsigned long long rebuilds = 1469598103934665603ull;
    int cur_build = 0;
    for (int it = 1; it < iters; ++it) {
        rebuilds = (rebuilds ^ (unsigned long long)(ctx->h_ip[it].rebuild ? 2 * it + 1 : 2 * it)) * 1099511628211ull;
        if (ctx->h_ip[it].rebuild) cur_build = it;
    }
    if (ctx->profiling || !opt->use_graph) {
        ctx->launches += ng_issue(ctx, g, run, tab, iters, N, s, sp);
    } else {
        FR_TRY(ng_graph_launch(ctx, g, run, tab, iters, N, cap, rebuilds));
    }
    FR_CUDA(ctx, cudaGetLastError());
    double st[4];
    unsigned long long inl = 0;
    std::vector<float> hb, hg;
    if (!run.solve) {
        hb.resize((size_t)g->nnzb * 36);
        hg.resize(6 * (size_t)g->K);
        FR_CUDA(ctx, cudaMemcpyAsync(hb.data(), g->blocks, hb.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
        FR_CUDA(ctx, cudaMemcpyAsync(hg.data(), g->g, hg.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
    }
    FR_CUDA(ctx, cudaMemcpyAsync(st, g->stats, sizeof st, cudaMemcpyDeviceToHost, s));
    FR_CUDA(ctx, cudaMemcpyAsync(&inl, g->inliers, sizeof inl, cudaMemcpyDeviceToHost, s));
    FR_CUDA(ctx, copy_async(ctx, hs, ctx->d_state, sizeof(DeviceState), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, copy_async(ctx, ctx->h_ip, ctx->d_ip, o.iters * sizeof(IterParams), cudaMemcpyDeviceToHost));
    std::vector<double> hT((size_t)g->K * 16);
    if (run.solve)
        FR_CUDA(ctx, cudaMemcpyAsync(hT.data(), g->node_T, hT.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    FR_CUDA(ctx, cudaStreamSynchronize(s));
    if (sp.n) collect_profile(ctx, sp.n);
    FR_TRY(check_flags(ctx, hs->flags));
    if (run.solve) std::copy(hT.begin(), hT.end(), node_T);
    if (!run.solve) {
        const size_t n = 6 * (size_t)g->K;
        if (A_out) {
            std::fill(A_out, A_out + n * n, 0.0);
            for (int q = 0; q < g->nnzb; ++q) {
                const size_t a0 = 6 * (size_t)g->h_blocks_a[q], b0 = 6 * (size_t)g->h_blocks_b[q];
                for (int r = 0; r < 6; ++r)
                    for (int c = 0; c < 6; ++c) {
                        const double v = hb[(size_t)q * 36 + 6 * r + c];
                        A_out[(a0 + r) * n + b0 + c] = v;
                        if (a0 != b0) A_out[(b0 + c) * n + a0 + r] = v;
                    }
            }
        }
        if (g_out)
            for (size_t i = 0; i < n; ++i) g_out[i] = hg[i];
    }
    if (rep) {
        *rep = fr_report{};
        rep->iters_run = run.solve ? iters : 0;
        rep->last_inliers = (int64_t)inl;
        rep->last_sum_w = st[0];
        rep->last_cost = st[1];
        rep->last_twist_norm = std::sqrt(st[2]);
        rep->lattice_vertices = ctx->h_ip[cur_build].nvert;
        rep->lattice_builds = hs->builds;
        rep->lattice_vertices_sum = hs->nvert_total;
    }
    return FR_OK;
}

}  // namespace

FR_API fr_status fr_register_nodegraph(fr_ctx *ctx, fr_nodegraph *g, const float *d_Y, const float *d_Yn,
                                       int64_t N, const fr_options *opt, double lambda, int pcg_iters,
                                       double *node_T, fr_report *rep) {
    fr::NvtxRange nvtx_("fr_register_nodegraph");
    FR_TRY(ng_validate(ctx, g, d_Y, d_Yn, N, opt, lambda, pcg_iters));
    if (!node_T) return ctx->fail(FR_EINVAL, "node_T must not be NULL");
    for (int64_t i = 0; i < 16 * (int64_t)g->K; ++i)
        if (!std::isfinite(node_T[i])) return ctx->fail(FR_EINVAL, "node poses must be finite");
    cudaSetDevice(ctx->device);
    NgRun run;
    run.pt2pl = opt->residual == FR_PT2PL;
    run.storage = opt->storage;
    run.iters = opt->iters;
    run.pcg_iters = pcg_iters;
    run.lambda = lambda;
    std::vector<double> T0(node_T, node_T + 16 * (size_t)g->K);
    fr_status st = ng_run(ctx, g, d_Y, d_Yn, N, opt, run, node_T, rep, false, nullptr, nullptr);
    if (st == FR_ECAPACITY) {  // the compact table overflowed: rerun at the safe size
        std::copy(T0.begin(), T0.end(), node_T);
        st = ng_run(ctx, g, d_Y, d_Yn, N, opt, run, node_T, rep, true, nullptr, nullptr);
    }
    return st;
}

FR_API fr_status fr_nodegraph_system(fr_ctx *ctx, fr_nodegraph *g, const float *d_Y, const float *d_Yn,
                                     int64_t N, const fr_options *opt, double lambda,
                                     const double *node_T, double *A_out, double *g_out, fr_report *rep) {
    fr::NvtxRange nvtx_("fr_nodegraph_system");
    FR_TRY(ng_validate(ctx, g, d_Y, d_Yn, N, opt, lambda, 0));
    if (!node_T) return ctx->fail(FR_EINVAL, "node_T must not be NULL");
    cudaSetDevice(ctx->device);
    NgRun run;
    run.pt2pl = opt->residual == FR_PT2PL;
    run.storage = opt->storage;
    run.lambda = lambda;
    run.solve = false;
    std::vector<double> T(node_T, node_T + 16 * (size_t)g->K);
    fr_status st = ng_run(ctx, g, d_Y, d_Yn, N, opt, run, T.data(), rep, false, A_out, g_out);
    if (st == FR_ECAPACITY) st = ng_run(ctx, g, d_Y, d_Yn, N, opt, run, T.data(), rep, true, A_out, g_out);
    return st;
}

FR_API fr_status fr_nodegraph_warp(fr_ctx *ctx, fr_nodegraph *g, const double *node_T, float *d_out) {
    fr::NvtxRange nvtx_("fr_nodegraph_warp");
    if (!ctx || !g || !node_T || !d_out) return FR_EINVAL;
    if (g->ctx != ctx) return ctx->fail(FR_EINVAL, "the node graph belongs to another context");
    if (!aligned16(d_out)) return ctx->fail(FR_EINVAL, "d_out must be 16-byte aligned (M x 4 floats)");
    cudaSetDevice(ctx->device);
    cudaStream_t s = ctx->stream;
    FR_CUDA(ctx, copy_async(ctx, g->node_T, node_T, (size_t)g->K * 16 * sizeof(double), cudaMemcpyHostToDevice));
    launch_ng_update(g->K, nullptr, g->node_T, g->node_dq, nullptr, s);
    NgPoints P{};
    P.X = g->X;
    P.w = g->w;
    P.perm = g->perm;
    P.seg_start = g->seg_start;
    P.seg_nodes = g->seg_nodes;
    P.S = g->S;
    P.node_dq = g->node_dq;
    P.warp_out = (float4 *)d_out;
    launch_ng_points(0, P, 1, s);
    ctx->launches += 2;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, cudaStreamSynchronize(s));
    return FR_OK;
}
