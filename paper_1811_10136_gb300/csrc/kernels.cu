// sm_103a kernels of the FilterReg hot path.
//
//   k_build_splat   Section 4.2 "Splat" of the observation Y with values
//                   [1, y] or [1, y, n_y] (Eq. 11), fused with the lattice
//                   build: elevate, simplex, hash insert (atomicCAS), float4
//                   atomic accumulation.  One thread per point, grid-stride.
//   k_clear_table   frees the occupied slots before a rebuild.
//   k_blur_pass     Section 4.2 "Blur" along one lattice axis (ping-pong).
//   k_rigid_step    one EM iteration minus the build: slice at x = T x_ref
//                   (E step, Eq. 6 / Eq. 9), outlier weight M0/(M0+c) and
//                   residuals (Eq. 7 / Eq. 10), twist Jacobian and the
//                   Gauss-Newton reduction of A and b (Eq. 17-18) -- warp
//                   shuffles, then one float64 partial per block -- and, in
//                   the last block to finish, the float64 Cholesky solve and
//                   the SE(3) exponential update T <- exp(dzeta^) T (Eq. 16).
//   primitives      embed / build / splat / slice / vertex listing kernels of
//                   the fr_lattice_* entry points.
#include <cuda_runtime.h>

#include "internal.h"
#include "lattice.cuh"

namespace fr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int grid_stride() { return gridDim.x * blockDim.x; }
__device__ __forceinline__ int gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }

// ---------------------------------------------------------------------------
// Small float64 linear algebra of the M step (one thread).
// ---------------------------------------------------------------------------

__device__ __forceinline__ int tri_index(int p, int q) {  // p <= q, row-major upper
    return p * 6 - p * (p - 1) / 2 + (q - p);
}

// Cholesky solve of the 6x6 normal equations A x = rhs.  A pivot below
// 1e-12 * max(diag A) means "not positive definite": returns false.
__device__ bool cholesky6(const double *tri, const double *rhs, double *x) {
    double L[6][6];
    double maxdiag = 0.0;
    for (int i = 0; i < 6; ++i) maxdiag = fmax(maxdiag, tri[tri_index(i, i)]);
    if (!(maxdiag > 0.0)) return false;
    const double floor_ = maxdiag * 1e-12;
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = tri[tri_index(j, i)];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > floor_)) return false;
                L[i][i] = sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[k][i] * x[k];
        x[i] = s / L[i][i];
    }
    return true;
}

// exp of the twist matrix of Eq. 16: R = I + A W + B W^2, t = (I + B W + C W^2) v.
__device__ void se3_exp(const double *z, double *T) {
    const double w0 = z[0], w1 = z[1], w2 = z[2];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    const double th = sqrt(th2);
    double A, B, C;
    if (th < 1e-3) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s, c;
        sincos(th, &s, &c);
        A = s / th;
        B = (1.0 - c) / th2;
        C = (th - s) / (th2 * th);
    }
    const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    double W2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            W2[3 * i + j] = W[3 * i] * W[j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j];
    for (int i = 0; i < 3; ++i) {
        double tv = 0.0;
        for (int j = 0; j < 3; ++j) {
            const double I = (i == j) ? 1.0 : 0.0;
            T[4 * i + j] = I + A * W[3 * i + j] + B * W2[3 * i + j];
            tv += (I + B * W[3 * i + j] + C * W2[3 * i + j]) * z[3 + j];
        }
        T[4 * i + 3] = tv;
    }
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}

// Gauss-Newton step from the reduced sums; updates the pose in st.
__device__ void solve_update(const double *tot, DeviceState *st, float stop_twist) {
    st->iters_run += 1;
    st->sum_w = tot[27];
    st->cost = tot[28];
    st->inliers = (long long)(tot[29] + 0.5);
    double rhs[6], dz[6];
    for (int p = 0; p < 6; ++p) rhs[p] = -tot[21 + p];
    if (!cholesky6(tot, rhs, dz)) {
        st->degenerate += 1;
        return;
    }
    double E[16], Tn[16];
    se3_exp(dz, E);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += E[4 * i + k] * st->T[4 * k + j];
            Tn[4 * i + j] = s;
        }
    for (int i = 0; i < 16; ++i) st->T[i] = Tn[i];
    double n2 = 0.0;
    for (int p = 0; p < 6; ++p) n2 += dz[p] * dz[p];
    st->twist_norm = sqrt(n2);
    if (stop_twist > 0.0f && st->twist_norm < (double)stop_twist) st->done = 1;
}

// Float accumulator with optional Kahan compensation.
template <bool KAHAN>
struct Acc {
    float s[kRigidVals];
    float c[KAHAN ? kRigidVals : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int v = 0; v < kRigidVals; ++v) s[v] = 0.0f;
        if (KAHAN) {
#pragma unroll
            for (int v = 0; v < (KAHAN ? kRigidVals : 1); ++v) c[v] = 0.0f;
        }
    }
    __device__ __forceinline__ void add(int v, float x) {
        if (KAHAN) {
            const float y = __fsub_rn(x, c[v]);
            const float t = __fadd_rn(s[v], y);
            c[v] = __fsub_rn(__fsub_rn(t, s[v]), y);
            s[v] = t;
        } else {
            s[v] += x;
        }
    }
};

// Block reduction of kRigidVals floats: warp shuffles, then shared memory;
// writes one float64 row per block.
template <bool KAHAN>
__device__ __forceinline__ void block_partial(Acc<KAHAN> &acc, double *partials) {
    __shared__ float sm[kBlock / 32][kRigidVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < kRigidVals; ++v) {
        float x = acc.s[v];
        if (KAHAN) x -= acc.c[KAHAN ? v : 0];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
        if (lane == 0) sm[warp][v] = x;
    }
    __syncthreads();
    if (threadIdx.x < kRigidVals) {
        double s = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) s += (double)sm[w][threadIdx.x];
        partials[(size_t)blockIdx.x * kRigidVals + threadIdx.x] = s;
    }
}

// The last block to arrive sums all partials in float64 and runs the solve.
__device__ __forceinline__ void grid_finish(double *partials, DeviceState *st, float stop_twist) {
    __shared__ int last;
    __shared__ double tot[kRigidVals];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(&st->ticket, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < kRigidVals) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b)
            s += __ldcg(partials + (size_t)b * kRigidVals + threadIdx.x);
        tot[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        solve_update(tot, st, stop_twist);
        st->ticket = 0;
    }
}

// ---------------------------------------------------------------------------
// Registration kernels
// ---------------------------------------------------------------------------

__global__ void k_init_state(const RigidJob *job, DeviceState *st) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < 16; ++i) st->T[i] = job->T0[i];
        st->sum_w = st->cost = st->twist_norm = 0.0;
        st->inliers = 0;
        st->iters_run = st->degenerate = 0;
        st->done = 0;
        st->ticket = 0;
        st->flags = 0;
        st->nvert = 0;
        st->builds = 0;
        st->nvert_total = 0;
    }
}

__global__ void k_clear_table(Table t, DeviceState *st, int full) {
    if (st && gtid() == 0) {
        st->nvert = 0;
        st->builds += 1;
    }
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t s = gtid(); s <= t.mask; s += grid_stride()) {
        if (full || __ldcg(t.keys + s) != kEmpty) {
            t.keys[s] = kEmpty;
            t.v0[s] = z;
            if (t.v1) t.v1[s] = z;
        }
    }
}

template <bool PT2PL>
__global__ void __launch_bounds__(kBlock) k_build_splat(const RigidJob *__restrict__ job,
                                                         const IterParams *__restrict__ ipa, int it,
                                                         Table t, DeviceState *st) {
    if (st->done) return;
    const IterParams ip = ipa[it];
    const int N = job->N;
    const float4 *__restrict__ Y = job->Y;
    const float4 *__restrict__ Yn = job->Yn;
    int claimed_here = 0, bad = 0;
    for (int i = gtid(); i < N; i += grid_stride()) {
        const float4 y = __ldg(Y + i);
        Simplex sx;
        if (!embed(y.x, y.y, y.z, ip.s1, ip.s2, ip.s3, sx)) {
            bad |= kFlagRange;
            continue;
        }
        float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PT2PL) n = __ldg(Yn + i);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            bool claimed;
            const int s = insert_key(t.keys, t.mask, sx.key[k], t.mask + 1, claimed);
            if (s < 0) {
                bad |= kFlagCapacity;
                continue;
            }
            claimed_here += claimed;
            const float b = sx.b[k];
            atomicAdd(t.v0 + s, make_float4(b, b * y.x, b * y.y, b * y.z));
            if (PT2PL) atomicAdd(t.v1 + s, make_float4(b * n.x, b * n.y, b * n.z, 0.f));
        }
    }
    // One counter update per warp.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        claimed_here += __shfl_xor_sync(kFull, claimed_here, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (claimed_here) {
            atomicAdd(&st->nvert, claimed_here);
            atomicAdd((unsigned long long *)&st->nvert_total, (unsigned long long)claimed_here);
        }
        if (bad) atomicOr(&st->flags, bad);
    }
}

__global__ void k_blur_pass(Table in, Table out, int dir, const DeviceState *st) {
    if (st && st->done) return;
    for (uint32_t s = gtid(); s <= in.mask; s += grid_stride()) {
        const unsigned long long key = __ldg(in.keys + s);
        if (key == kEmpty) continue;
        const int sm = find_key(in.keys, in.mask, neighbour_key(key, dir, -1));
        const int sp = find_key(in.keys, in.mask, neighbour_key(key, dir, +1));
        float4 a = __ldg(in.v0 + s);
        if (sm >= 0) {
            const float4 u = __ldg(in.v0 + sm);
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
        }
        if (sp >= 0) {
            const float4 u = __ldg(in.v0 + sp);
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
        }
        out.v0[s] = a;
        if (in.v1) {
            float4 c = __ldg(in.v1 + s);
            if (sm >= 0) {
                const float4 u = __ldg(in.v1 + sm);
                c.x += 0.5f * u.x; c.y += 0.5f * u.y; c.z += 0.5f * u.z; c.w += 0.5f * u.w;
            }
            if (sp >= 0) {
                const float4 u = __ldg(in.v1 + sp);
                c.x += 0.5f * u.x; c.y += 0.5f * u.y; c.z += 0.5f * u.z; c.w += 0.5f * u.w;
            }
            out.v1[s] = c;
        }
    }
}

// E-step sums of one moved model point: M0, M1 and (pt2pl) the normal sum.
struct Sums {
    float m0, m1x, m1y, m1z, nx, ny, nz;
};

template <bool PT2PL>
__device__ __forceinline__ bool slice_point(const Table &t, float x0, float x1, float x2,
                                            const IterParams &ip, Sums &o, int &bad) {
    Simplex sx;
    o = Sums{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!embed(x0, x1, x2, ip.s1, ip.s2, ip.s3, sx)) {
        bad |= kFlagRange;
        return false;
    }
    int slot[kD];
    find4(t.keys, t.mask, sx, slot);
    float4 a[kD], c[kD];
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        a[k] = slot[k] >= 0 ? __ldg(t.v0 + slot[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
        if (PT2PL) c[k] = slot[k] >= 0 ? __ldg(t.v1 + slot[k]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        const float b = sx.b[k];
        o.m0 += b * a[k].x;
        o.m1x += b * a[k].y;
        o.m1y += b * a[k].z;
        o.m1z += b * a[k].w;
        if (PT2PL) {
            o.nx += b * c[k].x;
            o.ny += b * c[k].y;
            o.nz += b * c[k].z;
        }
    }
    return true;
}

__device__ __forceinline__ void load_pose(const double *T, float *P) {
    // P: row-major 3x4 float copy of the pose, staged in shared memory.
    if (threadIdx.x < 12) P[threadIdx.x] = (float)T[(threadIdx.x / 4) * 4 + (threadIdx.x % 4)];
    __syncthreads();
}

template <bool PT2PL, bool KAHAN>
__global__ void __launch_bounds__(kBlock) k_rigid_step(const RigidJob *__restrict__ job,
                                                        const IterParams *__restrict__ ipa, int it,
                                                        Table t, double *partials,
                                                        DeviceState *st) {
    if (st->done) return;
    __shared__ float P[12];
    load_pose(st->T, P);
    const IterParams ip = ipa[it];
    const int M = job->M;
    const int renorm = job->renormalize;
    const float4 *__restrict__ X = job->X;
    Acc<KAHAN> acc;
    acc.zero();
    int bad = 0;
    for (int i = gtid(); i < M; i += grid_stride()) {
        const float4 r = __ldg(X + i);
        const float x0 = P[0] * r.x + P[1] * r.y + P[2] * r.z + P[3];
        const float x1 = P[4] * r.x + P[5] * r.y + P[6] * r.z + P[7];
        const float x2 = P[8] * r.x + P[9] * r.y + P[10] * r.z + P[11];
        Sums e;
        if (!slice_point<PT2PL>(t, x0, x1, x2, ip, e, bad)) continue;
        if (!(e.m0 > 0.0f)) continue;
        const float W = e.m0 / (e.m0 + ip.c_eff);
        const float ws = W * ip.inv_sigma2;
        const float inv = 1.0f / e.m0;
        const float e0 = x0 - e.m1x * inv, e1 = x1 - e.m1y * inv, e2 = x2 - e.m1z * inv;
        if (!PT2PL) {
            // J = [S, I], S = -[x]_x:  J^T J = [[|x|^2 I - x x^T, [x]_x], [-[x]_x, I]],
            // J^T e = [x cross e; e].
            const float xx = x0 * x0, yy = x1 * x1, zz = x2 * x2;
            acc.add(tri_index(0, 0), ws * (yy + zz));
            acc.add(tri_index(0, 1), -ws * x0 * x1);
            acc.add(tri_index(0, 2), -ws * x0 * x2);
            acc.add(tri_index(1, 1), ws * (xx + zz));
            acc.add(tri_index(1, 2), -ws * x1 * x2);
            acc.add(tri_index(2, 2), ws * (xx + yy));
            // upper-right block [x]_x = [[0,-z,y],[z,0,-x],[-y,x,0]]
            acc.add(tri_index(0, 4), -ws * x2);
            acc.add(tri_index(0, 5), ws * x1);
            acc.add(tri_index(1, 3), ws * x2);
            acc.add(tri_index(1, 5), -ws * x0);
            acc.add(tri_index(2, 3), -ws * x1);
            acc.add(tri_index(2, 4), ws * x0);
            acc.add(tri_index(3, 3), ws);
            acc.add(tri_index(4, 4), ws);
            acc.add(tri_index(5, 5), ws);
            acc.add(21, ws * (x1 * e2 - x2 * e1));
            acc.add(22, ws * (x2 * e0 - x0 * e2));
            acc.add(23, ws * (x0 * e1 - x1 * e0));
            acc.add(24, ws * e0);
            acc.add(25, ws * e1);
            acc.add(26, ws * e2);
            acc.add(28, ws * (e0 * e0 + e1 * e1 + e2 * e2));
        } else {
            float n0 = e.nx * inv, n1 = e.ny * inv, n2 = e.nz * inv;
            if (renorm) {
                const float nn = sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
                if (!(nn > 0.0f)) continue;
                n0 /= nn; n1 /= nn; n2 /= nn;
            }
            const float res = n0 * e0 + n1 * e1 + n2 * e2;
            // j = [x cross n, n]
            const float j[6] = {x1 * n2 - x2 * n1, x2 * n0 - x0 * n2, x0 * n1 - x1 * n0, n0, n1, n2};
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                const float wj = ws * j[p];
#pragma unroll
                for (int q = p; q < 6; ++q) acc.add(tri_index(p, q), wj * j[q]);
                acc.add(21 + p, wj * res);
            }
            acc.add(28, ws * res * res);
        }
        acc.add(27, W);
        acc.add(29, 1.0f);
    }
    if (bad) atomicOr(&st->flags, bad);
    block_partial<KAHAN>(acc, partials);
    grid_finish(partials, st, job->stop_twist);
}

// E-step sums at T x for every model point (the fr_estep entry point).
template <bool PT2PL>
__global__ void __launch_bounds__(kBlock) k_estep_out(const RigidJob *__restrict__ job,
                                                       const IterParams *__restrict__ ipa, Table t,
                                                       float *out, DeviceState *st) {
    __shared__ float P[12];
    load_pose(st->T, P);
    const IterParams ip = ipa[0];
    const int M = job->M;
    const int vd = PT2PL ? 7 : 4;
    int bad = 0;
    for (int i = gtid(); i < M; i += grid_stride()) {
        const float4 r = __ldg(job->X + i);
        const float x0 = P[0] * r.x + P[1] * r.y + P[2] * r.z + P[3];
        const float x1 = P[4] * r.x + P[5] * r.y + P[6] * r.z + P[7];
        const float x2 = P[8] * r.x + P[9] * r.y + P[10] * r.z + P[11];
        Sums e;
        slice_point<PT2PL>(t, x0, x1, x2, ip, e, bad);
        float *o = out + (size_t)i * vd;
        o[0] = e.m0; o[1] = e.m1x; o[2] = e.m1y; o[3] = e.m1z;
        if (PT2PL) { o[4] = e.nx; o[5] = e.ny; o[6] = e.nz; }
    }
    if (bad) atomicOr(&st->flags, bad);
}

// ---------------------------------------------------------------------------
// Lattice primitives
// ---------------------------------------------------------------------------

__global__ void k_embed(const float4 *__restrict__ P, int n, float s1, float s2, float s3,
                        int *keys, float *bary, int *flags) {
    for (int i = gtid(); i < n; i += grid_stride()) {
        const float4 p = __ldg(P + i);
        Simplex sx;
        const bool ok = embed(p.x, p.y, p.z, s1, s2, s3, sx);
        if (!ok) atomicOr(flags, kFlagRange);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            if (keys) {
                int c[3], sum = 0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    c[j] = ok ? unpack_coord(sx.key[k], j) : 0;
                    sum += c[j];
                }
                int4 v = make_int4(c[0], c[1], c[2], -sum);
                reinterpret_cast<int4 *>(keys)[(size_t)i * kD + k] = v;
            }
            if (bary) bary[(size_t)i * kD + k] = ok ? sx.b[k] : 0.0f;
        }
    }
}

__global__ void k_build_records(const float4 *__restrict__ P, int n, float s1, float s2, float s3,
                                Table t, int *rec_slot, float *rec_w, int *counters) {
    int claimed_here = 0, bad = 0;
    for (int i = gtid(); i < n; i += grid_stride()) {
        const float4 p = __ldg(P + i);
        Simplex sx;
        if (!embed(p.x, p.y, p.z, s1, s2, s3, sx)) {
            bad |= kFlagRange;
#pragma unroll
            for (int k = 0; k < kD; ++k) {
                rec_slot[(size_t)i * kD + k] = -1;
                rec_w[(size_t)i * kD + k] = 0.0f;
            }
            continue;
        }
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            bool claimed;
            const int s = insert_key(t.keys, t.mask, sx.key[k], t.mask + 1, claimed);
            if (s < 0) bad |= kFlagCapacity;
            claimed_here += claimed;
            rec_slot[(size_t)i * kD + k] = s;
            rec_w[(size_t)i * kD + k] = sx.b[k];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        claimed_here += __shfl_xor_sync(kFull, claimed_here, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (claimed_here) atomicAdd(counters + 0, claimed_here);
        if (bad) atomicOr(counters + 1, bad);
    }
}

__global__ void k_splat_records(const float *__restrict__ vals, int vdim, int n,
                                const int *__restrict__ rec_slot, const float *__restrict__ rec_w,
                                Table t) {
    for (int i = gtid(); i < n; i += grid_stride()) {
        float v[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = c < vdim ? __ldg(vals + (size_t)i * vdim + c) : 0.0f;
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const int s = rec_slot[(size_t)i * kD + k];
            if (s < 0) continue;
            const float b = rec_w[(size_t)i * kD + k];
            atomicAdd(t.v0 + s, make_float4(b * v[0], b * v[1], b * v[2], b * v[3]));
            if (vdim > 4) atomicAdd(t.v1 + s, make_float4(b * v[4], b * v[5], b * v[6], b * v[7]));
        }
    }
}

__global__ void k_slice_out(const float4 *__restrict__ Q, int m, float s1, float s2, float s3,
                            Table t, int vdim, float *out, int *flags) {
    for (int i = gtid(); i < m; i += grid_stride()) {
        const float4 p = __ldg(Q + i);
        Simplex sx;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (embed(p.x, p.y, p.z, s1, s2, s3, sx)) {
            int slot[kD];
            find4(t.keys, t.mask, sx, slot);
#pragma unroll
            for (int k = 0; k < kD; ++k) {
                if (slot[k] < 0) continue;
                const float b = sx.b[k];
                const float4 a = __ldg(t.v0 + slot[k]);
                acc[0] += b * a.x; acc[1] += b * a.y; acc[2] += b * a.z; acc[3] += b * a.w;
                if (vdim > 4) {
                    const float4 c = __ldg(t.v1 + slot[k]);
                    acc[4] += b * c.x; acc[5] += b * c.y; acc[6] += b * c.z; acc[7] += b * c.w;
                }
            }
        } else {
            atomicOr(flags, kFlagRange);
        }
        for (int c = 0; c < vdim; ++c) out[(size_t)i * vdim + c] = acc[c];
    }
}

__global__ void k_vertices(Table t, int vdim, int *keys_out, float *vals_out, int *count) {
    for (uint32_t s = gtid(); s <= t.mask; s += grid_stride()) {
        const unsigned long long key = t.keys[s];
        if (key == kEmpty) continue;
        const int o = atomicAdd(count, 1);
        int c[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) c[j] = unpack_coord(key, j);
        reinterpret_cast<int4 *>(keys_out)[o] = make_int4(c[0], c[1], c[2], -(c[0] + c[1] + c[2]));
        if (vals_out) {
            const float4 a = t.v0[s];
            const float4 b = t.v1 ? t.v1[s] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            for (int ch = 0; ch < vdim; ++ch) vals_out[(size_t)o * vdim + ch] = v[ch];
        }
    }
}

int grid_for(long long n, int cap_blocks) {
    long long g = (n + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > cap_blocks) g = cap_blocks;
    return (int)g;
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

void launch_init_state(const RigidJob *job, DeviceState *st, cudaStream_t s) {
    k_init_state<<<1, 32, 0, s>>>(job, st);
}

void launch_clear_table(Table t, DeviceState *st, int full, int grid, cudaStream_t s) {
    k_clear_table<<<grid, kBlock, 0, s>>>(t, st, full);
}

void launch_build_splat(int pt2pl, const RigidJob *job, const IterParams *ip, int it, Table t,
                        DeviceState *st, int grid, cudaStream_t s) {
    if (pt2pl)
        k_build_splat<true><<<grid, kBlock, 0, s>>>(job, ip, it, t, st);
    else
        k_build_splat<false><<<grid, kBlock, 0, s>>>(job, ip, it, t, st);
}

void launch_blur_pass(Table in, Table out, int dir, int grid, const DeviceState *st, cudaStream_t s) {
    k_blur_pass<<<grid, kBlock, 0, s>>>(in, out, dir, st);
}

void launch_rigid_step(int pt2pl, int kahan, const RigidJob *job, const IterParams *ip, int it,
                       Table t, double *partials, DeviceState *st, int grid, cudaStream_t s) {
    if (pt2pl) {
        if (kahan)
            k_rigid_step<true, true><<<grid, kBlock, 0, s>>>(job, ip, it, t, partials, st);
        else
            k_rigid_step<true, false><<<grid, kBlock, 0, s>>>(job, ip, it, t, partials, st);
    } else {
        if (kahan)
            k_rigid_step<false, true><<<grid, kBlock, 0, s>>>(job, ip, it, t, partials, st);
        else
            k_rigid_step<false, false><<<grid, kBlock, 0, s>>>(job, ip, it, t, partials, st);
    }
}

void launch_estep_out(int pt2pl, const RigidJob *job, const IterParams *ip, Table t, float *out,
                      DeviceState *st, int grid, cudaStream_t s) {
    if (pt2pl)
        k_estep_out<true><<<grid, kBlock, 0, s>>>(job, ip, t, out, st);
    else
        k_estep_out<false><<<grid, kBlock, 0, s>>>(job, ip, t, out, st);
}

void launch_embed(const float4 *P, int n, float s1, float s2, float s3, int *keys, float *bary,
                  int *flags, cudaStream_t s) {
    k_embed<<<grid_for(n, 4096), kBlock, 0, s>>>(P, n, s1, s2, s3, keys, bary, flags);
}

void launch_build_records(const float4 *P, int n, float s1, float s2, float s3, Table t,
                          int *rec_slot, float *rec_w, int *counters, cudaStream_t s) {
    k_build_records<<<grid_for(n, 4096), kBlock, 0, s>>>(P, n, s1, s2, s3, t, rec_slot, rec_w,
                                                         counters);
}

void launch_splat_records(const float *vals, int vdim, int n, const int *rec_slot,
                          const float *rec_w, Table t, cudaStream_t s) {
    k_splat_records<<<grid_for(n, 4096), kBlock, 0, s>>>(vals, vdim, n, rec_slot, rec_w, t);
}

void launch_slice_out(const float4 *Q, int m, float s1, float s2, float s3, Table t, int vdim,
                      float *out, int *flags, cudaStream_t s) {
    k_slice_out<<<grid_for(m, 4096), kBlock, 0, s>>>(Q, m, s1, s2, s3, t, vdim, out, flags);
}

void launch_vertices(Table t, int vdim, int *keys_out, float *vals_out, int *count,
                     cudaStream_t s) {
    k_vertices<<<grid_for((long long)t.mask + 1, 4096), kBlock, 0, s>>>(t, vdim, keys_out,
                                                                        vals_out, count);
}

}  // namespace fr
