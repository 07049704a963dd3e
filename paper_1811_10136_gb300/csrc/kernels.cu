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
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "lattice.cuh"

namespace fr {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int grid_stride() { return gridDim.x * blockDim.x; }
__device__ __forceinline__ int gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }

// ---------------------------------------------------------------------------
// Reductions: float accumulation per thread, double-float across blocks.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int tri_index(int p, int q) {  // p <= q, row-major upper, 6 x 6
    return p * 6 - p * (p - 1) / 2 + (q - p);
}

// Unevaluated sum hi + lo of two floats (about 48 significant bits), added
// with error-free transformations (Knuth's two-sum), all at float32 rate.
struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, lo);
    return DF{hi, __fsub_rn(lo, __fsub_rn(hi, s))};
}

// Float accumulator with optional Kahan compensation.
template <bool KAHAN>
struct Acc {
    float s[kRigidVals];
    float c[KAHAN ? kRigidVals : 1];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int v = 0; v < kRigidVals; ++v) s[v] = 0.0f;
#pragma unroll
        for (int v = 0; v < (KAHAN ? kRigidVals : 1); ++v) c[v] = 0.0f;
    }
    __device__ __forceinline__ void add(int v, float x) {
        if (KAHAN) {
            const float y = __fsub_rn(x, c[KAHAN ? v : 0]);
            const float t = __fadd_rn(s[v], y);
            c[KAHAN ? v : 0] = __fsub_rn(__fsub_rn(t, s[v]), y);
            s[v] = t;
        } else {
            s[v] += x;
        }
    }
    __device__ __forceinline__ float total(int v) const {
        return KAHAN ? __fsub_rn(s[v], c[KAHAN ? v : 0]) : s[v];
    }
};

// Warp sum of 32 values per lane by recursive halving: at the step of
// offset o a lane keeps the half of its values whose index has bit o equal to
// its own lane bit, and adds its partner's copy of that half; 16 + 8 + 4 + 2 +
// 1 shuffles instead of 32 x 5.  Lane l returns the sum of value l.
__device__ __forceinline__ float warp_sum32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, o);
        }
    }
    return v[0];
}

// Block reduction of kRigidVals floats -- warp sums, then the 8 warp sums
// combined as double-float -- written value-major: value v of block blk at
// partials[v * rows + blk].
template <bool KAHAN>
__device__ __forceinline__ void block_partial(const Acc<KAHAN> &acc, float2 *partials, int blk,
                                              int rows) {
    static_assert(kRigidVals <= 32, "one value per lane");
    __shared__ float sm[kBlock / 32][kRigidVals];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = i < kRigidVals ? acc.total(i) : 0.0f;
    const float x = warp_sum32(v);
    if (lane < kRigidVals) sm[warp][lane] = x;
    __syncthreads();
    if (threadIdx.x < kRigidVals) {
        DF a{0.0f, 0.0f};
        for (int w = 0; w < kBlock / 32; ++w) a = df_add(a, DF{sm[w][threadIdx.x], 0.0f});
        partials[(size_t)threadIdx.x * rows + blk] = make_float2(a.hi, a.lo);
    }
}

// ---------------------------------------------------------------------------
// The M-step solve in float64, spread over the lanes of one warp.
//
// GB300's float64 pipe is narrow, so the cost of float64 work is the number
// of warp instructions on its critical path; each lane therefore owns one
// matrix entry.  LDL^T of the 6 x 6 normal matrix (Eq. 18): lane
// tri_index(p, q) (p <= q) holds A[p][q], then D[p] (p == q) or L[q][p].
// ---------------------------------------------------------------------------

// 1/d in float64 from the float reciprocal refined by one Newton step (the
// relative error squares: ~1e-7 -> ~1e-14, far below what the solve's pivot
// floor of 1e-12 and the float32 sums it is fed need), two dependent float64
// operations instead of a full division sequence on the narrow float64 pipe.
__device__ __forceinline__ double rcp64(double d) {
    double r = (double)(1.0f / (float)d);
    r = fma(r, fma(-d, r, 1.0), r);
    return r;
}

struct Solved {
    bool ok;
    double dz;     // lane i < 6: delta zeta_i = -(A^{-1} b)_i
};

__device__ Solved warp_solve6(double t /* lane v: reduced value v */) {
    const int lane = threadIdx.x & 31;
    int p = 0, q = 0;
    {
        int l = lane;
        for (int r = 0; r < 6; ++r) {
            if (l < 6 - r) { p = r; q = r + l; break; }
            l -= 6 - r;
        }
    }
    const bool mine = lane < 21;
    double a = mine ? t : 0.0;
    // pivot floor relative to the largest diagonal entry
    double md = (mine && p == q) ? a : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(kFull, md, o));
    bool ok = md > 0.0;
    const double floor_ = md * 1e-12;
    for (int k = 0; k < 6 && ok; ++k) {
        const double dk = __shfl_sync(kFull, a, tri_index(k, k));
        const double akp = __shfl_sync(kFull, a, tri_index(k, p < k ? k : p));
        const double akq = __shfl_sync(kFull, a, tri_index(k, q < k ? k : q));
        ok = dk > floor_;
        if (!ok) break;
        const double inv = rcp64(dk);
        if (mine) {
            if (p == k && q > k) a = a * inv;            // L[q][k]
            else if (p > k) a = a - akp * akq * inv;      // Schur complement
        }
    }
    Solved r{ok, 0.0};
    if (!ok) return r;
    // rhs = -b: lane i < 6 takes reduced value 21 + i
    double y = -__shfl_sync(kFull, t, 21 + (lane < 6 ? lane : 0));
    for (int k = 0; k < 6; ++k) {          // L y = rhs (unit lower)
        const double yk = __shfl_sync(kFull, y, k);
        const double lik = __shfl_sync(kFull, a, tri_index(k, lane > k && lane < 6 ? lane : k));
        if (lane < 6 && lane > k) y -= lik * yk;
    }
    const int li = lane < 6 ? lane : 0;
    y = y * rcp64(__shfl_sync(kFull, a, tri_index(li, li)));   // D z = y
    for (int k = 5; k >= 0; --k) {         // L^T x = z
        const double xk = __shfl_sync(kFull, y, k);
        const double lki = __shfl_sync(kFull, a, tri_index(lane < k ? lane : k, k));
        if (lane < k) y -= lki * xk;
    }
    r.dz = y;
    return r;
}

// T <- exp(dzeta^) T (Eq. 16 applied as the SE(3) exponential), lanes of one
// warp: R = I + A W + B W^2 and V = I + B W + C W^2 with W = [omega]_x,
// W^2 = omega omega^T - th^2 I; A, B, C by their series for th < 0.25 (each
// term below 2e-17 at the cut-off), else from sin and cos.
__device__ void warp_se3_update_cols(double dz, double *T /* row-major 4x4, global */,
                                     double *smem /* 24 doubles */, double c0, double c1, double c2);
__device__ void warp_se3_update(double dz, double *T /* row-major 4x4, global */,
                                double *smem /* 24 doubles */) {
    const int lane = threadIdx.x & 31, j = lane & 3;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0;
    if (lane < 12) {
        c0 = T[j];
        c1 = T[4 + j];
        c2 = T[8 + j];
    }
    warp_se3_update_cols(dz, T, smem, c0, c1, c2);
}
// The same with lane l < 12's column entries T[j], T[4 + j], T[8 + j]
// (j = l mod 4) already loaded.
__device__ void warp_se3_update_cols(double dz, double *T /* row-major 4x4, global */,
                                     double *smem /* 24 doubles */, double c0, double c1, double c2) {
    const int lane = threadIdx.x & 31;
    double w[3], v[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        w[i] = __shfl_sync(kFull, dz, i);
        v[i] = __shfl_sync(kFull, dz, 3 + i);
    }
    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double coef;  // lane 0: A, lane 1: B, lane 2: C
    if (th2 < 0.0625) {
        // A = sum_n (-1)^n th^{2n} / (2n+1)!, B: / (2n+2)!, C: / (2n+3)!, n = 0..5
        const bool la = lane == 0, lb = lane == 1;
#define FR_SERIES(n, a, b, c) (la ? (a) : (lb ? (b) : (c)))
        coef = FR_SERIES(5, -1.0 / 39916800.0, -1.0 / 479001600.0, -1.0 / 6227020800.0);
        coef = coef * th2 + FR_SERIES(4, 1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0);
        coef = coef * th2 + FR_SERIES(3, -1.0 / 5040.0, -1.0 / 40320.0, -1.0 / 362880.0);
        coef = coef * th2 + FR_SERIES(2, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0);
        coef = coef * th2 + FR_SERIES(1, -1.0 / 6.0, -1.0 / 24.0, -1.0 / 120.0);
        coef = coef * th2 + FR_SERIES(0, 1.0, 0.5, 1.0 / 6.0);
#undef FR_SERIES
    } else {
        const double th = sqrt(th2);
        double s, cth;
        sincos(th, &s, &cth);
        coef = lane == 0 ? s / th : (lane == 1 ? (1.0 - cth) / th2 : (th - s) / (th2 * th));
    }
    const double A = __shfl_sync(kFull, coef, 0), B = __shfl_sync(kFull, coef, 1),
                 C = __shfl_sync(kFull, coef, 2);
    // lanes 0..8: R_ij ; lanes 9..17: V_ij v_j (elements picked by selects:
    // a lane-dependent index into w or v would put them in local memory)
    auto pick = [](const double (&x)[3], int n) { return n == 0 ? x[0] : (n == 1 ? x[1] : x[2]); };
    if (lane < 18) {
        const int r = lane < 9 ? lane : lane - 9;
        const int i = r / 3, j = r % 3;
        const double Wij = (i == j) ? 0.0 : ((j == (i + 1) % 3) ? -pick(w, (i + 2) % 3) : pick(w, (i + 1) % 3));
        const double W2ij = pick(w, i) * pick(w, j) - (i == j ? th2 : 0.0);
        const double I = (i == j) ? 1.0 : 0.0;
        if (lane < 9) smem[lane] = I + A * Wij + B * W2ij;
        else smem[lane] = (I + B * Wij + C * W2ij) * pick(v, j);
    }
    __syncwarp();
    if (lane < 3) smem[18 + lane] = smem[9 + 3 * lane] + smem[10 + 3 * lane] + smem[11 + 3 * lane];
    __syncwarp();
    double tn = 0.0;
    if (lane < 12) {
        const int i = lane / 4, j = lane % 4;
        tn = smem[3 * i] * c0 + smem[3 * i + 1] * c1 + smem[3 * i + 2] * c2;
        if (j == 3) tn += smem[18 + i];
    }
    __syncwarp();
    if (lane < 12) T[lane] = tn;
}

// The last step block: double-float sum of all block partials (warp w sums
// values w, w + 8, ...; each lane keeps 4 independent loads in flight), then
// the solve and the pose update in warp 0.
__device__ void finish_iteration(const float2 *partials, int rows, DeviceState *st,
                                 float stop_twist, const RigidJob *sig_job = nullptr,
                                 const IterParams *ip_cur = nullptr, IterParams *ip_next = nullptr) {
    __shared__ DF tot_s[32];
    __shared__ double sm_e[24];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the pose entries the update multiplies, loaded while the partials are summed
    double tc0 = 0.0, tc1 = 0.0, tc2 = 0.0;
    if (warp == 0 && lane < 12) {
        const int j = lane & 3;
        tc0 = st->T[j];
        tc1 = st->T[4 + j];
        tc2 = st->T[8 + j];
    }
    // Warp w reduces values w, w + 8, w + 16, w + 24: all of its loads are
    // issued before any of them is consumed.
    constexpr int kPer = 4;      // values per warp
    constexpr int kBatch = 4;    // rows per lane per batch
    DF acc[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) acc[j] = DF{0.0f, 0.0f};
    for (int b0 = lane; b0 < rows; b0 += 32 * kBatch) {
        float2 r[kPer][kBatch];
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int v = warp + 8 * j;
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int b = b0 + 32 * u;
                r[j][u] = (v < kRigidVals && b < rows) ? __ldcg(partials + (size_t)v * rows + b)
                                                       : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j)
#pragma unroll
            for (int u = 0; u < kBatch; ++u) acc[j] = df_add(acc[j], DF{r[j][u].x, r[j][u].y});
    }
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
        DF a = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const DF b{__shfl_xor_sync(kFull, a.hi, o), __shfl_xor_sync(kFull, a.lo, o)};
            a = df_add(a, b);
        }
        const int v = warp + 8 * j;
        if (lane == 0 && v < kRigidVals) tot_s[v] = a;
    }
    __syncthreads();
    if (warp != 0) return;
    const double t = (lane < kRigidVals) ? (double)tot_s[lane].hi + (double)tot_s[lane].lo : 0.0;
    if (lane == 27) st->sum_w = t;
    if (lane == 28) st->cost = t;
    if (lane == 29) st->inliers = (long long)(t + 0.5);
    if (lane < kRigidVals) st->sums[lane] = t;
    if (ip_next) {
        // sigma^2 = sum_i Q_i / (M0_i + c) / (3 kappa sum_i W_i) -- kappa the
        // lattice kernel's per-axis variance in units of sigma^2, so that sigma
        // is the width at which the kernel used matches the residuals --
        // (floored; kept when no point had observations), rounded to float, and
        // the parameters of the next iteration from it, as the host derives
        // them from a sigma.
        const double sw = __shfl_sync(kFull, t, 27), sq = __shfl_sync(kFull, t, 30);
        if (lane == 0) {
            double sig = (double)ip_cur->sigma;
            if (sw > 0.0) {
                const double s2 = sq / (3.0 * sw * sig_job->sig_kappa);
                const double sn = sqrt(s2 > 0.0 ? s2 : 0.0);
                sig = sn > sig_job->sig_floor ? sn : sig_job->sig_floor;
            }
            const float sf = (float)sig;
            const double sd = (double)sf;
            IterParams n = *ip_next;
            n.sigma = sf;
            n.s1 = (float)(sig_job->sig_alpha[0] / sd);
            n.s2 = (float)(sig_job->sig_alpha[1] / sd);
            n.s3 = (float)(sig_job->sig_alpha[2] / sd);
            n.c_eff = (float)(sig_job->sig_c * sd * sd * sd * sig_job->sig_G);
            n.inv_sigma2 = (float)(1.0 / (sd * sd));
            n.rebuild = 1;
            n.vscale = 1.0f;
            n.inv_vscale = 1.0f;
            n.ws1 = 1.0f / (2.0f * n.s1);
            n.ws2 = 1.0f / (6.0f * n.s2);
            n.ws3 = 1.0f / (12.0f * n.s3);
            *ip_next = n;
        }
    }
    const Solved r = warp_solve6(t);
    if (lane == 0) st->iters_run += 1;
    if (!r.ok) {
        if (lane == 0) st->degenerate += 1;
        return;
    }
    warp_se3_update_cols(r.dz, st->T, sm_e, tc0, tc1, tc2);
    // |delta zeta| (a diagnostic and the stop test) in float
    float n2 = lane < 6 ? (float)r.dz * (float)r.dz : 0.0f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(kFull, n2, o);
    if (lane == 0) {
        const float nrm = sqrtf(n2);
        st->twist_norm = nrm;
        if (stop_twist > 0.0f && nrm < stop_twist) st->done = 1;
    }
}

// ---------------------------------------------------------------------------
// Roles of the fused EM-iteration kernel
// ---------------------------------------------------------------------------

// World position of the lattice point whose stored key coordinates are
// z0..z2 (z3 = -(z0 + z1 + z2)), at the feature scales of ip: the elevation's
// inverse, c_1 = (z0 - z1)/2, c_2 = (z0 + z1 - 2 z2)/6,
// c_3 = (z0 + z1 + z2 - 3 z3)/12, p_{i-1} = c_i / s_i (the factors 1/(2 s1),
// 1/(6 s2), 1/(12 s3) come with the iteration's parameters).  Conversion and
// slice evaluate it alike: the p_v taken out of a record is the one put back.
__device__ __forceinline__ float3 vertex_position(unsigned long long key, const IterParams &ip) {
    const int z0 = unpack_coord(key, 0), z1 = unpack_coord(key, 1), z2 = unpack_coord(key, 2);
    const int z3 = -(z0 + z1 + z2);
    return make_float3((float)(z0 - z1) * ip.ws1, (float)(z0 + z1 - 2 * z2) * ip.ws2,
                       (float)(z0 + z1 + z2 - 3 * z3) * ip.ws3);
}

template <int ST>
__device__ __forceinline__ unsigned pack2(float a, float b) {
    if (ST == kStoreBF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const unsigned *>(&h);
    }
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const unsigned *>(&h);
}

template <int ST>
__device__ __forceinline__ float2 unpack2(unsigned u) {
    if (ST == kStoreBF16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}

// Compact record of a built vertex: [W, sum b (y - p_v), sum b n, 0] -- the
// float32 sums re-centred on the vertex (values of magnitude ~sigma instead of
// scene coordinates) and rounded to 16 bits.
template <int ST>
__device__ __forceinline__ uint4 compact_record(float4 a, float4 c, float3 p, float sc) {
    return make_uint4(pack2<ST>(a.x * sc, (a.y - a.x * p.x) * sc),
                      pack2<ST>((a.z - a.x * p.y) * sc, (a.w - a.x * p.z) * sc),
                      pack2<ST>(c.x * sc, c.y * sc), pack2<ST>(c.z * sc, 0.0f));
}

// Writes the 16-bit record over slot s's float32 v0 (already read).
__device__ __forceinline__ void store_compact(unsigned long long *keys, uint32_t s, uint4 r) {
    *rec_cv(keys, s) = r;
}

// Vector float atomic add without a returned value (a reduction at L2).
__device__ __forceinline__ void red_add4(float4 *p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Build: Section 4.2 "Splat" of the observation with values [1, y] or
// [1, y, n_y] (Eq. 11), fused with the lattice build (elevate, simplex, hash
// insert, float4 atomic accumulation).  One thread per point per round.
// Lanes of a warp whose points share a lattice vertex (neighbouring pixels
// of a depth image mostly do, in raster order) are merged first: runs of
// equal keys in consecutive lanes are summed by a segmented scan and only
// the run's last lane inserts the key and issues the atomics.  The slots a
// round claims are appended to `list` (one atomic per block and round on the
// build's vertex counter) so that the table can later be freed without
// scanning it.
// Lanes per merge chunk: runs of equal keys merge within aligned chunks of
// this many lanes (log2 of it shuffle steps per channel).  Measured on the
// batched depth-frame step with the inserts overlapped: 4 lanes 100.4 us per
// launch, 8 lanes 101.4, 16 lanes 103.5 -- fewer scan steps against ~30 % more
// atomics than 8.
constexpr int kMergeLanes = 4;

template <bool PT2PL, int ST, bool SIG = false>
__device__ __forceinline__ void build_role(const RigidJob *__restrict__ job, IterParams *ipp,
                                           Table t, int *list, DeviceState *st, int blk, int nblk) {
    // the sigma update (point-to-point) adds the moment b |y - p_v|^2 about
    // each vertex's position p_v, stored in v1.x
    constexpr int kCh = PT2PL ? 7 : (SIG ? 5 : 4);
    constexpr int kClaimCap = 1024;
    __shared__ int s_claim[kClaimCap];
    __shared__ int s_n, s_fit, s_base;
    if (threadIdx.x == 0) {
        s_n = 0;
        s_fit = 0;
    }
    __syncthreads();
    const IterParams ip = *ipp;
    const int N = job->N;
    const float4 *__restrict__ Y = job->Y;
    const float4 *__restrict__ Yn = job->Yn;
    const int lane = threadIdx.x & 31;
    const int per_round = nblk * kBlock;
    const int rounds = (N + per_round - 1) / per_round;
    int bad = 0;
    unsigned long long claimed_total = 0;
    for (int r = 0; r < rounds; ++r) {
        const int i = r * per_round + blk * kBlock + threadIdx.x;
        Simplex sx;
        bool valid = false;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f), n = y;
        if (i < N) {
            y = __ldg(Y + i);
            if (PT2PL) n = __ldg(Yn + i);
            valid = embed(y.x, y.y, y.z, ip.s1, ip.s2, ip.s3, sx);
            if (!valid) bad |= kFlagRange;
        }
        // Merge runs of equal keys across neighbouring lanes: a segmented
        // inclusive scan within kMergeLanes-lane chunks (lane order) leaves
        // each run's sum at its last lane, which alone inserts
        // the key and issues the atomics.  First the runs of all four
        // vertices (head bits by ballot) and the inserts of this lane's run
        // tails, their probes and claims in flight together (insert4); then
        // the sums one vertex at a time, so that only its seven sums are live
        // (holding all four vertices' sums spilled more than overlapping
        // their probes saved).
        int sl[kD];
        int mask = 0;
        unsigned hd[kD];
        unsigned want = 0;
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const unsigned long long key = valid ? sx.key[k] : kEmpty;
            const unsigned long long prev = __shfl_up_sync(kFull, key, 1);
            hd[k] = __ballot_sync(kFull, (lane & (kMergeLanes - 1)) == 0 || prev != key);
            const bool tail = lane == 31 || ((hd[k] >> (lane + 1)) & 1u);
            want |= (valid && tail) ? 1u << k : 0u;
        }
        {
            unsigned cl;
            insert4(t.keys, t.mask, sx, want, t.max_probe, sl, cl);
            mask = (int)cl;
        }
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            const unsigned heads = hd[k];
            const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
            const bool tail = (want >> k) & 1u;
            const unsigned long long key = valid ? sx.key[k] : kEmpty;
            const float b = valid ? sx.b[k] : 0.0f;
            float v[kCh];
            v[0] = b;
            v[1] = b * y.x;
            v[2] = b * y.y;
            v[3] = b * y.z;
            if (PT2PL) {
                v[4] = b * n.x;
                v[5] = b * n.y;
                v[6] = b * n.z;
            } else if (SIG) {
                const float3 pv = vertex_position(key, ip);
                const float dx = y.x - pv.x, dy = y.y - pv.y, dz = y.z - pv.z;
                v[kCh - 1] = b * (dx * dx + dy * dy + dz * dz);
            }
#pragma unroll
            for (int o = 1; o < kMergeLanes; o <<= 1) {
#pragma unroll
                for (int c = 0; c < kCh; ++c) {
                    const float tv = __shfl_up_sync(kFull, v[c], o);
                    if (lane - o >= head) v[c] += tv;
                }
            }
            if (tail) {
                if (sl[k] < 0) {
                    bad |= kFlagCapacity;
                } else {
                    red_add4(rec_v0(t.keys, sl[k]), v[0], v[1], v[2], v[3]);
                    if (PT2PL) red_add4(rec_v1(t.keys, sl[k]), v[4], v[5], v[6], 0.f);
                    else if (SIG) atomicAdd(reinterpret_cast<float *>(rec_v1(t.keys, sl[k])), v[kCh - 1]);
                }
            }
        }
        // The warp's claimed slots go to the block's buffer (a shared
        // counter, no barrier); a warp that would not fit appends to the list
        // itself.
        const int cnt = __popc(mask);
        int pre = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, pre, o);
            if (lane >= o) pre += v;
        }
        const int wtot = __shfl_sync(kFull, pre, 31);
        if (wtot) {
            int wbase = 0;
            if (lane == 31) wbase = atomicAdd(&s_n, wtot);
            wbase = __shfl_sync(kFull, wbase, 31);
            int o = pre - cnt;
            if (wbase + wtot <= kClaimCap) {
#pragma unroll
                for (int k = 0; k < kD; ++k)
                    if (mask & (1 << k)) s_claim[wbase + o++] = sl[k];
                if (lane == 31) atomicMax(&s_fit, wbase + wtot);
            } else {
                int g = 0;
                if (lane == 31) g = atomicAdd(&ipp->nvert, wtot);
                g = __shfl_sync(kFull, g, 31);
#pragma unroll
                for (int k = 0; k < kD; ++k)
                    if (mask & (1 << k)) list[g + o++] = sl[k];
                if (lane == 31) claimed_total += wtot;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        s_base = s_fit ? atomicAdd(&ipp->nvert, s_fit) : 0;
        claimed_total += s_fit;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < s_fit; e += kBlock) list[s_base + e] = s_claim[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad |= __shfl_xor_sync(kFull, bad, o);
    if (lane == 0 && bad) atomicOr(&st->flags, bad);
    if (claimed_total) atomicAdd((unsigned long long *)&st->nvert_total, claimed_total);
    if (threadIdx.x == 0 && blk == 0) atomicAdd(&st->builds, 1);
}

// Convert: once a build is complete (an earlier launch), turn each listed
// vertex's float32 sums into its 16-bit record (16-bit storage modes only).
template <bool PT2PL, int ST>
__device__ __forceinline__ void convert_role(Table t, const int *list, const IterParams *ipp, int blk,
                                             int nblk) {
    if constexpr (ST != kStoreF32) {
        const IterParams ip = *ipp;
        const int n = __ldcg(&ipp->nvert);
        for (int e = blk * kBlock + threadIdx.x; e < n; e += nblk * kBlock) {
            const int slot = __ldcg(list + e);
            const float4 a = __ldcg(rec_v0(t.keys, slot));
            const float4 c = PT2PL ? __ldcg(rec_v1(t.keys, slot)) : make_float4(0.f, 0.f, 0.f, 0.f);
            store_compact(t.keys, slot,
                          compact_record<ST>(a, c, vertex_position(__ldcg(rec_key(t.keys, slot)), ip), ip.vscale));
        }
    }
}

// Clear: free the slots a build listed by zeroing their records (two whole
// 32-byte sectors: key, values and 16-bit record).
__device__ __forceinline__ void clear_role(Table t, const int *list, int n, int blk, int nblk) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = blk * kBlock + threadIdx.x; e < n; e += nblk * kBlock) {
        float4 *r = reinterpret_cast<float4 *>(rec_key(t.keys, (uint32_t)__ldcg(list + e)));
        r[0] = z;
        r[1] = z;
        r[2] = z;
        r[3] = z;
    }
}

// E-step sums of one moved model point: M0, M1 and (pt2pl) the normal sum.
struct Sums {
    float m0, m1x, m1y, m1z, nx, ny, nz;
    float q;  // sigma update: sum_j K |x - y_j|^2
};

template <bool PT2PL, int ST, bool SIG = false>
__device__ __forceinline__ bool slice_point(const Table &t, float x0, float x1, float x2,
                                            const IterParams &ip, Sums &o, int &bad) {
    Simplex sx;
    o = Sums{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (!embed(x0, x1, x2, ip.s1, ip.s2, ip.s3, sx)) {
        bad |= kFlagRange;
        return false;
    }
    if constexpr (ST == kStoreF32) {
        // Key probes of the four vertices together, then their value sums
        // (v0 in the key's sector, v1 in the next) -- the four-sector form
        // (key and v0 in one 256-bit load) needs registers the step does not
        // have at four blocks per SM, and measured slower.
        int slot[kD];
        find4(t.keys, t.mask, sx, slot, t.max_probe);
        float4 a[kD], c[kD];
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            a[k] = slot[k] >= 0 ? __ldg(rec_v0(t.keys, slot[k])) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (PT2PL || SIG) c[k] = slot[k] >= 0 ? __ldg(rec_v1(t.keys, slot[k])) : make_float4(0.f, 0.f, 0.f, 0.f);
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
            if (SIG && slot[k] >= 0) {
                // sum over the vertex's observations of b |x - y|^2, from its
                // moments about the vertex position p (all of size ~sigma):
                // W |x - p|^2 - 2 (x - p).(V - W p) + sum b |y - p|^2
                const float3 p = vertex_position(sx.key[k], ip);
                const float dx = x0 - p.x, dy = x1 - p.y, dz = x2 - p.z;
                const float W = a[k].x;
                const float rx = a[k].y - W * p.x, ry = a[k].z - W * p.y, rz = a[k].w - W * p.z;
                o.q += b * (W * (dx * dx + dy * dy + dz * dz) - 2.0f * (dx * rx + dy * ry + dz * rz) + c[k].x);
            }
        }
        return true;
    } else {
        // Key probes, then one 16-byte record per vertex (beside its key);
        // positions restored in float32.
        int slot[kD];
        find4(t.keys, t.mask, sx, slot, t.max_probe);
        uint4 r[kD];
#pragma unroll
        for (int k = 0; k < kD; ++k) r[k] = slot[k] >= 0 ? __ldg(rec_cv(t.keys, slot[k])) : make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int k = 0; k < kD; ++k) {
            if (slot[k] < 0) continue;
            const float b = sx.b[k];
            const float2 w_rx = unpack2<ST>(r[k].x), ry_rz = unpack2<ST>(r[k].y);
            const float3 p = vertex_position(sx.key[k], ip);
            const float bw = b * w_rx.x;
            o.m0 += bw;
            o.m1x += b * w_rx.y + bw * p.x;
            o.m1y += b * ry_rz.x + bw * p.y;
            o.m1z += b * ry_rz.y + bw * p.z;
            if (PT2PL) {
                const float2 nx_ny = unpack2<ST>(r[k].z), nz_0 = unpack2<ST>(r[k].w);
                o.nx += b * nx_ny.x;
                o.ny += b * nx_ny.y;
                o.nz += b * nz_0.x;
            }
        }
        const float u = ip.inv_vscale;
        o.m0 *= u;
        o.m1x *= u;
        o.m1y *= u;
        o.m1z *= u;
        o.nx *= u;
        o.ny *= u;
        o.nz *= u;
        return true;
    }
}

// One model point's terms of the M step, handed to add(value index, value):
// outlier weight W = M0/(M0+c) (Eq. 7), the point-to-point (Eq. 7) or
// point-to-plane (Eq. 10) residual with Sigma^{-1} weighting, its twist
// Jacobian J = [-[x]_x, I] (Eq. 16) and the contributions to A = sum J^T J
// (upper triangle, 21 values), b = sum J^T r (6), the weight sum, the cost
// and the inlier count (Eq. 17-18).  Returns false for a point without
// observations nearby (M0 = 0).
template <bool PT2PL, bool SIG = false, typename Add>
__device__ __forceinline__ bool point_terms(float x0, float x1, float x2, const Sums &e,
                                            const IterParams &ip, int renorm, Add &&add) {
    if (!(e.m0 > 0.0f)) return false;
    const float W = e.m0 / (e.m0 + ip.c_eff);
    const float ws = W * ip.inv_sigma2;
    const float inv = 1.0f / e.m0;
    const float e0 = x0 - e.m1x * inv, e1 = x1 - e.m1y * inv, e2 = x2 - e.m1z * inv;
    if (!PT2PL) {
        // J = [S, I], S = -[x]_x:  J^T J = [[|x|^2 I - x x^T, [x]_x], [-[x]_x, I]],
        // J^T e = [x cross e; e].
        const float xx = x0 * x0, yy = x1 * x1, zz = x2 * x2;
        add(tri_index(0, 0), ws * (yy + zz));
        add(tri_index(0, 1), -ws * x0 * x1);
        add(tri_index(0, 2), -ws * x0 * x2);
        add(tri_index(1, 1), ws * (xx + zz));
        add(tri_index(1, 2), -ws * x1 * x2);
        add(tri_index(2, 2), ws * (xx + yy));
        // upper-right block [x]_x = [[0,-z,y],[z,0,-x],[-y,x,0]]
        add(tri_index(0, 4), -ws * x2);
        add(tri_index(0, 5), ws * x1);
        add(tri_index(1, 3), ws * x2);
        add(tri_index(1, 5), -ws * x0);
        add(tri_index(2, 3), -ws * x1);
        add(tri_index(2, 4), ws * x0);
        add(tri_index(3, 3), ws);
        add(tri_index(4, 4), ws);
        add(tri_index(5, 5), ws);
        add(21, ws * (x1 * e2 - x2 * e1));
        add(22, ws * (x2 * e0 - x0 * e2));
        add(23, ws * (x0 * e1 - x1 * e0));
        add(24, ws * e0);
        add(25, ws * e1);
        add(26, ws * e2);
        add(28, ws * (e0 * e0 + e1 * e1 + e2 * e2));
    } else {
        float n0 = e.nx * inv, n1 = e.ny * inv, n2 = e.nz * inv;
        if (renorm) {
            const float nn = sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
            if (!(nn > 0.0f)) return false;
            n0 /= nn; n1 /= nn; n2 /= nn;
        }
        const float res = n0 * e0 + n1 * e1 + n2 * e2;
        // j = [x cross n, n]
        const float j[6] = {x1 * n2 - x2 * n1, x2 * n0 - x0 * n2, x0 * n1 - x1 * n0, n0, n1, n2};
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            const float wj = ws * j[p];
#pragma unroll
            for (int q = p; q < 6; ++q) add(tri_index(p, q), wj * j[q]);
            add(21 + p, wj * res);
        }
        add(28, ws * res * res);
    }
    add(27, W);
    add(29, 1.0f);
    if (SIG) add(30, e.q / (e.m0 + ip.c_eff));  // Q_i / (M0_i + c): the sigma update's numerator
    return true;
}

// Row j of x = T x_ref in float, as ((P_j0 x + P_j1 y) + P_j2 z) + P_j3 with
// every operation rounded (no FMA), so that the moved positions -- which
// decide lattice keys -- are reproducible outside the kernel.
__device__ __forceinline__ float apply_row(const float *P, int j, float4 r) {
    const float a = __fadd_rn(__fmul_rn(P[4 * j], r.x), __fmul_rn(P[4 * j + 1], r.y));
    return __fadd_rn(__fadd_rn(a, __fmul_rn(P[4 * j + 2], r.z)), P[4 * j + 3]);
}

__device__ __forceinline__ void load_pose(const double *T, float *P) {
    // P: row-major 3x4 float copy of the pose, staged in shared memory.
    if (threadIdx.x < 12) P[threadIdx.x] = (float)T[(threadIdx.x / 4) * 4 + (threadIdx.x % 4)];
    __syncthreads();
}

// Step: one EM iteration minus the build.  Slice at x = T x_ref (E step,
// Eq. 6 / Eq. 9), outlier weight M0/(M0+c) and residuals (Eq. 7 / Eq. 10),
// twist Jacobian, reduction of A and b (Eq. 17-18); the last block to finish
// solves and updates the pose.
template <bool PT2PL, bool KAHAN, int ST, bool SIG = false>
__device__ __forceinline__ void step_role(const RigidJob *job, const IterParams *ipp, const Table t,
                                          float2 *partials, DeviceState *st, int blk, int nblk,
                                          int sig_next = 0) {
    __shared__ float P[12];
    __shared__ int last;
    // The iteration's constants stay in shared memory and are re-read where
    // used (volatile: not hoisted), instead of being held in registers
    // across the slice, where the step runs short of them.
    __shared__ IterParams s_ip;
    if (threadIdx.x == 0) s_ip = *ipp;
    const volatile IterParams *vip = &s_ip;
    load_pose(st->T, P);
    const int M = job->M;
    const int renorm = job->renormalize;
    const float4 *__restrict__ X = job->X;
    Acc<KAHAN> acc;
    acc.zero();
    int bad = 0;
    for (int i = blk * kBlock + threadIdx.x; i < M; i += nblk * kBlock) {
        const float4 r = __ldg(X + i);
        const float x0 = apply_row(P, 0, r), x1 = apply_row(P, 1, r), x2 = apply_row(P, 2, r);
        Sums e;
        IterParams ip;
        ip.s1 = vip->s1;
        ip.s2 = vip->s2;
        ip.s3 = vip->s3;
        if constexpr (ST != kStoreF32) {
            ip.vscale = vip->vscale;
            ip.inv_vscale = vip->inv_vscale;
        }
        if constexpr (ST != kStoreF32 || SIG) {
            ip.ws1 = vip->ws1;
            ip.ws2 = vip->ws2;
            ip.ws3 = vip->ws3;
        }
        if (!slice_point<PT2PL, ST, SIG>(t, x0, x1, x2, ip, e, bad)) continue;
        ip.c_eff = vip->c_eff;
        ip.inv_sigma2 = vip->inv_sigma2;
        point_terms<PT2PL, SIG>(x0, x1, x2, e, ip, renorm, [&](int v, float x) { acc.add(v, x); });
    }
    if (bad) atomicOr(&st->flags, bad);
    block_partial<KAHAN>(acc, partials, blk, nblk);
    // The block's partial row is published by one thread: the barrier orders
    // the row's stores before thread 0's fence, whose release covers them.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int done_blocks = atomicAdd(&st->ticket, 1);
        last = done_blocks == nblk - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    if (SIG && sig_next)
        finish_iteration(partials, nblk, st, job->stop_twist, job, ipp, const_cast<IterParams *>(ipp) + 1);
    else
        finish_iteration(partials, nblk, st, job->stop_twist);
    if (threadIdx.x == 0) st->ticket = 0;
}

// A registration stops early once stop_twist was reached or a compact table
// overflowed (its result is discarded and it is rerun at the safe size).
__device__ __forceinline__ bool stopped(const DeviceState *st) {
    return __ldcg(&st->done) || (__ldcg(&st->flags) & kFlagCapacity);
}

template <bool PT2PL, bool KAHAN, int ST>
__global__ void __launch_bounds__(kBlock, 4) k_em_iter(IterLaunch L) {
    int b = blockIdx.x;
    if (b < L.gs) {
        if (L.check_done && stopped(L.st)) return;
        step_role<PT2PL, KAHAN, ST>(L.job, L.ip + L.it, L.step, L.partials, L.st, b, L.gs);
        return;
    }
    b -= L.gs;
    if (b < L.gv) {
        convert_role<PT2PL, ST>(L.conv, L.conv_list, L.ip + L.conv_it, b, L.gv);
        return;
    }
    b -= L.gv;
    if (b < L.gb) {
        if (L.check_done && stopped(L.st)) return;
        build_role<PT2PL, ST>(L.job, L.ip + L.build_it, L.build, L.build_list, L.st, b, L.gb);
        return;
    }
    b -= L.gb;
    if (b < L.gc) clear_role(L.clear, L.clear_list, __ldcg(&L.ip[L.clear_it].nvert), b, L.gc);
}

// Sigma as a decision variable (point-to-point, float32 records): the step
// of iteration `it` (whose last block also writes ip[it + 1]), or the build
// of an iteration at the sigma the previous step chose, and a clear.  The
// next sigma is known only once a step finishes, so steps and builds are
// separate launches.
template <bool KAHAN>
__global__ void __launch_bounds__(kBlock, 4) k_em_iter_sigma(IterLaunch L) {
    int b = blockIdx.x;
    if (b < L.gs) {
        if (L.check_done && stopped(L.st)) return;
        step_role<false, KAHAN, kStoreF32, true>(L.job, L.ip + L.it, L.step, L.partials, L.st, b, L.gs, L.sig_next);
        return;
    }
    b -= L.gs;
    if (b < L.gb) {
        if (L.check_done && stopped(L.st)) return;
        build_role<false, kStoreF32, true>(L.job, L.ip + L.build_it, L.build, L.build_list, L.st, b, L.gb);
        return;
    }
    b -= L.gb;
    if (b < L.gc) clear_role(L.clear, L.clear_list, __ldcg(&L.ip[L.clear_it].nvert), b, L.gc);
}

// Many registrations per launch: block b runs segment blockseg[b] -- one role
// of one slot (registration) at that slot's own iteration.  Used by the
// batched entry point (all slots in lockstep) and the serving loop (slots at
// different iterations).
template <bool PT2PL, bool KAHAN, int ST>
__global__ void __launch_bounds__(kBlock, 4) k_em_multi(const Slot *__restrict__ slots,
                                                         const Seg *__restrict__ segs,
                                                         const unsigned short *__restrict__ blockseg,
                                                         int check_done) {
    const Seg sg = segs[blockseg[blockIdx.x]];
    if (sg.role == kRoleNone) return;
    const Slot &sl = slots[sg.slot];
    DeviceState *st = sl.st;
    const int b = blockIdx.x - sg.blk0;
    if (sg.role == kRoleStep) {
        if (check_done && stopped(st)) return;
        step_role<PT2PL, KAHAN, ST>(sl.job, sl.ip + sg.it, sl.tab[sg.tab], sl.partials, st, b, sg.nblk);
    } else if (sg.role == kRoleBuild) {
        if (check_done && stopped(st)) return;
        build_role<PT2PL, ST>(sl.job, sl.ip + sg.it, sl.tab[sg.tab], sl.list[sg.tab], st, b, sg.nblk);
    } else if (sg.role == kRoleClear) {
        clear_role(sl.tab[sg.tab], sl.list[sg.tab], __ldcg(&sl.ip[sg.it].nvert), b, sg.nblk);
    } else if (sg.role == kRoleConvert) {
        convert_role<PT2PL, ST>(sl.tab[sg.tab], sl.list[sg.tab], sl.ip + sg.it, b, sg.nblk);
    }
}

// ---------------------------------------------------------------------------
// Articulated model (Section 5.1, Eq. 20, Algorithm 1)
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool in_subtree(const ArtTree &t, int b, int a) {  // b under or = a
    return (t.sub[a] >> b) & 1u;
}

// 3 x 4 row-major product C = A * B (float), B's implicit last row 0 0 0 1.
__device__ __forceinline__ void mul34(const float *A, const float *B, float *C) {
    float t[12];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            t[4 * i + j] = A[4 * i] * B[j] + A[4 * i + 1] * B[4 + j] + A[4 * i + 2] * B[8 + j] +
                           (j == 3 ? A[4 * i + 3] : 0.0f);
#pragma unroll
    for (int k = 0; k < 12; ++k) C[k] = t[k];
}

// Shared memory of the articulated tail (the float32 inverse is dead once the
// kinematics start, which reuse its space).
struct ArtTailSmem {
    ArtTree tree;                      // staged copy of the kinematic tree
    double q[kMaxJoints];              // joint angles before the update
    double S[kMaxBodies][21];          // subtree sums of J^T J (upper triangle) ...
    double sv[kMaxBodies][6];          // ... and of J^T r
    double cj[kMaxJoints][6];          // twist column of each joint
    double wj[kMaxJoints][6];          // S_{b(j)} c_j
    double A[kMaxDof][kMaxDof + 1];    // lower triangle of the normal matrix
    double y[kMaxDof];                 // right-hand side, then the solution
    double xr[kMaxDof], rr[kMaxDof];   // refined solution and its residual
    double diag[3];                    // weight sum, cost, count
    double sm_e[24];
    float sc[kMaxDof];                 // Jacobi scale 1 / sqrt(A_ii)
    float rs[kMaxDof], dz[kMaxDof];
    union {
        struct {
            float Ai[kMaxDof][kMaxDof + 1];    // inverse of the scaled matrix
            float v[2][kMaxDof + 1], u[2][kMaxDof + 1];  // rank-1 factors (double-buffered); v[.][kMaxDof] = pivot
        } gj;
        struct {
            float T[2][kMaxBodies][12];        // partial chains (ping-pong)
            float R[kMaxJoints][12];           // joint rotations
            float ja[kMaxJoints][3], jp[kMaxJoints][3];  // joint axis / point in the parent's frame
            int anc[2][kMaxBodies];
        } fk;
    } u;
    int use32, done, ok;
};

// Last block of an articulated step: the normal equations of Algorithm 1 from
// the subtree sums, the solve, the parameter update and the kinematics of
// the new pose.  With H_b, h_b the body sums and S_b, s_b their sums over the
// subtree of b, and c_j = (a_j; p_j x a_j) the twist column of joint j
// (shared by every body under the joint):
//   A_rr = S_root,  A_r,j = S_{b(j)} c_j,  g_r = s_root,  g_j = c_j . s_{b(j)},
//   A_jk = c_j^T S_d c_k  (d the deeper of b(j), b(k) when one is under the
//   other, else 0) -- the sum of J_sp^T (J^T J)_b J_sp over bodies.  With
//   w_j = S_{b(j)} c_j every A_jk is a dot product: w_j . c_k when b(j) is the
//   deeper body, c_j . w_k otherwise.
__device__ void art_finish(const ArtJob *job, ArtState *st, float stop_twist) {
    __shared__ ArtTailSmem sm;
    const int nb = job->tree.nb, nj = job->tree.nj, nd = 6 + nj;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Every global input is requested up front (one round trip to L2): the
    // subtree sums, the tree, the joint angles and the joint axes and points
    // of the current pose.
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&job->tree);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sm.tree);
        for (int w = tid; w < (int)(sizeof(ArtTree) / 4); w += kBlock) dst[w] = __ldg(src + w);
    }
    for (int e = tid; e < nb * kArtVals; e += kBlock) {
        const int b = e / kArtVals, v = e % kArtVals;
        const double x = __ldcg(&st->acc[b][v]);
        st->acc[b][v] = 0.0;                       // ready for the next iteration
        if (v < 21) sm.S[b][v] = x;
        else if (v < 27) sm.sv[b][v - 21] = x;
        else if (b == 0) sm.diag[v - 27] = x;      // the root's subtree is every body
    }
    for (int j = tid; j < nj; j += kBlock) {
        sm.q[j] = __ldcg(&st->q[j]);
        const double a0 = __ldcg(&st->jaxis[j][0]), a1 = __ldcg(&st->jaxis[j][1]), a2 = __ldcg(&st->jaxis[j][2]);
        const double p0 = __ldcg(&st->jpoint[j][0]), p1 = __ldcg(&st->jpoint[j][1]), p2 = __ldcg(&st->jpoint[j][2]);
        sm.cj[j][0] = a0; sm.cj[j][1] = a1; sm.cj[j][2] = a2;
        sm.cj[j][3] = p1 * a2 - p2 * a1;
        sm.cj[j][4] = p2 * a0 - p0 * a2;
        sm.cj[j][5] = p0 * a1 - p1 * a0;
    }
    __syncthreads();
    const ArtTree &t = sm.tree;
    auto Sx = [&](int b, int p, int q) { return p <= q ? sm.S[b][tri_index(p, q)] : sm.S[b][tri_index(q, p)]; };
    for (int e = tid; e < nj * 6; e += kBlock) {
        const int j = e / 6, p = e % 6, b = t.joint_body[j];
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < 6; ++q) s += Sx(b, p, q) * sm.cj[j][q];
        sm.wj[j][p] = s;
    }
    __syncthreads();
    // lower triangle of A (i >= j) and g
    const int nlow = nd * (nd + 1) / 2;
    for (int e = tid; e < nlow + nd; e += kBlock) {
        if (e >= nlow) {
            const int i = e - nlow;
            double gi;
            if (i < 6) {
                gi = sm.sv[0][i];
            } else {
                const int j = i - 6, b = t.joint_body[j];
                gi = 0.0;
                for (int p = 0; p < 6; ++p) gi += sm.cj[j][p] * sm.sv[b][p];
            }
            sm.y[i] = -gi;
            continue;
        }
        int i = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
        while (i * (i + 1) / 2 > e) --i;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int j = e - i * (i + 1) / 2;
        double a = 0.0;
        if (i < 6) {
            a = Sx(0, i, j);
        } else if (j < 6) {
            a = sm.wj[i - 6][j];
        } else {
            const int k1 = i - 6, k2 = j - 6, b1 = t.joint_body[k1], b2 = t.joint_body[k2];
            const double *u = nullptr, *v = nullptr;
            if (in_subtree(t, b1, b2)) { u = sm.wj[k1]; v = sm.cj[k2]; }
            else if (in_subtree(t, b2, b1)) { u = sm.cj[k1]; v = sm.wj[k2]; }
            if (u)
                for (int p = 0; p < 6; ++p) a += u[p] * v[p];
        }
        sm.A[i][j] = a;
    }
    __syncthreads();

    // ---- solve A dtheta = -g -----------------------------------------------
    // float64 answer by iterative refinement on the whole block: the
    // Jacobi-scaled matrix B = D A D (D = diag(1/sqrt(A_ii)), unit diagonal)
    // is inverted in float32 by Gauss-Jordan elimination (no pivoting: B is
    // symmetric positive definite), then x += D B^-1 D (y - A x) with the
    // residual in float64 until the error is below 1e-9 |x|.  A diagonal
    // entry at most 1e-12 of the largest, an elimination pivot below 1e-5 or
    // no convergence in 12 rounds hands the system to the float64 LDL^T,
    // whose pivot test decides degeneracy.
    if (warp == 0) {
        float md = 0.0f;
        for (int i = lane; i < nd; i += 32) md = fmaxf(md, (float)sm.A[i][i]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(kFull, md, o));
        bool good = md > 0.0f && md < 1e30f;
        for (int i = lane; i < nd; i += 32) {
            const float d = (float)sm.A[i][i];
            good = good && d > md * 1e-12f;
            sm.sc[i] = good ? rsqrtf(d) : 0.0f;
        }
        good = __all_sync(kFull, good);
        if (lane == 0) {
            sm.use32 = good;
            sm.done = 0;
        }
    }
    __syncthreads();
    if (sm.use32) {
        // Gauss-Jordan in registers.  Warp w holds rows w, w + 8, ... (slot
        // s), lane l columns l, l + 32.  A pivot step is the rank-1 update
        // a_ij -= u_i v_j with u_i = a_ik (u_k = p - 1) and v_j = a_kj / p
        // (v_k = 1 + 1/p), which gives row k / p, column k * (-1/p) and 1/p
        // at (k, k) with no per-entry case.  The warp owning row k rotates
        // its slots after each of its pivots, so its next pivot row is always
        // slot 0 (registers are never indexed by a run-time value).
        constexpr int kRows = (kMaxDof + 7) / 8, kCols = (kMaxDof + 31) / 32;
        float a[kRows][kCols];
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                const int i = warp + 8 * r, j = lane + 32 * c;
                a[r][c] = (i < nd && j < nd)
                              ? (float)(j <= i ? sm.A[i][j] : sm.A[j][i]) * sm.sc[i] * sm.sc[j]
                              : 0.0f;
            }
        for (int e = tid; e < 2 * (kMaxDof + 1); e += kBlock) {
            sm.u.gj.u[e / (kMaxDof + 1)][e % (kMaxDof + 1)] = 0.0f;
            sm.u.gj.v[e / (kMaxDof + 1)][e % (kMaxDof + 1)] = 0.0f;
        }
        __syncthreads();
        int row[kRows];  // row held in each slot (rotated with the slots)
#pragma unroll
        for (int r = 0; r < kRows; ++r) row[r] = warp + 8 * r;
        bool inverted = true;
        for (int k = 0; k < nd; ++k) {
            const int buf = k & 1, ck = k >> 5;
            if (lane == (k & 31)) {  // column k: u_i = a_ik
#pragma unroll
                for (int r = 0; r < kRows; ++r) {
                    const float x = ck ? a[r][kCols - 1] : a[r][0];
                    if (row[r] < nd) sm.u.gj.u[buf][row[r]] = (row[r] == k) ? x - 1.0f : x;
                }
            }
            if (warp == (k & 7)) {  // row k sits in slot 0
                const float p = __shfl_sync(kFull, ck ? a[0][kCols - 1] : a[0][0], k & 31);
                const float ip = 1.0f / p;
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    const int j = lane + 32 * c;
                    if (j < nd) sm.u.gj.v[buf][j] = (j == k) ? 1.0f + ip : a[0][c] * ip;
                }
                if (lane == 0) sm.u.gj.v[buf][kMaxDof] = p;
            }
            __syncthreads();
            if (!(sm.u.gj.v[buf][kMaxDof] > 1e-5f)) {  // the same pivot in every thread
                inverted = false;
                break;
            }
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                const float ui = sm.u.gj.u[buf][row[r]];
#pragma unroll
                for (int c = 0; c < kCols; ++c) a[r][c] = fmaf(-ui, sm.u.gj.v[buf][lane + 32 * c], a[r][c]);
            }
            if (warp == (k & 7)) {
#pragma unroll
                for (int c = 0; c < kCols; ++c) {
                    const float t0 = a[0][c];
#pragma unroll
                    for (int r = 0; r + 1 < kRows; ++r) a[r][c] = a[r + 1][c];
                    a[kRows - 1][c] = t0;
                }
                const int r0 = row[0];
#pragma unroll
                for (int r = 0; r + 1 < kRows; ++r) row[r] = row[r + 1];
                row[kRows - 1] = r0;
            }
        }
#pragma unroll
        for (int r = 0; r < kRows; ++r)
#pragma unroll
            for (int c = 0; c < kCols; ++c) {
                const int j = lane + 32 * c;
                if (row[r] < nd && j < nd) sm.u.gj.Ai[row[r]][j] = a[r][c];
            }
        __syncthreads();
        if (tid == 0) sm.done = 0;
        for (int i = tid; i < nd; i += kBlock) {
            sm.xr[i] = 0.0;
            sm.rr[i] = sm.y[i];
        }
        __syncthreads();
        float prev = 0.0f;  // |dz|^2 of the previous round (warp 0)
        for (int it = 0; it < 12 && inverted; ++it) {
            for (int i = tid; i < nd; i += kBlock) sm.rs[i] = (float)sm.rr[i] * sm.sc[i];
            __syncthreads();
            for (int i = warp; i < nd; i += kBlock / 32) {  // dz = D B^-1 D r, a warp per row
                float s = 0.0f;
                for (int j = lane; j < nd; j += 32) s += sm.u.gj.Ai[i][j] * sm.rs[j];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
                if (lane == 0) sm.dz[i] = s * sm.sc[i];
            }
            __syncthreads();
            if (warp == 0) {
                float dx2 = 0.0f, x2 = 0.0f;
                for (int i = lane; i < nd; i += 32) {
                    const double xi = sm.xr[i] + (double)sm.dz[i];
                    sm.xr[i] = xi;
                    dx2 += sm.dz[i] * sm.dz[i];
                    x2 += (float)xi * (float)xi;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    dx2 += __shfl_xor_sync(kFull, dx2, o);
                    x2 += __shfl_xor_sync(kFull, x2, o);
                }
                // Converged when this correction is below 1e-9 |x|, or when the
                // error it leaves -- |dz|^2 / |dz_prev| under the observed
                // contraction, if that is below 1e-2 -- is.
                const bool small = dx2 <= 1e-18f * x2;
                const bool fast = prev > 0.0f && dx2 < 1e-4f * prev && dx2 * (dx2 / prev) <= 1e-18f * x2;
                prev = dx2;
                if (lane == 0) sm.done = small || fast;
            }
            __syncthreads();
            if (sm.done) break;
            // r = y - A x in float64: four threads per row, seven columns each
            if (tid < 4 * nd) {
                const int i = tid >> 2, q = tid & 3;
                double s = 0.0;
                for (int j = q; j < nd; j += 4) s += (j <= i ? sm.A[i][j] : sm.A[j][i]) * sm.xr[j];
                s += __shfl_xor_sync(0xffffffffu >> (32 - min(32, 4 * nd - (tid & ~31))), s, 1);
                s += __shfl_xor_sync(0xffffffffu >> (32 - min(32, 4 * nd - (tid & ~31))), s, 2);
                if (q == 0) sm.rr[i] = sm.y[i] - s;
            }
            __syncthreads();
        }
        if (sm.done)
            for (int i = tid; i < nd; i += kBlock) sm.y[i] = sm.xr[i];
        __syncthreads();
    }
    if (warp == 0) {
        const bool done32 = sm.use32 && sm.done;
        bool okw = true;
        if (!done32) {  // float64 LDL^T (lane i owns rows i, i + 32)
            double md = 0.0;
            for (int i = 0; i < nd; ++i) md = fmax(md, sm.A[i][i]);
            const double fl = md * 1e-12;
            okw = md > 0.0;
            for (int k = 0; k < nd && okw; ++k) {
                const double d = sm.A[k][k];
                okw = d > fl;
                if (!okw) break;
                const double inv = rcp64(d);
                for (int i = k + 1 + lane; i < nd; i += 32) {  // Schur update of row i
                    const double aik = sm.A[i][k] * inv;
                    for (int j = k + 1; j <= i; ++j) sm.A[i][j] -= aik * sm.A[j][k];
                }
                __syncwarp();
                for (int i = k + 1 + lane; i < nd; i += 32) sm.A[i][k] *= inv;
                __syncwarp();
            }
            if (okw) {
                for (int k = 0; k < nd; ++k) {  // L z = rhs
                    for (int i = k + 1 + lane; i < nd; i += 32) sm.y[i] -= sm.A[i][k] * sm.y[k];
                    __syncwarp();
                }
                for (int i = lane; i < nd; i += 32) sm.y[i] *= rcp64(sm.A[i][i]);  // D w = z
                __syncwarp();
                for (int k = nd - 1; k >= 0; --k) {  // L^T x = w
                    for (int i = lane; i < k; i += 32) sm.y[i] -= sm.A[k][i] * sm.y[k];
                    __syncwarp();
                }
            }
        }
        if (lane == 0) sm.ok = okw;
    }
    __syncthreads();
    const bool ok = sm.ok;
    // parameter update (warp 0 for the root exponential), diagnostics
    if (warp == 0) {
        if (lane == 0) {
            st->ds.iters_run += 1;
            st->ds.sum_w = sm.diag[0];
            st->ds.cost = sm.diag[1];
            st->ds.inliers = (long long)(sm.diag[2] + 0.5);
            if (!ok) st->ds.degenerate += 1;
        }
        if (ok) {
            warp_se3_update(lane < 6 ? sm.y[lane] : 0.0, st->root_T, sm.sm_e);
            float n2 = 0.0f;
            for (int i = lane; i < nd; i += 32) n2 += (float)sm.y[i] * (float)sm.y[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(kFull, n2, o);
            if (lane == 0) {
                st->ds.twist_norm = sqrtf(n2);
                if (stop_twist > 0.0f && sqrtf(n2) < stop_twist) st->ds.done = 1;
            }
        }
    } else if (ok) {
        for (int j = tid - 32; j < nj; j += kBlock - 32) {
            double qj = sm.q[j] + sm.y[6 + j];
            qj = fmin(fmax(qj, t.q_min[j]), t.q_max[j]);
            st->q[j] = qj;
            sm.q[j] = qj;
        }
    }
    __syncthreads();

    // ---- forward kinematics in float -----------------------------------------
    // Body b's pose is T_parent * L_b with L_b = offset_b * R(q_j) ... over its
    // joints (body 0: root_T * offset_0 * ...).  Every L_b is formed at once,
    // then the chains are composed by pointer jumping (log2 of the depth
    // rounds); each joint's world axis and point follow from its parent's pose.
    for (int j = tid; j < nj; j += kBlock) {
        const float *a = t.axis[j];
        float sn, cs;
        sincosf((float)sm.q[j], &sn, &cs);
        const float v = 1.0f - cs;
        float *R = sm.u.fk.R[j];
        R[0] = cs + a[0] * a[0] * v;        R[1] = a[0] * a[1] * v - a[2] * sn; R[2] = a[0] * a[2] * v + a[1] * sn;
        R[4] = a[1] * a[0] * v + a[2] * sn; R[5] = cs + a[1] * a[1] * v;        R[6] = a[1] * a[2] * v - a[0] * sn;
        R[8] = a[2] * a[0] * v - a[1] * sn; R[9] = a[2] * a[1] * v + a[0] * sn; R[10] = cs + a[2] * a[2] * v;
        R[3] = R[7] = R[11] = 0.0f;
    }
    __syncthreads();
    for (int b = tid; b < nb; b += kBlock) {
        float F[12];
        if (b == 0) {
            float Rt[12];
            for (int k = 0; k < 12; ++k) Rt[k] = (float)st->root_T[k];
            mul34(Rt, t.offset[0], F);
        } else {
            for (int k = 0; k < 12; ++k) F[k] = t.offset[b][k];
        }
        for (int j = t.joint_begin[b]; j < t.joint_begin[b + 1]; ++j) {
            const float *a = t.axis[j];
            for (int r = 0; r < 3; ++r) {  // in the parent's frame (world for body 0)
                sm.u.fk.ja[j][r] = F[4 * r] * a[0] + F[4 * r + 1] * a[1] + F[4 * r + 2] * a[2];
                sm.u.fk.jp[j][r] = F[4 * r + 3];
            }
            mul34(F, sm.u.fk.R[j], F);
        }
        for (int k = 0; k < 12; ++k) sm.u.fk.T[0][b][k] = F[k];
        sm.u.fk.anc[0][b] = b == 0 ? -1 : t.parent[b];
    }
    __syncthreads();
    int cur = 0;
    for (int round = 0; round < 5; ++round) {  // depth < 32
        for (int b = tid; b < nb; b += kBlock) {
            const int a = sm.u.fk.anc[cur][b];
            if (a >= 0) {
                mul34(sm.u.fk.T[cur][a], sm.u.fk.T[cur][b], sm.u.fk.T[cur ^ 1][b]);
                sm.u.fk.anc[cur ^ 1][b] = sm.u.fk.anc[cur][a];
            } else {
                for (int k = 0; k < 12; ++k) sm.u.fk.T[cur ^ 1][b][k] = sm.u.fk.T[cur][b][k];
                sm.u.fk.anc[cur ^ 1][b] = -1;
            }
        }
        __syncthreads();
        cur ^= 1;
    }
    for (int e = tid; e < nb * 12; e += kBlock) st->body_T[e / 12][e % 12] = sm.u.fk.T[cur][e / 12][e % 12];
    for (int j = tid; j < nj; j += kBlock) {
        const int b = t.joint_body[j];
        if (b == 0) {
            for (int r = 0; r < 3; ++r) {
                st->jaxis[j][r] = sm.u.fk.ja[j][r];
                st->jpoint[j][r] = sm.u.fk.jp[j][r];
            }
        } else {
            const float *P = sm.u.fk.T[cur][t.parent[b]];
            const float *a = sm.u.fk.ja[j], *p = sm.u.fk.jp[j];
            for (int r = 0; r < 3; ++r) {
                st->jaxis[j][r] = P[4 * r] * a[0] + P[4 * r + 1] * a[1] + P[4 * r + 2] * a[2];
                st->jpoint[j][r] = P[4 * r] * p[0] + P[4 * r + 1] * p[1] + P[4 * r + 2] * p[2] + P[4 * r + 3];
            }
        }
    }
}

// Articulated step: slice at x = T_{b(i)} x_ref (body poses staged in shared
// memory), the same point terms as the rigid step, summed per body (Algorithm
// 1): thread registers while the body is unchanged, then one warp reduction
// per body present in the warp into shared memory, then float64 atomics per
// touched body.  Each
// block takes a contiguous range of points (points sorted by body keep the
// flushes rare).
template <bool PT2PL, int ST>
__device__ void art_step_role(const ArtLaunch &L, int blk, int nblk) {
    __shared__ float Tb[kMaxBodies][12];
    __shared__ float sacc[kMaxBodies][kArtVals];
    __shared__ int last;
    const ArtJob *job = L.job;
    ArtState *st = L.st;
    const int nb = job->tree.nb;
    for (int e = threadIdx.x; e < nb * 12; e += kBlock) Tb[e / 12][e % 12] = st->body_T[e / 12][e % 12];
    for (int e = threadIdx.x; e < nb * kArtVals; e += kBlock) sacc[e / kArtVals][e % kArtVals] = 0.0f;
    __syncthreads();
    const IterParams ip = L.ip[L.it];
    const int M = job->base.M;
    const int renorm = job->base.renormalize;
    const int chunk = (M + nblk - 1) / nblk;
    const int start = blk * chunk, end = min(M, start + chunk);
    float acc[kArtVals];
#pragma unroll
    for (int v = 0; v < kArtVals; ++v) acc[v] = 0.0f;
    int cur = -1, bad = 0;
    auto flush_lane = [&](int b) {
#pragma unroll
        for (int v = 0; v < kArtVals; ++v) atomicAdd(&sacc[b][v], acc[v]);
    };
    for (int i = start + threadIdx.x; i < end; i += kBlock) {
        const int b = __ldg(job->body + i);
        if (b < 0 || b >= nb) {
            bad |= kFlagRange;
            continue;
        }
        if (b != cur) {
            if (cur >= 0) flush_lane(cur);
#pragma unroll
            for (int v = 0; v < kArtVals; ++v) acc[v] = 0.0f;
            cur = b;
        }
        const float4 r = __ldg(job->base.X + i);
        const float x0 = apply_row(Tb[b], 0, r), x1 = apply_row(Tb[b], 1, r), x2 = apply_row(Tb[b], 2, r);
        Sums e;
        if (!slice_point<PT2PL, ST>(L.step, x0, x1, x2, ip, e, bad)) continue;
        point_terms<PT2PL>(x0, x1, x2, e, ip, renorm, [&](int v, float x) { acc[v] += x; });
    }
    // One warp reduction per distinct body among the lanes (lanes without a
    // point, or of another body, add zeros): conflicting per-lane shared
    // atomics on one body's sums would serialise 32 ways.
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(kFull, cur >= 0);
    while (pending) {
        const int bb = __shfl_sync(kFull, cur, __ffs(pending) - 1);
        const bool mine = cur == bb;
        float x[32];
#pragma unroll
        for (int v = 0; v < 32; ++v) x[v] = (v < kArtVals && mine) ? acc[v] : 0.0f;
        const float sum = warp_sum32(x);
        if (lane < kArtVals) atomicAdd(&sacc[bb][lane], sum);
        pending &= ~__ballot_sync(kFull, mine);
    }
    if (bad) atomicOr(&st->ds.flags, bad);
    __syncthreads();
    // The tail needs only subtree sums (S_b over the bodies under b): each
    // block adds its sums of every subtree that holds one of its points.
    for (int e = threadIdx.x; e < nb * kArtVals; e += kBlock) {
        const int b = e / kArtVals, v = e % kArtVals;
        float sum = 0.0f, cnt = 0.0f;
        for (unsigned m = __ldg(&job->tree.sub[b]); m; m &= m - 1) {
            const int c = __ffs(m) - 1;
            sum += sacc[c][v];
            cnt += sacc[c][kArtVals - 1];
        }
        if (cnt > 0.0f) atomicAdd(&st->acc[b][v], (double)sum);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->ds.ticket, 1) == nblk - 1;
        if (last) __threadfence();
    }
    __syncthreads();
    if (!last) return;
    art_finish(job, st, job->base.stop_twist);
    if (threadIdx.x == 0) st->ds.ticket = 0;
}

template <bool PT2PL, int ST>
__global__ void __launch_bounds__(kBlock, 3) k_art_iter(ArtLaunch L) {
    int b = blockIdx.x;
    if (b < L.gs) {
        if (stopped(&L.st->ds)) return;
        art_step_role<PT2PL, ST>(L, b, L.gs);
        return;
    }
    b -= L.gs;
    if (b < L.gv) {
        convert_role<PT2PL, ST>(L.conv, L.conv_list, L.ip + L.conv_it, b, L.gv);
        return;
    }
    b -= L.gv;
    if (b < L.gb) {
        if (stopped(&L.st->ds)) return;
        build_role<PT2PL, ST>(&L.job->base, L.ip + L.build_it, L.build, L.build_list, &L.st->ds, b, L.gb);
        return;
    }
    b -= L.gb;
    if (b < L.gc) clear_role(L.clear, L.clear_list, __ldcg(&L.ip[L.clear_it].nvert), b, L.gc);
}

struct ClearSet {
    Table t[3];
    const int *list[3];
    const int *count[3];
};

__global__ void k_clear_lists(ClearSet c, int n) {
    const int per = gridDim.x / n;
    const int which = blockIdx.x / per;
    if (which >= n) return;
    clear_role(c.t[which], c.list[which], __ldcg(c.count[which]), blockIdx.x % per, per);
}

// One blur pass writes every record of `out` (a separate record array of at
// least in.mask + 1 slots): the key copied (free slots stay free) and the
// values v + (v(n-) + v(n+)) / 2 along axis `dir`, missing neighbours 0.
__global__ void k_blur_pass(Table in, Table out, int dir, const DeviceState *st) {
    if (st && st->done) return;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t s = gtid(); s <= in.mask; s += grid_stride()) {
        const unsigned long long key = __ldg(rec_key(in.keys, s));
        float4 *o = reinterpret_cast<float4 *>(rec_key(out.keys, s));
        if (key == kEmpty) {
            o[0] = z;
            o[1] = z;
            o[2] = z;
            o[3] = z;
            continue;
        }
        const int sm = find_key(in.keys, in.mask, neighbour_key(key, dir, -1), in.max_probe);
        const int sp = find_key(in.keys, in.mask, neighbour_key(key, dir, +1), in.max_probe);
        float4 a = __ldg(rec_v0(in.keys, s));
        if (sm >= 0) {
            const float4 u = __ldg(rec_v0(in.keys, sm));
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
        }
        if (sp >= 0) {
            const float4 u = __ldg(rec_v0(in.keys, sp));
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
        }
        float4 c = z;
        if (in.vals > 4) {
            c = __ldg(rec_v1(in.keys, s));
            if (sm >= 0) {
                const float4 u = __ldg(rec_v1(in.keys, sm));
                c.x += 0.5f * u.x; c.y += 0.5f * u.y; c.z += 0.5f * u.z; c.w += 0.5f * u.w;
            }
            if (sp >= 0) {
                const float4 u = __ldg(rec_v1(in.keys, sp));
                c.x += 0.5f * u.x; c.y += 0.5f * u.y; c.z += 0.5f * u.z; c.w += 0.5f * u.w;
            }
        }
        reinterpret_cast<unsigned long long *>(o)[0] = key;
        reinterpret_cast<unsigned long long *>(o)[1] = 0ull;
        o[1] = a;   // v0
        o[2] = c;   // v1
        o[3] = z;
    }
}

// The same pass over the slots a build listed (the table's every vertex)
// instead of the whole table: `out` holds the same keys at the same slots as
// `in` after the pass, so lookups in either find the same vertices, and it is
// empty elsewhere -- the caller frees the listed slots of the scratch table
// once the last pass has read it.
__global__ void k_blur_list(Table in, Table out, int dir, const int *list, const int *count,
                            const DeviceState *st) {
    if (st && st->done) return;
    const int n = __ldcg(count);
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = gtid(); e < n; e += grid_stride()) {
        const uint32_t s = (uint32_t)__ldcg(list + e);
        const unsigned long long key = __ldg(rec_key(in.keys, s));
        const int sm = find_key(in.keys, in.mask, neighbour_key(key, dir, -1), in.max_probe);
        const int sp = find_key(in.keys, in.mask, neighbour_key(key, dir, +1), in.max_probe);
        float4 a = __ldg(rec_v0(in.keys, s));
        float4 c = in.vals > 4 ? __ldg(rec_v1(in.keys, s)) : z;
        if (sm >= 0) {
            const float4 u = __ldg(rec_v0(in.keys, sm));
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
            if (in.vals > 4) {
                const float4 v = __ldg(rec_v1(in.keys, sm));
                c.x += 0.5f * v.x; c.y += 0.5f * v.y; c.z += 0.5f * v.z; c.w += 0.5f * v.w;
            }
        }
        if (sp >= 0) {
            const float4 u = __ldg(rec_v0(in.keys, sp));
            a.x += 0.5f * u.x; a.y += 0.5f * u.y; a.z += 0.5f * u.z; a.w += 0.5f * u.w;
            if (in.vals > 4) {
                const float4 v = __ldg(rec_v1(in.keys, sp));
                c.x += 0.5f * v.x; c.y += 0.5f * v.y; c.z += 0.5f * v.z; c.w += 0.5f * v.w;
            }
        }
        float4 *o = reinterpret_cast<float4 *>(rec_key(out.keys, s));
        reinterpret_cast<unsigned long long *>(o)[0] = key;
        reinterpret_cast<unsigned long long *>(o)[1] = 0ull;
        o[1] = a;
        o[2] = c;
        o[3] = z;
    }
}

// E-step sums at T x for every model point (the fr_estep entry point).
template <bool PT2PL, int ST>
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
        const float x0 = apply_row(P, 0, r), x1 = apply_row(P, 1, r), x2 = apply_row(P, 2, r);
        Sums e;
        slice_point<PT2PL, ST>(t, x0, x1, x2, ip, e, bad);
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
            red_add4(rec_v0(t.keys, s), b * v[0], b * v[1], b * v[2], b * v[3]);
            if (vdim > 4) red_add4(rec_v1(t.keys, s), b * v[4], b * v[5], b * v[6], b * v[7]);
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
            find4(t.keys, t.mask, sx, slot, t.max_probe);
#pragma unroll
            for (int k = 0; k < kD; ++k) {
                if (slot[k] < 0) continue;
                const float b = sx.b[k];
                const float4 a = __ldg(rec_v0(t.keys, slot[k]));
                acc[0] += b * a.x; acc[1] += b * a.y; acc[2] += b * a.z; acc[3] += b * a.w;
                if (vdim > 4) {
                    const float4 c = __ldg(rec_v1(t.keys, slot[k]));
                    acc[4] += b * c.x; acc[5] += b * c.y; acc[6] += b * c.z; acc[7] += b * c.w;
                }
            }
        } else {
            atomicOr(flags, kFlagRange);
        }
        for (int c = 0; c < vdim; ++c) out[(size_t)i * vdim + c] = acc[c];
    }
}

// Zeroes the values (and 16-bit record) of every slot, keeping the keys.
__global__ void k_zero_values(Table t) {
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t s = gtid(); s <= t.mask; s += grid_stride()) {
        *rec_v0(t.keys, s) = z;
        *rec_v1(t.keys, s) = z;
    }
}

__global__ void k_vertices(Table t, int vdim, int *keys_out, float *vals_out, int *count) {
    for (uint32_t s = gtid(); s <= t.mask; s += grid_stride()) {
        const unsigned long long key = *rec_key(t.keys, s);
        if (key == kEmpty) continue;
        const int o = atomicAdd(count, 1);
        int c[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) c[j] = unpack_coord(key, j);
        reinterpret_cast<int4 *>(keys_out)[o] = make_int4(c[0], c[1], c[2], -(c[0] + c[1] + c[2]));
        if (vals_out) {
            const float4 a = *rec_v0(t.keys, s);
            const float4 b = t.vals > 4 ? *rec_v1(t.keys, s) : make_float4(0.f, 0.f, 0.f, 0.f);
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


// ---------------------------------------------------------------------------
// Node-graph model (Section 5.2, Eq. 21)
// ---------------------------------------------------------------------------

// Tuple positions of the 10 node pairs, and row / column of the 21
// upper-triangle entries of a 6 x 6 block (tri_index order).
__constant__ unsigned char c_pair_i[kNgPairs] = {0, 0, 0, 0, 1, 1, 1, 2, 2, 3};
__constant__ unsigned char c_pair_j[kNgPairs] = {0, 1, 2, 3, 1, 2, 3, 2, 3, 3};
__constant__ unsigned char c_tri_r[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
__constant__ unsigned char c_tri_c[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};

// Eq. 21: the dual-quaternion blend of a point's 4 node poses -- each
// node's dual quaternion sign-aligned with the largest-weight node's (the
// first such), the sum divided by the norm of its real part -- as a
// rotation R (row-major) and a translation t = 2 (r0 d - d0 r + r x d).
__device__ __forceinline__ void ng_blend(const float (&q)[4][8], const float (&w)[4], float R[9],
                                         float t[3]) {
    int ref = 0;
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (w[k] > w[ref]) ref = k;
    float r0 = q[0][0], r1 = q[0][1], r2 = q[0][2], r3 = q[0][3];
#pragma unroll
    for (int k = 1; k < 4; ++k)
        if (ref == k) {
            r0 = q[k][0];
            r1 = q[k][1];
            r2 = q[k][2];
            r3 = q[k][3];
        }
    float b[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float dot = q[k][0] * r0 + q[k][1] * r1 + q[k][2] * r2 + q[k][3] * r3;
        const float sw = dot < 0.0f ? -w[k] : w[k];
#pragma unroll
        for (int a = 0; a < 8; ++a) b[a] += sw * q[k][a];
    }
    const float inv = 1.0f / sqrtf(b[0] * b[0] + b[1] * b[1] + b[2] * b[2] + b[3] * b[3]);
    const float qw = b[0] * inv, qx = b[1] * inv, qy = b[2] * inv, qz = b[3] * inv;
    const float d0 = b[4] * inv, dx = b[5] * inv, dy = b[6] * inv, dz = b[7] * inv;
    R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    R[1] = 2.0f * (qx * qy - qw * qz);
    R[2] = 2.0f * (qx * qz + qw * qy);
    R[3] = 2.0f * (qx * qy + qw * qz);
    R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
    R[5] = 2.0f * (qy * qz - qw * qx);
    R[6] = 2.0f * (qx * qz - qw * qy);
    R[7] = 2.0f * (qy * qz + qw * qx);
    R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
    t[0] = 2.0f * (qw * dx - d0 * qx + (qy * dz - qz * dy));
    t[1] = 2.0f * (qw * dy - d0 * qy + (qz * dx - qx * dz));
    t[2] = 2.0f * (qw * dz - d0 * qz + (qx * dy - qy * dx));
}

// One warp per segment (a run of points sharing their 4 nodes): each lane
// warps a point (Eq. 21), slices the lattice at it (E step) and forms its
// rigid-model terms H = J^T J (21), h = J^T r (6) (Eq. 7 / Eq. 10); the
// warp then sums, over the segment, w_i w_j H for the 10 node pairs and
// w_i h for the 4 nodes (the point twist is the weighted sum of its node
// twists, so d r / d zeta_k = w_k J) through shared memory -- 234 sums, 8
// per lane -- and adds them to the pair blocks of A and to g.  With
// warp_only the kernel writes the warped points and stops.
template <bool PT2PL, int ST>
__global__ void __launch_bounds__(kBlock) k_ng_points(NgPoints L, int warp_only) {
    constexpr int kWarps = kBlock / 32;
    __shared__ float sh[kWarps][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = blockIdx.x * kWarps + warp;
    if (seg >= L.S) return;  // whole warps only: no block-wide barrier below
    const int p0 = L.seg_start[seg], p1 = L.seg_start[seg + 1];
    const int4 nd = L.seg_nodes[seg];
    const int nodes[4] = {nd.x, nd.y, nd.z, nd.w};
    float q[4][8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(L.node_dq) + 2 * nodes[k]);
        const float4 c = __ldg(reinterpret_cast<const float4 *>(L.node_dq) + 2 * nodes[k] + 1);
        q[k][0] = a.x; q[k][1] = a.y; q[k][2] = a.z; q[k][3] = a.w;
        q[k][4] = c.x; q[k][5] = c.y; q[k][6] = c.z; q[k][7] = c.w;
    }
    // this lane's sums o = lane + 32 m: products of shared columns ca * cb * cv
    // (columns 0..20 H, 21..26 h, 27..30 weights, 31 the constant 1)
    int ca[8], cb[8], cv[8];
    float acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int o = lane + 32 * m;
        acc[m] = 0.0f;
        if (o < kNgPairs * 21) {
            const int pr = o / 21, e = o % 21;
            ca[m] = 27 + c_pair_i[pr];
            cb[m] = 27 + c_pair_j[pr];
            cv[m] = e;
        } else if (o < kNgPairs * 21 + 24) {
            const int n = (o - kNgPairs * 21) / 6, c = (o - kNgPairs * 21) % 6;
            ca[m] = 27 + n;
            cb[m] = 31;
            cv[m] = 21 + c;
        } else {
            ca[m] = cb[m] = cv[m] = 31;
        }
    }
    IterParams ip{};
    if (!warp_only) ip = *L.ip;
    float sum_w = 0.0f, cost = 0.0f;
    int inl = 0, bad = 0;
    float(*row)[33] = sh[warp];
    for (int base = p0; base < p1; base += 32) {
        const int i = base + lane;
        float v[31];
#pragma unroll
        for (int c = 0; c < 31; ++c) v[c] = 0.0f;
        if (i < p1) {
            const float4 xr = L.X[i];
            const float4 wt = L.w[i];
            const float w4[4] = {wt.x, wt.y, wt.z, wt.w};
            float R[9], t[3];
            ng_blend(q, w4, R, t);
            const float x0 = R[0] * xr.x + R[1] * xr.y + R[2] * xr.z + t[0];
            const float x1 = R[3] * xr.x + R[4] * xr.y + R[5] * xr.z + t[1];
            const float x2 = R[6] * xr.x + R[7] * xr.y + R[8] * xr.z + t[2];
            if (warp_only) {
                L.warp_out[L.perm[i]] = make_float4(x0, x1, x2, 0.0f);
            } else {
                Sums e;
                if (slice_point<PT2PL, ST>(L.tab, x0, x1, x2, ip, e, bad)) {
                    float tv[kRigidVals];
#pragma unroll
                    for (int c = 0; c < kRigidVals; ++c) tv[c] = 0.0f;
                    if (point_terms<PT2PL>(x0, x1, x2, e, ip, L.renorm, [&](int c, float a) { tv[c] += a; })) {
#pragma unroll
                        for (int c = 0; c < 27; ++c) v[c] = tv[c];
                        sum_w += tv[27];
                        cost += tv[28];
                        ++inl;
                    }
                }
                v[27] = w4[0];
                v[28] = w4[1];
                v[29] = w4[2];
                v[30] = w4[3];
            }
        }
        if (warp_only) continue;
#pragma unroll
        for (int c = 0; c < 31; ++c) row[lane][c] = v[c];
        row[lane][31] = 1.0f;
        __syncwarp();
        const int cnt = min(32, p1 - base);
        for (int pt = 0; pt < cnt; ++pt) {
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] += row[pt][ca[m]] * row[pt][cb[m]] * row[pt][cv[m]];
        }
        __syncwarp();
    }
    if (warp_only) return;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int o = lane + 32 * m;
        if (o < kNgPairs * 21) {
            const int pr = o / 21, e = o % 21;
            const int blk = L.seg_blk[seg * kNgPairs + pr];
            const float val = L.seg_coef[seg * kNgPairs + pr] * acc[m];
            const int r = c_tri_r[e], c = c_tri_c[e];
            atomicAdd(L.blocks + (size_t)blk * 36 + r * 6 + c, val);
            if (r != c) atomicAdd(L.blocks + (size_t)blk * 36 + c * 6 + r, val);
        } else if (o < kNgPairs * 21 + 24) {
            const int n = (o - kNgPairs * 21) / 6, c = (o - kNgPairs * 21) % 6;
            atomicAdd(L.g + 6 * nodes[n] + c, acc[m]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum_w += __shfl_xor_sync(kFull, sum_w, o);
        cost += __shfl_xor_sync(kFull, cost, o);
        inl += __shfl_xor_sync(kFull, inl, o);
        bad |= __shfl_xor_sync(kFull, bad, o);
    }
    if (lane == 0) {
        atomicAdd(L.stats, (double)sum_w);
        atomicAdd(L.stats + 1, (double)cost);
        if (inl) atomicAdd(L.inliers, (unsigned long long)inl);
        if (bad) atomicOr(L.flags, bad);
    }
}

// The regulariser, one thread per directed edge (j, k):
// r = s (T_j p_k - T_k p_k), s = sqrt(lambda) / sigma, with
// d r / d zeta_j = s [-[T_j p_k]_x, I] and d r / d zeta_k = -s [-[T_k p_k]_x, I];
// adds J_j^T J_j, J_k^T J_k, the cross block and J^T r.
__global__ void __launch_bounds__(kBlock) k_ng_edges(NgEdges L) {
    const int e = gtid();
    double rr = 0.0;
    if (e < L.E) {
        const int2 jk = L.edges[e];
        const double s = sqrt(L.lambda) / (double)L.ip->sigma;
        const double *Tj = L.node_T + 16 * jk.x, *Tk = L.node_T + 16 * jk.y;
        const double *pk = L.node_pos + 3 * jk.y;
        // the two predictions of node k's position and their difference in
        // float64 (they nearly cancel); the Jacobian terms in float32, which
        // is what the float block sums keep of them
        float a[3], b[3], r[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double ad = Tj[4 * c] * pk[0] + Tj[4 * c + 1] * pk[1] + Tj[4 * c + 2] * pk[2] + Tj[4 * c + 3];
            const double bd = Tk[4 * c] * pk[0] + Tk[4 * c + 1] * pk[1] + Tk[4 * c + 2] * pk[2] + Tk[4 * c + 3];
            const double rd = s * (ad - bd);
            rr += rd * rd;
            a[c] = (float)(s * ad);
            b[c] = (float)(s * bd);
            r[c] = (float)rd;
        }
        const float sf = (float)s;
        const float Jj[3][6] = {{0.0f, a[2], -a[1], sf, 0.0f, 0.0f},
                                {-a[2], 0.0f, a[0], 0.0f, sf, 0.0f},
                                {a[1], -a[0], 0.0f, 0.0f, 0.0f, sf}};
        const float Jk[3][6] = {{0.0f, -b[2], b[1], -sf, 0.0f, 0.0f},
                                {b[2], 0.0f, -b[0], 0.0f, -sf, 0.0f},
                                {-b[1], b[0], 0.0f, 0.0f, 0.0f, -sf}};
        const int *eb = L.edge_blk + 3 * e;
        float *Bjj = L.blocks + (size_t)eb[0] * 36, *Bkk = L.blocks + (size_t)eb[1] * 36;
        float *Bx = L.blocks + (size_t)eb[2] * 36;
        const bool j_first = jk.x < jk.y;
#pragma unroll
        for (int p = 0; p < 6; ++p) {
            float gj = 0.0f, gk = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gj += Jj[c][p] * r[c];
                gk += Jk[c][p] * r[c];
            }
            atomicAdd(L.g + 6 * jk.x + p, gj);
            atomicAdd(L.g + 6 * jk.y + p, gk);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                float mjj = 0.0f, mkk = 0.0f, mjk = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    mjj += Jj[c][p] * Jj[c][q];
                    mkk += Jk[c][p] * Jk[c][q];
                    mjk += Jj[c][p] * Jk[c][q];
                }
                atomicAdd(Bjj + 6 * p + q, mjj);
                atomicAdd(Bkk + 6 * p + q, mkk);
                // block (min, max) holds rows of the smaller node: J_j^T J_k, or its transpose
                atomicAdd(Bx + (j_first ? 6 * p + q : 6 * q + p), mjk);
            }
        }
    }
    // the regulariser's cost: one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rr += __shfl_xor_sync(kFull, rr, o);
    if ((threadIdx.x & 31) == 0 && rr != 0.0) atomicAdd(L.stats + 1, rr);
}

// Sum of v over the grid: every block adds its partial; the last block to
// finish totals the partials with all its threads (a fixed order: thread t
// takes partials t, t + blockDim, ..., then a fixed tree) and returns true
// in its thread 0 with *total set.
__device__ __forceinline__ bool ng_grid_sum(double v, double *partial, int *ticket, double &total) {
    __shared__ double s_w[kBlock / 32];
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_w[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += s_w[w];
        partial[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return false;
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partial + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    __syncthreads();
    if (lane == 0) s_w[warp] = t;
    __syncthreads();
    if (threadIdx.x != 0) return false;
    double tt = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += s_w[w];
    total = tt;
    *ticket = 0;
    return true;
}

// Lane layout of the per-node PCG kernels: node `node` (of warp-group grp)
// component `i`; `base` is the group's first lane.  Lanes past the last node
// (and lanes 30, 31) are inactive but still take part in the shuffles.
struct NgLane {
    int node, i, base;
    bool active;
};

__device__ __forceinline__ NgLane ng_lane(int K) {
    const int lane = threadIdx.x & 31, grp = lane / 6;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    NgLane l;
    l.node = warp * kNgNodesPerWarp + grp;
    l.i = lane - 6 * grp;
    l.base = 6 * grp;
    l.active = grp < kNgNodesPerWarp && l.node < K;
    return l;
}

// Component c of a node's 6-vector whose component i sits in lane base + i.
__device__ __forceinline__ double ng_comp(double v, const NgLane &l, int c) {
    return __shfl_sync(kFull, v, (l.base + c) & 31);
}

// PCG set-up: the float64 copy of the blocks, P_k = (A_kk)^-1 by Cholesky
// (pivot floor 1e-12 of the largest diagonal entry; a block below it gets
// 1 / that entry), x = 0, r = -g, z = P r, rz = r.z.  The six lanes of a
// node factor its block alike; lane i then solves for column i of the
// inverse.
__global__ void __launch_bounds__(kNgPcgBlock) k_ng_pcg_init(NgPcg L) {
    for (int e = gtid(); e < L.nnzb * 36; e += grid_stride()) L.blocks_d[e] = (double)L.blocks[e];
    const NgLane l = ng_lane(L.K);
    double dot = 0.0;
    double ri = 0.0, zi = 0.0;
    double Pc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // column i of P (= row i)
    if (l.active) {
        const float *B = L.blocks + (size_t)L.diag_blk[l.node] * 36;
        double Lc[36];
        double dmax = 0.0;
        for (int a = 0; a < 6; ++a) dmax = fmax(dmax, (double)B[7 * a]);
        bool ok = dmax > 0.0;
        const double fl = dmax * 1e-12;
        for (int r = 0; r < 6 && ok; ++r)
            for (int c = 0; c <= r; ++c) {
                double sacc = (double)B[6 * r + c];
                for (int m = 0; m < c; ++m) sacc -= Lc[6 * r + m] * Lc[6 * c + m];
                if (r == c) {
                    if (!(sacc > fl)) { ok = false; break; }
                    Lc[6 * r + r] = sqrt(sacc);
                } else {
                    Lc[6 * r + c] = sacc / Lc[6 * c + c];
                }
            }
        if (ok) {
            double y[6];
            for (int r = 0; r < 6; ++r) {  // L y = e_i
                double sacc = (r == l.i) ? 1.0 : 0.0;
                for (int m = 0; m < r; ++m) sacc -= Lc[6 * r + m] * y[m];
                y[r] = sacc / Lc[6 * r + r];
            }
            for (int r = 5; r >= 0; --r) {  // L^T x = y
                double sacc = y[r];
                for (int m = r + 1; m < 6; ++m) sacc -= Lc[6 * m + r] * Pc[m];
                Pc[r] = sacc / Lc[6 * r + r];
            }
        } else {
            for (int r = 0; r < 6; ++r) Pc[r] = (r == l.i) ? (dmax > 0.0 ? 1.0 / dmax : 1.0) : 0.0;
        }
        double *Pk = L.P + 36 * (size_t)l.node;
        for (int r = 0; r < 6; ++r) Pk[6 * r + l.i] = Pc[r];
        ri = -(double)L.g[6 * l.node + l.i];
        L.r[6 * l.node + l.i] = ri;
        L.x[6 * l.node + l.i] = 0.0;
    }
    __syncwarp();  // the node's P is complete (written by its six lanes)
    // z_i = sum_c P_ic r_c
    const double *Pk = L.P + 36 * (size_t)(l.active ? l.node : 0);
    for (int c = 0; c < 6; ++c) {
        const double rc = ng_comp(ri, l, c);
        if (l.active) zi += Pk[6 * l.i + c] * rc;
    }
    if (l.active) {
        L.z[6 * l.node + l.i] = zi;
        dot = ri * zi;
    }
    double total;
    if (ng_grid_sum(dot, L.partial, L.ticket, total)) {
        L.scal[0] = total;
        L.scal[1] = 0.0;
        L.scal[2] = 0.0;
        L.scal[3] = (total > 0.0) ? 0.0 : 1.0;
    }
}

// p = z + beta p_old (the previous iteration's direction update), Ap = A p:
// one warp per block row.  Its five six-lane groups take the row's blocks
// g, g + 5, ... (A_ab, or A_ba^T for the stored transpose): lane i of a group
// loads component i of the partner's direction, gathers the other five by
// shuffles and forms component i of the block's product; the five groups'
// sums meet in shared memory.  Then alpha = r.z / p.Ap.
__global__ void __launch_bounds__(kNgPcgBlock) k_ng_pcg_spmv(NgPcg L) {
    __shared__ double part[kNgPcgBlock / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int grp = lane / 6, i = lane - 6 * grp, base = 6 * grp;
    const bool stop = L.scal[3] != 0.0;
    const double beta = L.scal[2];
    double dot = 0.0;
    if (!stop && row < L.K) {  // warp-uniform
        const int e0 = L.row_ptr[row], e1 = L.row_ptr[row + 1];
        double y = 0.0;
        for (int t0 = e0; t0 < e1; t0 += kNgNodesPerWarp) {
            const int e = t0 + grp;
            const bool has = grp < kNgNodesPerWarp && e < e1;
            const int2 en = has ? L.ent[e] : make_int2(0, 0);
            const int blk = en.x & 0x7fffffff, b = en.y;
            const bool tr = en.x < 0;
            const double pbi = has ? L.z[6 * b + i] + beta * L.p_old[6 * b + i] : 0.0;
            double pb[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) pb[c] = __shfl_sync(kFull, pbi, (base + c) & 31);
            if (has) {
                const double *M = L.blocks_d + (size_t)blk * 36;
                double acc = 0.0;
#pragma unroll
                for (int c = 0; c < 6; ++c) acc += (tr ? M[6 * c + i] : M[6 * i + c]) * pb[c];
                y += acc;
            }
        }
        part[wib][lane] = y;  // lanes 30, 31 hold 0
        __syncwarp();
        if (lane < 6) {
            double s = 0.0;
#pragma unroll
            for (int g = 0; g < kNgNodesPerWarp; ++g) s += part[wib][6 * g + lane];
            const double pn = L.z[6 * row + lane] + beta * L.p_old[6 * row + lane];
            L.p_new[6 * row + lane] = pn;
            L.Ap[6 * row + lane] = s;
            dot = pn * s;
        }
    }
    double total;
    if (ng_grid_sum(dot, L.partial, L.ticket, total) && !stop) {
        if (total > 0.0) {
            L.scal[1] = L.scal[0] / total;
        } else {
            L.scal[1] = 0.0;
            L.scal[3] = 1.0;
        }
    }
}

// x += alpha p, r -= alpha Ap, z = P r, then beta = r.z / rz and rz = r.z
// (one lane per component).
__global__ void __launch_bounds__(kNgPcgBlock) k_ng_pcg_update(NgPcg L) {
    const NgLane l = ng_lane(L.K);
    const bool stop = L.scal[3] != 0.0;
    double dot = 0.0;
    if (!stop) {
        const double alpha = L.scal[1];
        double ri = 0.0;
        if (l.active) {
            const size_t o = 6 * (size_t)l.node + l.i;
            L.x[o] += alpha * L.p_new[o];
            ri = L.r[o] - alpha * L.Ap[o];
            L.r[o] = ri;
        }
        double zi = 0.0;
        const double *Pk = L.P + 36 * (size_t)(l.active ? l.node : 0);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double rc = ng_comp(ri, l, c);
            if (l.active) zi += Pk[6 * l.i + c] * rc;
        }
        if (l.active) {
            L.z[6 * (size_t)l.node + l.i] = zi;
            dot = ri * zi;
        }
    }
    double total;
    if (ng_grid_sum(dot, L.partial, L.ticket, total) && !stop) {
        L.scal[2] = total / L.scal[0];
        L.scal[0] = total;
        if (!(total > 0.0)) L.scal[3] = 1.0;
    }
}

// T_k <- exp(dx_k^) T_k (float64; A = sin(t)/t, B = (1 - cos t)/t^2,
// C = (t - sin t)/t^3, their series below t = 1e-3), then the node's dual
// quaternion (q_r from R, q_d = 1/2 (0, t) q_r) in float.
__global__ void __launch_bounds__(kBlock) k_ng_update(int K, const double *dx, double *node_T,
                                                      float *node_dq, double *twist2) {
    const int k = gtid();
    if (k >= K) return;
    double *T = node_T + 16 * (size_t)k;
    if (dx) {
        const double *z = dx + 6 * (size_t)k;
        const double w0 = z[0], w1 = z[1], w2 = z[2];
        const double th2 = w0 * w0 + w1 * w1 + w2 * w2, th = sqrt(th2);
        double A, B, C;
        if (th < 1e-3) {
            A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
            B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
            C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
        } else {
            double sn, cs;
            sincos(th, &sn, &cs);
            A = sn / th;
            B = (1.0 - cs) / th2;
            C = (th - sn) / (th2 * th);
        }
        const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
        double W2[9], E[16];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                W2[3 * i + j] = W[3 * i] * W[j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j];
        for (int i = 0; i < 3; ++i) {
            double tv = 0.0;
            for (int j = 0; j < 3; ++j) {
                const double I = (i == j) ? 1.0 : 0.0;
                E[4 * i + j] = I + A * W[3 * i + j] + B * W2[3 * i + j];
                tv += (I + B * W[3 * i + j] + C * W2[3 * i + j]) * z[3 + j];
            }
            E[4 * i + 3] = tv;
        }
        double Tn[12];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 4; ++j)
                Tn[4 * i + j] = E[4 * i] * T[j] + E[4 * i + 1] * T[4 + j] + E[4 * i + 2] * T[8 + j] +
                                (j == 3 ? E[4 * i + 3] : 0.0);
        for (int a = 0; a < 12; ++a) T[a] = Tn[a];
        atomicAdd(twist2, w0 * w0 + w1 * w1 + w2 * w2 + z[3] * z[3] + z[4] * z[4] + z[5] * z[5]);
    }
    // unit quaternion of R (the largest of w, x, y, z pivots)
    const double m00 = T[0], m01 = T[1], m02 = T[2], m10 = T[4], m11 = T[5], m12 = T[6];
    const double m20 = T[8], m21 = T[9], m22 = T[10], tr = m00 + m11 + m22;
    double q[4];
    if (tr >= m00 && tr >= m11 && tr >= m22) {
        const double s = sqrt(1.0 + tr) * 2.0;
        q[0] = 0.25 * s; q[1] = (m21 - m12) / s; q[2] = (m02 - m20) / s; q[3] = (m10 - m01) / s;
    } else if (m00 >= m11 && m00 >= m22) {
        const double s = sqrt(1.0 + m00 - m11 - m22) * 2.0;
        q[0] = (m21 - m12) / s; q[1] = 0.25 * s; q[2] = (m01 + m10) / s; q[3] = (m02 + m20) / s;
    } else if (m11 >= m22) {
        const double s = sqrt(1.0 + m11 - m00 - m22) * 2.0;
        q[0] = (m02 - m20) / s; q[1] = (m01 + m10) / s; q[2] = 0.25 * s; q[3] = (m12 + m21) / s;
    } else {
        const double s = sqrt(1.0 + m22 - m00 - m11) * 2.0;
        q[0] = (m10 - m01) / s; q[1] = (m02 + m20) / s; q[2] = (m12 + m21) / s; q[3] = 0.25 * s;
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int a = 0; a < 4; ++a) q[a] /= n;
    const double t0 = T[3], t1 = T[7], t2 = T[11];
    // (0, t) q_r / 2
    const double d[4] = {0.5 * (-t0 * q[1] - t1 * q[2] - t2 * q[3]),
                         0.5 * (t0 * q[0] + t1 * q[3] - t2 * q[2]),
                         0.5 * (t1 * q[0] + t2 * q[1] - t0 * q[3]),
                         0.5 * (t2 * q[0] + t0 * q[2] - t1 * q[1])};
    float4 *out = reinterpret_cast<float4 *>(node_dq) + 2 * (size_t)k;
    out[0] = make_float4((float)q[0], (float)q[1], (float)q[2], (float)q[3]);
    out[1] = make_float4((float)d[0], (float)d[1], (float)d[2], (float)d[3]);
}


}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

// Instantiated variants: {pt2pt, pt2pl} x {float32, bfloat16, half storage}
// x {plain, Kahan-compensated float partial sums}.
#define FR_VARIANTS(CALL)                                           \
    do {                                                            \
        if (pt2pl) {                                                \
            if (storage == kStoreBF16) {                            \
                if (kahan) CALL(true, true, 1); else CALL(true, false, 1);   \
            } else if (storage == kStoreF16) {                      \
                if (kahan) CALL(true, true, 2); else CALL(true, false, 2);   \
            } else {                                                \
                if (kahan) CALL(true, true, 0); else CALL(true, false, 0);   \
            }                                                       \
        } else {                                                    \
            if (storage == kStoreBF16) {                            \
                if (kahan) CALL(false, true, 1); else CALL(false, false, 1); \
            } else if (storage == kStoreF16) {                      \
                if (kahan) CALL(false, true, 2); else CALL(false, false, 2); \
            } else {                                                \
                if (kahan) CALL(false, true, 0); else CALL(false, false, 0); \
            }                                                       \
        }                                                           \
    } while (0)

void launch_em_iter(int pt2pl, int kahan, const IterLaunch &a, cudaStream_t s, int storage) {
    const int grid = a.gs + a.gv + a.gb + a.gc;
    if (grid <= 0) return;
#define FR_CALL(P, K, S) k_em_iter<P, K, S><<<grid, kBlock, 0, s>>>(a)
    FR_VARIANTS(FR_CALL);
#undef FR_CALL
}

void launch_em_iter_sigma(int kahan, const IterLaunch &a, cudaStream_t s) {
    const int grid = a.gs + a.gb + a.gc;
    if (grid <= 0) return;
    if (kahan)
        k_em_iter_sigma<true><<<grid, kBlock, 0, s>>>(a);
    else
        k_em_iter_sigma<false><<<grid, kBlock, 0, s>>>(a);
}

void launch_em_multi(int pt2pl, int kahan, const Slot *slots, const Seg *segs,
                     const unsigned short *blockseg, int grid, int check_done, cudaStream_t s,
                     int storage) {
    if (grid <= 0) return;
#define FR_CALL(P, K, S) k_em_multi<P, K, S><<<grid, kBlock, 0, s>>>(slots, segs, blockseg, check_done)
    FR_VARIANTS(FR_CALL);
#undef FR_CALL
}

void launch_art_iter(int pt2pl, const ArtLaunch &a, cudaStream_t s, int storage) {
    const int grid = a.gs + a.gv + a.gb + a.gc;
    if (grid <= 0) return;
    const int kahan = 0;
#define FR_CALL(P, K, S) k_art_iter<P, S><<<grid, kBlock, 0, s>>>(a)
    FR_VARIANTS(FR_CALL);
#undef FR_CALL
}

int em_iter_blocks_per_sm(int pt2pl, int kahan) {
    int n = 0;
    const void *f = pt2pl ? (kahan ? (const void *)k_em_iter<true, true, 0> : (const void *)k_em_iter<true, false, 0>)
                          : (kahan ? (const void *)k_em_iter<false, true, 0> : (const void *)k_em_iter<false, false, 0>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, f, kBlock, 0);
    return n > 0 ? n : 1;
}

void launch_clear_lists(const Table *tabs, int *const *lists, const int *const *counts, int n,
                        int grid, cudaStream_t s) {
    if (n <= 0) return;
    ClearSet c{};
    for (int i = 0; i < n && i < 3; ++i) {
        c.t[i] = tabs[i];
        c.list[i] = lists[i];
        c.count[i] = counts[i];
    }
    const int per = (grid + n - 1) / n;
    k_clear_lists<<<per * n, kBlock, 0, s>>>(c, n);
}

void launch_blur_pass(Table in, Table out, int dir, int grid, const DeviceState *st, cudaStream_t s) {
    k_blur_pass<<<grid, kBlock, 0, s>>>(in, out, dir, st);
}

void launch_blur_list(Table in, Table out, int dir, const int *list, const int *count, int grid,
                      const DeviceState *st, cudaStream_t s) {
    k_blur_list<<<grid, kBlock, 0, s>>>(in, out, dir, list, count, st);
}

void launch_estep_out(int pt2pl, const RigidJob *job, const IterParams *ip, Table t, float *out,
                      DeviceState *st, int grid, cudaStream_t s, int storage) {
    const int kahan = 0;
#define FR_CALL(P, K, S) k_estep_out<P, S><<<grid, kBlock, 0, s>>>(job, ip, t, out, st)
    FR_VARIANTS(FR_CALL);
#undef FR_CALL
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

void launch_ng_points(int pt2pl, const NgPoints &a, int warp_only, cudaStream_t s, int storage) {
    if (a.S <= 0) return;
    const int grid = (a.S + kBlock / 32 - 1) / (kBlock / 32);
    const int kahan = 0;
#define FR_CALL(P, K, S) k_ng_points<P, S><<<grid, kBlock, 0, s>>>(a, warp_only)
    FR_VARIANTS(FR_CALL);
#undef FR_CALL
}

void launch_ng_edges(const NgEdges &a, cudaStream_t s) {
    if (a.E <= 0) return;
    k_ng_edges<<<(a.E + 63) / 64, 64, 0, s>>>(a);  // small blocks: spread over the SMs
}

void launch_ng_pcg_init(const NgPcg &a, cudaStream_t s) {
    k_ng_pcg_init<<<ng_pcg_grid(a.K), kNgPcgBlock, 0, s>>>(a);
}

void launch_ng_pcg_spmv(const NgPcg &a, cudaStream_t s) {
    k_ng_pcg_spmv<<<ng_spmv_grid(a.K), kNgPcgBlock, 0, s>>>(a);
}

void launch_ng_pcg_update(const NgPcg &a, cudaStream_t s) {
    k_ng_pcg_update<<<ng_pcg_grid(a.K), kNgPcgBlock, 0, s>>>(a);
}

void launch_ng_update(int K, const double *dx, double *node_T, float *node_dq, double *twist2,
                      cudaStream_t s) {
    // one node per thread, 32-thread blocks: the float64 exponentials of a
    // thousand nodes spread over ~32 SMs instead of 4
    k_ng_update<<<(K + 31) / 32, 32, 0, s>>>(K, dx, node_T, node_dq, twist2);
}

void launch_zero_values(Table t, int grid, cudaStream_t s) {
    k_zero_values<<<grid, kBlock, 0, s>>>(t);
}

void launch_vertices(Table t, int vdim, int *keys_out, float *vals_out, int *count,
                     cudaStream_t s) {
    k_vertices<<<grid_for((long long)t.mask + 1, 4096), kBlock, 0, s>>>(t, vdim, keys_out,
                                                                        vals_out, count);
}

}  // namespace fr
