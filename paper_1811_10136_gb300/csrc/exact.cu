// The exact Gaussian E step on the GPU (Section 4.1, the Gauss transform
// that the permutohedral lattice approximates): for every moved model point
// x_i = T x_ref_i,
//   M0_i = sum_j K_ij,  M1_i = sum_j K_ij y_j,  N_i = sum_j K_ij n_j,
//   K_ij = exp(-|x_i - y_j|^2 / (2 sigma^2))   (unnormalised, as in Eq. 11),
// over all N observations -- O(N M) work, an accuracy and speed reference for
// the lattice at scale.  One thread per model point; observations staged
// through shared memory a tile at a time, each tile summed on its own before
// it joins the point's running totals (float32 rounding then grows with
// tile + N / tile terms, not N); the observation range is split across
// blocks when the model points alone cannot fill the GPU, the splits' totals
// combined with float atomics.  Arithmetic-bound: per pair 3 differences,
// the squared distance, one exp2 and 4 or 7 fused multiply-adds.
#include "context.h"

#include <algorithm>

using namespace fr;

namespace {

constexpr int kExThreads = 256;
constexpr int kExTile = 256;  // observations per shared-memory tile

struct ExPose {
    float p[12];  // rows of T (float), applied with explicit rounding as the slice does
};

__device__ __forceinline__ float ex_row(const ExPose &P, int j, float4 r) {
    const float a = __fadd_rn(__fmul_rn(P.p[4 * j], r.x), __fmul_rn(P.p[4 * j + 1], r.y));
    return __fadd_rn(__fadd_rn(a, __fmul_rn(P.p[4 * j + 2], r.z)), P.p[4 * j + 3]);
}

template <bool PT2PL>
__global__ void __launch_bounds__(kExThreads) k_gauss_exact(const float4 *__restrict__ X, int M, ExPose P,
                                                            const float4 *__restrict__ Y,
                                                            const float4 *__restrict__ Yn, int N,
                                                            float neg_log2e_over_2s2, int ysplit, int ychunk,
                                                            float *__restrict__ out) {
    __shared__ float4 sy[kExTile];
    __shared__ float4 sn[PT2PL ? kExTile : 1];
    const int xb = blockIdx.x / ysplit, ys = blockIdx.x % ysplit;
    const int i = xb * kExThreads + threadIdx.x;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (i < M) {
        const float4 r = __ldg(X + i);
        x0 = ex_row(P, 0, r);
        x1 = ex_row(P, 1, r);
        x2 = ex_row(P, 2, r);
    }
    const int j0 = ys * ychunk, j1 = min(N, j0 + ychunk);
    float tot[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t0 = j0; t0 < j1; t0 += kExTile) {
        const int nt = min(kExTile, j1 - t0);
        __syncthreads();
        if (threadIdx.x < nt) {
            sy[threadIdx.x] = __ldg(Y + t0 + threadIdx.x);
            if (PT2PL) sn[threadIdx.x] = __ldg(Yn + t0 + threadIdx.x);
        }
        __syncthreads();
        float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
        for (int j = 0; j < nt; ++j) {
            const float4 y = sy[j];
            const float d0 = x0 - y.x, d1 = x1 - y.y, d2 = x2 - y.z;
            const float q = fmaf(d2, d2, fmaf(d1, d1, d0 * d0));
            const float k = exp2f(q * neg_log2e_over_2s2);
            s[0] += k;
            s[1] = fmaf(k, y.x, s[1]);
            s[2] = fmaf(k, y.y, s[2]);
            s[3] = fmaf(k, y.z, s[3]);
            if (PT2PL) {
                const float4 n = sn[j];
                s[4] = fmaf(k, n.x, s[4]);
                s[5] = fmaf(k, n.y, s[5]);
                s[6] = fmaf(k, n.z, s[6]);
            }
        }
#pragma unroll
        for (int c = 0; c < 7; ++c) tot[c] += s[c];
    }
    if (i >= M) return;
    constexpr int vd = PT2PL ? 7 : 4;
    float *o = out + (size_t)i * vd;
    if (ysplit == 1) {
#pragma unroll
        for (int c = 0; c < vd; ++c) o[c] = tot[c];
    } else {
#pragma unroll
        for (int c = 0; c < vd; ++c) atomicAdd(o + c, tot[c]);
    }
}

}  // namespace

extern "C" FR_API fr_status fr_gauss_transform(fr_ctx *ctx, const float *d_X, int64_t M, const float *d_Y,
                                               const float *d_Yn, int64_t N, float sigma, const double T[16],
                                               float *d_out) {
    fr::NvtxRange nvtx_("fr_gauss_transform");
    if (!ctx) return FR_EINVAL;
    FR_TRY(validate_cloud(ctx, d_X, M, "d_X"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (d_Yn) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn"));
    if (!d_out) return ctx->fail(FR_EINVAL, "d_out is NULL");
    if (M > (1ll << 30) || N > (1ll << 30)) return ctx->fail(FR_EINVAL, "clouds above 2^30 points");
    if (!(sigma > 0.0f) || !std::isfinite(sigma)) return ctx->fail(FR_EINVAL, "sigma must be finite and > 0");
    ExPose P{};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) {
            const double v = T ? T[4 * r + c] : (r == c ? 1.0 : 0.0);
            if (!std::isfinite(v)) return ctx->fail(FR_EINVAL, "T must be finite");
            P.p[4 * r + c] = (float)v;
        }
    cudaSetDevice(ctx->device);
    const int vd = d_Yn ? 7 : 4;
    const long long xblocks = (M + kExThreads - 1) / kExThreads;
    // split the observations until the grid holds ~4 blocks per SM (each
    // split at least a few tiles long)
    long long ysplit = (4LL * ctx->num_sms + xblocks - 1) / xblocks;
    const long long ymax = ((long long)N + 4 * kExTile - 1) / (4 * kExTile);
    ysplit = std::max<long long>(1, std::min<long long>(ysplit, ymax));
    const long long ychunk = ((N + ysplit - 1) / ysplit + kExTile - 1) / kExTile * kExTile;
    ysplit = (N + ychunk - 1) / ychunk;
    if (xblocks * ysplit > (1LL << 31) - 1) return ctx->fail(FR_EINVAL, "grid too large");
    if (ysplit > 1) FR_CUDA(ctx, cudaMemsetAsync(d_out, 0, (size_t)M * vd * sizeof(float), ctx->stream));
    const float scale = (float)(-1.4426950408889634 / (2.0 * (double)sigma * (double)sigma));
    const int grid = (int)(xblocks * ysplit);
    if (d_Yn)
        k_gauss_exact<true><<<grid, kExThreads, 0, ctx->stream>>>(
            (const float4 *)d_X, (int)M, P, (const float4 *)d_Y, (const float4 *)d_Yn, (int)N, scale, (int)ysplit,
            (int)ychunk, d_out);
    else
        k_gauss_exact<false><<<grid, kExThreads, 0, ctx->stream>>>(
            (const float4 *)d_X, (int)M, P, (const float4 *)d_Y, nullptr, (int)N, scale, (int)ysplit, (int)ychunk,
            d_out);
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}
