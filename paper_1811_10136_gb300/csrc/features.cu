// Feature-space E step (Section 3.3, Eq. feature_estep): the E step's
// Gaussian taken over d-dimensional feature vectors with a diagonal
// covariance diag(sigma_f^2) -- position and normal, colour, or any per-point
// descriptor -- filtered on the permutohedral lattice of Section 4.2 for
// 1 <= d <= 7 (lattice dimension D = d + 1 <= 8), plus the exact sums over
// every pair for checking.
//
// Each observation feature g = f / sigma_f is elevated onto sum(z) = 0 in
// R^D, assigned the D vertices of its enclosing simplex with barycentric
// weights, and its values [1, y] (and n_y) are added to those vertices; each
// model feature is located the same way and reads the weighted sum of its
// vertices' values (the augmentation of Eq. 13-14: queries insert nothing).
// A vertex key's d free integer coordinates (the last is minus their sum) are
// packed into 128 bits and claimed in an open-addressing table with one
// 128-bit compare-and-swap; a record is the key and its values in one 32-byte
// sector (point-to-point) or two (with normals).  Slots a build claims are
// listed and cleared after the slice, so the table is empty between calls
// without a sweep over all of it.
//
// The embedding's float steps are single IEEE operations (explicit _rn
// intrinsics, no contraction) in a fixed order and z / D is a correctly
// rounded division, so keys and weights are reproducible bit for bit by any
// implementation that takes the same steps.
#include "context.h"

#include <algorithm>
#include <mutex>

using namespace fr;

namespace {

constexpr int kFDMax = 7;        // largest feature dimension d
constexpr int kFThreads = 256;   // threads per block of every kernel here
constexpr int kFMaxProbe = 512;  // longest probe sequence before the table counts as full
constexpr uint32_t kFMaxSlots = 1u << 27;

// Bits per packed key coordinate: d fields share 126 bits, at most 32 each.
__host__ __device__ constexpr int fkey_bits(int d) { return 126 / d > 32 ? 32 : 126 / d; }

// |z_j| bound: the oracle's integer range (1e6), tightened where the packed
// fields are narrower (d = 7: 18 bits hold |coordinate| < 2^17).
__host__ __device__ constexpr float fz_limit(int d) { return fkey_bits(d) >= 21 ? 1.0e6f : 131000.0f; }

struct FScale {
    float s[kFDMax];  // alpha / sqrt(i (i+1)) / sigma_f[i-1], alpha = sqrt(2/3) (d+1)
};

struct FTable {
    uint4 *rec;      // cap records of STRIDE uint4: [key, (W, sum b y), (sum b n, 0), pad]
    int *list;       // slots claimed by the current build
    int *count;      // [0] claimed slots, [1] flags
    uint32_t mask;   // cap - 1
};

template <int d>
struct FSimplex {
    int r0[d + 1];
    int rank[d + 1];
    float b[d + 1];
};

// Elevate one feature row and find its simplex (Section 4.2): false for a
// non-finite or out-of-range coordinate.
template <int d>
__device__ __forceinline__ bool fembed(const float *__restrict__ f, const FScale &S, FSimplex<d> &o) {
    constexpr int D = d + 1;
    float c[d + 1];
#pragma unroll
    for (int i = 1; i <= d; ++i) c[i] = __fmul_rn(__ldg(f + i - 1), S.s[i - 1]);
    float z[D];
    float t = 0.0f;
#pragma unroll
    for (int i = d; i >= 1; --i) {
        z[i] = __fsub_rn(t, __fmul_rn((float)i, c[i]));
        t = __fadd_rn(t, c[i]);
    }
    z[0] = t;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < D; ++j) ok = ok && (fabsf(z[j]) < fz_limit(d));
    if (!ok) return false;

    // nearest remainder-0 point coordinate by coordinate, and the residuals
    int sum = 0;
    float delta[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float q = rintf(__fdiv_rn(z[j], (float)D));
        o.r0[j] = (int)q * D;
        sum += (int)q;
        delta[j] = __fsub_rn(z[j], (float)o.r0[j]);
    }
    // descending rank of each residual, ties to the lower index: of each pair
    // exactly one outranks the other
#pragma unroll
    for (int j = 0; j < D; ++j) o.rank[j] = 0;
#pragma unroll
    for (int j = 0; j < D; ++j)
#pragma unroll
        for (int k = j + 1; k < D; ++k) {
            if (delta[k] > delta[j])
                ++o.rank[j];
            else
                ++o.rank[k];
        }
    // repair the coordinate sum to zero
    if (sum > D || sum < -D) return false;
    if (sum > 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (o.rank[j] >= D - sum) {
                o.r0[j] -= D;
                o.rank[j] += sum - D;
            } else {
                o.rank[j] += sum;
            }
        }
    } else if (sum < 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (o.rank[j] < -sum) {
                o.r0[j] += D;
                o.rank[j] += D + sum;
            } else {
                o.rank[j] += sum;
            }
        }
    }
    // barycentric weights: with v_r the scaled residual of rank r,
    // b_0 = v_{D-1} + (1 - v_0) and b_k = v_{D-1-k} - v_{D-k}
    float vr[D];
#pragma unroll
    for (int r = 0; r < D; ++r) vr[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float v = __fdiv_rn(__fsub_rn(z[j], (float)o.r0[j]), (float)D);
#pragma unroll
        for (int r = 0; r < D; ++r) vr[r] = (o.rank[j] == r) ? v : vr[r];
    }
    o.b[0] = __fadd_rn(vr[D - 1], __fsub_rn(1.0f, vr[0]));
#pragma unroll
    for (int k = 1; k < D; ++k) o.b[k] = __fsub_rn(vr[D - 1 - k], vr[D - k]);
    return true;
}

// Coordinate j of vertex k: every coordinate of vertex k is k mod D.
template <int d>
__device__ __forceinline__ int fvertex_coord(const FSimplex<d> &s, int k, int j) {
    constexpr int D = d + 1;
    return s.r0[j] + k - (s.rank[j] > D - 1 - k ? D : 0);
}

// Vertex k's d free coordinates, biased and packed into (lo, hi).
template <int d>
__device__ __forceinline__ void fpack(const FSimplex<d> &s, int k, unsigned long long &lo,
                                      unsigned long long &hi) {
    constexpr int B = fkey_bits(d);
    constexpr unsigned long long mask = B == 32 ? 0xFFFFFFFFull : ((1ull << B) - 1ull);
    constexpr unsigned int bias = 1u << (B - 1);
    unsigned __int128 acc = 0;
#pragma unroll
    for (int j = 0; j < d; ++j) {
        const unsigned long long fld = (unsigned long long)((unsigned int)fvertex_coord<d>(s, k, j) + bias) & mask;
        acc |= (unsigned __int128)fld << (j * B);
    }
    lo = (unsigned long long)acc;
    hi = (unsigned long long)(acc >> 64);
}

__device__ __forceinline__ uint32_t fslot(unsigned long long lo, unsigned long long hi, uint32_t mask) {
    unsigned long long h = lo * 0x9E3779B97F4A7C15ull ^ (hi + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
    h ^= h >> 31;
    return (uint32_t)(h >> 32) & mask;
}

constexpr unsigned long long kFEmpty = ~0ull;  // both halves of an empty slot's key

// 128-bit compare-and-swap of a slot's key; returns the previous key.
__device__ __forceinline__ void fcas128(uint4 *addr, unsigned long long cmp_lo, unsigned long long cmp_hi,
                                        unsigned long long new_lo, unsigned long long new_hi,
                                        unsigned long long &old_lo, unsigned long long &old_hi) {
    asm volatile(
        "{\n\t.reg .b128 c, n, o;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 n, {%4, %5};\n\t"
        "atom.global.cas.b128 o, [%6], c, n;\n\t"
        "mov.b128 {%0, %1}, o;\n\t}"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(addr)
        : "memory");
}

__device__ __forceinline__ void fred_add4(uint4 *p, float a, float b, float c, float e) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(e)
                 : "memory");
}

__device__ __forceinline__ unsigned long long lo_of(uint4 v) {
    return (unsigned long long)v.x | ((unsigned long long)v.y << 32);
}
__device__ __forceinline__ unsigned long long hi_of(uint4 v) {
    return (unsigned long long)v.z | ((unsigned long long)v.w << 32);
}

// Find or claim the slot of key (lo, hi), the first probe's key already read
// (cur, at slot s0); -1 when the probe limit is reached.  A packed key never
// has an all-ones half (every field stays below its maximum), so a key read
// with an all-ones half is empty or being written and is settled by the
// compare-and-swap; a key with two other halves is final.
template <int STRIDE>
__device__ __forceinline__ int finsert_from(const FTable &t, unsigned long long lo, unsigned long long hi,
                                            uint32_t s0, uint4 cur, bool &claimed) {
    claimed = false;
    const unsigned long long clo = lo_of(cur), chi = hi_of(cur);
    if (clo == lo && chi == hi) return (int)s0;
    uint32_t s = s0;
    for (int p = 0; p < kFMaxProbe; ++p) {
        uint4 *r = t.rec + (size_t)s * STRIDE;
        const uint4 c = p == 0 ? cur : __ldcg(r);
        const unsigned long long a = lo_of(c), b = hi_of(c);
        if (a == lo && b == hi) return (int)s;
        if (a == kFEmpty || b == kFEmpty) {
            unsigned long long olo, ohi;
            fcas128(r, kFEmpty, kFEmpty, lo, hi, olo, ohi);
            if (olo == kFEmpty && ohi == kFEmpty) {
                claimed = true;
                return (int)s;
            }
            if (olo == lo && ohi == hi) return (int)s;
        }
        s = (s + 1) & t.mask;
    }
    return -1;
}

// Slot of key (lo, hi) in a completed table; -1 if absent.
template <int STRIDE>
__device__ __forceinline__ int ffind(const FTable &t, unsigned long long lo, unsigned long long hi) {
    uint32_t s = fslot(lo, hi, t.mask);
    for (int p = 0; p < kFMaxProbe; ++p) {
        const uint4 cur = __ldg(t.rec + (size_t)s * STRIDE);
        const unsigned long long clo = lo_of(cur), chi = hi_of(cur);
        if (clo == lo && chi == hi) return (int)s;
        if (clo == kFEmpty && chi == kFEmpty) return -1;
        s = (s + 1) & t.mask;
    }
    return -1;
}

}  // namespace

namespace {

// Splat (Section 4.2) of the observation features with values [1, y] or
// [1, y, n_y]: one thread per observation, block-strided rounds.  For each
// vertex k in turn, runs of equal keys in neighbouring lanes (consecutive
// observations -- pixels of a depth image in raster order -- mostly share
// vertices) are merged by a segmented scan within 8-lane chunks, and only a
// run's last lane inserts the key and issues the vector reductions.  The
// slots a round claims are gathered in shared memory and appended to the
// list with one global atomic per block and round.
template <int d, bool PT2PL>
__global__ void __launch_bounds__(kFThreads) k_feat_build(const float *__restrict__ F, int N, FScale S,
                                                          const float4 *__restrict__ Y,
                                                          const float4 *__restrict__ Yn, FTable t) {
    constexpr int STRIDE = PT2PL ? 4 : 2;
    constexpr int kCh = PT2PL ? 7 : 4;
    constexpr unsigned kFull = 0xffffffffu;
    __shared__ int s_claim[kFThreads * (d + 1)];
    __shared__ int s_n, s_base;
    const int lane = threadIdx.x & 31;
    int bad = 0;
    for (int base = blockIdx.x * kFThreads; base < N; base += gridDim.x * kFThreads) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        const int i = base + threadIdx.x;
        FSimplex<d> sx;
        bool valid = false;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f), n = y;
        if (i < N) {
            valid = fembed<d>(F + (size_t)i * d, S, sx);
            if (!valid) bad |= kFlagRange;
            y = __ldg(Y + i);
            if (PT2PL) n = __ldg(Yn + i);
        }
        // pass 1: keys, run tails, and each tail's first probe in flight
        unsigned long long lo[d + 1], hi[d + 1];
        uint32_t s0[d + 1];
        uint4 cur[d + 1];
        unsigned tails = 0;
#pragma unroll
        for (int k = 0; k <= d; ++k) {
            lo[k] = hi[k] = kFEmpty;
            if (valid) fpack<d>(sx, k, lo[k], hi[k]);
            const unsigned long long plo = __shfl_up_sync(kFull, lo[k], 1), phi = __shfl_up_sync(kFull, hi[k], 1);
            const unsigned heads = __ballot_sync(kFull, (lane & 7) == 0 || plo != lo[k] || phi != hi[k]);
            const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
            if (valid && tail) tails |= 1u << k;
            s0[k] = fslot(lo[k], hi[k], t.mask);
            if (valid && tail) cur[k] = __ldcg(t.rec + (size_t)s0[k] * STRIDE);
        }
        // pass 2: settle each tail's slot (claiming new vertices)
        int slot[d + 1];
#pragma unroll
        for (int k = 0; k <= d; ++k) {
            slot[k] = -1;
            if ((tails >> k) & 1u) {
                bool claimed = false;
                slot[k] = finsert_from<STRIDE>(t, lo[k], hi[k], s0[k], cur[k], claimed);
                if (slot[k] < 0) bad |= kFlagCapacity;
                else if (claimed) s_claim[atomicAdd(&s_n, 1)] = slot[k];
            }
        }
        // pass 3: merge each run's values (segmented scan within 8-lane
        // chunks, heads recomputed from the run tails) and reduce at its tail
#pragma unroll
        for (int k = 0; k <= d; ++k) {
            const unsigned long long plo = __shfl_up_sync(kFull, lo[k], 1), phi = __shfl_up_sync(kFull, hi[k], 1);
            const unsigned heads = __ballot_sync(kFull, (lane & 7) == 0 || plo != lo[k] || phi != hi[k]);
            const int head = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
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
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
                for (int c = 0; c < kCh; ++c) {
                    const float tv = __shfl_up_sync(kFull, v[c], o);
                    if (lane - o >= head) v[c] += tv;
                }
            }
            if (slot[k] >= 0) {
                uint4 *r = t.rec + (size_t)slot[k] * STRIDE;
                fred_add4(r + 1, v[0], v[1], v[2], v[3]);
                if (PT2PL) fred_add4(r + 2, v[4], v[5], v[6], 0.f);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base = s_n ? atomicAdd(t.count, s_n) : 0;
        __syncthreads();
        for (int j = threadIdx.x; j < s_n; j += kFThreads) t.list[s_base + j] = s_claim[j];
        __syncthreads();  // s_n and s_claim are reused by the next round
    }
    if (bad) atomicOr(t.count + 1, bad);
}

// Slice at the model features: out_i = sum_k b_k value(vertex k), absent
// vertices contributing nothing.  One thread per model point, grid-stride.
template <int d, bool PT2PL>
__global__ void __launch_bounds__(kFThreads) k_feat_slice(const float *__restrict__ F, int M, FScale S, FTable t,
                                                          float *__restrict__ out) {
    constexpr int STRIDE = PT2PL ? 4 : 2;
    constexpr int VD = PT2PL ? 7 : 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        FSimplex<d> sx;
        if (fembed<d>(F + (size_t)i * d, S, sx)) {
            // first probe of every vertex, key and values, in flight at once
            unsigned long long lo[d + 1], hi[d + 1];
            uint32_t s0[d + 1];
            uint4 key[d + 1];
            float4 v0[d + 1], v1[d + 1];
#pragma unroll
            for (int k = 0; k <= d; ++k) {
                fpack<d>(sx, k, lo[k], hi[k]);
                s0[k] = fslot(lo[k], hi[k], t.mask);
            }
#pragma unroll
            for (int k = 0; k <= d; ++k) {
                const uint4 *r = t.rec + (size_t)s0[k] * STRIDE;
                key[k] = __ldg(r);
                v0[k] = __ldg(reinterpret_cast<const float4 *>(r + 1));
                if (PT2PL) v1[k] = __ldg(reinterpret_cast<const float4 *>(r + 2));
            }
#pragma unroll
            for (int k = 0; k <= d; ++k) {
                const unsigned long long a = lo_of(key[k]), c = hi_of(key[k]);
                if (!(a == lo[k] && c == hi[k])) {
                    // absent, or the slot holds another key: probe on
                    v0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (PT2PL) v1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (!(a == kFEmpty && c == kFEmpty)) {
                        const int s = ffind<STRIDE>(t, lo[k], hi[k]);
                        if (s >= 0) {
                            const uint4 *r = t.rec + (size_t)s * STRIDE;
                            v0[k] = __ldg(reinterpret_cast<const float4 *>(r + 1));
                            if (PT2PL) v1[k] = __ldg(reinterpret_cast<const float4 *>(r + 2));
                        }
                    }
                }
                const float b = sx.b[k];
                acc[0] = fmaf(b, v0[k].x, acc[0]);
                acc[1] = fmaf(b, v0[k].y, acc[1]);
                acc[2] = fmaf(b, v0[k].z, acc[2]);
                acc[3] = fmaf(b, v0[k].w, acc[3]);
                if (PT2PL) {
                    acc[4] = fmaf(b, v1[k].x, acc[4]);
                    acc[5] = fmaf(b, v1[k].y, acc[5]);
                    acc[6] = fmaf(b, v1[k].z, acc[6]);
                }
            }
        } else {
            atomicOr(t.count + 1, kFlagRange);
        }
        if (PT2PL) {
            float *o = out + (size_t)i * VD;
#pragma unroll
            for (int c = 0; c < VD; ++c) o[c] = acc[c];
        } else {
            reinterpret_cast<float4 *>(out)[i] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        }
    }
}

// Empty the slots the last build claimed (key all ones, values zero).
template <int STRIDE>
__global__ void __launch_bounds__(kFThreads) k_feat_clear(FTable t, int limit) {
    const int n = min(*t.count, limit);
    const uint4 empty = make_uint4(~0u, ~0u, ~0u, ~0u), zero = make_uint4(0u, 0u, 0u, 0u);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint4 *r = t.rec + (size_t)t.list[i] * STRIDE;
        r[0] = empty;
#pragma unroll
        for (int c = 1; c < STRIDE; ++c) r[c] = zero;
    }
}

// Empty a whole table laid out with `stride` uint4 per record.
__global__ void __launch_bounds__(kFThreads) k_feat_init(uint4 *rec, long long cap, int stride) {
    const uint4 empty = make_uint4(~0u, ~0u, ~0u, ~0u), zero = make_uint4(0u, 0u, 0u, 0u);
    const long long n = cap * stride;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        rec[i] = (i % stride) == 0 ? empty : zero;
}

// Keys (all D coordinates of each vertex) and weights of n feature rows.
template <int d>
__global__ void __launch_bounds__(kFThreads) k_feat_embed(const float *__restrict__ F, int n, FScale S,
                                                          int *__restrict__ keys, float *__restrict__ bary,
                                                          int *flags) {
    constexpr int D = d + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        FSimplex<d> sx;
        const bool ok = fembed<d>(F + (size_t)i * d, S, sx);
        if (!ok) atomicOr(flags, kFlagRange);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (keys)
#pragma unroll
                for (int j = 0; j < D; ++j) keys[((size_t)i * D + k) * D + j] = ok ? fvertex_coord<d>(sx, k, j) : 0;
            if (bary) bary[(size_t)i * D + k] = ok ? sx.b[k] : 0.0f;
        }
    }
}

constexpr int kFExTile = 128;  // observations per shared-memory tile of the exact sums

// Exact feature-space sums (Eq. feature_estep without the lattice):
// K_ij = exp(-sum_c ((fx_c - fy_c) / sigma_c)^2 / 2), one thread per model
// point, observation tiles staged in shared memory and summed per tile; the
// observations are split across blocks when the model alone cannot fill the
// GPU (the splits' totals then meet in float atomics).
template <int d, bool PT2PL>
__global__ void __launch_bounds__(kFThreads) k_feat_exact(const float *__restrict__ FX, int M,
                                                          const float *__restrict__ FY,
                                                          const float4 *__restrict__ Y,
                                                          const float4 *__restrict__ Yn, int N, FScale inv,
                                                          int ysplit, int ychunk, float *__restrict__ out) {
    __shared__ float sf[kFExTile * d];
    __shared__ float4 sy[kFExTile];
    __shared__ float4 sn[PT2PL ? kFExTile : 1];
    const int xb = blockIdx.x / ysplit, ys = blockIdx.x % ysplit;
    const int i = xb * kFThreads + threadIdx.x;
    float g[d];
#pragma unroll
    for (int c = 0; c < d; ++c) g[c] = i < M ? __ldg(FX + (size_t)i * d + c) * inv.s[c] : 0.f;
    const int j0 = ys * ychunk, j1 = min(N, j0 + ychunk);
    constexpr float kNegHalfLog2e = -0.72134752044448170f;  // -log2(e) / 2
    float tot[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t0 = j0; t0 < j1; t0 += kFExTile) {
        const int nt = min(kFExTile, j1 - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < nt * d; e += kFThreads) sf[e] = __ldg(FY + (size_t)t0 * d + e) * inv.s[e % d];
        if (threadIdx.x < nt) {
            sy[threadIdx.x] = __ldg(Y + t0 + threadIdx.x);
            if (PT2PL) sn[threadIdx.x] = __ldg(Yn + t0 + threadIdx.x);
        }
        __syncthreads();
        float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
        for (int j = 0; j < nt; ++j) {
            float q = 0.f;
#pragma unroll
            for (int c = 0; c < d; ++c) {
                const float u = g[c] - sf[j * d + c];
                q = fmaf(u, u, q);
            }
            const float k = exp2f(q * kNegHalfLog2e);
            const float4 y = sy[j];
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
    constexpr int VD = PT2PL ? 7 : 4;
    float *o = out + (size_t)i * VD;
    if (ysplit == 1) {
#pragma unroll
        for (int c = 0; c < VD; ++c) o[c] = tot[c];
    } else {
#pragma unroll
        for (int c = 0; c < VD; ++c) atomicAdd(o + c, tot[c]);
    }
}

}  // namespace

namespace fr {

// The feature lattice's table, kept by the context between calls (empty
// between calls: every build's claimed slots are cleared after its slice).
struct FeatWorkspace {
    uint4 *rec = nullptr;
    size_t rec_bytes = 0;
    uint32_t cap = 0;  // slots of the current layout (0: not initialised)
    int stride = 0;    // uint4 per record of the current layout
    int *list = nullptr;
    size_t list_cap = 0;
    int *count = nullptr;  // [0] claimed, [1] flags
    int *h_count = nullptr;
};

void free_feat_workspace(fr_ctx *ctx) {
    FeatWorkspace *w = ctx->feat;
    if (!w) return;
    cudaFree(w->rec);
    cudaFree(w->list);
    cudaFree(w->count);
    cudaFreeHost(w->h_count);
    delete w;
    ctx->feat = nullptr;
}

}  // namespace fr

namespace {

fr_status feat_validate(fr_ctx *ctx, const float *p, int64_t n, const char *name) {
    if (!p) return ctx->fail(FR_EINVAL, "%s is NULL", name);
    if (n < 1 || n > (1ll << 30)) return ctx->fail(FR_EINVAL, "%s: size %lld out of range", name, (long long)n);
    if (((uintptr_t)p & 3u) != 0) return ctx->fail(FR_EINVAL, "%s must be 4-byte aligned (rows of d floats)", name);
    return FR_OK;
}

fr_status feat_scales(fr_ctx *ctx, int d, const float *sigma_f, FScale *S, FScale *inv) {
    if (d < 1 || d > kFDMax) return ctx->fail(FR_EINVAL, "feature dimension d must lie in [1, %d]", kFDMax);
    if (!sigma_f) return ctx->fail(FR_EINVAL, "sigma_f is NULL");
    const double alpha = std::sqrt(2.0 / 3.0) * (double)(d + 1);
    *S = FScale{};
    if (inv) *inv = FScale{};
    for (int i = 1; i <= d; ++i) {
        const float sg = sigma_f[i - 1];
        if (!(sg > 0.0f) || !std::isfinite(sg)) return ctx->fail(FR_EINVAL, "sigma_f must be finite and > 0");
        S->s[i - 1] = (float)(alpha / std::sqrt((double)(i * (i + 1))) / (double)sg);
        if (inv) inv->s[i - 1] = (float)(1.0 / (double)sg);
    }
    return FR_OK;
}

int feat_grid(const fr_ctx *ctx, long long n) {
    const long long want = (n + kFThreads - 1) / kFThreads;
    const long long most = 8LL * ctx->num_sms;
    return (int)std::max<long long>(1, std::min(want, most));
}

// The device counters and their pinned host mirror.
fr_status feat_ensure_counts(fr_ctx *ctx) {
    if (!ctx->feat) ctx->feat = new FeatWorkspace();
    FeatWorkspace *w = ctx->feat;
    if (!w->count) {
        FR_CUDA(ctx, fr::dev_malloc((void **)&w->count, 4 * sizeof(int)));
        FR_CUDA(ctx, cudaMemsetAsync(w->count, 0, 4 * sizeof(int), ctx->stream));
    }
    if (!w->h_count) FR_CUDA(ctx, cudaMallocHost((void **)&w->h_count, 4 * sizeof(int)));
    return FR_OK;
}

// A table of `cap` slots with `stride` uint4 per record, empty.
fr_status feat_ensure(fr_ctx *ctx, uint32_t cap, int stride, long long list_len) {
    FR_TRY(feat_ensure_counts(ctx));
    FeatWorkspace *w = ctx->feat;
    const size_t bytes = (size_t)cap * stride * sizeof(uint4);
    if (ctx->ws_limit && bytes > ctx->ws_limit)
        return ctx->fail(FR_ENOMEM, "feature lattice table of %zu bytes exceeds the workspace limit", bytes);
    if ((size_t)list_len > w->list_cap) {
        cudaFree(w->list);
        w->list = nullptr;
        w->list_cap = 0;
        FR_CUDA(ctx, fr::dev_malloc((void **)&w->list, (size_t)list_len * sizeof(int)));
        w->list_cap = (size_t)list_len;
    }
    if (bytes > w->rec_bytes) {
        cudaFree(w->rec);
        w->rec = nullptr;
        w->rec_bytes = 0;
        w->cap = 0;
        FR_CUDA(ctx, fr::dev_malloc((void **)&w->rec, bytes));
        w->rec_bytes = bytes;
    }
    if (w->cap != cap || w->stride != stride) {
        w->cap = 0;
        k_feat_init<<<feat_grid(ctx, (long long)cap * stride), kFThreads, 0, ctx->stream>>>(w->rec, cap, stride);
        ctx->launches += 1;
        FR_CUDA(ctx, cudaGetLastError());
        w->cap = cap;
        w->stride = stride;
    }
    return FR_OK;
}

// With profiling on, an event pair around each of the three launches
// (classes FR_K_BUILD, FR_K_SLICE, FR_K_CLEAR), collected after the sync.
struct FeatTimer {
    fr_ctx *ctx;
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
        cudaEventRecord(ctx->events[2 * n], ctx->stream);
    }
    void end() {
        if (!ctx->profiling) return;
        cudaEventRecord(ctx->events[2 * n + 1], ctx->stream);
        ++n;
    }
};

template <int d>
void launch_feat(bool pt2pl, fr_ctx *ctx, FeatTimer &tm, const float *FX, int M, const float *FY, int N,
                 const FScale &S, const float4 *Y, const float4 *Yn, FTable t, float *out) {
    const int gb = feat_grid(ctx, N), gs = feat_grid(ctx, M);
    // a list entry per claimed slot: at most (d+1) N
    const int limit = (int)std::min<long long>((long long)(d + 1) * N, (long long)t.mask + 1);
    const int gc = feat_grid(ctx, limit);
    tm.begin(FR_K_BUILD);
    if (pt2pl)
        k_feat_build<d, true><<<gb, kFThreads, 0, ctx->stream>>>(FY, N, S, Y, Yn, t);
    else
        k_feat_build<d, false><<<gb, kFThreads, 0, ctx->stream>>>(FY, N, S, Y, nullptr, t);
    tm.end();
    tm.begin(FR_K_SLICE);
    if (pt2pl)
        k_feat_slice<d, true><<<gs, kFThreads, 0, ctx->stream>>>(FX, M, S, t, out);
    else
        k_feat_slice<d, false><<<gs, kFThreads, 0, ctx->stream>>>(FX, M, S, t, out);
    tm.end();
    tm.begin(FR_K_CLEAR);
    if (pt2pl)
        k_feat_clear<4><<<gc, kFThreads, 0, ctx->stream>>>(t, limit);
    else
        k_feat_clear<2><<<gc, kFThreads, 0, ctx->stream>>>(t, limit);
    tm.end();
}

template <int d>
void launch_embed(const fr_ctx *ctx, const float *F, int n, const FScale &S, int32_t *keys, float *bary, int *flags) {
    k_feat_embed<d><<<feat_grid(ctx, n), kFThreads, 0, ctx->stream>>>(F, n, S, keys, bary, flags);
}

template <int d>
void launch_exact(bool pt2pl, const float *FX, int M, const float *FY, const float4 *Y, const float4 *Yn, int N,
                  const FScale &inv, int ysplit, int ychunk, int grid, cudaStream_t s, float *out) {
    if (pt2pl)
        k_feat_exact<d, true><<<grid, kFThreads, 0, s>>>(FX, M, FY, Y, Yn, N, inv, ysplit, ychunk, out);
    else
        k_feat_exact<d, false><<<grid, kFThreads, 0, s>>>(FX, M, FY, Y, nullptr, N, inv, ysplit, ychunk, out);
}

#define FR_FEATURE_DISPATCH(d, CALL) \
    switch (d) {                     \
    case 1: CALL(1); break;          \
    case 2: CALL(2); break;          \
    case 3: CALL(3); break;          \
    case 4: CALL(4); break;          \
    case 5: CALL(5); break;          \
    case 6: CALL(6); break;          \
    default: CALL(7); break;         \
    }

}  // namespace

extern "C" FR_API fr_status fr_estep_features(fr_ctx *ctx, const float *d_FX, int64_t M, const float *d_FY,
                                              int64_t N, int32_t d, const float *sigma_f, const float *d_Y,
                                              const float *d_Yn, float *d_out, int64_t *n_vertices) {
    fr::NvtxRange nvtx_("fr_estep_features");
    if (!ctx) return FR_EINVAL;
    FScale S;
    FR_TRY(feat_scales(ctx, d, sigma_f, &S, nullptr));
    FR_TRY(feat_validate(ctx, d_FX, M, "d_FX"));
    FR_TRY(feat_validate(ctx, d_FY, N, "d_FY"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (d_Yn) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn"));
    if (!d_out) return ctx->fail(FR_EINVAL, "d_out is NULL");
    if (!d_Yn && !aligned16(d_out)) return ctx->fail(FR_EINVAL, "d_out must be 16-byte aligned (M x 4 floats)");
    const int D = d + 1;
    const long long want = 2LL * D * N;  // slots: at most D N vertices at load factor 1/2
    if (want > (long long)kFMaxSlots)
        return ctx->fail(FR_EINVAL, "observation count too large for the feature lattice (%lld slots)", want);
    cudaSetDevice(ctx->device);
    const uint32_t cap = pow2_at_least(want);
    const int stride = d_Yn ? 4 : 2;
    const long long list_len = std::min<long long>((long long)D * N, cap);
    FR_TRY(feat_ensure(ctx, cap, stride, list_len));
    FeatWorkspace *w = ctx->feat;
    FR_CUDA(ctx, cudaMemsetAsync(w->count, 0, 2 * sizeof(int), ctx->stream));
    FTable t{w->rec, w->list, w->count, cap - 1};
    const bool pt2pl = d_Yn != nullptr;
    FeatTimer tm{ctx};
#define FR_FEAT_CALL(DD)                                                                                   \
    launch_feat<DD>(pt2pl, ctx, tm, d_FX, (int)M, d_FY, (int)N, S, (const float4 *)d_Y, (const float4 *)d_Yn, \
                    t, d_out)
    FR_FEATURE_DISPATCH(d, FR_FEAT_CALL)
#undef FR_FEAT_CALL
    ctx->launches += 3;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        w->cap = 0;  // the table may hold this build's vertices: re-initialise on the next call
        return ctx->cuda(e, "feature lattice launch");
    }
    FR_CUDA(ctx, copy_async(ctx, w->h_count, w->count, 2 * sizeof(int), cudaMemcpyDeviceToHost));
    const cudaError_t se = cudaStreamSynchronize(ctx->stream);
    if (se != cudaSuccess) {
        w->cap = 0;
        return ctx->cuda(se, "feature lattice");
    }
    if (tm.n) collect_profile(ctx, tm.n);
    if (n_vertices) *n_vertices = w->h_count[0];
    return check_flags(ctx, w->h_count[1]);
}

extern "C" FR_API fr_status fr_feature_embed(fr_ctx *ctx, const float *d_F, int64_t n, int32_t d,
                                             const float *sigma_f, int32_t *d_keys, float *d_bary) {
    fr::NvtxRange nvtx_("fr_feature_embed");
    if (!ctx) return FR_EINVAL;
    FScale S;
    FR_TRY(feat_scales(ctx, d, sigma_f, &S, nullptr));
    FR_TRY(feat_validate(ctx, d_F, n, "d_F"));
    if (((uintptr_t)d_keys & 3u) || ((uintptr_t)d_bary & 3u)) return ctx->fail(FR_EINVAL, "outputs must be 4-byte aligned");
    cudaSetDevice(ctx->device);
    FR_TRY(feat_ensure_counts(ctx));
    FeatWorkspace *w = ctx->feat;
    FR_CUDA(ctx, cudaMemsetAsync(w->count + 1, 0, sizeof(int), ctx->stream));
#define FR_EMB_CALL(DD) launch_embed<DD>(ctx, d_F, (int)n, S, d_keys, d_bary, w->count + 1)
    FR_FEATURE_DISPATCH(d, FR_EMB_CALL)
#undef FR_EMB_CALL
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, copy_async(ctx, w->h_count + 1, w->count + 1, sizeof(int), cudaMemcpyDeviceToHost));
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_flags(ctx, w->h_count[1]);
}

extern "C" FR_API fr_status fr_gauss_transform_features(fr_ctx *ctx, const float *d_FX, int64_t M,
                                                        const float *d_FY, int64_t N, int32_t d,
                                                        const float *sigma_f, const float *d_Y,
                                                        const float *d_Yn, float *d_out) {
    fr::NvtxRange nvtx_("fr_gauss_transform_features");
    if (!ctx) return FR_EINVAL;
    FScale S, inv;
    FR_TRY(feat_scales(ctx, d, sigma_f, &S, &inv));
    FR_TRY(feat_validate(ctx, d_FX, M, "d_FX"));
    FR_TRY(feat_validate(ctx, d_FY, N, "d_FY"));
    FR_TRY(validate_cloud(ctx, d_Y, N, "d_Y"));
    if (d_Yn) FR_TRY(validate_cloud(ctx, d_Yn, N, "d_Yn"));
    if (!d_out || ((uintptr_t)d_out & 3u)) return ctx->fail(FR_EINVAL, "d_out is NULL or misaligned");
    cudaSetDevice(ctx->device);
    const int vd = d_Yn ? 7 : 4;
    const long long xblocks = (M + kFThreads - 1) / kFThreads;
    long long ysplit = (4LL * ctx->num_sms + xblocks - 1) / xblocks;
    const long long ymax = ((long long)N + 4 * kFExTile - 1) / (4 * kFExTile);
    ysplit = std::max<long long>(1, std::min<long long>(ysplit, ymax));
    const long long ychunk = ((N + ysplit - 1) / ysplit + kFExTile - 1) / kFExTile * kFExTile;
    ysplit = (N + ychunk - 1) / ychunk;
    if (xblocks * ysplit > (1LL << 31) - 1) return ctx->fail(FR_EINVAL, "grid too large");
    if (ysplit > 1) FR_CUDA(ctx, cudaMemsetAsync(d_out, 0, (size_t)M * vd * sizeof(float), ctx->stream));
    const int grid = (int)(xblocks * ysplit);
    const bool pt2pl = d_Yn != nullptr;
#define FR_EX_CALL(DD)                                                                                         \
    launch_exact<DD>(pt2pl, d_FX, (int)M, d_FY, (const float4 *)d_Y, (const float4 *)d_Yn, (int)N, inv,        \
                     (int)ysplit, (int)ychunk, grid, ctx->stream, d_out)
    FR_FEATURE_DISPATCH(d, FR_EX_CALL)
#undef FR_EX_CALL
    ctx->launches += 1;
    FR_CUDA(ctx, cudaGetLastError());
    FR_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return FR_OK;
}
