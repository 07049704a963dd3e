// fr_estep_noalloc: the E step (lattice build + splat over the observation,
// slice at the moved model points) on scratch memory compiled into the
// library, for callers that cannot call cudaMalloc.
//
// Who needs it: a caller whose device memory is owned by another allocator
// (a framework that has reserved the GPU's memory up front and forbids
// other allocations), or a real-time loop that must not take the
// device-wide synchronisation that cudaMalloc / cudaFree can cause.  Such a
// caller passes its own input and output buffers; the hash table, the list of
// claimed slots and two counters live in the file-scope array below.
//
// The array costs every GPU that loads the library about 4.5 MB until the
// process exits.  It bounds the observation cloud to FR_NOALLOC_MAX_OBS
// points (the table has 65,536 slots, at least 6 per possible point, which
// is more than the at most 4 vertices a point creates).
//
// Every call shares the one array.  A call leaves the table empty again
// (it frees the slots its build claimed) and zeroes the counters it uses at
// its start, so consecutive calls are independent; calls that overlap on the
// GPU (from several streams or threads at once) race on the array and give
// wrong results.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "filterreg.h"
#include "lattice.cuh"

namespace {

using fr::kD;
using fr::Simplex;

constexpr int kThreads = 256;
constexpr uint32_t kCap = 65536;  // table slots, a power of two >= 6 * FR_NOALLOC_MAX_OBS
static_assert(kCap >= 6u * FR_NOALLOC_MAX_OBS, "table too small for the point bound");

// Byte layout of the scratch array.
constexpr size_t kKeysOff = 0;                                       // kCap slot records
constexpr size_t kListOff = kKeysOff + kCap * fr::kRecWords * 8;     // kCap x int claimed slots
constexpr size_t kCountOff = kListOff + kCap * 4;         // int[2]: claimed count, flags
constexpr size_t kScratchBytes = kCountOff + 256;

constexpr int kFlagRange = 1, kFlagCapacity = 2;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct View {
    unsigned long long *keys;  // slot records (key, 16-bit record, v0, v1)
    int *list, *count, *flags;
};

View view_of(unsigned char *base) {
    View v;
    v.keys = reinterpret_cast<unsigned long long *>(base + kKeysOff);
    v.list = reinterpret_cast<int *>(base + kListOff);
    v.count = reinterpret_cast<int *>(base + kCountOff);
    v.flags = v.count + 1;
    return v;
}

// Splat [1, y] (and [n, 0] with normals) onto the lattice over Y.
__global__ void k_na_build(const float4 *__restrict__ Y, const float4 *__restrict__ Yn, int N,
                           float s1, float s2, float s3, View v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 y = __ldg(Y + i);
    Simplex sx;
    if (!fr::embed(y.x, y.y, y.z, s1, s2, s3, sx)) {
        atomicOr(v.flags, kFlagRange);
        return;
    }
    const float4 n = Yn ? __ldg(Yn + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        bool claimed;
        const int s = fr::insert_key(v.keys, kCap - 1, sx.key[k], kCap, claimed);
        if (s < 0) {
            atomicOr(v.flags, kFlagCapacity);
            continue;
        }
        if (claimed) v.list[atomicAdd(v.count, 1)] = s;
        const float b = sx.b[k];
        atomicAdd(fr::rec_v0(v.keys, s), make_float4(b, b * y.x, b * y.y, b * y.z));
        if (Yn) atomicAdd(fr::rec_v1(v.keys, s), make_float4(b * n.x, b * n.y, b * n.z, 0.f));
    }
}

struct Pose {
    float p[12];  // row-major 3 x 4
};

// Slice at x = T x_ref: out[i] = [M0, M1 (, Nsum)].  The moved position is
// formed as ((T_j0 x + T_j1 y) + T_j2 z) + T_j3 with every operation rounded.
__global__ void k_na_slice(const float4 *__restrict__ X, int M, Pose T, float s1, float s2,
                           float s3, View v, int with_normals, float *out) {
    const int vd = with_normals ? 7 : 4;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) {
        const float4 r = __ldg(X + i);
        float x[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float a = __fadd_rn(__fmul_rn(T.p[4 * j], r.x), __fmul_rn(T.p[4 * j + 1], r.y));
            x[j] = __fadd_rn(__fadd_rn(a, __fmul_rn(T.p[4 * j + 2], r.z)), T.p[4 * j + 3]);
        }
        float acc[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        Simplex sx;
        if (fr::embed(x[0], x[1], x[2], s1, s2, s3, sx)) {
            int slot[kD];
            fr::find4(v.keys, kCap - 1, sx, slot, kCap);
#pragma unroll
            for (int k = 0; k < kD; ++k) {
                if (slot[k] < 0) continue;
                const float b = sx.b[k];
                const float4 a = __ldcg(fr::rec_v0(v.keys, slot[k]));
                acc[0] += b * a.x; acc[1] += b * a.y; acc[2] += b * a.z; acc[3] += b * a.w;
                if (with_normals) {
                    const float4 c = __ldcg(fr::rec_v1(v.keys, slot[k]));
                    acc[4] += b * c.x; acc[5] += b * c.y; acc[6] += b * c.z;
                }
            }
        } else {
            atomicOr(v.flags, kFlagRange);
        }
        for (int c = 0; c < vd; ++c) out[(size_t)i * vd + c] = acc[c];
    }
}

// Leave the table empty for the next call: free every slot the build listed.
__global__ void k_na_clear(View v) {
    const int n = *v.count;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float4 *r = reinterpret_cast<float4 *>(fr::rec_key(v.keys, (uint32_t)v.list[e]));
        r[0] = z;
        r[1] = z;
        r[2] = z;
        r[3] = z;
    }
}

// Per-device set-up: the device address of the array (host code may not use
// the symbol itself) and an empty table.  It runs under a per-device mutex
// and is marked done only when it succeeded, so a failed set-up (say a first
// call made while the stream was being captured, which is refused) is tried
// again by the next call instead of failing every later one.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu[kMaxDevices];
unsigned char *g_base[kMaxDevices];  // written under the mutex, then only read
bool g_ready[kMaxDevices];

// FR_OK once device `dev` has its scratch address and an empty table.
fr_status setup_device(int dev, cudaStream_t stream) {
    std::lock_guard<std::mutex> lock(g_setup_mu[dev]);
    if (g_ready[dev]) return FR_OK;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return FR_EINVAL;  // set-up synchronises: not while capturing
    unsigned char *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, kScratchBytes, stream);  // free slots are zero
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    g_base[dev] = p;
    g_ready[dev] = true;
    return FR_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

extern "C" FR_API fr_status fr_estep_noalloc(const float *d_X, int64_t M, const float *d_Y,
                                             const float *d_Yn, int64_t N, float sigma,
                                             const double T[16], float *d_out,
                                             void *cuda_stream) {
    if (!d_X || !d_Y || !d_out || !T) return FR_EINVAL;
    if (M < 1 || M > (1ll << 30) || N < 1 || N > FR_NOALLOC_MAX_OBS) return FR_EINVAL;
    if (!aligned16(d_X) || !aligned16(d_Y) || (d_Yn && !aligned16(d_Yn))) return FR_EINVAL;
    if (!(sigma > 0.0f) || !std::isfinite(sigma)) return FR_EINVAL;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(T[i])) return FR_EINVAL;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    const fr_status ss = setup_device(dev, stream);
    if (ss != FR_OK) return ss;
    const View v = view_of(g_base[dev]);

    // Feature scales alpha / (sqrt(i (i+1)) sigma), alpha = sqrt(2/3) (d+1).
    const double alpha = std::sqrt(2.0 / 3.0) * 4.0;
    float s[3];
    for (int i = 1; i <= 3; ++i) s[i - 1] = (float)(alpha / std::sqrt((double)(i * (i + 1))) / (double)sigma);
    Pose P;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 4; ++c) P.p[4 * r + c] = (float)T[4 * r + c];

    cudaError_t e = cudaMemsetAsync(v.count, 0, 2 * sizeof(int), stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    k_na_build<<<(int)((N + kThreads - 1) / kThreads), kThreads, 0, stream>>>(
        (const float4 *)d_Y, (const float4 *)d_Yn, (int)N, s[0], s[1], s[2], v);
    long long gs = (M + kThreads - 1) / kThreads;
    if (gs > 4096) gs = 4096;
    k_na_slice<<<(int)gs, kThreads, 0, stream>>>((const float4 *)d_X, (int)M, P, s[0], s[1], s[2], v,
                                                 d_Yn ? 1 : 0, d_out);
    k_na_clear<<<(int)((4 * N + kThreads - 1) / kThreads), kThreads, 0, stream>>>(v);
    int flags = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, v.flags, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FR_ECUDA;
    }
    if (flags & kFlagCapacity) return FR_ECAPACITY;
    if (flags & kFlagRange) return FR_EINVAL;
    return FR_OK;
}
