// Device side of the permutohedral lattice (Section 4.2 of FilterReg; the
// filter of Adams et al. 2010 it adopts), d = 3 position features, lattice
// dimension D = d + 1 = 4.
//
// embed(): elevation of f = p / sigma onto the hyperplane sum(z) = 0,
// nearest remainder-0 lattice point, rank sort of the differences, coordinate
// sum repair, barycentric weights and the 4 vertex keys of the enclosing
// simplex.  Every float operation is an explicit round-to-nearest intrinsic
// (never contracted into an FMA) in a fixed order, so that the integer keys
// are reproducible bit for bit by any IEEE-754 implementation that performs
// the same operations.
//
// The hash table is open addressing with linear probing over a power-of-two
// array of 64-byte slot records (see Table) whose first word is the key:
// three 21-bit two's-complement coordinates (the fourth is minus their sum)
// and bit 63 set; kEmpty (0) marks a free slot.  Slots are claimed with
// atomicCAS; the record's values are accumulated with float4 atomics (sm_90+
// vector atomics).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace fr {

constexpr int kD = 4;                      // lattice dimension d + 1
constexpr float kKeyLimit = 1000000.0f;    // |z_j| bound: keys fit 21-bit fields

struct Simplex {
    unsigned long long key[kD];  // packed vertex keys, vertex k = remainder-k point
    float b[kD];                 // barycentric weight of vertex k
};

// Packs coordinates 0..2 of a vertex key (the 4th is implied by sum = 0).
__device__ __forceinline__ unsigned long long pack_key(int k0, int k1, int k2) {
    return (1ull << 63) | (unsigned long long)(k0 & 0x1FFFFF) | ((unsigned long long)(k1 & 0x1FFFFF) << 21) |
           ((unsigned long long)(k2 & 0x1FFFFF) << 42);
}

__device__ __forceinline__ int unpack_coord(unsigned long long key, int j) {
    int v = (int)((key >> (21 * j)) & 0x1FFFFF);
    return (v ^ 0x100000) - 0x100000;  // sign-extend 21 bits
}

// 64-bit mix (xor-shift-multiply finaliser) -> table slot.
__device__ __forceinline__ uint32_t slot_of(unsigned long long k, uint32_t mask) {
    uint32_t h = (uint32_t)k * 0x9E3779B1u ^ (uint32_t)(k >> 32) * 0x85EBCA77u;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h & mask;
}

// Elevated coordinates, ranks and remainder-0 point of position p under the
// per-axis feature scales s = alpha / (sqrt(i (i+1)) sigma).  Returns false for
// non-finite or out-of-range coordinates.
__device__ __forceinline__ bool embed(float px, float py, float pz, float s1, float s2, float s3,
                                      Simplex &out) {
    const float c1 = __fmul_rn(px, s1);
    const float c2 = __fmul_rn(py, s2);
    const float c3 = __fmul_rn(pz, s3);
    // z_j = sum_{i > j} c_i - j c_j, accumulated from the last axis down.
    float z[kD];
    z[3] = __fsub_rn(0.0f, __fmul_rn(3.0f, c3));
    float t = __fadd_rn(0.0f, c3);
    z[2] = __fsub_rn(t, __fmul_rn(2.0f, c2));
    t = __fadd_rn(t, c2);
    z[1] = __fsub_rn(t, __fmul_rn(1.0f, c1));
    t = __fadd_rn(t, c1);
    z[0] = t;

    bool ok = true;
#pragma unroll
    for (int j = 0; j < kD; ++j) ok = ok && (fabsf(z[j]) < kKeyLimit);
    if (!ok) return false;

    // Nearest remainder-0 point (round half to even), coordinate-wise.
    int r0[kD];
    int sum = 0;
#pragma unroll
    for (int j = 0; j < kD; ++j) {
        const float q = rintf(__fmul_rn(z[j], 0.25f));
        r0[j] = (int)q * kD;
        sum += (int)q;
    }
    float dl[kD];
#pragma unroll
    for (int j = 0; j < kD; ++j) dl[j] = __fsub_rn(z[j], (float)r0[j]);

    // Rank of each difference, descending, ties to the lower index.
    int rk[kD];
#pragma unroll
    for (int j = 0; j < kD; ++j) {
        int r = 0;
#pragma unroll
        for (int k = 0; k < kD; ++k) r += (dl[k] > dl[j]) || (k < j && dl[k] == dl[j]);
        rk[j] = r;
    }
    if (sum > kD || sum < -kD) return false;
    // Repair the coordinate sum to zero.
#pragma unroll
    for (int j = 0; j < kD; ++j) {
        if (sum > 0) {
            const bool mv = rk[j] >= kD - sum;
            r0[j] -= mv ? kD : 0;
            rk[j] += mv ? sum - kD : sum;
        } else if (sum < 0) {
            const bool mv = rk[j] < -sum;
            r0[j] += mv ? kD : 0;
            rk[j] += mv ? kD + sum : sum;
        }
    }
    // u_r = (z_j - r0_j) / D for the coordinate j of rank r.
    float u[kD];
#pragma unroll
    for (int r = 0; r < kD; ++r) u[r] = 0.0f;
#pragma unroll
    for (int j = 0; j < kD; ++j) {
        const float v = __fmul_rn(__fsub_rn(z[j], (float)r0[j]), 0.25f);
#pragma unroll
        for (int r = 0; r < kD; ++r) u[r] = (rk[j] == r) ? v : u[r];
    }
    // b_m = u_{D-1-m} - u_{D-m} (m = 1..3), b_0 = u_{D-1} + (1 - u_0).
    out.b[0] = __fadd_rn(u[3], __fadd_rn(1.0f, -u[0]));
    out.b[1] = __fsub_rn(u[2], u[3]);
    out.b[2] = __fsub_rn(u[1], u[2]);
    out.b[3] = __fsub_rn(u[0], u[1]);
    // Vertex k: coordinate j is r0_j + k, minus D where rank_j > D - 1 - k.
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        int c[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) c[j] = r0[j] + k - (rk[j] > kD - 1 - k ? kD : 0);
        out.key[k] = pack_key(c[0], c[1], c[2]);
    }
    return true;
}

// Inserts `key`; returns its slot (or -1 when max_probe slots were all taken
// by other keys).  *claimed is set when this call created the vertex.
__device__ __forceinline__ int insert_key(unsigned long long *keys, uint32_t mask,
                                          unsigned long long key, uint32_t max_probe,
                                          bool &claimed, int start = -1) {
    uint32_t s = start >= 0 ? (uint32_t)start : slot_of(key, mask);
    claimed = false;
    for (uint32_t p = 0; p < max_probe; ++p) {
        unsigned long long cur = __ldcg(rec_key(keys, s));
        if (cur == key) return (int)s;
        if (cur == kEmpty) {
            cur = atomicCAS(rec_key(keys, s), kEmpty, key);
            if (cur == kEmpty) {
                claimed = true;
                return (int)s;
            }
            if (cur == key) return (int)s;
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// Slot of `key`, or -1 if absent.  The table must not change during the call
// (read through the read-only path).  An insert never places a key more than
// max_probe slots past its home, so a lookup stops there too: a full table
// (one whose build overflowed) costs at most max_probe probes, not a scan.
__device__ __forceinline__ int find_key(const unsigned long long *__restrict__ keys, uint32_t mask,
                                        unsigned long long key, uint32_t max_probe) {
    uint32_t s = slot_of(key, mask);
    for (uint32_t p = 0; p < max_probe; ++p) {
        const unsigned long long cur = __ldg(rec_key(const_cast<unsigned long long *>(keys), s));
        if (cur == key) return (int)s;
        if (cur == kEmpty) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// Four lookups with the first probes issued together (independent loads in
// flight), then any collision chains walked one by one (max_probe slots at
// most, as find_key).
__device__ __forceinline__ void find4(const unsigned long long *__restrict__ keys, uint32_t mask,
                                      const Simplex &sx, int slot[kD], uint32_t max_probe) {
    uint32_t s[kD];
    unsigned long long cur[kD];
#pragma unroll
    for (int k = 0; k < kD; ++k) s[k] = slot_of(sx.key[k], mask);
#pragma unroll
    for (int k = 0; k < kD; ++k) cur[k] = __ldg(rec_key(const_cast<unsigned long long *>(keys), s[k]));
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        uint32_t p = 1;
        while (cur[k] != sx.key[k] && cur[k] != kEmpty && p < max_probe) {
            s[k] = (s[k] + 1) & mask;
            cur[k] = __ldg(rec_key(const_cast<unsigned long long *>(keys), s[k]));
            ++p;
        }
        slot[k] = (cur[k] == sx.key[k]) ? (int)s[k] : -1;
    }
}

// Offsets of the lattice neighbour along axis `dir` in the stored coordinates
// 0..2: +1 on every coordinate and -D on coordinate `dir` (sum stays 0).
__device__ __forceinline__ unsigned long long neighbour_key(unsigned long long key, int dir,
                                                            int sign) {
    int c[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) c[j] = unpack_coord(key, j) + sign * (j == dir ? 1 - kD : 1);
    return pack_key(c[0], c[1], c[2]);
}

}  // namespace fr
