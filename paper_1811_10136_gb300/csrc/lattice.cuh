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
// three 21-bit coordinates biased by 2^20 (the fourth is minus their sum) and
// bit 63 set; kEmpty (0) marks a free slot.  With non-negative fields, moving
// to a neighbouring vertex is one 64-bit addition of packed offsets.  Slots
// are claimed with atomicCAS; the record's values are accumulated with float4
// atomics (sm_90+ vector atomics).
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

constexpr int kKeyBias = 1 << 20;                      // stored field = coordinate + 2^20
constexpr unsigned long long kKeyOne = 1ull | (1ull << 21) | (1ull << 42);  // +1 on every field

// Packs coordinates 0..2 of a vertex key (the 4th is implied by sum = 0).
// |coordinate| < 2^20 (kKeyLimit keeps it so), so every field is in [0, 2^21).
__device__ __forceinline__ unsigned long long pack_key(int k0, int k1, int k2) {
    return (1ull << 63) | (unsigned long long)(unsigned)(k0 + kKeyBias) |
           ((unsigned long long)(unsigned)(k1 + kKeyBias) << 21) |
           ((unsigned long long)(unsigned)(k2 + kKeyBias) << 42);
}

__device__ __forceinline__ int unpack_coord(unsigned long long key, int j) {
    return (int)((key >> (21 * j)) & 0x1FFFFF) - kKeyBias;
}

// Key -> table slot: the two 32-bit halves multiplied by odd constants and
// summed, the high half folded onto the low bits.
__device__ __forceinline__ uint32_t slot_of(unsigned long long k, uint32_t mask) {
    uint32_t h = (uint32_t)k * 0x9E3779B1u + (uint32_t)(k >> 32) * 0x85EBCA77u;
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
    const float z3 = __fsub_rn(0.0f, __fmul_rn(3.0f, c3));
    float t = __fadd_rn(0.0f, c3);
    const float z2 = __fsub_rn(t, __fmul_rn(2.0f, c2));
    t = __fadd_rn(t, c2);
    const float z1 = __fsub_rn(t, __fmul_rn(1.0f, c1));
    t = __fadd_rn(t, c1);
    const float z0 = t;
    if (!(fabsf(z0) < kKeyLimit && fabsf(z1) < kKeyLimit && fabsf(z2) < kKeyLimit && fabsf(z3) < kKeyLimit))
        return false;

    // Nearest remainder-0 point (round half to even), coordinate-wise: 4 q_j.
    const float q0 = rintf(__fmul_rn(z0, 0.25f)), q1 = rintf(__fmul_rn(z1, 0.25f));
    const float q2 = rintf(__fmul_rn(z2, 0.25f)), q3 = rintf(__fmul_rn(z3, 0.25f));
    const int sum = (int)q0 + (int)q1 + (int)q2 + (int)q3;
    if (sum > kD || sum < -kD) return false;
    const float d0 = __fsub_rn(z0, 4.0f * q0), d1 = __fsub_rn(z1, 4.0f * q1);
    const float d2 = __fsub_rn(z2, 4.0f * q2), d3 = __fsub_rn(z3, 4.0f * q3);

    // Rank of each difference, descending, ties to the lower index: of a
    // pair j < k, j comes first iff d_j >= d_k.  The ranks start at the
    // coordinate sum, which the repair below adds to every rank.
    const bool p01 = d0 >= d1, p02 = d0 >= d2, p03 = d0 >= d3;
    const bool p12 = d1 >= d2, p13 = d1 >= d3, p23 = d2 >= d3;
    int r0 = sum + !p01 + !p02 + !p03;
    int r1 = sum + p01 + !p12 + !p13;
    int r2 = sum + p02 + p12 + !p23;
    int r3 = sum + p03 + p13 + p23;
    // Repair of the coordinate sum to zero: a coordinate whose shifted rank
    // leaves [0, D) wraps around (rank mod D) and its remainder-0 coordinate
    // moves by -D floor(rank / D).
    const int m0 = (int)q0 - (r0 >> 2), m1 = (int)q1 - (r1 >> 2);
    const int m2 = (int)q2 - (r2 >> 2), m3 = (int)q3 - (r3 >> 2);
    r0 &= 3; r1 &= 3; r2 &= 3; r3 &= 3;

    // u_r = (z_j - r0_j) / D for the coordinate j of rank r.
    const float v0 = __fmul_rn(__fsub_rn(z0, (float)(4 * m0)), 0.25f);
    const float v1 = __fmul_rn(__fsub_rn(z1, (float)(4 * m1)), 0.25f);
    const float v2 = __fmul_rn(__fsub_rn(z2, (float)(4 * m2)), 0.25f);
    const float v3 = __fmul_rn(__fsub_rn(z3, (float)(4 * m3)), 0.25f);
    auto of_rank = [&](int r) { return r0 == r ? v0 : (r1 == r ? v1 : (r2 == r ? v2 : v3)); };
    const float u0 = of_rank(0), u1 = of_rank(1), u2 = of_rank(2), u3 = of_rank(3);
    // b_m = u_{D-1-m} - u_{D-m} (m = 1..3), b_0 = u_{D-1} + (1 - u_0).
    out.b[0] = __fadd_rn(u3, __fadd_rn(1.0f, -u0));
    out.b[1] = __fsub_rn(u2, u3);
    out.b[2] = __fsub_rn(u1, u2);
    out.b[3] = __fsub_rn(u0, u1);
    // Vertex k: coordinate j is r0_j + k, minus D where rank_j > D - 1 - k.
    // Vertex k follows from vertex k - 1 by +1 on every coordinate and -D on
    // the coordinate of rank D - k (no stored field when that is coordinate 3).
    unsigned long long key = pack_key(4 * m0, 4 * m1, 4 * m2);
    out.key[0] = key;
#pragma unroll
    for (int k = 1; k < kD; ++k) {
        const int r = kD - k;
        const unsigned long long down = (r0 == r ? 4ull : 0ull) | (r1 == r ? 4ull << 21 : 0ull) |
                                        (r2 == r ? 4ull << 42 : 0ull);
        key = key + kKeyOne - down;
        out.key[k] = key;
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

// insert_key for the four vertices of one point, those in `want`: the four
// home-slot loads are in flight together, then the compare-and-swaps of the
// empty ones together; only a collision walks on (insert_key from the next
// slot, the remaining max_probe - 1 probes).  slot[k] = -1 for a vertex not
// wanted or not placed; bit k of *claimed set where this call created it.
__device__ __forceinline__ void insert4(unsigned long long *keys, uint32_t mask, const Simplex &sx,
                                        unsigned want, uint32_t max_probe, int slot[kD],
                                        unsigned &claimed) {
    uint32_t s[kD];
    unsigned long long cur[kD];
    claimed = 0;
#pragma unroll
    for (int k = 0; k < kD; ++k) s[k] = slot_of(sx.key[k], mask);
#pragma unroll
    for (int k = 0; k < kD; ++k) cur[k] = ((want >> k) & 1u) ? __ldcg(rec_key(keys, s[k])) : 0ull;
#pragma unroll
    for (int k = 0; k < kD; ++k)
        if (((want >> k) & 1u) && cur[k] == kEmpty) {
            cur[k] = atomicCAS(rec_key(keys, s[k]), kEmpty, sx.key[k]);
            if (cur[k] == kEmpty) {
                claimed |= 1u << k;
                cur[k] = sx.key[k];
            }
        }
#pragma unroll
    for (int k = 0; k < kD; ++k) {
        slot[k] = -1;
        if (!((want >> k) & 1u)) continue;
        if (cur[k] == sx.key[k]) {
            slot[k] = (int)s[k];
        } else if (max_probe > 1) {
            bool c;
            slot[k] = insert_key(keys, mask, sx.key[k], max_probe - 1, c, (int)((s[k] + 1) & mask));
            claimed |= c ? 1u << k : 0u;
        }
    }
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
