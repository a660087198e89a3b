// device.cuh -- device-side building blocks shared by the CUDA kernels:
// Philox4x32-10, the keyed collapse/init/noise masks, bounded grid barrier.
#pragma once

#include <cstdint>

#include "internal.h"

namespace stimgb {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// -> 64-bit multiplies; the key follows the Weyl sequence
// (k0, k1) += (0x9E3779B9, 0xBB67AE85) after every round.
// ---------------------------------------------------------------------------
// The key of round r is (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85).
struct Key {
    uint32_t k0, k1;
};

// ---- shared-memory helpers (32-bit shared-window addresses) ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t lds64(uint32_t a) {
    uint64_t v;
    asm volatile("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts64(uint32_t a, uint64_t v) {
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Round keys precomputed once per CTA in shared memory: 10 rounds as 5
// 16-byte vectors (k0_2i, k1_2i, k0_2i+1, k1_2i+1).
struct SmemKeys {
    uint32_t sa;
    __device__ __forceinline__ uint4 pair(int i) const { return lds128(sa + 16u * (uint32_t)i); }
};

// Round keys in the kernel's parameter space (constant bank): with the index
// known at compile time they are operands of the round's instructions, no
// loads at all.
struct ParamKeys {
    const uint32_t *rk;
    __device__ __forceinline__ uint4 pair(int i) const {
        return make_uint4(rk[4 * i], rk[4 * i + 1], rk[4 * i + 2], rk[4 * i + 3]);
    }
};

__device__ __forceinline__ void write_round_keys(uint32_t *dst, Key k) {
    // called by threads 0..9 of a CTA: dst[2r] = k0 + r W0, dst[2r + 1] = k1 + r W1
    const uint32_t r = threadIdx.x;
    if (r < 10) {
        dst[2 * r] = k.k0 + r * 0x9E3779B9u;
        dst[2 * r + 1] = k.k1 + r * 0xBB67AE85u;
    }
}

__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1,
                      (uint32_t)p0);
}

template <class K>
__device__ __forceinline__ uint4 philox_sched(uint4 c, K k) {
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const uint4 kk = k.pair(i);
        c = philox_round(c, kk.x, kk.y);
        c = philox_round(c, kk.z, kk.w);
    }
    return c;
}

// Counter layout: (draw block, slot, tag << 28 | instruction ordinal, 64-shot word).
constexpr uint32_t kTagNoise = 0u << 28;
constexpr uint32_t kTagCollapse = 1u << 28;
constexpr uint32_t kTagInit = 2u << 28;

// 64 fair bits for a collapse (tag COLLAPSE) or the initial frame (tag INIT):
// draws 0 and 1 of the keyed stream.
template <class K>
__device__ __forceinline__ uint64_t half_mask(K key, uint32_t tag_instr, uint32_t slot, uint32_t word) {
    const uint4 r = philox_sched(make_uint4(0u, slot, tag_instr, word), key);
    return (uint64_t)r.x | ((uint64_t)r.y << 32);
}

// Gap to the next error for a draw u with u < G[63]: min{k : u < G[k]}.
// With the channel's per-shot probability q, G[k] is about
// 2^32 (1 - (1 - q)^(k + 1)), so k is about floor(log2(1 - u / 2^32) /
// log2(1 - q)); inv = 1 / log2(1 - q) comes with the table. The estimate
// is checked against G[k - 1] <= u < G[k] (two independent loads) and moved
// a step at a time until it holds, so the result is the table's exactly;
// float rounding only decides how many steps that takes (almost always 0).
__device__ __forceinline__ int geo_gap(const uint64_t *__restrict__ G, uint32_t u, float inv) {
    const float y = __log2f(1.0f - (float)u * 2.3283064365386963e-10f) * inv;
    int k = (int)y;             // y >= 0; saturates for infinities
    k = k < 0 ? 0 : k > 63 ? 63 : k;
    const uint64_t lo = k > 0 ? __ldg(G + k - 1) : 0ull, hi = __ldg(G + k);
    if ((uint64_t)u < lo) {
        do k--;
        while (k > 0 && (uint64_t)u < __ldg(G + k - 1));
    } else if ((uint64_t)u >= hi) {
        do k++;
        while ((uint64_t)u >= __ldg(G + k));     // ends by k = 63: u < G[63]
    }
    return k;
}

// Pauli index of a channel hit: 1 + #{i : v >= T[i]} over the table's 15
// non-decreasing choice thresholds. A uniform (depolarizing) channel over m
// Paulis stores m in T[15] and thresholds ceil(i 2^32 / m), for which the
// count equals floor(m v / 2^32): one multiply instead of the scan.
__device__ __forceinline__ uint32_t pauli_choice(const uint64_t *__restrict__ T, uint32_t v) {
    const uint64_t m = __ldg(T + 15) & 0xFFFFFFFFull;
    if (m) return 1u + (uint32_t)((m * v) >> 32);
    uint32_t c = 1;
#pragma unroll 1
    while (c < 16u && (uint64_t)v >= __ldg(T + c - 1)) c++;
    return c;
}

// General procedure: exact geometric gaps. With G the table of the channel
// (kNoiseTableWords words: gap thresholds G[0..63], then Pauli-choice
// thresholds T[0..14] and T[15]), a draw u gives the gap min{k : u < G[k]} to the next error;
// the error process stops at the first draw with u >= G[remaining - 1] (next
// error beyond bit 63). The caller has drawn block 0 and found an error: its
// first word, draw 0, satisfies blk0.x < G[63]. X_ERROR, Y_ERROR and Z_ERROR
// put X, Y or Z at each error; the one-qubit channels (DEPOLARIZE1,
// PAULI_CHANNEL_1) spend one more draw v per error on the Pauli c =
// pauli_choice(v) (1 X, 2 Y, 3 Z), the two-qubit channels (DEPOLARIZE2,
// PAULI_CHANNEL_2) on c with first-qubit Pauli c >> 2 and second c & 3. For
// the depolarizing channels c = 1 + floor(3v / 2^32) and 1 + floor(15v / 2^32).
template <class K>
__device__ __forceinline__ void noise_masks_slow(uint32_t opc, const uint64_t *__restrict__ G, K key, uint32_t instr,
                                                 uint32_t slot, uint32_t word, uint4 blk0, uint64_t &xa,
                                                 uint64_t &za, uint64_t &xb, uint64_t &zb) {
    uint4 blk = blk0;
    uint32_t j = 1;                       // index of the next draw
    auto next = [&]() -> uint32_t {
        const uint32_t l = j & 3u;
        if (l == 0u) blk = philox_sched(make_uint4(j >> 2, slot, kTagNoise | instr, word), key);
        j++;
        return l == 0u ? blk.x : l == 1u ? blk.y : l == 2u ? blk.z : blk.w;
    };
    const float inv = __uint_as_float((uint32_t)(__ldg(G + 79) >> 32));    // T[15]'s high half
    xa = za = xb = zb = 0;
    uint32_t u = blk0.x;
    int pos = -1;
    for (;;) {
        pos += geo_gap(G, u, inv) + 1;
        const uint64_t bit = 1ull << pos;
        if (opc == OP_XERR) {
            xa |= bit;
        } else if (opc == OP_ZERR) {
            za |= bit;
        } else if (opc == OP_DEP1 || opc == OP_DEP2) {
            const uint32_t c = pauli_choice(G + 64, next());
            const uint32_t pa = opc == OP_DEP1 ? c : c >> 2, pb = opc == OP_DEP1 ? 0u : c & 3u;
            if (pa == 1u || pa == 2u) xa |= bit;
            if (pa >= 2u) za |= bit;
            if (pb == 1u || pb == 2u) xb |= bit;
            if (pb >= 2u) zb |= bit;
        } else {                // Y_ERROR
            xa |= bit;
            za |= bit;
        }
        if (pos >= 63) break;
        u = next();
        if ((uint64_t)u >= __ldg(G + (62 - pos))) break;    // G[remaining - 1], remaining = 63 - pos
    }
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace stimgb
