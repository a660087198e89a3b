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
// The key of round r is (k0 + r * 0x9E3779B9, k1 + r * 0xBB67AE85): each is
// one add of a compile-time constant to the seed words, off the dependency
// chain of the rounds.
struct Key {
    uint32_t k0, k1;
};

__device__ __forceinline__ uint4 philox_sched(uint4 c, Key k) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ (k.k0 + (uint32_t)r * 0x9E3779B9u), (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ (k.k1 + (uint32_t)r * 0xBB67AE85u), (uint32_t)p0);
    }
    return c;
}

// Counter layout: (draw block, slot, tag << 28 | instruction ordinal, 64-shot word).
constexpr uint32_t kTagNoise = 0u << 28;
constexpr uint32_t kTagCollapse = 1u << 28;
constexpr uint32_t kTagInit = 2u << 28;

// 64 fair bits for a collapse (tag COLLAPSE) or the initial frame (tag INIT):
// draws 0 and 1 of the keyed stream.
__device__ __forceinline__ uint64_t half_mask(Key key, uint32_t tag_instr, uint32_t slot, uint32_t word) {
    const uint4 r = philox_sched(make_uint4(0u, slot, tag_instr, word), key);
    return (uint64_t)r.x | ((uint64_t)r.y << 32);
}

// Sequential draws of one keyed stream; block j/4 is generated on demand.
struct DrawStream {
    uint4 blk;
    uint32_t j, slot, ti, word;
    Key key;

    __device__ __forceinline__ DrawStream(Key key_, uint32_t ti_, uint32_t slot_, uint32_t word_, uint4 blk0)
        : blk(blk0), j(0), slot(slot_), ti(ti_), word(word_), key(key_) {}

    __device__ __forceinline__ uint32_t next() {
        const uint32_t lane = j & 3u;
        if (lane == 0u && j != 0u) blk = philox_sched(make_uint4(j >> 2, slot, ti, word), key);
        j++;
        return lane == 0u ? blk.x : lane == 1u ? blk.y : lane == 2u ? blk.z : blk.w;
    }
};

// General procedure: exact geometric gaps. With G the threshold table of p, a
// draw u gives the gap min{k : u < G[k]} to the next error. The first test
// asks whether the next error falls beyond bit 63 (u >= G[remaining - 1]);
// only otherwise is the gap located by binary search. DEPOLARIZE1 spends one
// more draw v per error on the Pauli 1 + floor(3v / 2^32) (1 X, 2 Y, 3 Z);
// DEPOLARIZE2 on c = 1 + floor(15v / 2^32), first-qubit Pauli c >> 2, second c & 3.
template <uint32_t OP>
__device__ __forceinline__ void noise_masks_slow(const uint64_t *__restrict__ G, Key key, uint32_t instr,
                                                 uint32_t slot, uint32_t word, uint4 blk0, uint64_t &xa,
                                                 uint64_t &za, uint64_t &xb, uint64_t &zb) {
    DrawStream ds(key, kTagNoise | instr, slot, word, blk0);
    int pos = -1;
    xa = za = xb = zb = 0;
    for (;;) {
        const int remaining = 63 - pos;
        if (remaining <= 0) break;
        const uint32_t u = ds.next();
        if ((uint64_t)u >= __ldg(G + remaining - 1)) break;
        int lo = 0, hi = remaining - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((uint64_t)u < __ldg(G + mid)) hi = mid;
            else lo = mid + 1;
        }
        pos += lo + 1;
        const uint64_t bit = 1ull << pos;
        if (OP == OP_XERR) {
            xa |= bit;
        } else if (OP == OP_ZERR) {
            za |= bit;
        } else if (OP == OP_DEP1) {
            const uint32_t pa = 1u + (uint32_t)((3ull * ds.next()) >> 32);
            if (pa <= 2u) xa |= bit;
            if (pa >= 2u) za |= bit;
        } else {
            const uint32_t c = 1u + (uint32_t)((15ull * ds.next()) >> 32);
            const uint32_t pa = c >> 2, pb = c & 3u;
            if (pa == 1u || pa == 2u) xa |= bit;
            if (pa >= 2u) za |= bit;
            if (pb == 1u || pb == 2u) xb |= bit;
            if (pb >= 2u) zb |= bit;
        }
    }
}

// Error masks of one noise slot over the 64 shots of one word. The first draw
// alone decides the common case: no error in the word exactly when
// u0 >= G[63]. Only then is the general procedure run (out of line).
template <uint32_t OP>
__device__ __forceinline__ bool noise_masks(const uint64_t *__restrict__ G, Key key, uint32_t instr, uint32_t slot,
                                            uint32_t word, uint64_t &xa, uint64_t &za, uint64_t &xb,
                                            uint64_t &zb) {
    const uint4 blk0 = philox_sched(make_uint4(0u, slot, kTagNoise | instr, word), key);
    if ((uint64_t)blk0.x >= __ldg(G + 63)) return false;
    noise_masks_slow<OP>(G, key, instr, slot, word, blk0, xa, za, xb, zb);
    return true;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

}  // namespace stimgb
