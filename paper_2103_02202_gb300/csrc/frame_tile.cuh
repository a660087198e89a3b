// frame_tile.cuh -- device code of the Pauli-frame propagation, shared by
// the per-circuit kernel (frame.cu) and the batched persistent kernel
// (batch.cu).
//
// Dynamic shared memory of one tile (byte offsets from the region start;
// H = kTileHeaderBytes):
//   [0, 80)                  Philox round keys of the seed
//   [256, H)                 per-warp queues of deferred noise hits
//   [H, H + R)               program metadata (prog | rank_tab | segs) when it
//                            fits the R = meta_region bytes reserved for it
//   [H + R, ...)             frame rows (shared-memory layout)
// Frame layout (W 64-shot words per tile): each qubit owns a row of 2W words,
// its X words then its Z words,
//     shared memory:  row(q) = q * 2W;  X = word w, Z = word W + w of the row,
//                     16-byte chunks XOR-swizzled by q (row_word)
//     global memory:  row(q) = gframe + q * 2G + tile0;  Z = row[G + w]
// (G = words of the call), so one offset addresses both planes of a qubit.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace stimgb {
namespace frame_detail {


__device__ __forceinline__ DevOp as_op(uint4 v) { return DevOp{v.x, v.y, v.z, v.w}; }

// Layer barrier of the tile, split in two halves: arrive when this thread's
// frame writes of the layer are done, wait before the next layer touches the
// frame. A single CTA uses its CTA barrier; a cluster's release/acquire
// barrier also orders the CTA's own shared-memory accesses.
template <int C>
__device__ __forceinline__ void tile_arrive() {
    if constexpr (C > 1) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    else __syncthreads();
}
template <int C>
__device__ __forceinline__ void tile_wait() {
    if constexpr (C > 1) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The tile as seen from one CTA of the cluster.
template <int W, int C, bool GMEM>
struct Tile {
    uint32_t fsa;        // shared address of row 0 (shared layout)
    uint64_t *base;      // row 0, word 0 of the tile (global layout)
    uint64_t gstride;    // G (global layout)
    uint32_t rank;
};

// Words per thread: a thread applies each op to V consecutive words of the
// tile (W / V threads share a chain when W > V).
template <int W>
struct VecWidth {
    static constexpr int V = W < 4 ? W : 4;
};

// 16-byte shared-memory accesses: this CTA (shared::cta window) or a peer
// CTA of the cluster (shared::cluster window, address from mapa).
__device__ __forceinline__ void lds_v2(uint32_t a, uint64_t &v0, uint64_t &v1) {
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "r"(a) : "memory");
}
__device__ __forceinline__ void sts_v2(uint32_t a, uint64_t v0, uint64_t v1) {
    asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(v0), "l"(v1) : "memory");
}
__device__ __forceinline__ void ldc_v2(uint32_t a, uint64_t &v0, uint64_t &v1) {
    asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "r"(a) : "memory");
}
__device__ __forceinline__ void stc_v2(uint32_t a, uint64_t v0, uint64_t v1) {
    asm volatile("st.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(v0), "l"(v1) : "memory");
}
__device__ __forceinline__ uint64_t ldc64(uint32_t a) {
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void stc64(uint32_t a, uint64_t v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ uint32_t mapa_rank(uint32_t sa, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
    return ra;
}

// Shared-layout address of word widx (0..2W-1: X words, then Z words) of the
// row of local qubit q. The row's 16-byte chunks are XOR-swizzled by the low
// bits of q, so lanes reading the same word of different qubits spread over
// the banks instead of all starting on the same bank.
template <int W>
__device__ __forceinline__ uint32_t row_word(uint32_t fsa, uint32_t q, uint32_t widx) {
    const uint32_t chunk = (widx >> 1) ^ (q & (uint32_t)(W - 1));
    return fsa + q * (16u * W) + chunk * 16u + (widx & 1u) * 8u;
}

// V words of one qubit's X and Z planes.
template <int V>
struct Planes {
    uint64_t x[V], z[V];
};

// One qubit's V words at word offset wo of the tile; a qubit reference is
// (rank << 24 | local index), other ranks are reached through distributed
// shared memory.
template <int W, int C, bool GMEM>
struct Qubit;

template <int W, int C>
struct Qubit<W, C, false> {
    static constexpr int V = VecWidth<W>::V;
    // shared::cta (C == 1) or shared::cluster (mapa to the owning CTA) address
    // of the qubit's row, its local index q and the first word wo of the group
    uint32_t row, q, wo;

    __device__ __forceinline__ Qubit(const Tile<W, C, false> &t, uint32_t ref, uint32_t wo_) {
        q = ref & 0xFFFFFFu;
        wo = wo_;
        row = t.fsa + q * (16u * W);
        if constexpr (C > 1) row = mapa_rank(row, ref >> 24);
    }
    // address of word widx of the row (same swizzle as row_word)
    __device__ __forceinline__ uint32_t at(uint32_t widx) const {
        return row + (((widx >> 1) ^ (q & (uint32_t)(W - 1))) * 16u) + (widx & 1u) * 8u;
    }
    __device__ __forceinline__ void ld(uint32_t plane, uint64_t (&v)[V]) const {
        if constexpr (V == 1) {
            const uint32_t a = at(plane * W + wo);
            v[0] = C > 1 ? ldc64(a) : lds64(a);
        } else {
#pragma unroll
            for (int i = 0; i < V / 2; i++) {
                const uint32_t a = at(plane * W + wo + 2u * i);
                if constexpr (C > 1) ldc_v2(a, v[2 * i], v[2 * i + 1]);
                else lds_v2(a, v[2 * i], v[2 * i + 1]);
            }
        }
    }
    __device__ __forceinline__ void st(uint32_t plane, const uint64_t (&v)[V]) const {
        if constexpr (V == 1) {
            const uint32_t a = at(plane * W + wo);
            if constexpr (C > 1) stc64(a, v[0]);
            else sts64(a, v[0]);
        } else {
#pragma unroll
            for (int i = 0; i < V / 2; i++) {
                const uint32_t a = at(plane * W + wo + 2u * i);
                if constexpr (C > 1) stc_v2(a, v[2 * i], v[2 * i + 1]);
                else sts_v2(a, v[2 * i], v[2 * i + 1]);
            }
        }
    }
    __device__ __forceinline__ void load(const Tile<W, C, false> &, Planes<V> &p) const {
        if constexpr (W == 1) {      // X and Z of the word share one 16-byte chunk
            if constexpr (C > 1) ldc_v2(row, p.x[0], p.z[0]);
            else lds_v2(row, p.x[0], p.z[0]);
        } else {
            ld(0, p.x);
            ld(1, p.z);
        }
    }
    __device__ __forceinline__ void store(const Tile<W, C, false> &, const Planes<V> &p) const {
        if constexpr (W == 1) {
            if constexpr (C > 1) stc_v2(row, p.x[0], p.z[0]);
            else sts_v2(row, p.x[0], p.z[0]);
        } else {
            st(0, p.x);
            st(1, p.z);
        }
    }
    // word wo + i of the X and Z planes ^= (mx, mz); only this thread
    // touches the qubit in this layer
    __device__ __forceinline__ void xor_word(const Tile<W, C, false> &t, uint32_t i, uint64_t mx, uint64_t mz) const {
        if constexpr (W == 1) {
            Planes<1> p;
            load(t, p);
            p.x[0] ^= mx;
            p.z[0] ^= mz;
            store(t, p);
        } else {
            const uint32_t ax = at(wo + i), az = at(W + wo + i);
            if constexpr (C > 1) {
                stc64(ax, ldc64(ax) ^ mx);
                stc64(az, ldc64(az) ^ mz);
            } else {
                sts64(ax, lds64(ax) ^ mx);
                sts64(az, lds64(az) ^ mz);
            }
        }
    }
    __device__ __forceinline__ void store_x(const Tile<W, C, false> &, const uint64_t (&x)[V]) const { st(0, x); }
    __device__ __forceinline__ void store_z(const Tile<W, C, false> &, const uint64_t (&z)[V]) const { st(1, z); }
};

template <int W, int C>
struct Qubit<W, C, true> {
    static constexpr int V = VecWidth<W>::V;
    uint64_t *p;

    __device__ __forceinline__ Qubit(const Tile<W, C, true> &t, uint32_t ref, uint32_t wo) {
        p = t.base + (uint64_t)(ref & 0xFFFFFFu) * (2 * t.gstride) + wo;
    }
    __device__ __forceinline__ void load(const Tile<W, C, true> &t, Planes<V> &q) const {
#pragma unroll
        for (int i = 0; i < V; i++) {
            q.x[i] = p[i];
            q.z[i] = p[t.gstride + i];
        }
    }
    __device__ __forceinline__ void store(const Tile<W, C, true> &t, const Planes<V> &q) const {
#pragma unroll
        for (int i = 0; i < V; i++) {
            p[i] = q.x[i];
            p[t.gstride + i] = q.z[i];
        }
    }
    __device__ __forceinline__ void xor_word(const Tile<W, C, true> &t, uint32_t i, uint64_t mx, uint64_t mz) const {
        p[i] ^= mx;
        p[t.gstride + i] ^= mz;
    }
    __device__ __forceinline__ void store_x(const Tile<W, C, true> &, const uint64_t (&x)[V]) const {
#pragma unroll
        for (int i = 0; i < V; i++) p[i] = x[i];
    }
    __device__ __forceinline__ void store_z(const Tile<W, C, true> &t, const uint64_t (&z)[V]) const {
#pragma unroll
        for (int i = 0; i < V; i++) p[t.gstride + i] = z[i];
    }
};

// One noise op on V words. Every word draws block 0 of its stream; only a
// word whose first draw shows an error in its 64 shots (probability about
// 64p) runs the general gap procedure, one word at a time.
template <int W, int C, bool GMEM, class K>
__device__ __forceinline__ void noise_op(const FrameArgs &a, const K key, const Tile<W, C, GMEM> &t,
                                         const DevOp op, uint32_t wo, uint32_t gw0, uint32_t instr_off) {
    constexpr int V = VecWidth<W>::V;
    const uint32_t opc = op.a >> 28;
    const bool pair = opc == OP_DEP2;
    const uint32_t tbl = pair ? (op.slot >> 24) : op.b;
    const uint32_t slot = pair ? (op.slot & 0xFFFFFFu) : op.slot;
    const uint32_t instr = op.instr + instr_off;
    const uint64_t *G = a.geo + kNoiseTableWords * tbl;
    const uint64_t g63 = __ldg(G + 63);
    uint4 blk[V];
    uint32_t hits = 0;
#pragma unroll
    for (int i = 0; i < V; i++) {
        blk[i] = philox_sched(make_uint4(0u, slot, kTagNoise | instr, gw0 + i), key);
        if ((uint64_t)blk[i].x < g63) hits |= 1u << i;
    }
    if (!hits) return;
    // masks first, then one read-modify-write of each hit word: the frame
    // words are not held across the gap procedure
    while (hits) {
        const int w = __ffs((int)hits) - 1;
        hits &= hits - 1u;
        uint4 b0 = blk[0];
#pragma unroll
        for (int i = 1; i < V; i++)
            if (w == i) b0 = blk[i];
        uint64_t mxa, mza, mxb, mzb;
        noise_masks_slow(opc, G, key, instr, slot, gw0 + (uint32_t)w, b0, mxa, mza, mxb, mzb);
        const Qubit<W, C, GMEM> qa(t, op.a & 0x0FFFFFFFu, wo);
        qa.xor_word(t, (uint32_t)w, mxa, mza);
        if (pair) {
            const Qubit<W, C, GMEM> qb(t, op.b, wo);
            qb.xor_word(t, (uint32_t)w, mxb, mzb);
        }
    }
}

// Applies one op to the V words at word offset wo of the tile (word tile0 + wo
// of the call). DETS: detection events are computed in the kernel, so
// measurements write their flips into the ring rows of a.rec.
template <int W, int C, bool GMEM, bool DETS, class K>
__device__ __forceinline__ void frame_op(const FrameArgs &a, const K key, const Tile<W, C, GMEM> &t,
                                         const DevOp op, uint32_t wo, uint32_t tile0, uint32_t instr_off,
                                         uint32_t meas_off) {
    constexpr int V = VecWidth<W>::V;
    const uint32_t opc = op.a >> 28;
    const uint32_t lw0 = tile0 + wo;                   // first word within the call
    const uint32_t gw0 = (uint32_t)a.word0 + lw0;      // first global 64-shot word (RNG counter)
    if (opc - OP_XERR <= OP_YERR - OP_XERR) {      // noise channels
        noise_op<W, C, GMEM, K>(a, key, t, op, wo, gw0, instr_off);
        return;
    }
    const Qubit<W, C, GMEM> qa(t, op.a & 0x0FFFFFFFu, wo);
    Planes<V> pa;
    switch (opc) {
        case OP_H: {
            qa.load(t, pa);
            Planes<V> sw;
#pragma unroll
            for (int i = 0; i < V; i++) {
                sw.x[i] = pa.z[i];
                sw.z[i] = pa.x[i];
            }
            qa.store(t, sw);
            break;
        }
        case OP_S: {
            qa.load(t, pa);
#pragma unroll
            for (int i = 0; i < V; i++) pa.z[i] ^= pa.x[i];
            qa.store_z(t, pa.z);
            break;
        }
        case OP_CX: {
            const Qubit<W, C, GMEM> qb(t, op.b, wo);
            Planes<V> pb;
            qa.load(t, pa);
            qb.load(t, pb);
#pragma unroll
            for (int i = 0; i < V; i++) {
                pa.z[i] ^= pb.z[i];
                pb.x[i] ^= pa.x[i];
            }
            qa.store_z(t, pa.z);
            qb.store_x(t, pb.x);
            break;
        }
        case OP_CZ: {
            const Qubit<W, C, GMEM> qb(t, op.b, wo);
            Planes<V> pb;
            qa.load(t, pa);
            qb.load(t, pb);
#pragma unroll
            for (int i = 0; i < V; i++) {
                pa.z[i] ^= pb.x[i];
                pb.z[i] ^= pa.x[i];
            }
            qa.store_z(t, pa.z);
            qb.store_z(t, pb.z);
            break;
        }
        case OP_M:
        case OP_MR:
        case OP_R: {
            if (opc != OP_R) qa.load(t, pa);
            if (opc != OP_R && a.rec != nullptr) {
                // the record (reference xor flip), or with in-kernel detection
                // events the flip alone, in ring row m & rec_mask
                const uint32_t m = op.b + meas_off;
                uint64_t refm = 0;
                uint64_t *row;
                if constexpr (DETS) {
                    row = a.rec + (uint64_t)(m & a.rec_mask) * a.rec_stride;
                } else {
                    refm = 0ull - ((__ldg(a.ref + (m >> 6)) >> (m & 63)) & 1ull);
                    row = a.rec + (uint64_t)m * a.rec_stride;
                }
#pragma unroll
                for (int i = 0; i < V; i++) {
                    const uint32_t lw = lw0 + i;
                    if (lw < a.nwords) {
                        uint64_t v = pa.x[i] ^ refm;
                        if (lw == a.nwords - 1) v &= a.last_mask;
                        row[lw] = v;
                    }
                }
            }
            const uint32_t ti = kTagCollapse | (op.instr + instr_off);
            if (opc == OP_M) {
#pragma unroll
                for (int i = 0; i < V; i++) pa.z[i] ^= half_mask(key, ti, op.slot, gw0 + i);
                qa.store_z(t, pa.z);
            } else {
#pragma unroll
                for (int i = 0; i < V; i++) {
                    pa.x[i] = 0;
                    pa.z[i] = half_mask(key, ti, op.slot, gw0 + i);
                }
                qa.store(t, pa);
            }
            break;
        }
        case OP_FFX:
        case OP_FFZ: {
            // classically controlled X / Z: applied where the shot's record
            // differs from the reference (the record row was written in an
            // earlier merged layer, before the layer barrier)
            if (a.rec == nullptr) break;
            const uint32_t m = op.b + meas_off;
            const uint64_t refm = 0ull - ((__ldg(a.ref + (m >> 6)) >> (m & 63)) & 1ull);
            const uint64_t *row = a.rec + (uint64_t)m * a.rec_stride;
            uint64_t f[V];
#pragma unroll
            for (int i = 0; i < V; i++) f[i] = lw0 + i < a.nwords ? row[lw0 + i] ^ refm : 0ull;
            qa.load(t, pa);
            if (opc == OP_FFX) {
#pragma unroll
                for (int i = 0; i < V; i++) pa.x[i] ^= f[i];
                qa.store_x(t, pa.x);
            } else {
#pragma unroll
                for (int i = 0; i < V; i++) pa.z[i] ^= f[i];
                qa.store_z(t, pa.z);
            }
            break;
        }
        default:
            break;
    }
}

__device__ __forceinline__ uint32_t lds32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_xor_smem(uint32_t a, uint64_t v) {
    asm volatile("red.shared.xor.b64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}
__device__ __forceinline__ void red_xor_cluster(uint32_t a, uint64_t v) {
    asm volatile("red.shared::cluster.xor.b64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

// XORs error masks into word w of one qubit. Atomic: two deferred hits of one
// chain (say DEPOLARIZE2 then X_ERROR on a shared qubit) may meet in one word.
template <int W, int C, bool GMEM>
__device__ __forceinline__ void xor_qubit_word(const Tile<W, C, GMEM> &t, uint32_t ref, uint32_t w, uint64_t mx,
                                               uint64_t mz) {
    if constexpr (GMEM) {
        uint64_t *p = t.base + (uint64_t)(ref & 0xFFFFFFu) * (2 * t.gstride) + w;
        if (mx) atomicXor(reinterpret_cast<unsigned long long *>(p), (unsigned long long)mx);
        if (mz) atomicXor(reinterpret_cast<unsigned long long *>(p + t.gstride), (unsigned long long)mz);
    } else {
        const uint32_t q = ref & 0xFFFFFFu;
        uint32_t ax = row_word<W>(t.fsa, q, w), az = row_word<W>(t.fsa, q, W + w);
        if constexpr (C > 1) {
            ax = mapa_rank(ax, ref >> 24);
            az = mapa_rank(az, ref >> 24);
            if (mx) red_xor_cluster(ax, mx);
            if (mz) red_xor_cluster(az, mz);
        } else {
            if (mx) red_xor_smem(ax, mx);
            if (mz) red_xor_smem(az, mz);
        }
    }
}

// First draws of a noise op on V words: bit i set when word i has an error.
template <int V, class K>
__device__ __forceinline__ uint32_t noise_hits(const FrameArgs &a, const K key, const DevOp op, uint32_t gw0,
                                               uint32_t instr_off) {
    const uint32_t opc = op.a >> 28;
    const bool pair = opc == OP_DEP2;
    const uint32_t tbl = pair ? (op.slot >> 24) : op.b;
    const uint32_t slot = pair ? (op.slot & 0xFFFFFFu) : op.slot;
    const uint32_t ti = kTagNoise | (op.instr + instr_off);
    const uint64_t g63 = __ldg(a.geo + kNoiseTableWords * tbl + 63u);
    uint32_t hits = 0;
#pragma unroll
    for (int i = 0; i < V; i++) {
        const uint4 blk = philox_sched(make_uint4(0u, slot, ti, gw0 + (uint32_t)i), key);
        if ((uint64_t)blk.x < g63) hits |= 1u << i;
    }
    return hits;
}

// A deferred hit: entry = (op index within the CTA's layer) << 3 | word of the
// tile. Redraws block 0, runs the general procedure and XORs the masks in.
template <int W, int C, bool GMEM, class K>
__device__ __forceinline__ void deferred_hit(const FrameArgs &a, const K key, const Tile<W, C, GMEM> &t,
                                             uint32_t e, uint32_t first, uint32_t tile0, uint32_t instr_off) {
    const uint32_t oi = e >> 3, w = e & 7u;
    const uint4 ov = __ldg(reinterpret_cast<const uint4 *>(a.ops) + first + oi);
    const uint32_t opc = ov.x >> 28;
    if (opc - OP_XERR > OP_YERR - OP_XERR) return;      // only noise ops are queued
    const bool pair = opc == OP_DEP2;
    const uint32_t tbl = pair ? (ov.w >> 24) : ov.y;
    const uint32_t slot = pair ? (ov.w & 0xFFFFFFu) : ov.w;
    const uint32_t instr = ov.z + instr_off;
    const uint32_t gw = (uint32_t)a.word0 + tile0 + w;
    const uint4 blk0 = philox_sched(make_uint4(0u, slot, kTagNoise | instr, gw), key);
    uint64_t mxa, mza, mxb, mzb;
    noise_masks_slow(opc, a.geo + kNoiseTableWords * tbl, key, instr, slot, gw, blk0, mxa, mza, mxb, mzb);
    xor_qubit_word<W, C, GMEM>(t, ov.x & 0x0FFFFFFFu, w, mxa, mza);
    if (pair) xor_qubit_word<W, C, GMEM>(t, ov.y, w, mxb, mzb);
}

// Detection events of the DETS entry items [first, first + n) for this tile:
// each detector is the XOR of its records' flips, read from the ring rows of
// a.rec (written by every CTA of the tile before the barrier this follows);
// observables XOR into their rows. The tile's items x words are spread over
// the cluster's CTAs and their threads, four items per thread at a time so
// that their ring loads (L2: other SMs wrote them) are in flight together.
// Padding bits of the last word are cleared.
template <int W, int C>
__device__ __forceinline__ void eval_dets(const FrameArgs &a, uint32_t rank, uint32_t tile0, uint32_t first,
                                          uint32_t n, uint32_t meas_off, uint32_t det_off) {
    constexpr uint32_t kBatch = 4;
    const uint32_t total = n * W, stride = C * blockDim.x;
    const uint4 *items = reinterpret_cast<const uint4 *>(a.det_items) + first;
    const unsigned long long *ring = reinterpret_cast<const unsigned long long *>(a.rec);
    for (uint32_t u0 = rank * blockDim.x + threadIdx.x; u0 < total; u0 += kBatch * stride) {
        uint4 it[kBatch];
        uint64_t lw[kBatch], v[kBatch];
        bool ok[kBatch];
        uint32_t maxl = 0;
#pragma unroll
        for (uint32_t b = 0; b < kBatch; b++) {
            const uint32_t u = u0 + b * stride;
            lw[b] = (uint64_t)tile0 + u % W;
            ok[b] = u < total && lw[b] < a.nwords;
            it[b] = ok[b] ? __ldg(items + u / W) : make_uint4(0u, 0u, 0u, 0u);
            v[b] = 0;
            maxl = max(maxl, it[b].z);
        }
        for (uint32_t j = 0; j < maxl; j++) {
#pragma unroll
            for (uint32_t b = 0; b < kBatch; b++) {
                if (j < it[b].z) {
                    const uint32_t m = __ldg(a.det_looks + it[b].y + j) + meas_off;
                    v[b] ^= __ldcg(ring + (uint64_t)(m & a.rec_mask) * a.rec_stride + lw[b]);
                }
            }
        }
#pragma unroll
        for (uint32_t b = 0; b < kBatch; b++) {
            if (!ok[b]) continue;
            uint64_t x = v[b];
            if (lw[b] == a.nwords - 1) x &= a.last_mask;
            if (it[b].x & kObsRow)
                atomicXor(reinterpret_cast<unsigned long long *>(
                              a.det + (a.num_dets + (uint64_t)(it[b].x & ~kObsRow)) * a.det_stride + lw[b]),
                          (unsigned long long)x);
            else
                a.det[(uint64_t)(it[b].x + det_off) * a.det_stride + lw[b]] = x;
        }
    }
}

__device__ __forceinline__ uint64_t to_global(const void *p) {
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
    return g;
}

// Propagates the frames of one tile (W words, this CTA's qubit slice) through
// the whole program. dyn = start of the tile's dynamic shared memory (layout
// above). DETS: evaluate the program's DETS entries from the flip ring
// (a.det set); otherwise they are skipped. Returns false on a malformed program.
template <class K>
__device__ __forceinline__ K tile_keys(const FrameArgs &a, uint32_t sbase);
template <>
__device__ __forceinline__ SmemKeys tile_keys<SmemKeys>(const FrameArgs &, uint32_t sbase) {
    return SmemKeys{sbase};
}
template <>
__device__ __forceinline__ ParamKeys tile_keys<ParamKeys>(const FrameArgs &a, uint32_t) {
    return ParamKeys{a.rk};
}

// K: where the Philox round keys are read (SmemKeys: the tile header, written
// at the start; ParamKeys: a.rk in the kernel's parameter space).
template <int W, int C, bool GMEM, bool DETS, class K = SmemKeys>
__device__ __forceinline__ bool run_tile(const FrameArgs &a, unsigned char *dyn, uint32_t rank, uint64_t tile) {
    constexpr int V = VecWidth<W>::V;
    if (blockDim.x % 32u != 0u) {       // partial warps would stall the hit-queue ballots
        if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
        return false;
    }
    const uint32_t tile0 = (uint32_t)(tile * W);
    const uint32_t sbase = smem_addr(dyn);
    const K key = tile_keys<K>(a, sbase);
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t qsa = sbase + kHitQueueOffset + (threadIdx.x >> 5) * (4u * kHitQueueCap);   // this warp's queue
    const uint32_t qlo = rank * a.Q;
    const uint32_t nq = a.n > qlo ? min(a.Q, a.n - qlo) : 0u;
    Tile<W, C, GMEM> t;
    t.rank = rank;
    t.gstride = a.gstride;
    t.fsa = sbase + kTileHeaderBytes + a.meta_region;
    t.base = a.gframe + tile0;
    write_round_keys(reinterpret_cast<uint32_t *>(dyn), Key{(uint32_t)a.seed, (uint32_t)(a.seed >> 32)});
    // program metadata (prog | rank_tab | segs): a shared copy when it fits
    const unsigned char *meta_g = reinterpret_cast<const unsigned char *>(a.prog);
    const bool meta_shared = a.meta_bytes != 0 && a.meta_bytes <= a.meta_region;
    const unsigned char *meta = meta_shared ? dyn + kTileHeaderBytes : meta_g;
    if (meta_shared) {
        for (uint32_t i = threadIdx.x; i < a.meta_bytes / 16u; i += blockDim.x)
            reinterpret_cast<uint4 *>(dyn + kTileHeaderBytes)[i] = __ldg(reinterpret_cast<const uint4 *>(meta_g) + i);
    }
    const ProgEntry *prog = reinterpret_cast<const ProgEntry *>(meta);
    const uint32_t *rank_tab =
        reinterpret_cast<const uint32_t *>(meta + (reinterpret_cast<const unsigned char *>(a.rank_tab) - meta_g));
    const uint4 *segs = reinterpret_cast<const uint4 *>(meta + (reinterpret_cast<const unsigned char *>(a.segs) - meta_g));
    __syncthreads();   // round keys and metadata visible before use
    for (uint32_t i = threadIdx.x; i < nq * W; i += blockDim.x) {
        const uint32_t l = i / W, w = i % W;
        const uint64_t coin = half_mask(key, kTagInit, qlo + l, (uint32_t)a.word0 + tile0 + w);
        if constexpr (GMEM) {
            uint64_t *p = t.base + (uint64_t)l * (2 * a.gstride) + w;
            p[0] = 0;
            p[a.gstride] = coin;
        } else {
            sts64(row_word<W>(t.fsa, l, w), 0);
            sts64(row_word<W>(t.fsa, l, W + w), coin);
        }
    }
    tile_arrive<C>();

    const uint4 *ops = reinterpret_cast<const uint4 *>(a.ops);
    bool ok = true;
    uint32_t instr_off = 0, meas_off = 0;
    // a DETS entry waiting for the next barrier: its item count here, its
    // first item and the offsets of its loop iteration in shared memory (the
    // same values in every thread). Two slots (header bytes 80..103), used in
    // turn: with a cluster the end-of-layer arrive does not wait, so a fast
    // thread may record the next DETS entry while a slow one still evaluates
    // the pending one -- never further ahead, since the next layer's wait
    // needs the slow thread's arrive.
    uint32_t dets_n = 0, dets_slot = 0;
#define STIMGB_DETS_AT (reinterpret_cast<uint32_t *>(dyn + 80 + 12 * dets_slot))
    uint32_t loop_pc[kMaxLoopDepth];
    uint32_t loop_iter[kMaxLoopDepth];
    int sp = 0;
    uint32_t pc = 0;
    while (pc < a.nprog) {
        const ProgEntry e = prog[pc];
        if (e.kind == ENT_LAYER) {
            const uint32_t sb = rank_tab[e.op_begin + rank];
            const uint32_t se = rank_tab[e.op_begin + rank + 1];
            tile_wait<C>();      // the previous layer is complete in every CTA of the cluster
            if (sb < se && ok) {
                // Items are (chain, V-word group) pairs, numbered across this
                // CTA's segments of the merged layer. Each segment's items are
                // padded to whole warps, so a warp stays inside one segment and
                // all its lanes run the same chain step together (padding lanes
                // replay chain 0 without effect). Noise steps in a chain's
                // deferrable tail only take the first draw; hits are queued per
                // warp and resolved 32 at a time, one per lane.
                const uint32_t first = segs[sb].y;
                uint32_t qn = 0;
                auto flush = [&](uint32_t n) {
                    __syncwarp();
                    if (lane < n) deferred_hit<W, C, GMEM, K>(a, key, t, lds32(qsa + 4u * lane), first, tile0, instr_off);
                    __syncwarp();
                };
                uint32_t g = threadIdx.x, seg_start = 0;
                for (uint32_t s = sb; s < se; s++) {
                    const uint4 sv = segs[s];
                    const uint32_t len = sv.x, items = sv.z * (W / V), span = (items + 31u) & ~31u;
                    const uint32_t dfrom = sv.w;
                    bool have_next = false;      // nxt holds this item's first op
                    uint4 nxt = make_uint4(0u, 0u, 0u, 0u);
                    for (; g < seg_start + span; g += blockDim.x) {
                        const uint32_t it = g - seg_start;
                        const bool act = it < items;
                        const uint32_t wo = act ? (it % (W / V)) * V : 0u;
                        // ops are step-major: step j of the segment's chain c at sv.y + j * sv.z + c
                        const uint32_t op0 = sv.y + (act ? it / (W / V) : 0u);
                        if (!have_next) nxt = __ldg(ops + op0);
                        // the thread's next item of this segment, if any
                        const uint32_t it2 = it + blockDim.x;
                        have_next = g + blockDim.x < seg_start + span;
                        const uint32_t op2 = sv.y + (it2 < items ? it2 / (W / V) : 0u);
                        for (uint32_t j = 0; j < len; j++) {
                            const uint4 ov = nxt;
                            if (j + 1 < len) nxt = __ldg(ops + op0 + (j + 1) * sv.z);     // one op ahead
                            else if (have_next) nxt = __ldg(ops + op2);                 // across items
                            if (j < dfrom) {
                                if (act) frame_op<W, C, GMEM, DETS, K>(a, key, t, as_op(ov), wo, tile0, instr_off, meas_off);
                            } else {
                                const uint32_t hits =
                                    act ? noise_hits<V, K>(a, key, as_op(ov), (uint32_t)a.word0 + tile0 + wo, instr_off)
                                        : 0u;
                                const uint32_t oi = op0 + j * sv.z - first;      // index within the CTA's layer
#pragma unroll
                                for (int i = 0; i < V; i++) {
                                    const bool h = (hits >> i) & 1u;
                                    const uint32_t m = __ballot_sync(0xFFFFFFFFu, h);
                                    if (m) {
                                        const uint32_t cnt = __popc(m);
                                        if (qn + cnt > kHitQueueCap) {
                                            flush(qn);
                                            qn = 0;
                                        }
                                        if (h)
                                            sts32(qsa + 4u * (qn + __popc(m & ((1u << lane) - 1u))),
                                                  (oi << 3) | (wo + (uint32_t)i));
                                        qn += cnt;
                                    }
                                }
                            }
                        }
                    }
                    seg_start += span;
                }
                if (qn) flush(qn);
            }
            if (DETS && dets_n) {
                // the last stretch's flips were in the ring at this layer's
                // barrier; this layer's measurements do not reach their rows
                eval_dets<W, C>(a, rank, tile0, STIMGB_DETS_AT[0], dets_n, STIMGB_DETS_AT[1], STIMGB_DETS_AT[2]);
                dets_n = 0;
            }
            tile_arrive<C>();
            pc++;
        } else if (e.kind == ENT_DETS) {
            if constexpr (DETS) {
                if (dets_n) {       // two DETS entries without a layer between: a barrier of its own
                    tile_wait<C>();
                    eval_dets<W, C>(a, rank, tile0, STIMGB_DETS_AT[0], dets_n, STIMGB_DETS_AT[1], STIMGB_DETS_AT[2]);
                    tile_arrive<C>();
                }
                // detector offset of this loop iteration: iterations so far
                // times each enclosing loop's detector count
                uint32_t det_off = 0;
                for (int k = 0; k < sp; k++) det_off += loop_iter[k] * prog[loop_pc[k]].n_noise;
                dets_slot ^= 1u;
                STIMGB_DETS_AT[0] = e.op_begin;
                STIMGB_DETS_AT[1] = meas_off;
                STIMGB_DETS_AT[2] = det_off;
                dets_n = e.n_gate;
            }
            pc++;
        } else if (e.kind == ENT_LOOP_BEGIN) {
            if (sp >= kMaxLoopDepth) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                ok = false;
                break;
            }
            loop_pc[sp] = pc;
            loop_iter[sp] = 0;
            sp++;
            pc++;
        } else {
            if (sp <= 0) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                ok = false;
                break;
            }
            const uint32_t it = ++loop_iter[sp - 1];
            if (it < e.reps) {
                instr_off += e.instr_stride;
                meas_off += e.meas_stride;
                pc = loop_pc[sp - 1] + 1;
            } else {
                instr_off -= e.instr_stride * (e.reps - 1);
                meas_off -= e.meas_stride * (e.reps - 1);
                sp--;
                pc++;
            }
        }
    }
    tile_wait<C>();
    if (DETS && dets_n && ok) eval_dets<W, C>(a, rank, tile0, STIMGB_DETS_AT[0], dets_n, STIMGB_DETS_AT[1], STIMGB_DETS_AT[2]);
#undef STIMGB_DETS_AT
    return ok;
}

}  // namespace frame_detail
}  // namespace stimgb
