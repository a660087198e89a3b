// frame_tile.cuh -- device code of the Pauli-frame propagation, shared by
// the per-circuit kernel (frame.cu) and the batched persistent kernel
// (batch.cu).
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace stimgb {
namespace frame_detail {

__device__ __forceinline__ DevOp as_op(uint4 v) { return DevOp{v.x, v.y, v.z, v.w}; }

template <int C>
__device__ __forceinline__ void sync_tile() {
    if constexpr (C == 1) {
        __syncthreads();
    } else {
        cg::this_cluster().sync();
    }
}

// Word of a peer CTA's shared memory (same offset, CTA `rank` of the cluster).
__device__ __forceinline__ uint64_t ld_peer(const uint64_t *p, uint32_t rank) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    uint64_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
    return v;
}

__device__ __forceinline__ void st_peer(uint64_t *p, uint32_t rank, uint64_t v) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(v) : "memory");
}

// The X and Z planes of one tile as seen from one CTA. A qubit reference is
// (rank << 24 | local index); references to other CTAs of the cluster go
// through distributed shared memory.
template <int C, bool GMEM>
struct Tile {
    uint64_t *X, *Z;
    uint64_t qstride;
    uint32_t rank;

    __device__ __forceinline__ uint64_t *at(uint64_t *P, uint32_t ref, uint32_t w) const {
        return P + (uint64_t)(ref & 0xFFFFFFu) * qstride + w;
    }
    __device__ __forceinline__ uint64_t ld(uint64_t *P, uint32_t ref, uint32_t w) const {
        uint64_t *p = at(P, ref, w);
        if constexpr (C > 1) {
            if ((ref >> 24) != rank) return ld_peer(p, ref >> 24);
        }
        return *p;
    }
    __device__ __forceinline__ void st(uint64_t *P, uint32_t ref, uint32_t w, uint64_t v) const {
        uint64_t *p = at(P, ref, w);
        if constexpr (C > 1) {
            if ((ref >> 24) != rank) {
                st_peer(p, ref >> 24, v);
                return;
            }
        }
        *p = v;
    }
};

// Applies one op to word w of the tile.
template <int C, bool GMEM>
__device__ __forceinline__ void frame_op(const FrameArgs &a, const Key key, const Tile<C, GMEM> &t, const DevOp op,
                                         uint32_t w, uint64_t lw, uint32_t instr_off, uint32_t meas_off) {
    const uint32_t opc = op.a >> 28;
    const uint32_t ra = op.a & 0x0FFFFFFFu;
    const uint32_t gw = (uint32_t)(a.word0 + lw);     // global 64-shot word (RNG counter)
    switch (opc) {
        case OP_H: {
            const uint64_t x = t.ld(t.X, ra, w), z = t.ld(t.Z, ra, w);
            t.st(t.X, ra, w, z);
            t.st(t.Z, ra, w, x);
            break;
        }
        case OP_S:
            t.st(t.Z, ra, w, t.ld(t.Z, ra, w) ^ t.ld(t.X, ra, w));
            break;
        case OP_CX: {
            const uint32_t rb = op.b;
            const uint64_t xa = t.ld(t.X, ra, w), za = t.ld(t.Z, ra, w);
            const uint64_t xb = t.ld(t.X, rb, w), zb = t.ld(t.Z, rb, w);
            t.st(t.Z, ra, w, za ^ zb);
            t.st(t.X, rb, w, xb ^ xa);
            break;
        }
        case OP_CZ: {
            const uint32_t rb = op.b;
            const uint64_t xa = t.ld(t.X, ra, w), za = t.ld(t.Z, ra, w);
            const uint64_t xb = t.ld(t.X, rb, w), zb = t.ld(t.Z, rb, w);
            t.st(t.Z, ra, w, za ^ xb);
            t.st(t.Z, rb, w, zb ^ xa);
            break;
        }
        case OP_M:
        case OP_MR:
        case OP_R: {
            if (opc != OP_R && a.rec != nullptr && lw < a.nwords) {
                const uint32_t m = op.b + meas_off;
                const uint64_t refm = 0ull - ((__ldg(a.ref + (m >> 6)) >> (m & 63)) & 1ull);
                uint64_t v = t.ld(t.X, ra, w) ^ refm;
                if (lw == a.nwords - 1) v &= a.last_mask;
                a.rec[(uint64_t)m * a.rec_stride + lw] = v;
            }
            const uint64_t coin = half_mask(key, kTagCollapse | (op.instr + instr_off), op.slot, gw);
            if (opc == OP_M) {
                t.st(t.Z, ra, w, t.ld(t.Z, ra, w) ^ coin);
            } else {
                t.st(t.X, ra, w, 0);
                t.st(t.Z, ra, w, coin);
            }
            break;
        }
        case OP_XERR:
        case OP_ZERR:
        case OP_DEP1: {
            uint64_t mx, mz, u1, u2;
            const uint64_t *G = a.geo + 64u * op.b;
            const uint32_t instr = op.instr + instr_off;
            bool hit;
            if (opc == OP_XERR) hit = noise_masks<OP_XERR>(G, key, instr, op.slot, gw, mx, mz, u1, u2);
            else if (opc == OP_ZERR) hit = noise_masks<OP_ZERR>(G, key, instr, op.slot, gw, mx, mz, u1, u2);
            else hit = noise_masks<OP_DEP1>(G, key, instr, op.slot, gw, mx, mz, u1, u2);
            if (hit) {
                if (mx) t.st(t.X, ra, w, t.ld(t.X, ra, w) ^ mx);
                if (mz) t.st(t.Z, ra, w, t.ld(t.Z, ra, w) ^ mz);
            }
            break;
        }
        case OP_DEP2: {
            uint64_t m0x, m0z, m1x, m1z;
            if (noise_masks<OP_DEP2>(a.geo + 64u * (op.slot >> 24), key, op.instr + instr_off,
                                     op.slot & 0xFFFFFFu, gw, m0x, m0z, m1x, m1z)) {
                const uint32_t rb = op.b;
                t.st(t.X, ra, w, t.ld(t.X, ra, w) ^ m0x);
                t.st(t.Z, ra, w, t.ld(t.Z, ra, w) ^ m0z);
                t.st(t.X, rb, w, t.ld(t.X, rb, w) ^ m1x);
                t.st(t.Z, rb, w, t.ld(t.Z, rb, w) ^ m1z);
            }
            break;
        }
        default:
            break;
    }
}

// Propagates the frames of one tile (W words, this CTA's qubit slice) through
// the whole program. Returns false on a malformed program.
template <int W, int C, bool GMEM>
__device__ __forceinline__ bool run_tile(const FrameArgs &a, uint64_t *smem, uint32_t rank, uint64_t tile) {
    const uint64_t tile0 = tile * W;
    const uint32_t qlo = rank * a.Q;
    const uint32_t nq = a.n > qlo ? min(a.Q, a.n - qlo) : 0u;
    const Key key{(uint32_t)a.seed, (uint32_t)(a.seed >> 32)};
    Tile<C, GMEM> t;
    t.rank = rank;
    if (GMEM) {
        t.X = a.gframe + tile0;
        t.Z = a.gframe + (uint64_t)a.n * a.gstride + tile0;
        t.qstride = a.gstride;
    } else {
        t.X = smem;
        t.Z = smem + (uint64_t)a.Q * W;
        t.qstride = W;
    }
    for (uint32_t i = threadIdx.x; i < nq * W; i += blockDim.x) {
        const uint32_t l = i / W, w = i % W;
        t.X[(uint64_t)l * t.qstride + w] = 0;
        t.Z[(uint64_t)l * t.qstride + w] =
            half_mask(key, kTagInit, qlo + l, (uint32_t)(a.word0 + tile0 + w));
    }
    sync_tile<C>();

    uint32_t instr_off = 0, meas_off = 0;
    uint32_t loop_pc[kMaxLoopDepth];
    uint32_t loop_iter[kMaxLoopDepth];
    int sp = 0;
    uint32_t pc = 0;
    while (pc < a.nprog) {
        const ProgEntry e = a.prog[pc];
        if (e.kind == ENT_LAYER) {
            // Items are (chain, word) pairs, numbered across this CTA's
            // segments of the merged layer; the W words of a chain sit on
            // adjacent threads, which share its op fetches.
            const uint32_t sb = __ldg(a.rank_tab + e.op_begin + rank);
            const uint32_t se = __ldg(a.rank_tab + e.op_begin + rank + 1);
            uint32_t g = threadIdx.x, seg_start = 0;
            for (uint32_t s = sb; s < se; s++) {
                const uint4 sv = __ldg(reinterpret_cast<const uint4 *>(a.segs) + s);
                const uint32_t len = sv.x, op0 = sv.y, items = sv.z * W;
                for (; g < seg_start + items; g += blockDim.x) {
                    const uint32_t it = g - seg_start;
                    const uint32_t w = it % W;
                    const uint4 *cp = reinterpret_cast<const uint4 *>(a.ops) + op0 + (it / W) * len;
                    for (uint32_t j = 0; j < len; j++)
                        frame_op<C, GMEM>(a, key, t, as_op(__ldg(cp + j)), w, tile0 + w, instr_off, meas_off);
                }
                seg_start += items;
            }
            sync_tile<C>();
            pc++;
        } else if (e.kind == ENT_LOOP_BEGIN) {
            if (sp >= kMaxLoopDepth) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return false;
            }
            loop_pc[sp] = pc;
            loop_iter[sp] = 0;
            sp++;
            pc++;
        } else {
            if (sp <= 0) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return false;
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
    return true;
}

}  // namespace frame_detail
}  // namespace stimgb
