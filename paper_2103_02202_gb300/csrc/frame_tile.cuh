// frame_tile.cuh -- device code of the Pauli-frame propagation, shared by
// the per-circuit kernel (frame.cu) and the batched persistent kernel
// (batch.cu).
//
// Dynamic shared memory of one tile (byte offsets from the region start):
//   [0, 80)                  Philox round keys of the seed
//   [128, 136)               mbarrier of the op-staging copy
//   [256, 256 + 16 op_cap)   the current layer's ops of this CTA, copied in
//                            by the TMA engine (cp.async.bulk) at the start of
//                            the layer
//   [256 + 16 op_cap, ...)   frame rows (shared-memory layout)
// Frame layout (W 64-shot words per tile): each qubit owns a row of 2W words,
// its X words then its Z words,
//     shared memory:  row(q) = q * 2W;  X = row[w], Z = row[W + w]
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

constexpr uint64_t kStageTimeoutNs = 2000000000ull;   // bounded wait for a staging copy

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
__device__ __forceinline__ uint64_t ld_peer(uint32_t sa, uint32_t rank) {
    uint32_t ra;
    uint64_t v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(ra) : "memory");
    return v;
}

__device__ __forceinline__ void st_peer(uint32_t sa, uint32_t rank, uint64_t v) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(sa), "r"(rank));
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(ra), "l"(v) : "memory");
}

// The tile as seen from one CTA of the cluster.
template <int W, int C, bool GMEM>
struct Tile {
    uint32_t fsa;        // shared address of row 0 (shared layout)
    uint64_t *base;      // row 0, word 0 of the tile (global layout)
    uint64_t gstride;    // G (global layout)
    uint32_t rank;
};

// One qubit's X and Z words at word w of the tile; a qubit reference is
// (rank << 24 | local index), other ranks are reached through distributed
// shared memory.
template <int W, int C, bool GMEM>
struct Qubit;

template <int W, int C>
struct Qubit<W, C, false> {
    uint32_t sa;         // shared address of the X word
    uint32_t peer;       // owning CTA when remote, else 0xFFFFFFFF

    __device__ __forceinline__ Qubit(const Tile<W, C, false> &t, uint32_t ref, uint32_t w) {
        sa = t.fsa + ((ref & 0xFFFFFFu) * (2u * W) + w) * 8u;
        peer = 0xFFFFFFFFu;
        if constexpr (C > 1) {
            if ((ref >> 24) != t.rank) peer = ref >> 24;
        }
    }
    __device__ __forceinline__ uint64_t get(uint32_t off) const {
        if constexpr (C > 1) {
            if (peer != 0xFFFFFFFFu) return ld_peer(sa + off, peer);
        }
        return lds64(sa + off);
    }
    __device__ __forceinline__ void put(uint32_t off, uint64_t v) const {
        if constexpr (C > 1) {
            if (peer != 0xFFFFFFFFu) {
                st_peer(sa + off, peer, v);
                return;
            }
        }
        sts64(sa + off, v);
    }
    __device__ __forceinline__ uint64_t x(const Tile<W, C, false> &) const { return get(0); }
    __device__ __forceinline__ uint64_t z(const Tile<W, C, false> &) const { return get(8u * W); }
    __device__ __forceinline__ void set_x(const Tile<W, C, false> &, uint64_t v) const { put(0, v); }
    __device__ __forceinline__ void set_z(const Tile<W, C, false> &, uint64_t v) const { put(8u * W, v); }
};

template <int W, int C>
struct Qubit<W, C, true> {
    uint64_t *p;

    __device__ __forceinline__ Qubit(const Tile<W, C, true> &t, uint32_t ref, uint32_t w) {
        p = t.base + (uint64_t)(ref & 0xFFFFFFu) * (2 * t.gstride) + w;
    }
    __device__ __forceinline__ uint64_t x(const Tile<W, C, true> &) const { return *p; }
    __device__ __forceinline__ uint64_t z(const Tile<W, C, true> &t) const { return p[t.gstride]; }
    __device__ __forceinline__ void set_x(const Tile<W, C, true> &, uint64_t v) const { *p = v; }
    __device__ __forceinline__ void set_z(const Tile<W, C, true> &t, uint64_t v) const { p[t.gstride] = v; }
};

// One noise op on word w. Every lane draws block 0 of its stream; only when
// its first draw shows an error in the 64 shots (probability about 64p) does
// it run the general gap procedure.
template <int W, int C, bool GMEM>
__device__ __forceinline__ void noise_op(const FrameArgs &a, const SmemKeys key, const Tile<W, C, GMEM> &t,
                                         const DevOp op, uint32_t w, uint32_t gw, uint32_t instr_off) {
    const uint32_t opc = op.a >> 28;
    const bool pair = opc == OP_DEP2;
    const uint32_t tbl = pair ? (op.slot >> 24) : op.b;
    const uint32_t slot = pair ? (op.slot & 0xFFFFFFu) : op.slot;
    const uint32_t ti = kTagNoise | (op.instr + instr_off);
    const uint64_t *G = a.geo + 64u * tbl;
    const uint4 blk0 = philox_sched(make_uint4(0u, slot, ti, gw), key);
    if ((uint64_t)blk0.x < __ldg(G + 63)) {
        uint64_t xa, za, xb, zb;
        const uint32_t instr = op.instr + instr_off;
        if (opc == OP_XERR) noise_masks_slow<OP_XERR>(G, key, instr, slot, gw, blk0, xa, za, xb, zb);
        else if (opc == OP_ZERR) noise_masks_slow<OP_ZERR>(G, key, instr, slot, gw, blk0, xa, za, xb, zb);
        else if (opc == OP_DEP1) noise_masks_slow<OP_DEP1>(G, key, instr, slot, gw, blk0, xa, za, xb, zb);
        else noise_masks_slow<OP_DEP2>(G, key, instr, slot, gw, blk0, xa, za, xb, zb);
        const Qubit<W, C, GMEM> qa(t, op.a & 0x0FFFFFFFu, w);
        if (xa) qa.set_x(t, qa.x(t) ^ xa);
        if (za) qa.set_z(t, qa.z(t) ^ za);
        if (pair) {
            const Qubit<W, C, GMEM> qb(t, op.b, w);
            if (xb) qb.set_x(t, qb.x(t) ^ xb);
            if (zb) qb.set_z(t, qb.z(t) ^ zb);
        }
    }
}

// Applies one op to word w of the tile; lw = word within the call. Padding
// lanes (act false) do nothing.
template <int W, int C, bool GMEM>
__device__ __forceinline__ void frame_op(const FrameArgs &a, const SmemKeys key, const Tile<W, C, GMEM> &t,
                                         const DevOp op, uint32_t w, uint32_t lw, uint32_t instr_off,
                                         uint32_t meas_off, bool act) {
    if (!act) return;
    const uint32_t opc = op.a >> 28;
    const uint32_t gw = (uint32_t)a.word0 + lw;       // global 64-shot word (RNG counter)
    if (opc >= OP_XERR) {
        noise_op<W, C, GMEM>(a, key, t, op, w, gw, instr_off);
        return;
    }
    const Qubit<W, C, GMEM> qa(t, op.a & 0x0FFFFFFFu, w);
    switch (opc) {
        case OP_H: {
            const uint64_t x = qa.x(t), z = qa.z(t);
            qa.set_x(t, z);
            qa.set_z(t, x);
            break;
        }
        case OP_S:
            qa.set_z(t, qa.z(t) ^ qa.x(t));
            break;
        case OP_CX: {
            const Qubit<W, C, GMEM> qb(t, op.b, w);
            const uint64_t xa = qa.x(t), za = qa.z(t), xb = qb.x(t), zb = qb.z(t);
            qa.set_z(t, za ^ zb);
            qb.set_x(t, xb ^ xa);
            break;
        }
        case OP_CZ: {
            const Qubit<W, C, GMEM> qb(t, op.b, w);
            const uint64_t xa = qa.x(t), za = qa.z(t), xb = qb.x(t), zb = qb.z(t);
            qa.set_z(t, za ^ xb);
            qb.set_z(t, zb ^ xa);
            break;
        }
        case OP_M:
        case OP_MR:
        case OP_R: {
            if (opc != OP_R && a.rec != nullptr && lw < a.nwords) {
                const uint32_t m = op.b + meas_off;
                const uint64_t refm = 0ull - ((__ldg(a.ref + (m >> 6)) >> (m & 63)) & 1ull);
                uint64_t v = qa.x(t) ^ refm;
                if (lw == a.nwords - 1) v &= a.last_mask;
                a.rec[(uint64_t)m * a.rec_stride + lw] = v;
            }
            const uint64_t coin = half_mask(key, kTagCollapse | (op.instr + instr_off), op.slot, gw);
            if (opc == OP_M) {
                qa.set_z(t, qa.z(t) ^ coin);
            } else {
                qa.set_x(t, 0);
                qa.set_z(t, coin);
            }
            break;
        }
        default:
            break;
    }
}

__device__ __forceinline__ uint64_t to_global(const void *p) {
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
    return g;
}

// Propagates the frames of one tile (W words, this CTA's qubit slice) through
// the whole program. dyn = start of the tile's dynamic shared memory (layout
// above). Returns false on a malformed program or a staging timeout.
template <int W, int C, bool GMEM>
__device__ __forceinline__ bool run_tile(const FrameArgs &a, unsigned char *dyn, uint32_t rank, uint64_t tile) {
    const uint32_t tile0 = (uint32_t)(tile * W);
    const uint32_t sbase = smem_addr(dyn);
    const SmemKeys key{sbase};
    const uint32_t mb = sbase + 128u;
    const uint32_t opbuf = sbase + kTileHeaderBytes;
    const uint32_t op_cap = a.op_cap;
    const uint32_t qlo = rank * a.Q;
    const uint32_t nq = a.n > qlo ? min(a.Q, a.n - qlo) : 0u;
    Tile<W, C, GMEM> t;
    t.rank = rank;
    t.gstride = a.gstride;
    t.fsa = opbuf + 16u * op_cap;
    t.base = a.gframe + tile0;
    write_round_keys(reinterpret_cast<uint32_t *>(dyn), Key{(uint32_t)a.seed, (uint32_t)(a.seed >> 32)});
    if (threadIdx.x == 0) {
        mbar_init(mb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();   // round keys visible before the first draw
    for (uint32_t i = threadIdx.x; i < nq * W; i += blockDim.x) {
        const uint32_t l = i / W, w = i % W;
        const uint64_t coin = half_mask(key, kTagInit, qlo + l, (uint32_t)a.word0 + tile0 + w);
        if constexpr (GMEM) {
            uint64_t *p = t.base + (uint64_t)l * (2 * a.gstride) + w;
            p[0] = 0;
            p[a.gstride] = coin;
        } else {
            const uint32_t sa = t.fsa + (l * (2u * W) + w) * 8u;
            sts64(sa, 0);
            sts64(sa + 8u * W, coin);
        }
    }
    sync_tile<C>();

    const uint64_t ops_g = to_global(a.ops);
    uint32_t phase = 0;
    bool ok = true, pending = false;
    uint32_t instr_off = 0, meas_off = 0;
    uint32_t loop_pc[kMaxLoopDepth];
    uint32_t loop_iter[kMaxLoopDepth];
    int sp = 0;
    uint32_t pc = 0;
    while (pc < a.nprog) {
        const ProgEntry e = a.prog[pc];
        if (e.kind == ENT_LAYER) {
            const uint32_t sb = __ldg(a.rank_tab + e.op_begin + rank);
            const uint32_t se = __ldg(a.rank_tab + e.op_begin + rank + 1);
            if (sb < se && ok) {
                // this CTA's ops of the layer are contiguous: stage them in shared memory
                const uint4 s0 = __ldg(reinterpret_cast<const uint4 *>(a.segs) + sb);
                const uint4 s1 = __ldg(reinterpret_cast<const uint4 *>(a.segs) + se - 1);
                const uint32_t first = s0.y;
                const uint32_t nops = s1.y + s1.z * s1.x - first;
                const uint32_t staged = nops < op_cap ? nops : op_cap;
                if (staged) {
                    if (threadIdx.x == 0) {
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(mb, staged * 16u);
                        bulk_g2s(opbuf, reinterpret_cast<const void *>(ops_g + (uint64_t)first * 16u), staged * 16u,
                                 mb);
                    }
                    const uint64_t t0 = globaltimer_ns();
                    while (!mbar_try_wait(mb, phase)) {
                        if (globaltimer_ns() - t0 > kStageTimeoutNs) {
                            ok = false;
                            pending = true;        // the copy may still land: wait for it before leaving
                            atomicExch(a.status, DEV_TIMEOUT);
                            break;
                        }
                    }
                    if (!pending) phase ^= 1u;
                }
                if (ok) {
                    // Items are (chain, word) pairs, numbered across this CTA's
                    // segments of the merged layer; the W words of a chain sit
                    // on adjacent threads.
                    // Each segment's items are padded to whole warps, so a warp
                    // stays inside one segment: its lanes run the same opcode at
                    // every chain step (padding lanes replay chain 0, inactive).
                    uint32_t g = threadIdx.x, seg_start = 0;
                    for (uint32_t s = sb; s < se; s++) {
                        const uint4 sv = __ldg(reinterpret_cast<const uint4 *>(a.segs) + s);
                        const uint32_t len = sv.x, items = sv.z * W, span = (items + 31u) & ~31u;
                        for (; g < seg_start + span; g += blockDim.x) {
                            const uint32_t it = g - seg_start;
                            const bool act = it < items;
                            const uint32_t w = it % W;
                            uint32_t oi = sv.y + (act ? it / W : 0u) * len - first;     // index within the layer
                            for (uint32_t j = 0; j < len; j++, oi++) {
                                const uint4 ov = oi < staged ? lds128(opbuf + oi * 16u)
                                                             : __ldg(reinterpret_cast<const uint4 *>(a.ops) + first + oi);
                                frame_op<W, C, GMEM>(a, key, t, as_op(ov), w, tile0 + w, instr_off, meas_off, act);
                            }
                        }
                        seg_start += span;
                    }
                }
            }
            sync_tile<C>();
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
    if (pending) {
        const uint64_t t0 = globaltimer_ns();
        while (!mbar_try_wait(mb, phase) && globaltimer_ns() - t0 < kStageTimeoutNs) {
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mb) : "memory");
    __syncthreads();
    return ok;
}

}  // namespace frame_detail
}  // namespace stimgb
