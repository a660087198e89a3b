// frame.cu -- batched Pauli-frame propagation (Section 3 of the paper).
//
// Work unit: a tile of W 64-shot words for all n qubits, owned by a cluster
// of C CTAs (C = 1: a single CTA). The qubits are split into C contiguous
// slices of Q = ceil(n / C); CTA r of the cluster keeps the X and Z planes of
// its slice -- the paper's separate "XXXX...ZZZZ" planes (Section 5.1) --
// resident in shared memory for the whole circuit:
//     X[l * W + w], Z[l * W + w]      l = local qubit, w = word of the tile
// so a row of W words per qubit is contiguous.
// (When even one 64-shot word of the largest slice does not fit, a C = 1
// variant keeps the same rows in a global-memory frame instead.)
//
// The CTA walks the compiled program. Consecutive fused layers are folded
// into chains (an op that acts only on qubits of one earlier op runs right
// after it on the same thread); for each merged layer the threads take
// (chain, word) items of the CTA's own chains and apply each chain's ops:
//   H: swap(x, z)   S: z ^= x   CX(c,t): z_c ^= z_t, x_t ^= x_c
//   CZ(a,b): z_a ^= x_b, z_b ^= x_a
//   M:  record = ref[m] ^ x, then z ^= collapse coin
//   MR: record = ref[m] ^ x, then x = 0, z = collapse coin
//   R:  x = 0, z = collapse coin
//   noise: keyed geometric masks multiplied into the frame.
// The second qubit of a two-qubit op may belong to another CTA of the
// cluster; it is then read and written in that CTA's shared memory through
// the cluster's distributed shared memory. Layers end with a cluster barrier
// (a block barrier when C = 1). Frames start as x = 0, z = fair coin (step 2
// of the algorithm in Section 3).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace stimgb {

namespace {

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
__device__ __forceinline__ void frame_op(const FrameArgs &a, const Tile<C, GMEM> &t, const DevOp op, uint32_t w,
                                         uint64_t lw, uint32_t instr_off, uint32_t meas_off) {
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
            const uint64_t coin = half_mask(a.rk0, a.rk1, kTagCollapse | (op.instr + instr_off), op.slot, gw);
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
            if (opc == OP_XERR) hit = noise_masks<OP_XERR>(G, a.rk0, a.rk1, instr, op.slot, gw, mx, mz, u1, u2);
            else if (opc == OP_ZERR) hit = noise_masks<OP_ZERR>(G, a.rk0, a.rk1, instr, op.slot, gw, mx, mz, u1, u2);
            else hit = noise_masks<OP_DEP1>(G, a.rk0, a.rk1, instr, op.slot, gw, mx, mz, u1, u2);
            if (hit) {
                if (mx) t.st(t.X, ra, w, t.ld(t.X, ra, w) ^ mx);
                if (mz) t.st(t.Z, ra, w, t.ld(t.Z, ra, w) ^ mz);
            }
            break;
        }
        case OP_DEP2: {
            uint64_t m0x, m0z, m1x, m1z;
            if (noise_masks<OP_DEP2>(a.geo + 64u * (op.slot >> 24), a.rk0, a.rk1, op.instr + instr_off,
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

}  // namespace

template <int W, int C, bool GMEM>
__global__ void __launch_bounds__(1024, 1) frame_kernel(const __grid_constant__ FrameArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t rank = C > 1 ? (uint32_t)(blockIdx.x % C) : 0u;
    const uint64_t tile0 = (uint64_t)(blockIdx.x / C) * W;
    const uint32_t qlo = rank * a.Q;
    const uint32_t nq = a.n > qlo ? min(a.Q, a.n - qlo) : 0u;
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
            half_mask(a.rk0, a.rk1, kTagInit, qlo + l, (uint32_t)(a.word0 + tile0 + w));
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
                        frame_op<C, GMEM>(a, t, as_op(__ldg(cp + j)), w, tile0 + w, instr_off, meas_off);
                }
                seg_start += items;
            }
            sync_tile<C>();
            pc++;
        } else if (e.kind == ENT_LOOP_BEGIN) {
            if (sp >= kMaxLoopDepth) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return;
            }
            loop_pc[sp] = pc;
            loop_iter[sp] = 0;
            sp++;
            pc++;
        } else {
            if (sp <= 0) {
                if (threadIdx.x == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return;
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
}

template <int W, int C, bool GMEM>
static cudaError_t launch_frame_t(const FrameArgs &a, uint32_t tiles, uint32_t threads, size_t smem,
                                  cudaStream_t stream) {
    auto kern = frame_kernel<W, C, GMEM>;
    if (!GMEM && smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles * C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = GMEM ? 0 : smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int C, bool GMEM>
static cudaError_t launch_frame_w(const FrameArgs &a, int W, uint32_t tiles, uint32_t threads, size_t smem,
                                  cudaStream_t stream) {
    switch (W) {
        case 1: return launch_frame_t<1, C, GMEM>(a, tiles, threads, smem, stream);
        case 2: return launch_frame_t<2, C, GMEM>(a, tiles, threads, smem, stream);
        case 4: return launch_frame_t<4, C, GMEM>(a, tiles, threads, smem, stream);
        case 8: return launch_frame_t<8, C, GMEM>(a, tiles, threads, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_frame(const FrameArgs &a, int W, int C, bool gmem, uint32_t tiles, uint32_t threads, size_t smem,
                         cudaStream_t stream) {
    if (gmem) return C == 1 ? launch_frame_w<1, true>(a, W, tiles, threads, smem, stream) : cudaErrorInvalidValue;
    switch (C) {
        case 1: return launch_frame_w<1, false>(a, W, tiles, threads, smem, stream);
        case 2: return launch_frame_w<2, false>(a, W, tiles, threads, smem, stream);
        case 4: return launch_frame_w<4, false>(a, W, tiles, threads, smem, stream);
        case 8: return launch_frame_w<8, false>(a, W, tiles, threads, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

void philox_key_schedule(uint64_t seed, uint32_t rk0[10], uint32_t rk1[10]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; r++) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

}  // namespace stimgb
