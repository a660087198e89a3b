// frame.cu -- batched Pauli-frame propagation (Section 3 of the paper).
//
// Each CTA owns W 64-shot words of frames for all n qubits. The X and Z
// planes are kept separately (the paper's "XXXX...ZZZZ" layout, Section 5.1),
// qubit-major with the CTA's W words contiguous per qubit:
//     X[q * qstride + w], Z[q * qstride + w]
// in shared memory for the whole circuit when n * W * 16 bytes fit
// (qstride = W), otherwise in a global-memory frame of all words of the call
// (qstride = words of the call). The CTA walks the compiled program: for
// every fused layer its threads take (op, word) items -- ops of a layer touch
// disjoint qubits -- and a block barrier separates layers.
//
// Per item:
//   H: swap(x, z)   S: z ^= x   CX(c,t): z_c ^= z_t, x_t ^= x_c
//   CZ(a,b): z_a ^= x_b, z_b ^= x_a
//   M:  record = ref[m] ^ x, then z ^= collapse coin
//   MR: record = ref[m] ^ x, then x = 0, z = collapse coin
//   R:  x = 0, z = collapse coin
//   noise: keyed geometric masks multiplied into the frame.
// Frames start as x = 0 and z = a fair coin per qubit (step 2 of the
// algorithm in Section 3).
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace stimgb {

template <int W>
__device__ __forceinline__ void frame_apply(const FrameArgs &a, const DevOp op, uint32_t w,
                                            uint64_t *__restrict__ X, uint64_t *__restrict__ Z,
                                            uint64_t qstride, uint64_t tile0, uint32_t instr_off,
                                            uint32_t meas_off) {
    const uint32_t opc = op.a >> 24;
    const uint64_t ia = (uint64_t)(op.a & kQubitMask) * qstride + w;
    const uint64_t lw = tile0 + w;                       // word index within this call
    const uint32_t gw = (uint32_t)(a.word0 + lw);        // global 64-shot word (RNG counter)
    switch (opc) {
        case OP_H: {
            const uint64_t t = X[ia];
            X[ia] = Z[ia];
            Z[ia] = t;
            break;
        }
        case OP_S:
            Z[ia] ^= X[ia];
            break;
        case OP_CX: {
            const uint64_t ib = (uint64_t)(op.b & kQubitMask) * qstride + w;
            Z[ia] ^= Z[ib];
            X[ib] ^= X[ia];
            break;
        }
        case OP_CZ: {
            const uint64_t ib = (uint64_t)(op.b & kQubitMask) * qstride + w;
            Z[ia] ^= X[ib];
            Z[ib] ^= X[ia];
            break;
        }
        case OP_M:
        case OP_MR: {
            const uint32_t m = op.b + meas_off;
            if (a.rec != nullptr && lw < a.nwords) {
                const uint64_t refm = 0ull - ((__ldg(a.ref + (m >> 6)) >> (m & 63)) & 1ull);
                uint64_t v = X[ia] ^ refm;
                if (lw == a.nwords - 1) v &= a.last_mask;
                a.rec[(uint64_t)m * a.rec_stride + lw] = v;
            }
            const uint64_t coin = half_mask(a.k0, a.k1, kTagCollapse | (op.instr + instr_off), op.slot, gw);
            if (opc == OP_M) {
                Z[ia] ^= coin;
            } else {
                X[ia] = 0;
                Z[ia] = coin;
            }
            break;
        }
        case OP_R: {
            X[ia] = 0;
            Z[ia] = half_mask(a.k0, a.k1, kTagCollapse | (op.instr + instr_off), op.slot, gw);
            break;
        }
        case OP_XERR: {
            uint64_t xa, za, xb, zb;
            noise_masks<OP_XERR>(a.geo + 64u * (op.b >> 24), a.k0, a.k1, op.instr + instr_off, op.slot, gw,
                                 xa, za, xb, zb);
            X[ia] ^= xa;
            break;
        }
        case OP_ZERR: {
            uint64_t xa, za, xb, zb;
            noise_masks<OP_ZERR>(a.geo + 64u * (op.b >> 24), a.k0, a.k1, op.instr + instr_off, op.slot, gw,
                                 xa, za, xb, zb);
            Z[ia] ^= za;
            break;
        }
        case OP_DEP1: {
            uint64_t xa, za, xb, zb;
            noise_masks<OP_DEP1>(a.geo + 64u * (op.b >> 24), a.k0, a.k1, op.instr + instr_off, op.slot, gw,
                                 xa, za, xb, zb);
            X[ia] ^= xa;
            Z[ia] ^= za;
            break;
        }
        case OP_DEP2: {
            uint64_t xa, za, xb, zb;
            noise_masks<OP_DEP2>(a.geo + 64u * (op.b >> 24), a.k0, a.k1, op.instr + instr_off, op.slot, gw,
                                 xa, za, xb, zb);
            const uint64_t ib = (uint64_t)(op.b & kQubitMask) * qstride + w;
            X[ia] ^= xa;
            Z[ia] ^= za;
            X[ib] ^= xb;
            Z[ib] ^= zb;
            break;
        }
        default:
            break;
    }
}

template <int W, bool GMEM>
__global__ void __launch_bounds__(1024) frame_kernel(FrameArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    const uint32_t n = a.n;
    const uint64_t tile0 = (uint64_t)blockIdx.x * W;
    uint64_t *X, *Z;
    uint64_t qstride;
    if (GMEM) {
        X = a.gframe + tile0;
        Z = a.gframe + (uint64_t)n * a.gstride + tile0;
        qstride = a.gstride;
    } else {
        X = smem;
        Z = smem + (uint64_t)n * W;
        qstride = W;
    }
    for (uint32_t i = threadIdx.x; i < n * W; i += blockDim.x) {
        const uint32_t q = i / W, w = i % W;
        X[(uint64_t)q * qstride + w] = 0;
        Z[(uint64_t)q * qstride + w] = half_mask(a.k0, a.k1, kTagInit, q, (uint32_t)(a.word0 + tile0 + w));
    }
    __syncthreads();

    uint32_t instr_off = 0, meas_off = 0;
    uint32_t loop_pc[kMaxLoopDepth];
    uint32_t loop_iter[kMaxLoopDepth];
    int sp = 0;
    uint32_t pc = 0;
    while (pc < a.nprog) {
        const ProgEntry e = a.prog[pc];
        if (e.kind == ENT_LAYER) {
            const uint32_t items = (e.n_gate + e.n_noise + e.n_collapse) * W;
            const DevOp *ops = a.ops + e.op_begin;
            for (uint32_t i = threadIdx.x; i < items; i += blockDim.x)
                frame_apply<W>(a, ops[i / W], i % W, X, Z, qstride, tile0, instr_off, meas_off);
            __syncthreads();
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

template <int W, bool GMEM>
static cudaError_t launch_frame_t(const FrameArgs &a, uint32_t grid, uint32_t threads, size_t smem,
                                  cudaStream_t stream) {
    auto kern = frame_kernel<W, GMEM>;
    if (!GMEM && smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    kern<<<grid, threads, GMEM ? 0 : smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_frame(const FrameArgs &a, int W, bool gmem, uint32_t grid, uint32_t threads, size_t smem,
                         cudaStream_t stream) {
#define STIMGB_CASE(w)                                                             \
    case w:                                                                        \
        return gmem ? launch_frame_t<w, true>(a, grid, threads, smem, stream)      \
                    : launch_frame_t<w, false>(a, grid, threads, smem, stream);
    switch (W) {
        STIMGB_CASE(1)
        STIMGB_CASE(2)
        STIMGB_CASE(4)
        STIMGB_CASE(8)
        STIMGB_CASE(16)
        default:
            return cudaErrorInvalidValue;
    }
#undef STIMGB_CASE
}

}  // namespace stimgb
