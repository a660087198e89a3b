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
#include <cuda_runtime.h>

#include "frame_tile.cuh"

namespace stimgb {

template <int W, int C, bool GMEM, bool DETS>
__global__ void __launch_bounds__(frame_max_threads(W), frame_min_ctas(W)) frame_kernel(const __grid_constant__ FrameArgs a) {
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    const uint32_t rank = C > 1 ? (uint32_t)(blockIdx.x % C) : 0u;
    frame_detail::run_tile<W, C, GMEM, DETS, ParamKeys>(a, dyn_smem, rank, blockIdx.x / C);
}

template <int W, int C, bool GMEM>
static cudaError_t launch_frame_t(const FrameArgs &a, uint32_t tiles, uint32_t threads, size_t smem,
                                  cudaStream_t stream) {
    // detection events in the kernel: shared-memory frames of 1 or 8 words
    // per tile only (the shapes the tile chooser picks by itself)
    constexpr bool kDets = !GMEM && (W == 1 || W == 8);
    if (a.det != nullptr && !kDets) return cudaErrorInvalidValue;
    auto kern = a.det != nullptr ? frame_kernel<W, C, GMEM, kDets> : frame_kernel<W, C, GMEM, false>;
    if (smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles * C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
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
    // the kernel's warp collectives (hit-queue ballots) name all 32 lanes of every warp
    if (threads == 0 || threads % 32 != 0) return cudaErrorInvalidValue;
    if (gmem) return C == 1 ? launch_frame_w<1, true>(a, W, tiles, threads, smem, stream) : cudaErrorInvalidValue;
    switch (C) {
        case 1: return launch_frame_w<1, false>(a, W, tiles, threads, smem, stream);
        case 2: return launch_frame_w<2, false>(a, W, tiles, threads, smem, stream);
        case 4: return launch_frame_w<4, false>(a, W, tiles, threads, smem, stream);
        case 8: return launch_frame_w<8, false>(a, W, tiles, threads, smem, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace stimgb
