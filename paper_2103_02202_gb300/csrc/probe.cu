// probe.cu -- shared-memory bandwidth of this GPU, measured with the frame
// kernel's own access widths (measurement support; no counterpart in the
// paper). The frame kernel keeps its Pauli frames in shared memory (local,
// or a peer CTA's through distributed shared memory), so the roofline that
// bounds its gate work is shared-memory bandwidth, not HBM; this probe gives
// that roofline's denominator on the box it runs on.
//
// Each CTA owns a 64 KiB buffer; every thread streams 16-byte loads and
// stores (ld.shared.v2.u64 / st.shared.v2.u64, the frame kernel's access
// width) over its own conflict-free column, XOR-folding what it reads into a
// register that is written out once, so nothing can be elided. The cluster
// variant reads and writes the buffer of the next CTA of its 2-CTA cluster
// (ld/st.shared::cluster). Bytes = loads + stores.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/stimgb.h"
#include "internal.h"

namespace stimgb {
namespace {

constexpr uint32_t kProbeBytes = 64 * 1024;
constexpr uint32_t kProbeThreads = 512;
constexpr uint32_t kProbeIters = 4096;

template <bool REMOTE>
__global__ void __launch_bounds__(kProbeThreads) smem_probe_kernel(uint64_t *sink) {
    extern __shared__ __align__(128) unsigned char buf[];
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    for (uint32_t i = threadIdx.x; i < kProbeBytes / 8; i += blockDim.x)
        reinterpret_cast<uint64_t *>(buf)[i] = i * 0x9E3779B97F4A7C15ull;
    uint32_t peer = base;
    if constexpr (REMOTE) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
        uint32_t rank;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(peer) : "r"(base), "r"(rank ^ 1u));
    } else {
        __syncthreads();
    }
    // thread t walks 16-byte chunk t, t + 512, ... (64 KiB = 4096 chunks, 8 per thread)
    uint64_t acc0 = 0, acc1 = 0;
    uint32_t a = peer + 16u * threadIdx.x;
    const uint32_t wrap = peer + kProbeBytes;
#pragma unroll 4
    for (uint32_t it = 0; it < kProbeIters; it++) {
        uint64_t v0, v1;
        if constexpr (REMOTE) {
            asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "r"(a) : "memory");
            asm volatile("st.shared::cluster.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(v1 ^ it), "l"(v0) : "memory");
        } else {
            asm volatile("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "r"(a) : "memory");
            asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(a), "l"(v1 ^ it), "l"(v0) : "memory");
        }
        acc0 ^= v0;
        acc1 += v1;
        a += 16u * kProbeThreads;
        if (a >= wrap) a -= kProbeBytes;
    }
    if constexpr (REMOTE)
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    sink[blockIdx.x * blockDim.x + threadIdx.x] = acc0 ^ acc1;
}

template <bool REMOTE>
cudaError_t run_probe(uint64_t *sink, uint32_t blocks, cudaStream_t st) {
    auto kern = smem_probe_kernel<REMOTE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kProbeBytes);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kProbeThreads);
    cfg.dynamicSmemBytes = kProbeBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = REMOTE ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, sink);
}

}  // namespace
}  // namespace stimgb

using namespace stimgb;

extern "C" int stim_probe_smem_bandwidth(double *local_gbs, double *cluster_gbs) {
    if (!local_gbs || !cluster_gbs) return report_error(STIM_E_INVALID_ARG, "stim_probe_smem_bandwidth: null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return report_error(STIM_E_CUDA, std::string("probe: ") + cudaGetErrorString(e));
    // three 64 KiB CTAs per SM (192 KiB of the 228 KiB), an even count for the 2-CTA clusters
    const uint32_t blocks = (uint32_t)sms * 3u & ~1u;
    uint64_t *sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double out[2] = {0, 0};
    e = cudaMalloc((void **)&sink, (size_t)blocks * kProbeThreads * 8);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int remote = 0; remote < 2 && e == cudaSuccess; remote++) {
        float best = 0;
        for (int rep = 0; rep < 4 && e == cudaSuccess; rep++) {      // the first run warms up
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = remote ? run_probe<true>(sink, blocks, st) : run_probe<false>(sink, blocks, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0 && (best == 0 || ms < best)) best = ms;
        }
        const double bytes = (double)blocks * kProbeThreads * kProbeIters * 32.0;
        if (e == cudaSuccess && best > 0) out[remote] = bytes / (best * 1e-3) / 1e9;
    }
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) return report_error(STIM_E_CUDA, std::string("probe: ") + cudaGetErrorString(e));
    *local_gbs = out[0];
    *cluster_gbs = out[1];
    return STIM_OK;
}
