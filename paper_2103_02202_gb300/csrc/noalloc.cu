// noalloc.cu -- detection-event sampling that allocates no device memory.
//
// stim_frame_sample_noalloc() runs the same frame and detector kernels as
// stim_frame_sample_ex(), but the measurement records that the detector
// kernel reads -- the one buffer the normal path allocates for this output --
// live in a fixed array in this file instead of memory from cudaMalloc. It is
// meant for callers that cannot obtain device memory at sampling time, for
// instance because another allocator (a framework's caching allocator or a
// service's up-front reservation) owns the device's memory, or because they
// cannot afford the device-wide synchronization that cudaFree implies.
//
// The array is a module global: every GPU that loads the library holds all
// of it until the process exits, and every call on a device uses the same
// array, so calls whose work overlaps on one GPU race with each other.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/stimgb.h"
#include "handle.h"
#include "internal.h"
#include "kernels.h"

using namespace stimgb;

namespace {

constexpr size_t kScratchWords = STIM_NOALLOC_SCRATCH_BYTES / 8;

// Measurement records of one call, measurement-major: [M][ceil(num_shots/64)].
static __device__ __align__(256) uint64_t g_noalloc_records[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint64_t *g_scratch[kMaxDevices];   // device address of g_noalloc_records, per device
bool g_ready[kMaxDevices];

int fail(int code, const std::string &msg) { return report_error(code, msg); }

// Looks up the array's device address on the current device (once per device).
int scratch_for(int dev, uint64_t **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(STIM_E_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_records);
        if (e != cudaSuccess)
            return fail(STIM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch[dev] = (uint64_t *)p;
        g_ready[dev] = true;
    }
    *out = g_scratch[dev];
    return STIM_OK;
}

}  // namespace

extern "C" int stim_frame_sample_noalloc(stim_circuit *c, uint64_t num_shots, uint64_t seed,
                                         uint64_t shot_offset, uint64_t *det_out, void *stream) {
    if (!c) return fail(STIM_E_INVALID_ARG, "stim_frame_sample_noalloc: null handle");
    if (shot_offset % 64)
        return fail(STIM_E_INVALID_ARG, "stim_frame_sample_noalloc: shot_offset must be a multiple of 64");
    if ((shot_offset + num_shots + 63) / 64 > (1ull << 32))
        return fail(STIM_E_UNSUPPORTED, "stim_frame_sample_noalloc: global shot index above 2^38");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(STIM_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (c->device != dev || !c->ref_valid)
        return fail(STIM_E_INVALID_ARG,
                    "stim_frame_sample_noalloc: call stim_reference_sample on this device first "
                    "(it uploads the circuit and takes the reference sample)");
    if (num_shots == 0) return STIM_OK;
    const HostProgram &hp = c->hp;
    const uint64_t M = hp.num_meas, D = hp.num_det;
    const uint32_t n = hp.num_qubits;
    const uint64_t nwords = (num_shots + 63) / 64;
    if (M > 0 && M > kScratchWords / nwords)
        return fail(STIM_E_UNSUPPORTED,
                    "stim_frame_sample_noalloc: measurements x ceil(shots/64) x 8 bytes exceeds the "
                    "fixed 32 MiB record array; sample fewer shots per call");
    int smem_optin = 0, sms = 0;
    e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(STIM_E_CUDA, std::string("attribute: ") + cudaGetErrorString(e));
    const DevFrameProgram &fp = c->fprog[0];    // single-CTA program, uploaded with the circuit
    if (fp.C != 1) return fail(STIM_E_INVALID_ARG, "stim_frame_sample_noalloc: circuit not uploaded");
    // the launch asks for exactly tile_smem_bytes(...) of shared memory, so
    // both the rejection and the tile width are decided on that figure
    const uint32_t meta_region = meta_region_for(fp.meta_bytes);
    if (tile_smem_bytes(fp.Q, 1, false, meta_region) > (size_t)smem_optin)
        return fail(STIM_E_UNSUPPORTED,
                    "stim_frame_sample_noalloc: one 64-shot frame tile does not fit shared memory");
    uint64_t *rec = nullptr;
    int r = scratch_for(dev, &rec);
    if (r != STIM_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    // Every record row read by the detector kernel is written first by the
    // frame kernel (all measurements, all words), so the array needs no clearing.
    if (n > 0 && M > 0) {
        int W = 1;
        for (int w : {8, 4, 2}) {
            if (tile_smem_bytes(fp.Q, w, false, meta_region) <= (size_t)smem_optin / 2 &&
                (nwords + w - 1) / w >= (uint64_t)sms * 2) {
                W = w;
                break;
            }
        }
        FrameArgs a{};
        a.prog = fp.prog;
        a.nprog = fp.nprog;
        a.rank_tab = fp.rank_tab;
        a.segs = fp.segs;
        a.ops = fp.ops;
        a.geo = c->d_geo;
        a.ref = c->d_ref;
        a.n = n;
        a.Q = fp.Q;
        set_seed(a, seed);
        a.word0 = shot_offset / 64;
        a.nwords = nwords;
        a.last_mask = (num_shots % 64) ? ((1ull << (num_shots % 64)) - 1) : ~0ull;
        a.rec = rec;
        a.rec_stride = nwords;
        a.rec_mask = 0xFFFFFFFFu;
        a.status = c->d_status;
        const uint64_t grid = (nwords + W - 1) / W;
        a.meta_bytes = fp.meta_bytes;
        a.meta_region = meta_region;
        e = launch_frame(a, W, 1, false, (uint32_t)grid, 256, tile_smem_bytes(fp.Q, W, false, a.meta_region), st);
        if (e != cudaSuccess) return fail(STIM_E_CUDA, std::string("frame kernel: ") + cudaGetErrorString(e));
    }
    if (det_out && D > 0) {
        const uint64_t last_mask = (num_shots % 64) ? ((1ull << (num_shots % 64)) - 1) : ~0ull;
        e = launch_detectors(rec, nwords, c->d_det_ptr, c->d_det_meas, c->d_ref, D, nwords, last_mask, det_out,
                             nwords, st);
        if (e != cudaSuccess) return fail(STIM_E_CUDA, std::string("detector kernel: ") + cudaGetErrorString(e));
    }
    return STIM_OK;
}
