// batch.cu -- many compiled circuits in one persistent launch.
//
// A batch plan lists the (circuit, word tile) work items of k circuits, most
// expensive circuits first, and launches one persistent frame kernel sized to
// the GPU: each CTA (or cluster of CTAs splitting the qubits) takes the next
// item from an atomic counter, copies that circuit's descriptor into shared
// memory and runs the same per-tile code as the single-circuit kernel. A
// batched detector kernel follows. Both launches and the upload of the
// per-call descriptors (seeds, output pointers) are captured once into a
// CUDA graph and replayed. The tile shape is chosen by a small autotuner that
// times candidate shapes on a prefix of the work list and remembers the
// winner per batch shape (optionally in a file named by STIMGB_TUNE_CACHE).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/stimgb.h"
#include "frame_tile.cuh"
#include "handle.h"

namespace cg = cooperative_groups;

namespace stimgb {

struct BatchItem {
    uint32_t circuit;
    uint32_t tile;
};

struct DetDesc {
    const uint64_t *rec;
    uint64_t rec_stride;
    const uint64_t *det_ptr;
    const uint32_t *det_meas;
    const uint64_t *ref;
    uint64_t ndet, nwords, last_mask;
    uint64_t *det;
    uint64_t row_begin;    // detector rows of earlier circuits
};

constexpr uint32_t kDescBytes = 384;   // FrameArgs copy at the start of dynamic smem
static_assert(sizeof(FrameArgs) <= kDescBytes, "descriptor does not fit its slot");

template <int W, int C>
__global__ void __launch_bounds__(batch_max_threads(W), frame_min_ctas(W)) batch_frame_kernel(const FrameArgs *__restrict__ descs,
                                                              const BatchItem *__restrict__ items, uint32_t nitems,
                                                              uint32_t *counter) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint32_t s_item;
    FrameArgs *sa = reinterpret_cast<FrameArgs *>(smem);
    unsigned char *tile_dyn = smem + kDescBytes;
    const uint32_t rank = C > 1 ? (uint32_t)(blockIdx.x % C) : 0u;
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        if constexpr (C > 1) {
            cg::cluster_group cl = cg::this_cluster();
            cl.sync();
            uint32_t k = 0;
            if (threadIdx.x == 0) k = *cl.map_shared_rank(&s_item, 0);
            cl.sync();                      // rank 0's slot is read before anyone moves on
            if (threadIdx.x == 0 && rank != 0) s_item = k;
            __syncthreads();
        } else {
            __syncthreads();
        }
        const uint32_t k = s_item;
        if (k >= nitems) break;
        const BatchItem it = items[k];
        const uint32_t *src = reinterpret_cast<const uint32_t *>(descs + it.circuit);
        for (uint32_t i = threadIdx.x; i < sizeof(FrameArgs) / 4; i += blockDim.x)
            reinterpret_cast<uint32_t *>(sa)[i] = __ldg(src + i);
        __syncthreads();
        frame_detail::run_tile<W, C, false, false>(*sa, tile_dyn, rank, it.tile);
        __syncthreads();
    }
}

// One warp per detector row of the batch (rows numbered across circuits):
// the owning circuit is found once per row, then the lanes sweep the row's
// words as in the single-circuit detector kernel.
__global__ void __launch_bounds__(256) batch_detector_kernel(const DetDesc *__restrict__ d, uint32_t k,
                                                             uint64_t rows) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < rows; i += warps) {
        uint32_t lo = 0, hi = k - 1;        // last circuit with row_begin <= i
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (d[mid].row_begin <= i) lo = mid;
            else hi = mid - 1;
        }
        const DetDesc &c = d[lo];
        const uint64_t det = i - c.row_begin;
        const uint64_t b = __ldg(c.det_ptr + det), e = __ldg(c.det_ptr + det + 1);
        uint64_t *out = c.det + det * c.nwords;
        for (uint64_t w = lane; w < c.nwords; w += 32) {
            uint64_t v = 0;
            for (uint64_t t = b; t < e; t++) {
                const uint32_t m = __ldg(c.det_meas + t);
                const uint64_t refm = 0ull - ((__ldg(c.ref + (m >> 6)) >> (m & 63)) & 1ull);
                v ^= __ldg(c.rec + (uint64_t)m * c.rec_stride + w) ^ refm;
            }
            if (w == c.nwords - 1) v &= c.last_mask;
            out[w] = v;
        }
    }
}

template <int W, int C>
static cudaError_t launch_batch_t(const FrameArgs *descs, const BatchItem *items, uint32_t nitems, uint32_t *counter,
                                  uint32_t blocks, uint32_t threads, size_t smem, cudaStream_t st) {
    auto kern = batch_frame_kernel<W, C>;      // smem attribute set by max_resident_ctas
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, descs, items, nitems, counter);
}

template <int W, int C>
static int max_resident_ctas_t(uint32_t threads, size_t smem, int sms) {
    auto kern = batch_frame_kernel<W, C>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (C == 1) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, smem) != cudaSuccess) return 0;
        return per_sm * sms;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms * C));
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) return 0;
    return clusters * C;
}

#define STIMGB_BATCH_DISPATCH(FN, ...)                                            \
    switch (C) {                                                                  \
        case 1: switch (W) { case 1: return FN<1, 1>(__VA_ARGS__); case 2: return FN<2, 1>(__VA_ARGS__); \
                             case 4: return FN<4, 1>(__VA_ARGS__); default: break; } break;            \
        case 2: switch (W) { case 1: return FN<1, 2>(__VA_ARGS__); case 2: return FN<2, 2>(__VA_ARGS__); \
                             case 4: return FN<4, 2>(__VA_ARGS__); default: break; } break;            \
        case 4: switch (W) { case 1: return FN<1, 4>(__VA_ARGS__); case 2: return FN<2, 4>(__VA_ARGS__); \
                             case 4: return FN<4, 4>(__VA_ARGS__); default: break; } break;            \
        case 8: switch (W) { case 1: return FN<1, 8>(__VA_ARGS__); case 2: return FN<2, 8>(__VA_ARGS__); \
                             case 4: return FN<4, 8>(__VA_ARGS__); default: break; } break;            \
        default: break;                                                           \
    }

static cudaError_t launch_batch(int W, int C, const FrameArgs *descs, const BatchItem *items, uint32_t nitems,
                                uint32_t *counter, uint32_t blocks, uint32_t threads, size_t smem, cudaStream_t st) {
    // the kernel's warp collectives (hit-queue ballots) name all 32 lanes of every warp
    if (threads == 0 || threads % 32 != 0) return cudaErrorInvalidValue;
    STIMGB_BATCH_DISPATCH(launch_batch_t, descs, items, nitems, counter, blocks, threads, smem, st)
    return cudaErrorInvalidValue;
}

static int max_resident_ctas(int W, int C, uint32_t threads, size_t smem, int sms) {
    STIMGB_BATCH_DISPATCH(max_resident_ctas_t, threads, smem, sms)
    return 0;
}

}  // namespace stimgb

using namespace stimgb;

struct stim_batch {
    int device = -1;
    size_t k = 0;
    std::vector<stim_circuit *> cs;
    std::vector<uint64_t> shots;
    int W = 1, C = 1;
    uint32_t threads = 256, blocks = 0;
    size_t smem = 0;
    uint32_t nitems = 0;
    std::vector<BatchItem> items_host;
    BatchItem *d_items = nullptr;
    uint32_t *d_counter = nullptr;
    FrameArgs *d_descs = nullptr;
    FrameArgs *h_descs = nullptr;          // pinned
    DetDesc *d_det = nullptr;
    DetDesc *h_det = nullptr;              // pinned
    uint64_t det_total = 0;
    std::vector<uint64_t *> rec_scratch;
    std::vector<size_t> rec_cap;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool launched = false;
    bool tuned = false;
    std::string tune_key;
    bool hinted = false;
    uint32_t meta_region = 0;              // shared bytes for the largest program metadata that fits
    std::vector<uint8_t> out_sig;          // which outputs the captured graph serves
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, uint32_t>> g_tune;   // batch shape -> (W, threads)
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("STIMGB_TUNE_CACHE");
    if (!path || !*path) return;
    std::ifstream in(path);
    std::string key;
    int W;
    uint32_t th;
    while (in >> key >> W >> th) g_tune[key] = {W, th};
}

void tune_store_locked() {
    const char *path = getenv("STIMGB_TUNE_CACHE");
    if (!path || !*path) return;
    std::ofstream out(path, std::ios::trunc);
    for (const auto &kv : g_tune) out << kv.first << " " << kv.second.first << " " << kv.second.second << "\n";
}

int bfail(int code, const std::string &msg) { return report_error(code, msg); }

#define STIMGB_BCK(call, what)                                                                   \
    do {                                                                                         \
        cudaError_t _e = (call);                                                                 \
        if (_e != cudaSuccess)                                                                   \
            return bfail(_e == cudaErrorMemoryAllocation ? STIM_E_OOM : STIM_E_CUDA,             \
                         std::string(what) + ": " + cudaGetErrorString(_e));                     \
    } while (0)

uint64_t words_of(uint64_t shots) { return (shots + 63) / 64; }

// Work list for tile width W: circuits by decreasing cost per word, all tiles of each.
void build_items(stim_batch *b, int W) {
    std::vector<size_t> order(b->k);
    for (size_t i = 0; i < b->k; i++) order[i] = i;
    auto cost = [&](size_t i) {
        const HostProgram &hp = b->cs[i]->hp;
        return (double)(hp.num_gate_targets + hp.num_noise_targets) * (double)words_of(b->shots[i]);
    };
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost(x) > cost(y); });
    b->items_host.clear();
    for (size_t i : order) {
        const uint64_t tiles = (words_of(b->shots[i]) + W - 1) / W;
        for (uint64_t t = 0; t < tiles; t++) b->items_host.push_back({(uint32_t)i, (uint32_t)t});
    }
    b->nitems = (uint32_t)b->items_host.size();
}

int upload_items(stim_batch *b) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    STIMGB_BCK(cudaMalloc((void **)&b->d_items, std::max<size_t>(b->nitems, 1) * sizeof(BatchItem)), "batch items");
    if (b->nitems)
        STIMGB_BCK(cudaMemcpy(b->d_items, b->items_host.data(), b->nitems * sizeof(BatchItem), cudaMemcpyHostToDevice),
                   "batch items");
    return STIM_OK;
}

// Largest qubit slice of any circuit in the batch.
uint32_t batch_max_slice(const stim_batch *b, int C) {
    uint32_t maxq = 1;
    for (stim_circuit *c : b->cs) {
        const uint32_t n = c->hp.num_qubits ? c->hp.num_qubits : 1;
        maxq = std::max(maxq, (n + (uint32_t)C - 1) / (uint32_t)C);
    }
    return maxq;
}

// Dynamic shared memory of the persistent kernel: descriptor + tile region.
size_t batch_smem(const stim_batch *b, int W, int C, uint32_t meta_region) {
    return kDescBytes + tile_smem_bytes(batch_max_slice(b, C), W, false, meta_region);
}

}  // namespace

namespace {

int fill_descs(stim_batch *b, const uint64_t *seeds, const uint64_t *offsets, uint64_t *const *meas_out,
               uint64_t *const *det_out, int C) {
    b->det_total = 0;
    for (size_t i = 0; i < b->k; i++) {
        stim_circuit *c = b->cs[i];
        const HostProgram &hp = c->hp;
        const uint64_t nwords = words_of(b->shots[i]);
        const uint64_t S = b->shots[i];
        const uint64_t last_mask = (S % 64) ? ((1ull << (S % 64)) - 1) : ~0ull;
        uint64_t *meas = meas_out ? meas_out[i] : nullptr;
        uint64_t *det = det_out ? det_out[i] : nullptr;
        uint64_t *rec = meas;
        if (!rec && hp.num_meas > 0 && ((det && hp.num_det > 0) || hp.num_feedforward > 0)) {
            const size_t need = hp.num_meas * nwords;
            if (b->rec_cap[i] < need) {
                cudaFree(b->rec_scratch[i]);
                b->rec_scratch[i] = nullptr;
                b->rec_cap[i] = 0;
                STIMGB_BCK(cudaMalloc((void **)&b->rec_scratch[i], need * 8), "batch record scratch");
                b->rec_cap[i] = need;
            }
            rec = b->rec_scratch[i];
        }
        const DevFrameProgram *fp = nullptr;
        int r = stimgb_frame_program(c, C, &fp);
        if (r != STIM_OK) return r;
        FrameArgs a{};
        a.prog = fp->prog;
        a.nprog = fp->nprog;
        a.rank_tab = fp->rank_tab;
        a.segs = fp->segs;
        a.ops = fp->ops;
        a.geo = c->d_geo;
        a.ref = c->d_ref;
        a.n = hp.num_qubits;
        a.Q = fp->Q;
        a.word0 = (offsets ? offsets[i] : 0) / 64;
        a.nwords = nwords;
        a.last_mask = last_mask;
        a.rec = hp.num_meas ? rec : nullptr;
        a.rec_stride = nwords;
        a.rec_mask = 0xFFFFFFFFu;
        a.status = c->d_status;
        set_seed(a, seeds[i]);
        a.meta_bytes = fp->meta_bytes;
        a.meta_region = b->meta_region;
        b->h_descs[i] = a;
        DetDesc d{};
        d.rec = rec;
        d.rec_stride = nwords;
        d.det_ptr = c->d_det_ptr;
        d.det_meas = c->d_det_meas;
        d.ref = c->d_ref;
        d.ndet = (det && hp.num_det) ? hp.num_det : 0;
        d.nwords = nwords;
        d.last_mask = last_mask;
        d.det = det;
        d.row_begin = b->det_total;
        b->det_total += d.ndet;
        b->h_det[i] = d;
    }
    return STIM_OK;
}

// The replayed work of one call: descriptor upload, counter reset, frames, detectors.
int enqueue(stim_batch *b, cudaStream_t st, uint32_t nitems_limit) {
    STIMGB_BCK(cudaMemcpyAsync(b->d_descs, b->h_descs, b->k * sizeof(FrameArgs), cudaMemcpyHostToDevice, st),
               "batch descriptors");
    STIMGB_BCK(cudaMemcpyAsync(b->d_det, b->h_det, b->k * sizeof(DetDesc), cudaMemcpyHostToDevice, st),
               "batch descriptors");
    STIMGB_BCK(cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), st), "batch counter");
    STIMGB_BCK(launch_batch(b->W, b->C, b->d_descs, b->d_items, nitems_limit, b->d_counter, b->blocks, b->threads,
                            b->smem, st),
               "batch frame kernel");
    if (b->det_total) {
        uint64_t grid = (b->det_total + 7) / 8;      // 8 warps (rows) per block
        if (grid > 65535ull * 32) grid = 65535ull * 32;
        batch_detector_kernel<<<(unsigned)grid, 256, 0, st>>>(b->d_det, (uint32_t)b->k, b->det_total);
        STIMGB_BCK(cudaGetLastError(), "batch detector kernel");
    }
    return STIM_OK;
}

int configure(stim_batch *b, int W, uint32_t threads) {
    int sms = 0;
    STIMGB_BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "attr");
    if (threads == 0 || threads % 32 != 0)
        return bfail(STIM_E_INVALID_ARG, "batch: threads per CTA must be a multiple of 32");
    if ((int)threads > batch_max_threads(W))
        return bfail(STIM_E_INVALID_ARG, "batch: too many threads per CTA for this many words per tile (448 for 1, 768 for 2, 512 for 4 or 8)");
    b->W = W;
    b->threads = threads;
    int smem_optin = 0;
    STIMGB_BCK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device), "attr");
    uint32_t meta_region = 0;
    for (stim_circuit *c : b->cs) {
        const DevFrameProgram *fp;
        int r = stimgb_frame_program(c, b->C, &fp);
        if (r != STIM_OK) return r;
        meta_region = std::max(meta_region, meta_region_for(fp->meta_bytes));
    }
    // the metadata region is part of this shape's shared memory: a circuit
    // larger than it reads its metadata from global memory
    if (batch_smem(b, W, b->C, meta_region) > (size_t)smem_optin) meta_region = 0;
    b->meta_region = meta_region;
    b->smem = batch_smem(b, W, b->C, meta_region);
    for (size_t i = 0; i < b->k; i++) b->h_descs[i].meta_region = meta_region;
    const int ctas = max_resident_ctas(W, b->C, threads, b->smem, sms);
    if (ctas <= 0) return bfail(STIM_E_UNSUPPORTED, "batch: tile shape does not fit an SM");
    b->blocks = (uint32_t)ctas;
    build_items(b, W);
    return upload_items(b);
}

// Times candidate tile shapes on the whole work list; keeps the fastest.
int autotune(stim_batch *b, cudaStream_t st) {
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(b->tune_key);
        if (it != g_tune.end()) return configure(b, it->second.first, it->second.second);
    }
    int smem_optin = 0;
    STIMGB_BCK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device), "attr");
    // Each candidate shape runs the whole batch once (after one warm-up run of
    // the first shape): prefixes of the largest-first queue misjudge mixes of
    // large and small circuits.
    const int cand_w[4] = {1, 2, 4, 8};
    const uint32_t cand_t[3] = {256, 448, 512};
    bool warm = false;
    double best = -1;
    int bw = 1;
    uint32_t bt = 256;
    cudaEvent_t e0, e1;
    STIMGB_BCK(cudaEventCreate(&e0), "event");
    STIMGB_BCK(cudaEventCreate(&e1), "event");
    for (int w : cand_w) {
        if (batch_smem(b, w, b->C, 0) > (size_t)smem_optin) continue;
        for (uint32_t t : cand_t) {
            if (configure(b, w, t) != STIM_OK) continue;
            if (!warm) {
                if (enqueue(b, st, b->nitems) != STIM_OK) continue;
                warm = true;
            }
            cudaEventRecord(e0, st);
            if (enqueue(b, st, b->nitems) != STIM_OK) continue;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) continue;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            const double rate = ms > 0 ? 1.0 / ms : 0;
            if (rate > best) {
                best = rate;
                bw = w;
                bt = t;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[b->tune_key] = {bw, bt};
        tune_store_locked();
    }
    return configure(b, bw, bt);
}

}  // namespace

extern "C" {

int stim_batch_create(stim_circuit *const *circuits, const uint64_t *num_shots, size_t k, const stim_tile_hint *hint,
                      void *stream, stim_batch **out) {
    if (!out || !circuits || !num_shots || k == 0) return bfail(STIM_E_INVALID_ARG, "stim_batch_create: bad arguments");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    stim_batch *b = new (std::nothrow) stim_batch();
    if (!b) return bfail(STIM_E_OOM, "stim_batch_create: out of host memory");
    int dev = 0;
    cudaGetDevice(&dev);
    b->device = dev;
    b->k = k;
    b->cs.assign(circuits, circuits + k);
    b->shots.assign(num_shots, num_shots + k);
    b->rec_scratch.assign(k, nullptr);
    b->rec_cap.assign(k, 0);
    int r = STIM_OK;
    int smem_optin = 0;
    cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    uint32_t maxn = 1;
    uint64_t ops = 0, words = 0;
    for (size_t i = 0; i < k && r == STIM_OK; i++) {
        if (!circuits[i]) r = bfail(STIM_E_INVALID_ARG, "stim_batch_create: null circuit");
        else if ((num_shots[i] + 63) / 64 > (1ull << 31)) r = bfail(STIM_E_UNSUPPORTED, "stim_batch_create: too many shots");
    }
    // reference samples of all circuits, side by side
    if (r == STIM_OK) r = stimgb_ensure_references(circuits, k);
    for (size_t i = 0; i < k && r == STIM_OK; i++) {
        r = stimgb_ensure_reference(circuits[i], st);
        if (r == STIM_OK) {
            maxn = std::max(maxn, circuits[i]->hp.num_qubits);
            ops += circuits[i]->hp.num_gate_targets + circuits[i]->hp.num_noise_targets;
            words += words_of(num_shots[i]);
        }
    }
    if (r == STIM_OK) {
        // smallest cluster whose largest slice fits with two tiles per SM
        b->C = 0;
        for (int C : {1, 2, 4, 8})
            if ((size_t)((maxn + C - 1) / C) * 16 * 2 + 2 * (kDescBytes + kTileHeaderBytes) <= (size_t)smem_optin) {
                b->C = C;
                break;
            }
        if (hint && hint->cluster_size) b->C = (int)hint->cluster_size;
        if (b->C == 0) r = bfail(STIM_E_UNSUPPORTED, "stim_batch_create: a circuit is too wide for the batched kernel");
    }
    if (r == STIM_OK) {
        b->h_descs = nullptr;
        if (cudaMallocHost((void **)&b->h_descs, k * sizeof(FrameArgs)) != cudaSuccess ||
            cudaMallocHost((void **)&b->h_det, k * sizeof(DetDesc)) != cudaSuccess ||
            cudaMalloc((void **)&b->d_descs, k * sizeof(FrameArgs)) != cudaSuccess ||
            cudaMalloc((void **)&b->d_det, k * sizeof(DetDesc)) != cudaSuccess ||
            cudaMalloc((void **)&b->d_counter, sizeof(uint32_t)) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
            r = bfail(STIM_E_OOM, "stim_batch_create: allocation failed");
    }
    if (r == STIM_OK) {
        for (size_t i = 0; i < k && r == STIM_OK; i++) {
            const DevFrameProgram *fp;
            r = stimgb_frame_program(circuits[i], b->C, &fp);
        }
    }
    if (r == STIM_OK) {
        std::ostringstream key;
        key << "C" << b->C << "_n" << (maxn + 63) / 64 << "_k" << k << "_o" << (ops >> 14) << "_w" << (words >> 10);
        b->tune_key = key.str();
        if (hint && hint->words_per_cta) {
            b->hinted = true;
            const uint32_t th = hint->threads ? hint->threads : 256;
            r = configure(b, (int)hint->words_per_cta, th);
            b->tuned = true;
        }
    }
    if (r != STIM_OK) {
        stim_batch_free(b);
        return r;
    }
    *out = b;
    return STIM_OK;
}

int stim_batch_sample(stim_batch *b, const uint64_t *seeds, const uint64_t *shot_offsets, uint64_t *const *meas_out,
                      uint64_t *const *det_out, void *stream) {
    if (!b || !seeds) return bfail(STIM_E_INVALID_ARG, "stim_batch_sample: bad arguments");
    if (shot_offsets)
        for (size_t i = 0; i < b->k; i++)
            if (shot_offsets[i] % 64) return bfail(STIM_E_INVALID_ARG, "stim_batch_sample: shot offsets must be multiples of 64");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return bfail(STIM_E_INVALID_ARG, "stim_batch_sample: plan belongs to another device");
    if (b->launched) STIMGB_BCK(cudaEventSynchronize(b->done), "batch previous launch");
    const int C = b->C;
    int r = fill_descs(b, seeds, shot_offsets, meas_out, det_out, C);
    if (r != STIM_OK) return r;
    if (!b->tuned) {
        r = autotune(b, st);
        if (r != STIM_OK) return r;
        b->tuned = true;
        STIMGB_BCK(cudaStreamSynchronize(st), "batch autotune");
    }
    std::vector<uint8_t> sig(b->k);
    for (size_t i = 0; i < b->k; i++)
        sig[i] = (uint8_t)((meas_out && meas_out[i] ? 1 : 0) | (det_out && det_out[i] ? 2 : 0));
    if (b->exec && sig != b->out_sig) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
    }
    if (!b->exec) {
        // capture the replayed work once per output configuration; later calls
        // refill the pinned descriptors (seeds, offsets, output pointers)
        b->out_sig = sig;
        cudaStream_t cap;
        STIMGB_BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream");
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            r = enqueue(b, cap, b->nitems);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(cap, &g);
            if (r == STIM_OK && e == cudaSuccess) {
                b->graph = g;
                e = cudaGraphInstantiate(&b->exec, g, 0);
            }
        }
        cudaStreamDestroy(cap);
        if (r != STIM_OK) return r;
        if (e != cudaSuccess) return bfail(STIM_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    STIMGB_BCK(cudaGraphLaunch(b->exec, st), "batch graph launch");
    STIMGB_BCK(cudaEventRecord(b->done, st), "batch event");
    b->launched = true;
    return STIM_OK;
}

int stim_batch_info(const stim_batch *b, uint32_t *words_per_tile, uint32_t *threads, uint32_t *cluster_size,
                    uint32_t *ctas, uint64_t *work_items) {
    if (!b) return bfail(STIM_E_INVALID_ARG, "stim_batch_info: null plan");
    if (words_per_tile) *words_per_tile = (uint32_t)b->W;
    if (threads) *threads = b->threads;
    if (cluster_size) *cluster_size = (uint32_t)b->C;
    if (ctas) *ctas = b->blocks;
    if (work_items) *work_items = b->nitems;
    return STIM_OK;
}

void stim_batch_free(stim_batch *b) {
    if (!b) return;
    if (b->device >= 0) {
        cudaDeviceSynchronize();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        if (b->done) cudaEventDestroy(b->done);
        cudaFree(b->d_items);
        cudaFree(b->d_counter);
        cudaFree(b->d_descs);
        cudaFree(b->d_det);
        if (b->h_descs) cudaFreeHost(b->h_descs);
        if (b->h_det) cudaFreeHost(b->h_det);
        for (uint64_t *p : b->rec_scratch) cudaFree(p);
    }
    delete b;
}

}  // extern "C"
