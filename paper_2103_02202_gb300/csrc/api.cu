// api.cu -- the C ABI declared in include/stimgb.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/stimgb.h"
#include "internal.h"
#include "handle.h"
#include "kernels.h"

using namespace stimgb;

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(e == cudaErrorMemoryAllocation ? STIM_E_OOM : STIM_E_CUDA, msg);
}

#define STIMGB_CK(call, what)                       \
    do {                                            \
        cudaError_t _e = (call);                    \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// Device allocations of the single-circuit paths go through dev_malloc, so a
// test can make the next few fail as if the device were out of memory
// (stim_debug_fail_allocations) and check that every error path leaves the
// handle usable.
std::mutex g_inject_mu;
int g_inject_skip = 0, g_inject_fail = 0;
std::atomic<bool> g_inject_armed{false};

bool injected_failure() {
    if (!g_inject_armed.load()) return false;
    std::lock_guard<std::mutex> g(g_inject_mu);
    if (g_inject_skip > 0) {
        g_inject_skip--;
        return false;
    }
    if (g_inject_fail > 0) {
        g_inject_fail--;
        if (g_inject_fail == 0) g_inject_armed.store(false);
        return true;
    }
    return false;
}

// Tableau grid-barrier settings (stim_debug_tableau_barrier): the limit of
// one wait and, for tests, arrivals the barrier waits for beyond its CTAs.
constexpr uint64_t kBarrierTimeoutNs = 2000000000ull;   // 2 s per wait
std::atomic<uint32_t> g_bar_extra{0};
std::atomic<uint64_t> g_bar_timeout_ns{kBarrierTimeoutNs};

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t st) {
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, st);
}

template <typename T>
int upload(T **dst, const std::vector<T> &src, const char *what) {
    size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
    if (*dst) {         // left by an earlier attempt that failed part way
        cudaFree(*dst);
        *dst = nullptr;
    }
    STIMGB_CK(dev_malloc((void **)dst, bytes), what);
    if (!src.empty()) STIMGB_CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return STIM_OK;
}

// Grow-only device scratch buffer (words of 8 bytes).
int grow(uint64_t **p, size_t *cap, size_t words, const char *what) {
    if (words <= *cap) return STIM_OK;
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
        *cap = 0;
    }
    STIMGB_CK(dev_malloc((void **)p, std::max<size_t>(words, 1) * 8), what);
    *cap = words;
    return STIM_OK;
}

// ---- kernel timing (stim_profile) ----
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec {
    int kernel;
    cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof_pending;
uint64_t g_prof_launches[STIM_KERNEL_COUNT];
double g_prof_ms[STIM_KERNEL_COUNT];

// Records an event pair around one kernel launch when profiling is on.
class ProfScope {
  public:
    ProfScope(int kernel, cudaStream_t st) : kernel_(kernel), st_(st) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_on) return;
        if (cudaEventCreate(&a_) != cudaSuccess) return;
        if (cudaEventCreate(&b_) != cudaSuccess) {
            cudaEventDestroy(a_);
            return;
        }
        active_ = cudaEventRecord(a_, st_) == cudaSuccess;
    }
    ~ProfScope() {
        if (!active_) return;
        std::lock_guard<std::mutex> lk(g_prof_mu);
        cudaEventRecord(b_, st_);
        g_prof_pending.push_back({kernel_, a_, b_});
    }

  private:
    int kernel_;
    cudaStream_t st_;
    cudaEvent_t a_{}, b_{};
    bool active_ = false;
};

void prof_drain_locked() {
    for (ProfRec &r : g_prof_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_prof_launches[r.kernel]++;
            g_prof_ms[r.kernel] += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_prof_pending.clear();
}

}  // namespace



namespace {

int cluster_slot(int C) { return C == 1 ? 0 : C == 2 ? 1 : C == 4 ? 2 : 3; }

// Builds and uploads the frame program for cluster size C (once per handle).
int frame_program(stim_circuit *c, int C, const DevFrameProgram **out) {
    DevFrameProgram &d = c->fprog[cluster_slot(C)];
    if (d.C != C) {
        FrameProgram fp;
        try {
            build_frame_program(c->hp, C, &fp);
        } catch (const std::bad_alloc &) {
            return fail(STIM_E_OOM, "out of host memory building the frame program");
        }
        // deferred noise hits name their op by a 29-bit index within the CTA's layer
        if (fp.max_rank_ops >= (1u << 29))
            return fail(STIM_E_UNSUPPORTED, "a layer holds 2^29 or more ops for one CTA");
        int r;
        // prog | rank_tab | segs, each starting on a 16-byte boundary
        auto pad16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
        const size_t off_rt = pad16(fp.prog.size() * sizeof(ProgEntry));
        const size_t off_sg = off_rt + pad16(fp.rank_tab.size() * sizeof(uint32_t));
        const size_t total = off_sg + pad16(fp.segs.size() * sizeof(FrameSeg));
        if (total >= (1ull << 32)) return fail(STIM_E_UNSUPPORTED, "frame program metadata above 4 GiB");
        std::vector<unsigned char> meta(std::max<size_t>(total, 16), 0);
        if (!fp.prog.empty()) std::memcpy(meta.data(), fp.prog.data(), fp.prog.size() * sizeof(ProgEntry));
        if (!fp.rank_tab.empty())
            std::memcpy(meta.data() + off_rt, fp.rank_tab.data(), fp.rank_tab.size() * sizeof(uint32_t));
        if (!fp.segs.empty()) std::memcpy(meta.data() + off_sg, fp.segs.data(), fp.segs.size() * sizeof(FrameSeg));
        if ((r = upload(&d.meta, meta, "upload frame program")) != STIM_OK) return r;
        d.meta_bytes = (uint32_t)meta.size();
        d.prog = reinterpret_cast<ProgEntry *>(d.meta);
        d.rank_tab = reinterpret_cast<uint32_t *>(d.meta + off_rt);
        d.segs = reinterpret_cast<FrameSeg *>(d.meta + off_sg);
        if ((r = upload(&d.ops, fp.ops, "upload frame program")) != STIM_OK) return r;
        d.Q = fp.Q;
        d.nprog = (uint32_t)fp.prog.size();
        d.max_rank_ops = fp.max_rank_ops;
        d.C = C;
    }
    *out = &d;
    return STIM_OK;
}

int ensure_device(stim_circuit *c) {
    int dev = 0;
    STIMGB_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (c->device >= 0) {
        if (c->device != dev) return fail(STIM_E_INVALID_ARG, "circuit handle was uploaded to another device");
        if (c->fprog[0].C == 1) return STIM_OK;
        const DevFrameProgram *fp1;     // an earlier upload stopped before the single-CTA program
        return frame_program(c, 1, &fp1);
    }
    const HostProgram &hp = c->hp;
    // a failure part way frees what was uploaded, so a later call starts afresh
    auto drop = [&](int r) {
        for (void **p : {(void **)&c->d_prog, (void **)&c->d_ops, (void **)&c->d_geo, (void **)&c->d_det_ptr,
                         (void **)&c->d_det_meas, (void **)&c->d_det_items, (void **)&c->d_det_looks,
                         (void **)&c->d_ref, (void **)&c->d_detflag, (void **)&c->d_status}) {
            cudaFree(*p);
            *p = nullptr;
        }
        return r;
    };
    int r;
    if ((r = upload(&c->d_prog, hp.prog, "upload program")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_ops, hp.ops, "upload ops")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_geo, hp.geo, "upload noise tables")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_det_ptr, hp.det_ptr, "upload detectors")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_det_meas, hp.det_meas, "upload detectors")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_det_items, hp.det_items, "upload detectors")) != STIM_OK) return drop(r);
    if ((r = upload(&c->d_det_looks, hp.det_looks, "upload detectors")) != STIM_OK) return drop(r);
    c->ref_words = std::max<size_t>((hp.num_meas + 63) / 64, 1);
    cudaError_t e = dev_malloc((void **)&c->d_ref, c->ref_words * 8);
    if (e == cudaSuccess) e = dev_malloc((void **)&c->d_detflag, c->ref_words * 8);
    if (e == cudaSuccess) e = dev_malloc((void **)&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_ref, 0, c->ref_words * 8);
    if (e == cudaSuccess) e = cudaMemset(c->d_detflag, 0, c->ref_words * 8);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return drop(cuda_fail(e, "alloc reference"));
    c->device = dev;
    const DevFrameProgram *fp1;
    return frame_program(c, 1, &fp1);     // the single-CTA program is always resident
}

// Reference samples by noiseless skeleton, process-wide: a circuit that
// differs from an earlier one only in its noise channels, detectors or
// observables (a sweep of noise strengths, say) takes the earlier reference
// sample instead of running the tableau again -- the reuse of work across
// slight variations of a circuit that the paper's conclusion (Section 7)
// suggests. Least recently used entries leave first when the byte budget is
// exceeded; a budget of 0 turns the cache off.
struct RefCache {
    struct Entry {
        std::vector<uint32_t> skeleton;
        std::vector<uint64_t> ref, detflag;
        uint64_t last_use = 0;
        size_t bytes() const { return skeleton.size() * 4 + (ref.size() + detflag.size()) * 8 + 64; }
    };
    std::mutex mu;
    std::multimap<uint64_t, Entry> map;     // skeleton hash -> entries
    size_t bytes = 0, cap = (size_t)256 << 20;
    uint64_t clock = 0, hits = 0, misses = 0;

    bool enabled() {
        std::lock_guard<std::mutex> g(mu);
        return cap > 0;
    }
    void evict_to(size_t limit) {          // lock held
        while (bytes > limit && !map.empty()) {
            auto old = map.begin();
            for (auto it = map.begin(); it != map.end(); ++it)
                if (it->second.last_use < old->second.last_use) old = it;
            bytes -= old->second.bytes();
            map.erase(old);
        }
    }
    bool lookup(const HostProgram &hp, size_t words, std::vector<uint64_t> *ref, std::vector<uint64_t> *det) {
        std::lock_guard<std::mutex> g(mu);
        if (cap == 0) return false;
        auto range = map.equal_range(hp.skeleton_hash);
        for (auto it = range.first; it != range.second; ++it)
            if (it->second.ref.size() == words && it->second.skeleton == hp.skeleton) {
                it->second.last_use = ++clock;
                *ref = it->second.ref;
                *det = it->second.detflag;
                hits++;
                return true;
            }
        misses++;
        return false;
    }
    void insert(const HostProgram &hp, std::vector<uint64_t> ref, std::vector<uint64_t> det) {
        std::lock_guard<std::mutex> g(mu);
        if (cap == 0) return;
        auto range = map.equal_range(hp.skeleton_hash);
        for (auto it = range.first; it != range.second; ++it)
            if (it->second.skeleton == hp.skeleton) return;
        Entry e;
        e.skeleton = hp.skeleton;
        e.ref = std::move(ref);
        e.detflag = std::move(det);
        e.last_use = ++clock;
        if (e.bytes() > cap) return;
        bytes += e.bytes();
        map.emplace(hp.skeleton_hash, std::move(e));
        evict_to(cap);
    }
};

RefCache &ref_cache() {
    static RefCache c;
    return c;
}

// Device-resident inverse-tableau states at top-level REPEAT boundaries (the
// cut points of HostProgram). The state there is a function of the noiseless
// skeleton of the source before the cut and of the qubit count alone, so a
// circuit sharing that skeleton prefix resumes its tableau there instead of
// at the identity: memories that differ only in what follows their REPEAT
// block (the final readout, extra rounds of a different kind) recompute only
// that part. An entry holds the tableau columns, signs and permutation, the
// control words, and the reference and determinism words of the measurements
// before the cut. Entries are taken in least-recently-used order under a
// device-memory budget; copies out of an entry are ordered by events that
// eviction waits for.
struct PrefixCache {
    struct Entry {
        std::vector<uint32_t> skeleton;   // skeleton words of the prefix
        uint32_t n = 0;
        uint64_t meas = 0;
        int device = -1;
        char *buf = nullptr;              // state | control words | ref words | detflag words
        size_t state_bytes = 0, ctl_off = 0, ref_off = 0, det_off = 0, words = 0, bytes = 0;
        // stored after a top-level REPEAT block (see HostProgram::CutPoint)
        bool after_loop = false;
        uint64_t loop_hash = 0, loop_reps = 0, reps_pos = 0;
        uint64_t last_use = 0;
        std::vector<cudaEvent_t> reads;   // copies out of buf that may still be in flight
    };
    std::mutex mu;
    std::multimap<uint64_t, Entry> map;   // prefix hash -> entries
    size_t bytes = 0, cap = (size_t)1 << 30;
    uint64_t clock = 0, resumes = 0, saves = 0;

    static void release(Entry &e) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (e.device >= 0 && e.device != cur) cudaSetDevice(e.device);
        for (cudaEvent_t ev : e.reads) {
            cudaEventSynchronize(ev);
            cudaEventDestroy(ev);
        }
        e.reads.clear();
        if (e.buf) cudaFreeAsync(e.buf, nullptr);
        e.buf = nullptr;
        if (e.device >= 0 && e.device != cur) cudaSetDevice(cur);
    }
    void evict_to(size_t limit) {          // lock held
        while (bytes > limit && !map.empty()) {
            auto old = map.begin();
            for (auto it = map.begin(); it != map.end(); ++it)
                if (it->second.last_use < old->second.last_use) old = it;
            bytes -= old->second.bytes;
            release(old->second);
            map.erase(old);
        }
    }
    // Entry for cut k of hp on device, or nullptr (lock held).
    Entry *find(const HostProgram &hp, size_t k, int device) {
        const HostProgram::CutPoint &ct = hp.cuts[k];
        auto range = map.equal_range(ct.prefix_hash);
        for (auto it = range.first; it != range.second; ++it) {
            Entry &e = it->second;
            if (e.device != device || e.n != hp.num_qubits || e.meas != ct.meas ||
                e.skeleton.size() != ct.skeleton_len ||
                !std::equal(e.skeleton.begin(), e.skeleton.end(), hp.skeleton.begin()))
                continue;
            return &e;
        }
        return nullptr;
    }
    // Entry holding the state after the most iterations (fewer than the
    // circuit's own) of the REPEAT block before cut k of hp, with the same
    // body and the same source before it; nullptr if none (lock held).
    Entry *find_in_loop(const HostProgram &hp, size_t k, int device) {
        const HostProgram::CutPoint &ct = hp.cuts[k];
        if (ct.loop_begin == UINT32_MAX) return nullptr;
        const uint64_t meas0 = ct.meas - ct.loop_reps * ct.loop_meas;     // before the block
        Entry *best = nullptr;
        for (auto &kv : map) {
            Entry &e = kv.second;
            if (!e.after_loop || e.loop_hash != ct.loop_hash || e.loop_reps == 0 || e.loop_reps >= ct.loop_reps ||
                e.device != device || e.n != hp.num_qubits || e.reps_pos != ct.reps_pos ||
                e.meas != meas0 + e.loop_reps * ct.loop_meas || e.skeleton.size() != ct.skeleton_len)
                continue;
            bool same = true;
            for (size_t i = 0; i < e.skeleton.size() && same; i++)
                same = i == ct.reps_pos || i == ct.reps_pos + 1 || e.skeleton[i] == hp.skeleton[i];
            if (same && (!best || e.loop_reps > best->loop_reps)) best = &e;
        }
        return best;
    }
};

PrefixCache &prefix_cache() {
    static PrefixCache c;
    return c;
}

// One reference-sample computation in flight: its stream and tableau scratch
// (or the cached sample being copied in).
struct RefJob {
    cudaStream_t st = nullptr;
    char *blob = nullptr;
    bool launched = false;
    bool from_cache = false;
    bool to_cache = false;
    std::vector<uint64_t> ref, detflag;     // host copies (cache hit: source; miss: destination)
    size_t state_bytes = 0;     // tableau columns, signs and permutation at the front of blob
    int resume_cut = -1;        // cut of the circuit the tableau resumed at (a stored prefix state)
    int save_cut = -1;          // cut whose state this computation stores
    char *snap = nullptr;       // that state, until the kernel has succeeded (see PrefixCache)
    size_t snap_ctl = 0, snap_ref = 0, snap_det = 0, snap_words = 0, snap_bytes = 0;
};

// Resumes the tableau of c at the latest cut whose prefix state is stored,
// or part way through the REPEAT block before a cut when a circuit with the
// same source before the block and the same body stored its state after
// fewer iterations: copies the state into the scratch behind a and sets
// a->pc_begin (and a->iter_begin). Leaves a untouched when none is stored.
cudaError_t prefix_resume(stim_circuit *c, RefJob *job, TabArgs *a, cudaStream_t st, bool *resumed) {
    *resumed = false;
    PrefixCache &pc = prefix_cache();
    std::lock_guard<std::mutex> g(pc.mu);
    if (pc.cap == 0) return cudaSuccess;
    const HostProgram &hp = c->hp;
    for (size_t k = hp.cuts.size(); k-- > 0;) {
        const HostProgram::CutPoint &ct = hp.cuts[k];
        // the state at the cut itself, else part way through the block before it
        uint32_t pc_begin = ct.prog_index, iter_begin = 0;
        PrefixCache::Entry *en = ct.prog_index > 0 ? pc.find(hp, k, c->device) : nullptr;
        if (!en && (en = pc.find_in_loop(hp, k, c->device)) != nullptr) {
            pc_begin = ct.loop_begin;
            iter_begin = (uint32_t)en->loop_reps;
        }
        if (!en || en->state_bytes != job->state_bytes) continue;
        cudaError_t e = cudaMemcpyAsync(job->blob, en->buf, en->state_bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(a->ctl, en->buf + en->ctl_off, sizeof(TabCtl), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && en->words)
            e = cudaMemcpyAsync(c->d_ref, en->buf + en->ref_off, en->words * 8, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && en->words)
            e = cudaMemcpyAsync(c->d_detflag, en->buf + en->det_off, en->words * 8, cudaMemcpyDeviceToDevice, st);
        cudaEvent_t ev = nullptr;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ev, st);
        if (ev) {
            for (size_t i = 0; i < en->reads.size();) {
                if (cudaEventQuery(en->reads[i]) == cudaSuccess) {
                    cudaEventDestroy(en->reads[i]);
                    en->reads[i] = en->reads.back();
                    en->reads.pop_back();
                } else {
                    i++;
                }
            }
            en->reads.push_back(ev);
        }
        if (e != cudaSuccess) return e;
        en->last_use = ++pc.clock;
        pc.resumes++;
        a->pc_begin = pc_begin;
        a->iter_begin = iter_begin;
        job->resume_cut = (int)k;
        *resumed = true;
        return cudaSuccess;
    }
    return cudaSuccess;
}

// The cut whose state a computation of c starting at pc_begin stores: the
// last one after pc_begin, unless it is stored already (-1: none).
int prefix_save_choice(const stim_circuit *c, uint32_t pc_begin) {
    const HostProgram &hp = c->hp;
    if (hp.cuts.empty() || hp.cuts.back().prog_index <= pc_begin) return -1;
    PrefixCache &pc = prefix_cache();
    std::lock_guard<std::mutex> g(pc.mu);
    if (pc.cap == 0) return -1;
    const size_t k = hp.cuts.size() - 1;
    return pc.find(hp, k, c->device) ? -1 : (int)k;
}

// Moves the state a successful computation stored (job->snap) into the
// prefix cache, or frees it when an equal one got there first or it exceeds
// the budget.
void prefix_store(stim_circuit *c, RefJob *job) {
    PrefixCache &pc = prefix_cache();
    std::lock_guard<std::mutex> g(pc.mu);
    const HostProgram &hp = c->hp;
    const HostProgram::CutPoint &ct = hp.cuts[(size_t)job->save_cut];
    if (pc.cap == 0 || job->snap_bytes > pc.cap || pc.find(hp, (size_t)job->save_cut, c->device)) {
        cudaFreeAsync(job->snap, job->st);
        job->snap = nullptr;
        return;
    }
    PrefixCache::Entry en;
    en.skeleton.assign(hp.skeleton.begin(), hp.skeleton.begin() + (long)ct.skeleton_len);
    en.n = hp.num_qubits;
    en.meas = ct.meas;
    en.device = c->device;
    en.buf = job->snap;
    en.state_bytes = job->state_bytes;
    en.ctl_off = job->snap_ctl;
    en.ref_off = job->snap_ref;
    en.det_off = job->snap_det;
    en.words = job->snap_words;
    en.bytes = job->snap_bytes;
    en.after_loop = ct.loop_begin != UINT32_MAX;
    en.loop_hash = ct.loop_hash;
    en.loop_reps = ct.loop_reps;
    en.reps_pos = ct.reps_pos;
    en.last_use = ++pc.clock;
    job->snap = nullptr;
    pc.evict_to(pc.cap - en.bytes);
    pc.bytes += en.bytes;
    pc.saves++;
    pc.map.emplace(ct.prefix_hash, std::move(en));
}

// CTAs of the inverse-tableau kernel for c: ~1024 column words per CTA
// (measured best for random circuits; d=100 uses all SMs either way), at most
// the co-resident maximum maxb. alone: the circuit has the GPU to itself (one
// reference computation, not a share of a batched launch); from 128 qubits it
// then takes at least 32 CTAs, which measured faster than the 2-16 the word
// count gives for 150-500 qubits (random Clifford n=250: 0.12 -> 0.05 s;
// n=500: 0.15 -> 0.13 s; surface code d=15: 2.2 -> 2.0 ms), while smaller
// circuits keep the single-CTA kernel without grid barriers.
uint32_t tableau_blocks(const stim_circuit *c, int maxb, bool alone = false) {
    const uint32_t n = c->hp.num_qubits;
    const uint64_t col_words = (uint64_t)2 * n * ((n + 63) / 64);
    uint64_t want = (col_words + 1023) / 1024;
    if (want < 1) want = 1;
    if (alone && n >= 128 && want < 32) want = 32;
    return (uint32_t)std::min<uint64_t>(want, (uint64_t)std::max(maxb, 1));
}

// First half of a reference computation on st: a cached sample of an equal
// skeleton is copied in (job->from_cache), or the tableau scratch is
// allocated, cleared and initialised into *a (*needs_kernel = true). Trivial
// circuits (no qubits or no measurements) need neither.
int reference_prepare(stim_circuit *c, cudaStream_t st, bool use_cache, RefJob *job, TabArgs *a, bool *needs_kernel) {
    const HostProgram &hp = c->hp;
    const uint32_t n = hp.num_qubits;
    *needs_kernel = false;
    job->st = st;
    job->blob = nullptr;
    job->launched = false;
    job->from_cache = false;
    job->to_cache = false;
    job->resume_cut = -1;
    job->save_cut = -1;
    job->snap = nullptr;
    if (n > 0 && hp.num_meas > 0 && use_cache && ref_cache().lookup(hp, c->ref_words, &job->ref, &job->detflag)) {
        STIMGB_CK(cudaMemcpyAsync(c->d_ref, job->ref.data(), c->ref_words * 8, cudaMemcpyHostToDevice, st), "copy reference");
        STIMGB_CK(cudaMemcpyAsync(c->d_detflag, job->detflag.data(), c->ref_words * 8, cudaMemcpyHostToDevice, st),
                  "copy reference");
        job->from_cache = true;
        return STIM_OK;
    }
    job->to_cache = use_cache;
    STIMGB_CK(cudaMemsetAsync(c->d_ref, 0, c->ref_words * 8, st), "memset");
    STIMGB_CK(cudaMemsetAsync(c->d_detflag, 0, c->ref_words * 8, st), "memset");
    if (n == 0 || hp.num_meas == 0) return STIM_OK;
    const uint32_t nw = (n + 63) / 64;
    const size_t col_words = (size_t)2 * n * nw;
    *a = TabArgs{};
    a->prog = c->d_prog;
    a->nprog = (uint32_t)hp.prog.size();
    a->pc_begin = 0;
    a->pc_end = a->nprog;
    a->bclu = 1;
    a->ops = c->d_ops;
    a->n = n;
    a->nw = nw;
    a->ref = c->d_ref;
    a->detflag = c->d_detflag;
    a->status = c->d_status;
    a->bar_extra = g_bar_extra.load();
    a->bar_timeout_ns = g_bar_timeout_ns.load();
    const size_t bytes_tx = col_words * 8, bytes_sign = (size_t)2 * n * 4, bytes_klist = (size_t)n * 4 + 64;
    const size_t bytes_kmask = (size_t)nw * 8 + 64, bytes_rnd = (size_t)std::max<uint32_t>(hp.max_layer_ops, 1) * 4 + 64;
    // Every part starts on a 256-byte boundary; the allocation is the sum of
    // the rounded part sizes, so the last part (the control words, which the
    // memset below must clear) lies wholly inside it.
    auto round256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // row-major copy for bursts of random measurements (circuits of 256 qubits or more)
    const uint32_t nw2 = (2 * n + 63) / 64;
    const bool rows = n >= 256;
    const size_t bytes_rows = rows ? (size_t)n * nw2 * 8 : 0, bytes_rsign = rows ? (size_t)nw2 * 8 : 0;
    const size_t total = 2 * round256(bytes_tx) + 2 * round256(bytes_sign) + round256(bytes_klist) +
                         round256(bytes_kmask) + round256(bytes_rnd) + round256(sizeof(TabCtl)) +
                         (rows ? 2 * round256(bytes_rows) + round256(bytes_rsign) : 0);
    STIMGB_CK(dev_malloc_async((void **)&job->blob, total, st), "alloc tableau");
    size_t off = 0;
    auto take = [&](size_t b) {
        char *p = job->blob + off;
        off += round256(b);
        return p;
    };
    a->tx = (uint64_t *)take(bytes_tx);
    a->tz = (uint64_t *)take(bytes_tx);
    a->sign = (uint32_t *)take(bytes_sign);
    a->perm = (uint32_t *)take(bytes_sign);
    a->klist = (uint32_t *)take(bytes_klist);
    a->kmask = (uint64_t *)take(bytes_kmask);
    a->rnd = (uint32_t *)take(bytes_rnd);
    a->ctl = (TabCtl *)take(sizeof(TabCtl));
    if (rows) {
        a->rx = (uint64_t *)take(bytes_rows);
        a->rz = (uint64_t *)take(bytes_rows);
        a->rsign = (uint64_t *)take(bytes_rsign);
        a->nw2 = nw2;
    }
    if (off != total) {
        cudaFreeAsync(job->blob, st);
        job->blob = nullptr;
        return fail(STIM_E_CUDA, "reference sample: tableau scratch layout mismatch");
    }
    job->state_bytes = 2 * round256(bytes_tx) + 2 * round256(bytes_sign);
    cudaError_t e = cudaMemsetAsync(job->blob, 0, total, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
    // a stored state of the longest shared skeleton prefix, else the identity
    bool resumed = false;
    if (e == cudaSuccess && use_cache) e = prefix_resume(c, job, a, st, &resumed);
    if (e == cudaSuccess && !resumed) e = launch_tableau_init(*a, st);
    if (e == cudaSuccess && use_cache) job->save_cut = prefix_save_choice(c, a->pc_begin);
    if (e != cudaSuccess) {
        cudaFreeAsync(job->blob, st);
        job->blob = nullptr;
        return cuda_fail(e, "reference sample");
    }
    *needs_kernel = true;
    return STIM_OK;
}

// The tableau of c in two launches split at cut job->save_cut, with the
// state at the cut copied into job->snap between them (when the allocation
// fails the computation goes on without storing it).
cudaError_t launch_tableau_saving(stim_circuit *c, RefJob *job, const TabArgs &a, uint32_t blocks, cudaStream_t st) {
    const HostProgram::CutPoint &ct = c->hp.cuts[(size_t)job->save_cut];
    TabArgs head = a;
    head.pc_end = ct.prog_index;
    cudaError_t e = launch_tableau(head, blocks, kTableauThreads, st);
    if (e != cudaSuccess) return e;
    auto round256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t words = (size_t)((ct.meas + 63) / 64);
    job->snap_words = words;
    job->snap_ctl = round256(job->state_bytes);
    job->snap_ref = job->snap_ctl + round256(sizeof(TabCtl));
    job->snap_det = job->snap_ref + round256(words * 8);
    job->snap_bytes = job->snap_det + round256(words * 8);
    if (dev_malloc_async((void **)&job->snap, job->snap_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        job->snap = nullptr;
    } else {
        e = cudaMemcpyAsync(job->snap, job->blob, job->state_bytes, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(job->snap + job->snap_ctl, a.ctl, sizeof(TabCtl), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && words)
            e = cudaMemcpyAsync(job->snap + job->snap_ref, c->d_ref, words * 8, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && words)
            e = cudaMemcpyAsync(job->snap + job->snap_det, c->d_detflag, words * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    if (ct.prog_index >= a.nprog) return cudaSuccess;
    TabArgs tail = a;
    tail.pc_begin = ct.prog_index;
    tail.iter_begin = 0;
    return launch_tableau(tail, blocks, kTableauThreads, st);
}

// Launches the inverse-tableau kernel of c on st with at most max_blocks CTAs
// (0: the library's choice; 1: the single-CTA variant, which keeps the tableau
// in its L1 and needs no grid barrier). Scratch comes from the stream-ordered
// allocator, so launches on several streams do not serialize on allocation.
int reference_launch(stim_circuit *c, cudaStream_t st, uint32_t max_blocks, bool use_cache, RefJob *job) {
    TabArgs a;
    bool needs_kernel = false;
    const int r = reference_prepare(c, st, use_cache, job, &a, &needs_kernel);
    if (r != STIM_OK || !needs_kernel) return r;
    uint32_t blocks = tableau_blocks(c, tableau_max_blocks(kTableauThreads, c->device), max_blocks == 0);
    if (max_blocks && blocks > max_blocks) blocks = max_blocks;
    cudaError_t e;
    {
        ProfScope ps(STIM_KERNEL_TABLEAU, st);
        e = job->save_cut >= 0 ? launch_tableau_saving(c, job, a, blocks, st) : launch_tableau(a, blocks, kTableauThreads, st);
    }
    if (e != cudaSuccess) {
        cudaFreeAsync(job->blob, st);
        job->blob = nullptr;
        if (job->snap) cudaFreeAsync(job->snap, st);
        job->snap = nullptr;
        return cuda_fail(e, "reference sample");
    }
    job->launched = true;
    return STIM_OK;
}

// Waits for a launched job, checks the kernel's status word, frees the scratch
// and marks the reference valid.
int reference_finish(stim_circuit *c, RefJob *job) {
    int status = 0;
    cudaError_t e = cudaSuccess;
    if (job->launched) e = cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, job->st);
    const bool keep = job->launched && job->to_cache && ref_cache().enabled();
    if (keep && e == cudaSuccess) {
        job->ref.resize(c->ref_words);
        job->detflag.resize(c->ref_words);
        e = cudaMemcpyAsync(job->ref.data(), c->d_ref, c->ref_words * 8, cudaMemcpyDeviceToHost, job->st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(job->detflag.data(), c->d_detflag, c->ref_words * 8, cudaMemcpyDeviceToHost, job->st);
    }
    if (job->blob) {
        const cudaError_t f = cudaFreeAsync(job->blob, job->st);
        if (e == cudaSuccess) e = f;
        job->blob = nullptr;
    }
    const cudaError_t s = cudaStreamSynchronize(job->st);
    if (e == cudaSuccess) e = s;
    if (job->snap) {        // the state stored at a cut is kept only from a kernel that succeeded
        if (e == cudaSuccess && status == 0) {
            prefix_store(c, job);
        } else {
            cudaFreeAsync(job->snap, job->st);
            job->snap = nullptr;
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "reference sample");
    if (status == DEV_TIMEOUT) return fail(STIM_E_TIMEOUT, "tableau grid barrier timed out");
    if (status != 0) return fail(STIM_E_CUDA, "tableau kernel reported a malformed program");
    if (keep) ref_cache().insert(c->hp, std::move(job->ref), std::move(job->detflag));
    c->ref_valid = true;
    return STIM_OK;
}

// use_cache: take the sample of an equal noiseless skeleton when one is cached
// (and cache a freshly computed one); false recomputes with the tableau.
int compute_reference(stim_circuit *c, cudaStream_t st, bool use_cache) {
    RefJob job;
    const int r = reference_launch(c, st, 0, use_cache, &job);
    if (r != STIM_OK) return r;
    return reference_finish(c, &job);
}

// Multi-CTA tableaus of several circuits in one cooperative launch on st:
// circuit i gets blocks[i] CTAs (the sum co-resident), meeting only at its
// own barrier. One launch, so no two cooperative grids run side by side.
int reference_batch(const std::vector<stim_circuit *> &cs, const std::vector<uint32_t> &blocks, bool use_cache,
                    cudaStream_t st) {
    std::vector<RefJob> jobs(cs.size());
    std::vector<TabArgs> args;
    std::vector<size_t> which;       // index into cs of each args entry
    std::vector<uint32_t> first, job_of;
    size_t prepared = 0;             // cs[0 .. prepared) went through reference_prepare
    int rc = STIM_OK;
    for (size_t i = 0; i < cs.size() && rc == STIM_OK; i++) {
        TabArgs a;
        bool needs = false;
        rc = reference_prepare(cs[i], st, use_cache, &jobs[i], &a, &needs);
        if (rc != STIM_OK) break;
        prepared = i + 1;
        if (!needs) continue;
        a.nblk = blocks[i];
        first.push_back((uint32_t)job_of.size());
        for (uint32_t b = 0; b < blocks[i]; b++) job_of.push_back((uint32_t)args.size());
        args.push_back(a);
        which.push_back(i);
    }
    char *dev = nullptr;
    if (rc == STIM_OK && !args.empty()) {
        const size_t b_args = args.size() * sizeof(TabArgs), b_first = first.size() * 4, b_of = job_of.size() * 4;
        const size_t o_first = (b_args + 255) & ~(size_t)255, o_of = o_first + ((b_first + 255) & ~(size_t)255);
        cudaError_t e = dev_malloc_async((void **)&dev, o_of + b_of, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dev, args.data(), b_args, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dev + o_first, first.data(), b_first, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dev + o_of, job_of.data(), b_of, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) {
            ProfScope ps(STIM_KERNEL_TABLEAU, st);
            e = launch_tableau_batch(reinterpret_cast<const TabArgs *>(dev), reinterpret_cast<const uint32_t *>(dev + o_of),
                                     reinterpret_cast<const uint32_t *>(dev + o_first), (uint32_t)job_of.size(),
                                     kTableauThreads, st);
        }
        if (e == cudaSuccess)
            for (size_t k : which) jobs[k].launched = true;
        else
            rc = cuda_fail(e, "reference sample (batched tableau)");
    }
    // prepared circuits: the launched ones and those that needed no kernel are
    // finished (and become valid); a tableau that never ran only frees its scratch
    std::vector<bool> needs_kernel(cs.size(), false);
    for (size_t k : which) needs_kernel[k] = true;
    for (size_t i = 0; i < prepared; i++) {
        if (needs_kernel[i] && !jobs[i].launched) {
            if (jobs[i].blob) cudaFreeAsync(jobs[i].blob, st);
            jobs[i].blob = nullptr;
            continue;
        }
        const int r = reference_finish(cs[i], &jobs[i]);
        if (rc == STIM_OK) rc = r;
    }
    if (dev) {
        cudaFreeAsync(dev, st);
        cudaStreamSynchronize(st);
    }
    return rc;
}

// Reference samples of many circuits. Circuits whose tableau wants at most
// kSideBySideBlocks CTAs run the single-CTA tableau (no grid barrier) side by
// side on internal streams; the others share batched cooperative launches
// (reference_batch), each circuit with CTAs in proportion to what it wants,
// the total within the co-resident maximum.
constexpr uint32_t kSideBySideBlocks = 2;
constexpr size_t kReferenceStreams = 32;

int references_many(stim_circuit *const *cs, size_t k, bool recompute) {
    std::vector<stim_circuit *> small, large;
    for (size_t i = 0; i < k; i++) {
        stim_circuit *c = cs[i];
        if (!c) return fail(STIM_E_INVALID_ARG, "stim_reference_many: null circuit");
        const int r = ensure_device(c);
        if (r != STIM_OK) return r;
        if ((c->ref_valid && !recompute) || std::find(small.begin(), small.end(), c) != small.end() ||
            std::find(large.begin(), large.end(), c) != large.end())
            continue;
        const int maxb = tableau_max_blocks(kTableauThreads, c->device);
        (tableau_blocks(c, maxb) <= kSideBySideBlocks ? small : large).push_back(c);
    }
    int rc = STIM_OK;
    if (!small.empty()) {
        std::vector<cudaStream_t> streams(std::min(small.size(), kReferenceStreams), nullptr);
        for (cudaStream_t &st : streams)
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
                st = nullptr;
                rc = fail(STIM_E_CUDA, "stim_reference_many: stream creation failed");
            }
        std::vector<RefJob> jobs(small.size());
        std::vector<bool> started(small.size(), false);
        for (size_t i = 0; i < small.size() && rc == STIM_OK; i++) {
            rc = reference_launch(small[i], streams[i % streams.size()], 1, !recompute, &jobs[i]);
            started[i] = rc == STIM_OK;
        }
        for (size_t i = 0; i < small.size(); i++) {
            if (!started[i]) continue;
            const int r = reference_finish(small[i], &jobs[i]);
            if (rc == STIM_OK) rc = r;
        }
        for (cudaStream_t st : streams)
            if (st) cudaStreamDestroy(st);
        if (rc != STIM_OK) return rc;
    }
    if (large.empty()) return STIM_OK;
    const int maxb = tableau_batch_max_blocks(kTableauThreads, large[0]->device);
    // waves of at most maxb circuits; CTAs in proportion to each circuit's want
    for (size_t w0 = 0; w0 < large.size(); w0 += (size_t)maxb) {
        const size_t w1 = std::min(large.size(), w0 + (size_t)maxb);
        std::vector<stim_circuit *> wave(large.begin() + (long)w0, large.begin() + (long)w1);
        std::vector<uint32_t> want(wave.size());
        uint64_t sum = 0;
        for (size_t i = 0; i < wave.size(); i++) sum += (want[i] = tableau_blocks(wave[i], maxb));
        std::vector<uint32_t> blocks(wave.size());
        uint64_t used = 0;
        for (size_t i = 0; i < wave.size(); i++) {
            blocks[i] = sum <= (uint64_t)maxb ? want[i]
                                              : std::max<uint32_t>(1, (uint32_t)((uint64_t)want[i] * (uint64_t)maxb / sum));
            used += blocks[i];
        }
        // rounding up to one CTA each can exceed maxb by a little: trim the largest
        while (used > (uint64_t)maxb) {
            size_t big = 0;
            for (size_t i = 1; i < wave.size(); i++)
                if (blocks[i] > blocks[big]) big = i;
            if (blocks[big] <= 1) break;
            blocks[big]--;
            used--;
        }
        const int r = reference_batch(wave, blocks, !recompute, nullptr);
        if (r != STIM_OK) return r;
    }
    return STIM_OK;
}

// Tile shape: the smallest cluster whose qubit slice fits shared memory, then
// the widest word tile that keeps at least two CTAs per SM busy; hints override.
int choose_tile(uint32_t n, uint64_t nwords, int sms, size_t smem_optin, const stim_tile_hint *hint,
                TileChoice *out) {
    TileChoice t;
    const uint32_t hW = hint ? hint->words_per_cta : 0, hC = hint ? hint->cluster_size : 0;
    if (hW && hW != 1 && hW != 2 && hW != 4 && hW != 8)
        return fail(STIM_E_INVALID_ARG, "tile hint: words_per_cta must be 1, 2, 4 or 8");
    if (hC && hC != 1 && hC != 2 && hC != 4 && hC != 8)
        return fail(STIM_E_INVALID_ARG, "tile hint: cluster_size must be 1, 2, 4 or 8");
    if (hint && hint->threads && (hint->threads < 32 || hint->threads > 1024 || hint->threads % 32))
        return fail(STIM_E_INVALID_ARG, "tile hint: threads must be a multiple of 32 in [32, 1024]");
    const uint32_t nn = n ? n : 1;
    auto slice = [&](int C) { return (size_t)((nn + C - 1) / C) * 16; };   // bytes per word of a slice
    if (hint && hint->frame_in_global) {
        if (hC > 1) return fail(STIM_E_INVALID_ARG, "tile hint: a global-memory frame uses cluster_size 1");
        t.gmem = true;
        t.C = 1;
    } else if (hC) {
        t.C = (int)hC;
        if (slice(t.C) + kTileHeaderBytes > smem_optin) return fail(STIM_E_INVALID_ARG, "tile hint: slice does not fit shared memory");
    } else {
        // smallest cluster whose slice leaves room for two CTAs per SM
        t.C = 0;
        for (int C : {1, 2, 4, 8})
            if (slice(C) * 2 + 2048 <= smem_optin) {
                t.C = C;
                break;
            }
        if (t.C == 0)
            for (int C : {1, 2, 4, 8})
                if (slice(C) + kTileHeaderBytes <= smem_optin) {
                    t.C = C;
                    break;
                }
        if (t.C == 0) {
            t.C = 1;
            t.gmem = true;
        }
    }
    if (hW) {
        t.W = (int)hW;
        if (!t.gmem && slice(t.C) * t.W + kTileHeaderBytes > smem_optin)
            return fail(STIM_E_INVALID_ARG, "tile hint: words_per_cta does not fit shared memory");
    } else if (t.C == 1 && !t.gmem && n >= 1024 && nwords >= (uint64_t)8 * sms &&
               slice(1) * 8 + kTileHeaderBytes + kMetaCap + 1024 <= smem_optin) {
        // a large circuit whose 8-word tile fits one CTA: threads apply each op
        // to 4 words (independent Philox streams in flight), two per chain
        t.W = 8;
    } else {
        // one 64-shot word per tile: a thread's Philox chains stay independent
        t.W = t.gmem ? 2 : 1;
    }
    if (hint && hint->threads) {
        if ((int)hint->threads > frame_max_threads(t.W))
            return fail(STIM_E_INVALID_ARG, "tile hint: too many threads per CTA for this many words per tile (512 for 1 or 4 or 8, 768 for 2)");
        t.threads = hint->threads;
    } else if (t.gmem) {
        t.threads = 256;
    } else if (t.W >= 4) {
        t.threads = 512;
    } else {
        const size_t per_cta = slice(t.C) * t.W + 1024;
        const size_t per_sm = (size_t)smem_optin + 1024;
        size_t ctas = per_sm / per_cta;
        if (ctas < 1) ctas = 1;
        uint32_t th = (uint32_t)(2048 / ctas);
        if (th > (uint32_t)frame_max_threads(t.W)) th = (uint32_t)frame_max_threads(t.W);
        if (th < 256) th = 256;
        t.threads = th & ~31u;      // whole warps: the kernel's warp collectives name all 32 lanes
    }
    *out = t;
    return STIM_OK;
}

// Frame kernel (records into rec, may be null) and detector kernel (events
// into det, may be null) for one call, with caller-provided buffers. With a
// ring (stimgb_ring_words words), detection events are computed inside the
// frame kernel from the ring of recent flips instead, and rec may be null.
int launch_sampling(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset, const TileChoice &tc,
                    uint64_t *rec, uint64_t *det, uint64_t *gframe, uint64_t *ring, cudaStream_t st) {
    const HostProgram &hp = c->hp;
    const uint32_t n = hp.num_qubits;
    const uint64_t D = hp.num_det;
    const uint64_t nwords = (num_shots + 63) / 64;
    const uint64_t last_mask = (num_shots % 64) ? ((1ull << (num_shots % 64)) - 1) : ~0ull;
    const int W = tc.W, C = tc.C;
    const bool gmem = tc.gmem;
    const uint32_t threads = tc.threads;
    const uint64_t grid = (nwords + W - 1) / W;
    const uint64_t gstride = grid * W;
    int r;
    if (n > 0) {
        const DevFrameProgram *fp = nullptr;
        if ((r = frame_program(c, C, &fp)) != STIM_OK) return r;
        FrameArgs a{};
        a.prog = fp->prog;
        a.nprog = fp->nprog;
        a.rank_tab = fp->rank_tab;
        a.segs = fp->segs;
        a.ops = fp->ops;
        a.geo = c->d_geo;
        a.ref = c->d_ref;
        a.n = n;
        a.Q = fp->Q;
        a.word0 = shot_offset / 64;
        a.nwords = nwords;
        a.last_mask = last_mask;
        a.rec = hp.num_meas ? rec : nullptr;
        a.rec_stride = nwords;
        a.rec_mask = 0xFFFFFFFFu;
        a.gframe = gframe;
        a.gstride = gstride;
        a.status = c->d_status;
        set_seed(a, seed);
        a.meta_bytes = fp->meta_bytes;
        a.meta_region = meta_region_for(fp->meta_bytes);
        if (ring && det && D > 0) {
            a.rec = ring;
            a.rec_mask = (uint32_t)(hp.ring_len - 1);
            a.num_dets = (uint32_t)(D - hp.num_obs);
            a.det = det;
            a.det_stride = nwords;
            a.det_items = c->d_det_items;
            a.det_looks = c->d_det_looks;
            if (hp.num_obs)      // observables accumulate over the whole circuit
                STIMGB_CK(cudaMemsetAsync(det + (D - hp.num_obs) * nwords, 0, hp.num_obs * nwords * 8, st),
                          "clear observables");
        }
        ProfScope ps(STIM_KERNEL_FRAME, st);
        STIMGB_CK(launch_frame(a, W, C, gmem, (uint32_t)grid, threads, tile_smem_bytes(fp->Q, W, gmem, a.meta_region), st),
                  "frame kernel");
    }
    if (det && D > 0 && !(ring && n > 0)) {
        ProfScope ps(STIM_KERNEL_DETECTORS, st);
        STIMGB_CK(launch_detectors(rec, nwords, c->d_det_ptr, c->d_det_meas, c->d_ref, D, nwords, last_mask, det,
                                   nwords, st),
                  "detector kernel");
    }
    return STIM_OK;
}

bool valid_flags(int flags, int allowed) { return (flags & ~allowed) == 0; }

}  // namespace

size_t stimgb_ring_words(const stim_circuit *c, uint64_t num_shots, const TileChoice &tc) {
    const HostProgram &hp = c->hp;
    if (hp.ring_len == 0 || hp.num_det == 0 || hp.num_feedforward > 0 || hp.num_qubits == 0) return 0;
    if (hp.ring_len > (1ull << 31)) return 0;
    if (tc.gmem || (tc.W != 1 && tc.W != 8)) return 0;      // the frame kernel shapes that evaluate DETS entries
    const uint64_t nwords = (num_shots + 63) / 64;
    const uint64_t ring = nwords * hp.ring_len;
    if (ring * 4 > hp.num_meas * nwords) return 0;     // a ring is worth it only when far smaller than the records
    return (size_t)ring;
}

// Used by the batched launch (batch.cu).
int stimgb_frame_program(stim_circuit *c, int C, const DevFrameProgram **out) {
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    return frame_program(c, C, out);
}

int stimgb_sampling_layout(stim_circuit *c, uint64_t num_shots, TileChoice *tc, size_t *gframe_words) {
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    int sms = 0, smem_optin = 0;
    STIMGB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
    STIMGB_CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device), "attr");
    const uint64_t nwords = (num_shots + 63) / 64;
    r = choose_tile(c->hp.num_qubits, nwords, sms, (size_t)smem_optin, nullptr, tc);
    if (r != STIM_OK) return r;
    const uint64_t grid = (nwords + tc->W - 1) / tc->W;
    *gframe_words = tc->gmem ? 2 * (size_t)c->hp.num_qubits * grid * tc->W : 0;
    const DevFrameProgram *fp;
    return frame_program(c, tc->C, &fp);
}

int stimgb_sample_into(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset, const TileChoice &tc,
                       uint64_t *rec, uint64_t *det, uint64_t *gframe, cudaStream_t st) {
    return launch_sampling(c, num_shots, seed, shot_offset, tc, rec, det, gframe, nullptr, st);
}

int stimgb_ensure_references(stim_circuit *const *cs, size_t k) { return references_many(cs, k, false); }

int stimgb_ensure_reference(stim_circuit *c, cudaStream_t st) {
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    if (!c->ref_valid) return compute_reference(c, st, true);
    return STIM_OK;
}

namespace stimgb {
int report_error(int code, const std::string &msg) { return fail(code, msg); }
}  // namespace stimgb

extern "C" {

int stim_last_error(char *buf, size_t len) {
    if (buf && len) {
        size_t k = std::min(len - 1, g_last_error.size());
        memcpy(buf, g_last_error.data(), k);
        buf[k] = 0;
    }
    return (int)g_last_error.size();
}

int stim_compile(const char *text, size_t len, stim_circuit **out) {
    if (!out || (!text && len)) return fail(STIM_E_INVALID_ARG, "stim_compile: null argument");
    *out = nullptr;
    stim_circuit *c = new (std::nothrow) stim_circuit();
    if (!c) return fail(STIM_E_OOM, "stim_compile: out of host memory");
    std::string err;
    int r = compile_circuit(text ? text : "", len, &c->hp, &err);
    if (r != 0) {
        delete c;
        return fail(r, err);
    }
    *out = c;
    return STIM_OK;
}

int stim_info_get(const stim_circuit *c, stim_info *out) {
    if (!c || !out) return fail(STIM_E_INVALID_ARG, "stim_info_get: null argument");
    const HostProgram &hp = c->hp;
    out->num_qubits = hp.num_qubits;
    out->num_measurements = hp.num_meas;
    out->num_detectors = hp.num_det - hp.num_obs;
    out->num_observables = hp.num_obs;
    out->num_gate_targets = hp.num_gate_targets;
    out->num_noise_targets = hp.num_noise_targets;
    out->num_instructions = hp.num_instr;
    out->num_layers = hp.num_layers_exec;
    out->num_program_layers = hp.num_layers_stored;
    out->reference_key = hp.skeleton_hash;
    out->flip_ring_rows = hp.ring_len;
    return STIM_OK;
}

int stim_frame_program_info_get(const stim_circuit *c, int cluster_size, stim_frame_program_info *out) {
    if (!c || !out) return fail(STIM_E_INVALID_ARG, "stim_frame_program_info_get: null argument");
    if (cluster_size != 1 && cluster_size != 2 && cluster_size != 4 && cluster_size != 8)
        return fail(STIM_E_INVALID_ARG, "stim_frame_program_info_get: cluster_size must be 1, 2, 4 or 8");
    FrameProgram fp;
    try {
        build_frame_program(c->hp, cluster_size, &fp);
    } catch (const std::bad_alloc &) {
        return fail(STIM_E_OOM, "out of host memory building the frame program");
    }
    *out = stim_frame_program_info{};
    out->cluster_size = (uint32_t)cluster_size;
    out->qubits_per_cta = fp.Q;
    out->merged_layers = fp.merged_layers_exec;
    for (const ProgEntry &e : fp.prog) out->stored_layers += e.kind == ENT_LAYER;
    out->segments = fp.segs.size();
    out->ops = fp.ops.size();
    out->max_cta_ops = fp.max_rank_ops;
    auto global_q = [&](uint32_t ref) { return (ref >> 24) * fp.Q + (ref & 0xFFFFFFu); };
    for (const FrameSeg &sg : fp.segs) {
        out->chains += sg.count;
        out->max_chain_ops = std::max(out->max_chain_ops, sg.len);
        out->deferred_ops += (uint64_t)sg.count * (sg.len - sg.defer_from);
        for (uint32_t k = 0; k < sg.count; k++) {
            std::vector<uint32_t> qs;
            for (uint32_t j = 0; j < sg.len; j++) {
                const DevOp &op = fp.ops[sg.op_begin + (size_t)j * sg.count + k];      // step-major
                const uint32_t opc = op.a >> 28;
                if ((opc == OP_FFX || opc == OP_FFZ) && j > 0) out->feedforward_not_first++;
                if (j < sg.defer_from) continue;
                qs.push_back(global_q(op.a & 0x0FFFFFFFu));
                if (opc == OP_DEP2) qs.push_back(global_q(op.b));
            }
            std::sort(qs.begin(), qs.end());
            if (std::adjacent_find(qs.begin(), qs.end()) != qs.end()) out->tails_repeating_qubit++;
        }
    }
    return STIM_OK;
}

int stim_debug_fail_allocations(int skip, int count) {
    if (skip < 0 || count < 0) return fail(STIM_E_INVALID_ARG, "stim_debug_fail_allocations: negative argument");
    std::lock_guard<std::mutex> g(g_inject_mu);
    g_inject_skip = skip;
    g_inject_fail = count;
    g_inject_armed.store(count > 0);
    return STIM_OK;
}

int stim_debug_tableau_barrier(uint32_t extra_arrivals, uint64_t timeout_ns) {
    g_bar_extra.store(extra_arrivals);
    g_bar_timeout_ns.store(timeout_ns ? timeout_ns : kBarrierTimeoutNs);
    return STIM_OK;
}

int stim_reference_cache_set(size_t budget_bytes) {
    RefCache &rc = ref_cache();
    std::lock_guard<std::mutex> g(rc.mu);
    rc.cap = budget_bytes;
    rc.evict_to(budget_bytes);
    return STIM_OK;
}

int stim_prefix_cache_set(size_t budget_bytes) {
    PrefixCache &pc = prefix_cache();
    std::lock_guard<std::mutex> g(pc.mu);
    pc.cap = budget_bytes;
    pc.evict_to(budget_bytes);
    return STIM_OK;
}

int stim_prefix_cache_stats(uint64_t *resumes, uint64_t *saves, uint64_t *entries, uint64_t *bytes) {
    PrefixCache &pc = prefix_cache();
    std::lock_guard<std::mutex> g(pc.mu);
    if (resumes) *resumes = pc.resumes;
    if (saves) *saves = pc.saves;
    if (entries) *entries = pc.map.size();
    if (bytes) *bytes = pc.bytes;
    return STIM_OK;
}

int stim_reference_cache_stats(uint64_t *hits, uint64_t *misses, uint64_t *entries, uint64_t *bytes) {
    RefCache &rc = ref_cache();
    std::lock_guard<std::mutex> g(rc.mu);
    if (hits) *hits = rc.hits;
    if (misses) *misses = rc.misses;
    if (entries) *entries = rc.map.size();
    if (bytes) *bytes = rc.bytes;
    return STIM_OK;
}

void stim_free(stim_circuit *c) {
    if (!c) return;
    if (c->device >= 0) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != c->device) cudaSetDevice(c->device);
        cudaDeviceSynchronize();
        cudaFree(c->d_prog);
        cudaFree(c->d_ops);
        cudaFree(c->d_geo);
        cudaFree(c->d_det_ptr);
        cudaFree(c->d_det_meas);
        cudaFree(c->d_det_items);
        cudaFree(c->d_det_looks);
        cudaFree(c->d_ref);
        cudaFree(c->d_detflag);
        cudaFree(c->d_status);
        if (c->kernels_done) cudaEventDestroy(c->kernels_done);
        for (auto &sc : c->scratch) {
            cudaFree(sc.rec);
            cudaFree(sc.det);
            cudaFree(sc.tr);
            cudaFree(sc.gframe);
            cudaFree(sc.hits);
            cudaFree(sc.hits_out);
            cudaFree(sc.ring);
            if (sc.done) cudaEventDestroy(sc.done);
        }
        for (DevFrameProgram &d : c->fprog) {
            cudaFree(d.meta);
            cudaFree(d.ops);
        }
        if (cur >= 0 && cur != c->device) cudaSetDevice(cur);
    }
    delete c;
}

int stim_reference_sample(stim_circuit *c, uint64_t *ref_bits, uint64_t *det_bits, int flags, void *stream) {
    if (!c) return fail(STIM_E_INVALID_ARG, "stim_reference_sample: null handle");
    if (!valid_flags(flags, STIM_HOST | STIM_RECOMPUTE))
        return fail(STIM_E_INVALID_ARG, "stim_reference_sample: unknown flags");
    cudaStream_t st = (cudaStream_t)stream;
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    if (!c->ref_valid || (flags & STIM_RECOMPUTE)) {
        r = compute_reference(c, st, (flags & STIM_RECOMPUTE) == 0);
        if (r != STIM_OK) return r;
    }
    const size_t words = (c->hp.num_meas + 63) / 64;
    const cudaMemcpyKind kind = (flags & STIM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (ref_bits && words) STIMGB_CK(cudaMemcpyAsync(ref_bits, c->d_ref, words * 8, kind, st), "copy reference");
    if (det_bits && words) STIMGB_CK(cudaMemcpyAsync(det_bits, c->d_detflag, words * 8, kind, st), "copy flags");
    if (flags & STIM_HOST) STIMGB_CK(cudaStreamSynchronize(st), "sync");
    return STIM_OK;
}

int stim_reference_many(stim_circuit *const *circuits, size_t k, int flags) {
    if (!circuits && k) return fail(STIM_E_INVALID_ARG, "stim_reference_many: null array");
    if (!valid_flags(flags, STIM_RECOMPUTE)) return fail(STIM_E_INVALID_ARG, "stim_reference_many: unknown flags");
    return references_many(circuits, k, (flags & STIM_RECOMPUTE) != 0);
}

int stim_frame_sample_ex(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset,
                         uint64_t *meas_out, uint64_t *det_out, int flags, const stim_tile_hint *hint,
                         void *stream) {
    if (!c) return fail(STIM_E_INVALID_ARG, "stim_frame_sample: null handle");
    if (!valid_flags(flags, STIM_HOST | STIM_SHOT_MAJOR | STIM_ASYNC | STIM_EVENTS_IN_KERNEL))
        return fail(STIM_E_INVALID_ARG, "stim_frame_sample: unknown flags");
    if (shot_offset % 64) return fail(STIM_E_INVALID_ARG, "stim_frame_sample: shot_offset must be a multiple of 64");
    if ((shot_offset + num_shots + 63) / 64 > (1ull << 32))
        return fail(STIM_E_UNSUPPORTED, "stim_frame_sample: global shot index above 2^38");
    cudaStream_t st = (cudaStream_t)stream;
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    if (!c->ref_valid) {
        r = compute_reference(c, st, true);
        if (r != STIM_OK) return r;
    }
    if (num_shots == 0) return STIM_OK;
    const HostProgram &hp = c->hp;
    const uint32_t n = hp.num_qubits;
    const uint64_t M = hp.num_meas, D = hp.num_det;
    const uint64_t nwords = (num_shots + 63) / 64;
    const bool shot_major = (flags & STIM_SHOT_MAJOR) != 0, host = (flags & STIM_HOST) != 0;

    // ---- tile choice ----
    int sms = 0, smem_optin = 0;
    STIMGB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device), "attr");
    STIMGB_CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device), "attr");
    TileChoice tc;
    r = choose_tile(n, nwords, sms, (size_t)smem_optin, hint, &tc);
    if (r != STIM_OK) return r;
    const int W = tc.W, C = tc.C;
    const bool gmem = tc.gmem;
    const uint64_t grid = (nwords + W - 1) / W;     // word tiles (clusters)
    if (grid * C > 0x7FFFFFFFull) return fail(STIM_E_UNSUPPORTED, "too many shots for one call");

    // ---- staging set (two alternate under STIM_ASYNC) ----
    const bool async = (flags & STIM_ASYNC) != 0;
    stim_circuit::Scratch &sc = c->scratch[async ? (c->next_scratch++ & 1u) : 0u];
    if (!sc.done) STIMGB_CK(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming), "event");
    if (sc.used) STIMGB_CK(cudaStreamWaitEvent(st, sc.done, 0), "wait for staging");
    if (async) {
        if (!c->kernels_done)
            STIMGB_CK(cudaEventCreateWithFlags(&c->kernels_done, cudaEventDisableTiming), "event");
        if (c->kernels_pending) STIMGB_CK(cudaStreamWaitEvent(st, c->kernels_done, 0), "wait for kernels");
    }

    // ---- record buffers ----
    const bool meas_direct = meas_out && !shot_major && !host;
    // detection events alone: computed inside the frame kernel from a ring of
    // recent flips when the circuit allows it, so no record buffer is written
    constexpr uint64_t kRecordBytesForRing = 8ull << 30;     // records above this take the ring by themselves
    const bool want_ring = (flags & STIM_EVENTS_IN_KERNEL) || M * nwords * 8 > kRecordBytesForRing;
    const size_t ring_words = (det_out && !meas_out && D > 0 && want_ring) ? stimgb_ring_words(c, num_shots, tc) : 0;
    // classically controlled ops read the records back inside the frame kernel
    const bool need_rec = (meas_out || (det_out && !ring_words) || hp.num_feedforward > 0) && M > 0;
    uint64_t *rec = nullptr;
    if (need_rec) {
        if (meas_direct) {
            rec = meas_out;
        } else {
            if ((r = grow(&sc.rec, &sc.rec_cap, M * nwords, "alloc records")) != STIM_OK) return r;
            rec = sc.rec;
        }
    }
    uint64_t *gframe = nullptr;
    const uint64_t gstride = grid * W;
    if (gmem && n > 0) {
        if ((r = grow(&sc.gframe, &sc.gframe_cap, 2 * (size_t)n * gstride, "alloc frame")) != STIM_OK) return r;
        gframe = sc.gframe;
    }

    uint64_t *det = nullptr;
    const bool det_direct = det_out && !shot_major && !host;
    if (det_out && D > 0) {
        if (det_direct) {
            det = det_out;
        } else {
            if ((r = grow(&sc.det, &sc.det_cap, D * nwords, "alloc detectors")) != STIM_OK) return r;
            det = sc.det;
        }
    }
    uint64_t *ring = nullptr;
    if (ring_words) {
        if ((r = grow(&sc.ring, &sc.ring_cap, ring_words, "alloc flip ring")) != STIM_OK) return r;
        ring = sc.ring;
    }
    if ((r = launch_sampling(c, num_shots, seed, shot_offset, tc, rec, det, gframe, ring, st)) != STIM_OK) return r;
    if (async) {
        STIMGB_CK(cudaEventRecord(c->kernels_done, st), "record kernels");
        c->kernels_pending = true;
    }

    // ---- output layouts ----
    auto emit = [&](uint64_t *src, uint64_t rows, uint64_t *dst) -> int {
        if (!dst || rows == 0) return STIM_OK;
        if (shot_major) {
            const uint64_t out_stride = (rows + 63) / 64;
            uint64_t *tgt = dst;
            if (host) {
                int rr = grow(&sc.tr, &sc.tr_cap, num_shots * out_stride, "alloc transpose");
                if (rr != STIM_OK) return rr;
                tgt = sc.tr;
            }
            {
                ProfScope ps(STIM_KERNEL_TRANSPOSE, st);
                STIMGB_CK(launch_transpose(src, rows, nwords, num_shots, tgt, out_stride, st), "transpose kernel");
            }
            if (host)
                STIMGB_CK(cudaMemcpyAsync(dst, tgt, num_shots * out_stride * 8, cudaMemcpyDeviceToHost, st), "copy out");
        } else if (host) {
            STIMGB_CK(cudaMemcpyAsync(dst, src, rows * nwords * 8, cudaMemcpyDeviceToHost, st), "copy out");
        }
        return STIM_OK;
    };
    if (meas_out && !meas_direct && (r = emit(rec, M, meas_out)) != STIM_OK) return r;
    if (det_out && !det_direct && (r = emit(det, D, det_out)) != STIM_OK) return r;
    STIMGB_CK(cudaEventRecord(sc.done, st), "record staging");
    sc.used = true;
    if (host && !async) STIMGB_CK(cudaStreamSynchronize(st), "sync");
    return STIM_OK;
}

int stim_frame_sample_detections(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset,
                                 uint64_t *shot_begin, uint32_t *detectors, uint64_t capacity, uint64_t *count,
                                 int flags, void *stream) {
    if (!c || !count) return fail(STIM_E_INVALID_ARG, "stim_frame_sample_detections: null argument");
    if (!valid_flags(flags, STIM_HOST))
        return fail(STIM_E_INVALID_ARG, "stim_frame_sample_detections: unknown flags");
    *count = 0;
    cudaStream_t st = (cudaStream_t)stream;
    int r = ensure_device(c);
    if (r != STIM_OK) return r;
    const bool host = (flags & STIM_HOST) != 0;
    const uint64_t D = c->hp.num_det;
    const uint64_t S = num_shots, nwords = (S + 63) / 64, dw = (D + 63) / 64;
    stim_circuit::Scratch &sc = c->scratch[0];
    if (!sc.done) STIMGB_CK(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming), "event");
    if (sc.used) STIMGB_CK(cudaStreamWaitEvent(st, sc.done, 0), "wait for staging");
    // dense events [D][nwords] -> shot-major rows [S][dw] -> per-shot lists
    if (D > 0 && S > 0 && (r = grow(&sc.det, &sc.det_cap, D * nwords, "alloc detectors")) != STIM_OK) return r;
    if (D > 0 && S > 0 && (r = grow(&sc.tr, &sc.tr_cap, S * dw, "alloc transpose")) != STIM_OK) return r;
    const uint64_t nblocks = (S + 1023) / 1024;
    const size_t w_counts = (S + 1) / 2, w_part = S, w_tot = nblocks + 1;
    const bool begin_here = host || !shot_begin;     // offsets staged in the pool
    if ((r = grow(&sc.hits, &sc.hits_cap, w_counts + w_part + w_tot + (begin_here ? S + 1 : 0) + 1,
                  "alloc event lists")) != STIM_OK)
        return r;
    uint32_t *counts = reinterpret_cast<uint32_t *>(sc.hits);
    uint64_t *part = sc.hits + w_counts, *tot = part + w_part;
    uint64_t *begin = begin_here ? tot + w_tot : shot_begin;
    if (D > 0 && S > 0) {
        r = stim_frame_sample_ex(c, S, seed, shot_offset, nullptr, sc.det, STIM_MEAS_MAJOR | STIM_DEVICE, nullptr,
                                 stream);
        if (r != STIM_OK) return r;
        {
            ProfScope ps(STIM_KERNEL_TRANSPOSE, st);
            STIMGB_CK(launch_transpose(sc.det, D, nwords, S, sc.tr, dw, st), "transpose kernel");
        }
        STIMGB_CK(launch_hits(sc.tr, S, dw, counts, part, tot, begin, st), "event list kernels");
    } else {
        if (shot_offset % 64) return fail(STIM_E_INVALID_ARG, "stim_frame_sample: shot_offset must be a multiple of 64");
        STIMGB_CK(cudaMemsetAsync(begin, 0, (S + 1) * sizeof(uint64_t), st), "event list offsets");
    }
    uint64_t total = 0;
    STIMGB_CK(cudaMemcpyAsync(&total, begin + S, sizeof(uint64_t), cudaMemcpyDeviceToHost, st), "copy count");
    STIMGB_CK(cudaStreamSynchronize(st), "sync");
    *count = total;
    const uint64_t keep = std::min<uint64_t>(total, detectors ? capacity : 0);
    if (detectors && keep > 0) {
        uint32_t *dst = detectors;
        if (host) {      // a separate buffer: growing sc.hits would drop the offsets
            if ((r = grow(&sc.hits_out, &sc.hits_out_cap, (keep + 1) / 2, "alloc event lists")) != STIM_OK) return r;
            dst = reinterpret_cast<uint32_t *>(sc.hits_out);
        }
        STIMGB_CK(launch_hits_write(sc.tr, S, dw, begin, dst, keep, st), "event list kernel");
        if (host) STIMGB_CK(cudaMemcpyAsync(detectors, dst, keep * sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                            "copy events");
    }
    if (host && shot_begin)
        STIMGB_CK(cudaMemcpyAsync(shot_begin, begin, (S + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st),
                  "copy offsets");
    STIMGB_CK(cudaEventRecord(sc.done, st), "record staging");
    sc.used = true;
    if (host) STIMGB_CK(cudaStreamSynchronize(st), "sync");
    if (detectors && total > capacity)
        return fail(STIM_E_CAPACITY, "stim_frame_sample_detections: " + std::to_string(total) +
                                         " events exceed the capacity of " + std::to_string(capacity));
    return STIM_OK;
}

int stim_profile(int enable) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (enable) {
        prof_drain_locked();
        for (int k = 0; k < STIM_KERNEL_COUNT; k++) {
            g_prof_launches[k] = 0;
            g_prof_ms[k] = 0;
        }
    }
    g_prof_on = enable != 0;
    return STIM_OK;
}

int stim_profile_read(stim_kernel_stat *out, int n) {
    if (!out || n < 0) return fail(STIM_E_INVALID_ARG, "stim_profile_read: bad arguments");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    prof_drain_locked();
    for (int k = 0; k < n && k < STIM_KERNEL_COUNT; k++) {
        out[k].launches = g_prof_launches[k];
        out[k].total_ms = g_prof_ms[k];
    }
    return STIM_OK;
}

int stim_frame_sample(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t *meas_out, uint64_t *det_out,
                      int flags, void *stream) {
    return stim_frame_sample_ex(c, num_shots, seed, 0, meas_out, det_out, flags, nullptr, stream);
}

}  // extern "C"
