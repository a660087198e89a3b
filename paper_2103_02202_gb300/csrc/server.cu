// server.cu -- continuous-batching sampling server.
//
// Requests (circuit, shots, seed, outputs) are queued by any thread. One
// dispatcher thread owns a pool of CUDA streams and an arena of device memory
// (the HBM budget, reserved once): whenever a stream slot is free and the
// arena can hold the next queued request's outputs and scratch, that request
// is admitted and its frame and detector kernels are launched on the free
// stream, so requests that arrive while others run start at once and their
// work overlaps on the GPU. Compiled circuits and their reference samples stay
// resident on the device across requests. Completion is observed through a
// CUDA event per request; latency is measured from submission to completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/stimgb.h"
#include "handle.h"

using namespace stimgb;

namespace {

using Clock = std::chrono::steady_clock;

// Best-fit allocator over one device range; 256-byte granules.
class Arena {
  public:
    int init(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        if (cudaMalloc((void **)&base_, bytes) != cudaSuccess) return -1;
        size_ = bytes;
        free_[0] = bytes;
        return 0;
    }
    void release() {
        if (base_) cudaFree(base_);
        base_ = nullptr;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

    // Returns offset or SIZE_MAX.
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        if (bytes == 0) bytes = 256;
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes && (best == free_.end() || it->second < best->second)) best = it;
        if (best == free_.end()) return SIZE_MAX;
        const size_t off = best->first, len = best->second;
        free_.erase(best);
        if (len > bytes) free_[off + bytes] = len - bytes;
        taken_[off] = bytes;
        used_ += bytes;
        peak_ = std::max(peak_, used_);
        return off;
    }
    void free(size_t off) {
        auto t = taken_.find(off);
        if (t == taken_.end()) return;
        size_t len = t->second;
        taken_.erase(t);
        used_ -= len;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += len;
                return;
            }
        }
        free_[off] = len;
    }
    uint64_t *ptr(size_t off) const { return (uint64_t *)(base_ + off); }

  private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
    std::unordered_map<size_t, size_t> taken_;
};

enum ReqState { RQ_QUEUED, RQ_RUNNING, RQ_DONE, RQ_FAILED, RQ_CANCELLED };

struct Request {
    uint64_t id = 0;
    stim_circuit *c = nullptr;
    uint64_t shots = 0, seed = 0, shot_offset = 0;
    int outputs = 0;
    ReqState state = RQ_QUEUED;
    int error = STIM_OK;
    std::string message;
    TileChoice tc;
    bool planned = false;
    size_t meas_words = 0, det_words = 0, rec_words = 0, gframe_words = 0;
    size_t off_meas = SIZE_MAX, off_det = SIZE_MAX, off_rec = SIZE_MAX, off_gframe = SIZE_MAX;
    int slot = -1;
    cudaEvent_t ev = nullptr;
    cudaEvent_t copy_ev = nullptr;      // after the last device copy out of the result buffers
    Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct stim_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int device = 0;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::deque<Request *> queue;
    std::vector<Request *> running;
    std::unordered_map<uint64_t, Request *> reqs;
    uint64_t next_id = 1;
    // statistics of completed requests
    std::vector<double> latencies;
    uint64_t done_count = 0, failed_count = 0, shots_done = 0;
    double gate_shots_done = 0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    cudaStream_t setup_stream = nullptr;
};

namespace {

int sfail(int code, const std::string &msg) { return report_error(code, msg); }

size_t words_of(uint64_t shots) { return (size_t)((shots + 63) / 64); }

void free_scratch(stim_server *s, Request *r) {
    if (r->off_rec != SIZE_MAX) s->arena.free(r->off_rec);
    if (r->off_gframe != SIZE_MAX) s->arena.free(r->off_gframe);
    r->off_rec = r->off_gframe = SIZE_MAX;
}

void free_outputs(stim_server *s, Request *r) {
    if (r->off_meas != SIZE_MAX) s->arena.free(r->off_meas);
    if (r->off_det != SIZE_MAX) s->arena.free(r->off_det);
    r->off_meas = r->off_det = SIZE_MAX;
}

// Plans a request (reference sample, tile shape, buffer sizes). Lock held.
void plan(stim_server *s, Request *r) {
    r->planned = true;
    int rc = stimgb_ensure_reference(r->c, s->setup_stream);
    if (rc == STIM_OK) rc = stimgb_sampling_layout(r->c, r->shots, &r->tc, &r->gframe_words);
    if (rc != STIM_OK) {
        r->error = rc;
        char buf[256];
        stim_last_error(buf, sizeof buf);
        r->message = buf;
        return;
    }
    const HostProgram &hp = r->c->hp;
    const size_t w = words_of(r->shots);
    const bool want_meas = (r->outputs & STIM_OUT_MEAS) != 0, want_det = (r->outputs & STIM_OUT_DET) != 0;
    r->meas_words = want_meas ? hp.num_meas * w : 0;
    r->det_words = want_det ? hp.num_det * w : 0;
    r->rec_words = (!want_meas && ((want_det && hp.num_det) || hp.num_feedforward)) ? hp.num_meas * w : 0;
    const size_t total = 8 * (r->meas_words + r->det_words + r->rec_words + r->gframe_words) + 4 * 256;
    if (total > s->arena.size()) {
        r->error = STIM_E_UNSUPPORTED;
        r->message = "request needs more device memory than the server's budget";
    }
}

bool reserve(stim_server *s, Request *r) {
    size_t got[4] = {SIZE_MAX, SIZE_MAX, SIZE_MAX, SIZE_MAX};
    const size_t need[4] = {r->meas_words, r->det_words, r->rec_words, r->gframe_words};
    for (int k = 0; k < 4; k++) {
        if (!need[k]) continue;
        got[k] = s->arena.alloc(need[k] * 8);
        if (got[k] == SIZE_MAX) {
            for (int j = 0; j < k; j++)
                if (got[j] != SIZE_MAX) s->arena.free(got[j]);
            return false;
        }
    }
    r->off_meas = got[0];
    r->off_det = got[1];
    r->off_rec = got[2];
    r->off_gframe = got[3];
    return true;
}

void finish(stim_server *s, Request *r, ReqState st) {
    r->state = st;
    r->t_done = Clock::now();
    if (st == RQ_DONE) {
        s->done_count++;
        s->shots_done += r->shots;
        s->gate_shots_done += (double)r->c->hp.num_gate_targets * (double)r->shots;
        s->latencies.push_back(std::chrono::duration<double>(r->t_done - r->t_submit).count());
        s->t_last = r->t_done;
    } else if (st == RQ_FAILED) {
        s->failed_count++;
        free_outputs(s, r);
    }
    free_scratch(s, r);
}

void dispatcher(stim_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // completions
        for (size_t i = 0; i < s->running.size();) {
            Request *r = s->running[i];
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) {
                i++;
                continue;
            }
            if (q != cudaSuccess) {
                r->error = STIM_E_CUDA;
                r->message = cudaGetErrorString(q);
            }
            s->slot_busy[r->slot] = false;
            finish(s, r, q == cudaSuccess ? RQ_DONE : RQ_FAILED);
            s->running[i] = s->running.back();
            s->running.pop_back();
            s->cv_done.notify_all();
        }
        // admissions, in arrival order, while a stream slot and memory are free
        while (!s->queue.empty()) {
            int slot = -1;
            for (size_t k = 0; k < s->slot_busy.size(); k++)
                if (!s->slot_busy[k]) {
                    slot = (int)k;
                    break;
                }
            if (slot < 0) break;
            Request *r = s->queue.front();
            if (!r->planned) plan(s, r);
            if (r->error != STIM_OK) {
                s->queue.pop_front();
                finish(s, r, RQ_FAILED);
                s->cv_done.notify_all();
                continue;
            }
            if (!reserve(s, r)) break;      // wait for memory to free up
            s->queue.pop_front();
            cudaStream_t st = s->streams[slot];
            uint64_t *meas = r->off_meas != SIZE_MAX ? s->arena.ptr(r->off_meas) : nullptr;
            uint64_t *det = r->off_det != SIZE_MAX ? s->arena.ptr(r->off_det) : nullptr;
            uint64_t *rec = meas ? meas : (r->off_rec != SIZE_MAX ? s->arena.ptr(r->off_rec) : nullptr);
            uint64_t *gframe = r->off_gframe != SIZE_MAX ? s->arena.ptr(r->off_gframe) : nullptr;
            r->t_start = Clock::now();
            int rc = stimgb_sample_into(r->c, r->shots, r->seed, r->shot_offset, r->tc, rec, det, gframe, st);
            if (rc == STIM_OK && !r->ev && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
                rc = STIM_E_CUDA;
            if (rc == STIM_OK && cudaEventRecord(r->ev, st) != cudaSuccess) rc = STIM_E_CUDA;
            if (rc != STIM_OK) {
                r->error = rc;
                char buf[256];
                stim_last_error(buf, sizeof buf);
                r->message = buf;
                finish(s, r, RQ_FAILED);
                s->cv_done.notify_all();
                continue;
            }
            r->state = RQ_RUNNING;
            r->slot = slot;
            s->slot_busy[slot] = true;
            s->running.push_back(r);
        }
        if (s->stop && s->queue.empty() && s->running.empty()) break;
        if (s->running.empty() && s->queue.empty()) {
            s->cv_work.wait(lk);
        } else {
            // poll running requests' events; new submissions wake us early
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

int fill_result(stim_server *s, Request *r, stim_result *out) {
    memset(out, 0, sizeof(*out));
    out->status = r->state == RQ_DONE ? STIM_OK : r->error != STIM_OK ? r->error : STIM_E_BUSY;
    out->num_shots = r->shots;
    out->words_per_row = words_of(r->shots);
    out->meas = r->off_meas != SIZE_MAX ? s->arena.ptr(r->off_meas) : nullptr;
    out->det = r->off_det != SIZE_MAX ? s->arena.ptr(r->off_det) : nullptr;
    out->queue_s = r->state >= RQ_RUNNING && r->state != RQ_CANCELLED
                       ? std::chrono::duration<double>(r->t_start - r->t_submit).count() : 0;
    out->latency_s = (r->state == RQ_DONE || r->state == RQ_FAILED)
                         ? std::chrono::duration<double>(r->t_done - r->t_submit).count() : 0;
    return out->status;
}

}  // namespace

extern "C" {

int stim_server_create(size_t hbm_budget_bytes, int streams, stim_server **out) {
    if (!out || streams < 0 || streams > 64) return sfail(STIM_E_INVALID_ARG, "stim_server_create: bad arguments");
    *out = nullptr;
    stim_server *s = new (std::nothrow) stim_server();
    if (!s) return sfail(STIM_E_OOM, "stim_server_create: out of host memory");
    cudaGetDevice(&s->device);
    if (s->arena.init(hbm_budget_bytes) != 0) {
        delete s;
        return sfail(STIM_E_OOM, "stim_server_create: cannot reserve the HBM budget");
    }
    const int n = streams ? streams : 8;
    for (int i = 0; i < n; i++) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            s->arena.release();
            delete s;
            return sfail(STIM_E_CUDA, "stim_server_create: stream creation failed");
        }
        s->streams.push_back(st);
    }
    cudaStreamCreateWithFlags(&s->setup_stream, cudaStreamNonBlocking);
    s->slot_busy.assign(s->streams.size(), false);
    s->worker = std::thread(dispatcher, s);
    *out = s;
    return STIM_OK;
}

int stim_server_submit(stim_server *s, stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset,
                       int outputs, stim_request_id *id) {
    if (!s || !c || !id) return sfail(STIM_E_INVALID_ARG, "stim_server_submit: null argument");
    if (shot_offset % 64) return sfail(STIM_E_INVALID_ARG, "stim_server_submit: shot_offset must be a multiple of 64");
    if (outputs & ~(STIM_OUT_MEAS | STIM_OUT_DET)) return sfail(STIM_E_INVALID_ARG, "stim_server_submit: bad outputs");
    if (num_shots == 0) return sfail(STIM_E_INVALID_ARG, "stim_server_submit: zero shots");
    Request *r = new (std::nothrow) Request();
    if (!r) return sfail(STIM_E_OOM, "stim_server_submit: out of host memory");
    r->c = c;
    r->shots = num_shots;
    r->seed = seed;
    r->shot_offset = shot_offset;
    r->outputs = outputs;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return sfail(STIM_E_BUSY, "stim_server_submit: server is shutting down");
        }
        r->id = s->next_id++;
        if (!s->have_first) {
            s->have_first = true;
            s->t_first = r->t_submit;
        }
        s->reqs[r->id] = r;
        s->queue.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_one();
    return STIM_OK;
}

int stim_server_poll(stim_server *s, stim_request_id id, stim_result *out) {
    if (!s || !out) return sfail(STIM_E_INVALID_ARG, "stim_server_poll: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(STIM_E_INVALID_ARG, "stim_server_poll: unknown request");
    return fill_result(s, it->second, out);
}

int stim_server_wait(stim_server *s, stim_request_id id, uint64_t timeout_ns, stim_result *out) {
    if (!s || !out) return sfail(STIM_E_INVALID_ARG, "stim_server_wait: null argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(STIM_E_INVALID_ARG, "stim_server_wait: unknown request");
    Request *r = it->second;
    const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns);
    while (r->state == RQ_QUEUED || r->state == RQ_RUNNING) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            (r->state == RQ_QUEUED || r->state == RQ_RUNNING)) {
            fill_result(s, r, out);
            return sfail(STIM_E_TIMEOUT, "stim_server_wait: request not finished within the timeout");
        }
    }
    return fill_result(s, r, out);
}

int stim_server_cancel(stim_server *s, stim_request_id id) {
    if (!s) return sfail(STIM_E_INVALID_ARG, "stim_server_cancel: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(STIM_E_INVALID_ARG, "stim_server_cancel: unknown request");
    Request *r = it->second;
    if (r->state != RQ_QUEUED) return sfail(STIM_E_BUSY, "stim_server_cancel: request already started");
    s->queue.erase(std::find(s->queue.begin(), s->queue.end(), r));
    r->state = RQ_CANCELLED;
    r->error = STIM_E_BUSY;
    r->t_done = Clock::now();
    s->cv_done.notify_all();
    return STIM_OK;
}

int stim_server_release(stim_server *s, stim_request_id id) {
    if (!s) return sfail(STIM_E_INVALID_ARG, "stim_server_release: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return sfail(STIM_E_INVALID_ARG, "stim_server_release: unknown request");
    Request *r = it->second;
    if (r->state == RQ_QUEUED || r->state == RQ_RUNNING)
        return sfail(STIM_E_BUSY, "stim_server_release: request still in progress");
    // an asynchronous device copy out of the result buffers may still be in
    // flight on the caller's stream: the buffers return to the arena (and to
    // the next request's kernels) only once it is done
    if (r->copy_ev) {
        cudaEventSynchronize(r->copy_ev);
        cudaEventDestroy(r->copy_ev);
        r->copy_ev = nullptr;
    }
    free_outputs(s, r);
    if (r->ev) cudaEventDestroy(r->ev);
    s->reqs.erase(it);
    delete r;
    s->cv_work.notify_one();    // memory freed: queued requests may now fit
    return STIM_OK;
}

int stim_server_copy_result(stim_server *s, stim_request_id id, uint64_t *meas_dst, uint64_t *det_dst, int flags,
                            void *stream) {
    if (!s) return sfail(STIM_E_INVALID_ARG, "stim_server_copy_result: null server");
    if (flags & ~STIM_HOST) return sfail(STIM_E_INVALID_ARG, "stim_server_copy_result: bad flags");
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t *meas = nullptr, *det = nullptr;
    size_t mb = 0, db = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) return sfail(STIM_E_INVALID_ARG, "stim_server_copy_result: unknown request");
        Request *r = it->second;
        if (r->state != RQ_DONE) return sfail(STIM_E_BUSY, "stim_server_copy_result: request not finished");
        if (r->off_meas != SIZE_MAX) meas = s->arena.ptr(r->off_meas);
        if (r->off_det != SIZE_MAX) det = s->arena.ptr(r->off_det);
        mb = r->meas_words * 8;
        db = r->det_words * 8;
    }
    const cudaMemcpyKind kind = (flags & STIM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (meas_dst && meas && mb && cudaMemcpyAsync(meas_dst, meas, mb, kind, st) != cudaSuccess)
        return sfail(STIM_E_CUDA, "stim_server_copy_result: copy failed");
    if (det_dst && det && db && cudaMemcpyAsync(det_dst, det, db, kind, st) != cudaSuccess)
        return sfail(STIM_E_CUDA, "stim_server_copy_result: copy failed");
    if ((flags & STIM_HOST) && cudaStreamSynchronize(st) != cudaSuccess)
        return sfail(STIM_E_CUDA, "stim_server_copy_result: sync failed");
    if (!(flags & STIM_HOST)) {
        // remember where the copy ends, so that stim_server_release waits for it
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(id);
        if (it != s->reqs.end()) {
            Request *r = it->second;
            if (!r->copy_ev && cudaEventCreateWithFlags(&r->copy_ev, cudaEventDisableTiming) != cudaSuccess)
                return sfail(STIM_E_CUDA, "stim_server_copy_result: event creation failed");
            if (cudaEventRecord(r->copy_ev, st) != cudaSuccess)
                return sfail(STIM_E_CUDA, "stim_server_copy_result: event record failed");
        }
    }
    return STIM_OK;
}

int stim_server_stats(stim_server *s, stim_server_statistics *out) {
    if (!s || !out) return sfail(STIM_E_INVALID_ARG, "stim_server_stats: null argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->completed = s->done_count;
    out->failed = s->failed_count;
    out->queued = s->queue.size();
    out->running = s->running.size();
    out->shots = s->shots_done;
    out->gate_shots = s->gate_shots_done;
    out->budget_bytes = s->arena.size();
    out->bytes_in_use = s->arena.used();
    out->peak_bytes_in_use = s->arena.peak();
    if (!s->latencies.empty()) {
        std::vector<double> l = s->latencies;
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[(size_t)std::min<double>(l.size() - 1, f * (l.size() - 1) + 0.5)]; };
        out->p50_latency_s = q(0.50);
        out->p99_latency_s = q(0.99);
        out->max_latency_s = l.back();
    }
    if (s->have_first && s->done_count)
        out->wall_s = std::chrono::duration<double>(s->t_last - s->t_first).count();
    return STIM_OK;
}

void stim_server_destroy(stim_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : s->reqs) {
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        if (kv.second->copy_ev) cudaEventDestroy(kv.second->copy_ev);
        delete kv.second;
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    if (s->setup_stream) cudaStreamDestroy(s->setup_stream);
    s->arena.release();
    delete s;
}

}  // extern "C"
