// handle.h -- the library-owned circuit handle (host view).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "kernels.h"

// Device copy of a FrameProgram for one cluster size.
struct DevFrameProgram {
    int C = 0;                          // 0: not built
    uint32_t Q = 0;
    uint32_t nprog = 0;
    uint32_t max_rank_ops = 0;
    // prog, rank_tab and segs live in one allocation (meta, meta_bytes, a
    // multiple of 16) that kernels copy into shared memory when it is small
    unsigned char *meta = nullptr;
    uint32_t meta_bytes = 0;
    stimgb::ProgEntry *prog = nullptr;
    uint32_t *rank_tab = nullptr;
    stimgb::FrameSeg *segs = nullptr;
    stimgb::DevOp *ops = nullptr;
};

struct stim_circuit {
    stimgb::HostProgram hp;
    int device = -1;
    stimgb::ProgEntry *d_prog = nullptr;
    stimgb::DevOp *d_ops = nullptr;
    uint64_t *d_geo = nullptr;
    uint64_t *d_det_ptr = nullptr;
    uint32_t *d_det_meas = nullptr;
    stimgb::DetItem *d_det_items = nullptr;    // DETS entries' detectors (see HostProgram)
    uint32_t *d_det_looks = nullptr;
    uint64_t *d_ref = nullptr;
    uint64_t *d_detflag = nullptr;
    int *d_status = nullptr;
    bool ref_valid = false;
    size_t ref_words = 1;
    // Device staging of stim_frame_sample_ex (records, detection events,
    // transposes, spilled frames). Calls with STIM_ASYNC alternate between the
    // two sets so one call's copies overlap the next call's kernels; every
    // call waits on the GPU for the previous user of its set (done event).
    struct Scratch {
        uint64_t *rec = nullptr;
        size_t rec_cap = 0;
        uint64_t *det = nullptr;
        size_t det_cap = 0;
        uint64_t *tr = nullptr;
        size_t tr_cap = 0;
        uint64_t *gframe = nullptr;
        size_t gframe_cap = 0;
        uint64_t *hits = nullptr;         // per-shot event lists: counts, scans, offsets
        size_t hits_cap = 0;
        uint64_t *hits_out = nullptr;     // per-shot event lists: host-bound detector indices
        size_t hits_out_cap = 0;
        uint64_t *ring = nullptr;         // recent measurement flips (detection events in the frame kernel)
        size_t ring_cap = 0;
        cudaEvent_t done = nullptr;
        bool used = false;
    } scratch[2];
    unsigned next_scratch = 0;
    // Asynchronous calls run their kernels in call order, even on different
    // streams: each waits for the previous asynchronous call's kernels (not
    // its copies), so kernels never share the GPU with each other while the
    // copies of earlier calls overlap them.
    cudaEvent_t kernels_done = nullptr;
    bool kernels_pending = false;
    DevFrameProgram fprog[4];           // cluster sizes 1, 2, 4, 8
};

// Frame-kernel launch shape.
struct TileChoice {
    int W = 1, C = 1;
    bool gmem = false;
    uint32_t threads = 256;
};


// Library-internal entry points shared by the batched and serving paths.
int stimgb_frame_program(stim_circuit *c, int C, const DevFrameProgram **out);
int stimgb_ensure_reference(stim_circuit *c, cudaStream_t st);
// Reference samples of k circuits: small ones side by side (single-CTA
// tableaus on internal streams), the others one at a time; blocks until done.
int stimgb_ensure_references(stim_circuit *const *cs, size_t k);
// Tile shape for num_shots shots and the global-frame scratch it needs (words).
int stimgb_sampling_layout(stim_circuit *c, uint64_t num_shots, TileChoice *tc, size_t *gframe_words);
// Frame and detector launches into caller-provided buffers (rec: M rows of
// ceil(num_shots/64) words, required when det is given; any may be null).
int stimgb_sample_into(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset, const TileChoice &tc,
                       uint64_t *rec, uint64_t *det, uint64_t *gframe, cudaStream_t st);
// Words of the flip ring for detection events computed inside the frame
// kernel, or 0 when that path does not apply (no detectors, classically
// controlled ops, or a ring no smaller than a quarter of the records).
size_t stimgb_ring_words(const stim_circuit *c, uint64_t num_shots, const TileChoice &tc);
