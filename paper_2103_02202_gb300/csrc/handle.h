// handle.h -- the library-owned circuit handle (host view).
#pragma once

#include <cstddef>
#include <cstdint>

#include "internal.h"

// Device copy of a FrameProgram for one cluster size.
struct DevFrameProgram {
    int C = 0;                          // 0: not built
    uint32_t Q = 0;
    uint32_t nprog = 0;
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
    uint64_t *d_ref = nullptr;
    uint64_t *d_detflag = nullptr;
    int *d_status = nullptr;
    bool ref_valid = false;
    size_t ref_words = 1;
    uint64_t *d_rec = nullptr;
    size_t rec_cap = 0;
    uint64_t *d_det = nullptr;
    size_t det_cap = 0;
    uint64_t *d_tr = nullptr;
    size_t tr_cap = 0;
    uint64_t *d_gframe = nullptr;
    size_t gframe_cap = 0;
    DevFrameProgram fprog[4];           // cluster sizes 1, 2, 4, 8
};
