// kernels.h -- argument blocks and launchers of the CUDA kernels (host view).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace stimgb {

struct FrameArgs {
    const ProgEntry *prog;     // FrameProgram::prog (LAYER.op_begin indexes rank_tab)
    uint32_t nprog;
    const uint32_t *rank_tab;  // per merged layer: C + 1 segment offsets
    const FrameSeg *segs;      // FrameProgram::segs
    const DevOp *ops;          // FrameProgram::ops (qubit references)
    const uint64_t *geo;       // [tables][kNoiseTableWords] noise tables
    const uint64_t *ref;       // packed reference sample (ceil(M/64) words)
    uint32_t n;                // qubits
    uint32_t Q;                // qubits per CTA slice
    uint64_t word0;            // global 64-shot word of this call's word 0
    uint64_t nwords;           // words written by this call
    uint64_t last_mask;        // valid bits of the last word
    uint64_t *rec;             // measurement-major records [M][rec_stride], or null
    uint64_t rec_stride;
    uint64_t *gframe;          // global frame [2][n][gstride] when the tile is not in smem
    uint64_t gstride;
    int *status;
    uint64_t seed;             // Philox key = (seed lo, seed hi)
    uint32_t rk[20];           // its round keys: rk[2r] = lo + r 0x9E3779B9, rk[2r + 1] = hi + r 0xBB67AE85 (set_seed)
    uint32_t meta_bytes;       // bytes of prog + rank_tab + segs (one buffer starting at prog)
    uint32_t meta_region;      // shared bytes reserved for them; copied there when meta_bytes fits
    // Detection events inside the frame kernel (det null: DETS entries are
    // skipped and the detector kernel reads the records instead). With det
    // set, rec holds each measurement's flip (x before the collapse; the
    // record xor the reference) in a ring of the rec_mask + 1 most recent
    // measurements, row m & rec_mask; a DETS entry XORs its detectors' ring
    // words into det rows [num_dets][det_stride] (observables XOR into rows
    // num_dets + k, cleared before the launch). rec_mask is all ones otherwise.
    uint32_t rec_mask;
    uint32_t num_dets;         // DETECTOR rows (observables follow)
    uint64_t *det;
    uint64_t det_stride;
    const DetItem *det_items;
    const uint32_t *det_looks;
};

// Sets a.seed and the round keys derived from it.
inline void set_seed(FrameArgs &a, uint64_t seed) {
    a.seed = seed;
    for (uint32_t r = 0; r < 10; r++) {
        a.rk[2 * r] = (uint32_t)seed + r * 0x9E3779B9u;
        a.rk[2 * r + 1] = (uint32_t)(seed >> 32) + r * 0xBB67AE85u;
    }
}

// Dynamic shared memory of a frame tile: a header (round keys, then 32
// queues of 32 deferred noise hits, one per warp), the program metadata
// (meta_region bytes), then (shared layout) the frame rows of Q qubits x 2W
// words.
constexpr uint32_t kHitQueueOffset = 256;
constexpr uint32_t kHitQueueCap = 32;          // entries per warp
constexpr uint32_t kTileHeaderBytes = kHitQueueOffset + 32 * kHitQueueCap * 4;

// Largest CTA of a frame kernel with W words per tile: threads that apply ops
// to two or four words at once need more registers. One-word tiles are sized
// for two CTAs of up to 512 threads per SM (64 registers, no spills).
constexpr int frame_max_threads(int W) { return W >= 4 ? 512 : W == 2 ? 768 : 512; }
// The batched kernel keeps per-circuit state besides: its one-word tiles stay
// at 448 threads (72 registers).
constexpr int batch_max_threads(int W) { return W == 1 ? 448 : frame_max_threads(W); }
constexpr int frame_min_ctas(int W) { return W == 1 ? 2 : 1; }
inline size_t tile_smem_bytes(uint32_t Q, int W, bool gmem, uint32_t meta_region) {
    return kTileHeaderBytes + meta_region + (gmem ? 0 : (size_t)Q * 2 * W * 8);
}

// Program metadata up to this size is read from shared memory.
constexpr uint32_t kMetaCap = 16384;
inline uint32_t meta_region_for(uint32_t meta_bytes) { return meta_bytes <= kMetaCap ? meta_bytes : 0u; }

// tiles = word tiles (clusters); the grid has tiles * C CTAs.
cudaError_t launch_frame(const FrameArgs &a, int W, int C, bool gmem, uint32_t tiles, uint32_t threads, size_t smem,
                         cudaStream_t stream);

struct TabCtl {
    unsigned bar_count;
    unsigned bar_gen;
    int abort;
    uint32_t next_j;
    uint32_t has_random;
    uint32_t pivot;
    uint32_t nk;
    uint32_t pivot_is_y;
    uint32_t fix_x;
    uint32_t use_mask;
    uint32_t nk_sum, nk_cnt;   // CNOT targets of the random measurements resolved so far (burst choice)
};

struct TabArgs {
    const ProgEntry *prog;
    uint32_t nprog;
    const DevOp *ops;
    uint32_t n, nw;            // qubits, words per column plane
    uint64_t *tx, *tz;         // [2n][nw] physical columns
    uint32_t *sign;            // [2n] physical
    uint32_t *perm;            // [2n] logical column -> physical column
    uint64_t *ref;             // packed outcomes (zeroed before launch)
    uint64_t *detflag;         // packed deterministic flags (zeroed before launch)
    uint32_t *klist;           // [n] scratch: CNOT targets of the current random measurement
    uint64_t *kmask;           // [nw] scratch: the same targets as a mask
    uint32_t *rnd;             // [max collapse ops per layer] scratch: random flags
    TabCtl *ctl;               // zeroed before launch
    int *status;
    uint32_t nblk;             // CTAs working on this circuit (set by the launchers)
    // Row-major copy for bursts of random measurements (null: bursts off):
    // rx/rz[row k][nw2 words], bit c = the x/z bit of physical column c at
    // start-of-time qubit k; rsign[nw2] the column signs. nw2 = ceil(2n / 64).
    uint64_t *rx, *rz, *rsign;
    uint32_t nw2;
    // program entries [pc_begin, pc_end) are walked (a top-level stretch: the
    // tableau of an earlier prefix may be resumed, or saved part way); with
    // iter_begin > 0, pc_begin is a top-level LOOP_BEGIN entered at that
    // iteration (the state of the earlier iterations resumed)
    uint32_t pc_begin, pc_end, iter_begin;
    // CTAs that walk a row-major burst together: the first bclu CTAs, one
    // thread-block cluster (1: CTA 0 alone, no cluster launch)
    uint32_t bclu;
    uint32_t bar_extra;        // test knob: arrivals a barrier waits for beyond nblk (0 in normal use)
    uint64_t bar_timeout_ns;   // limit of one barrier wait
};

constexpr uint32_t kTableauThreads = 512;     // threads per CTA of the tableau kernel

cudaError_t launch_tableau_init(const TabArgs &a, cudaStream_t stream);
// Cooperative launch; blocks * threads must be co-resident.
cudaError_t launch_tableau(const TabArgs &a, uint32_t blocks, uint32_t threads, cudaStream_t stream);
int tableau_max_blocks(uint32_t threads, int device);
// One cooperative launch for several circuits: jobs[j] (device array, nblk set)
// gets CTAs first[j] .. first[j] + jobs[j].nblk - 1; job_of[b] names CTA b's
// circuit. blocks (the sum) must be co-resident: tableau_batch_max_blocks.
cudaError_t launch_tableau_batch(const TabArgs *jobs, const uint32_t *job_of, const uint32_t *first, uint32_t blocks,
                                 uint32_t threads, cudaStream_t stream);
int tableau_batch_max_blocks(uint32_t threads, int device);

// det[k][w] = XOR over m in D_k of rec[m][w] ^ ref(m), padding bits cleared.
cudaError_t launch_detectors(const uint64_t *rec, uint64_t rec_stride, const uint64_t *det_ptr,
                             const uint32_t *det_meas, const uint64_t *ref, uint64_t ndet, uint64_t nwords,
                             uint64_t last_mask, uint64_t *det, uint64_t det_stride, cudaStream_t stream);

// Bit transpose: in has `rows` rows of in_stride words (bit s of a row = column s);
// out gets `cols` rows of out_stride = ceil(rows/64) words.
cudaError_t launch_transpose(const uint64_t *in, uint64_t rows, uint64_t in_stride, uint64_t cols,
                             uint64_t *out, uint64_t out_stride, cudaStream_t stream);

// Per-row lists of set bits (CSR): begin[0] = 0, begin[r + 1] = begin[r] +
// popcount(row r), for nrows rows of `stride` words. Scratch: counts[nrows],
// part[nrows], tot[ceil(nrows / 1024)]. launch_hits_write then stores the bit
// indices of row r at out[begin[r] ...] in ascending order, skipping entries at
// or beyond capacity.
cudaError_t launch_hits(const uint64_t *rows, uint64_t nrows, uint64_t stride, uint32_t *counts, uint64_t *part,
                        uint64_t *tot, uint64_t *begin, cudaStream_t stream);
cudaError_t launch_hits_write(const uint64_t *rows, uint64_t nrows, uint64_t stride, const uint64_t *begin,
                              uint32_t *out, uint64_t capacity, cudaStream_t stream);

}  // namespace stimgb
