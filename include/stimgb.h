/*
 * stimgb.h -- C ABI of the GB300 bulk stabilizer-circuit sampler.
 *
 * The library implements the bulk-sampling path of Gidney, "Stim: a fast
 * stabilizer circuit simulator" (Quantum 2021): a circuit is compiled once,
 * one noiseless reference sample is taken with the inverse-tableau simulator
 * (Section 4), and then many shots are sampled by propagating bit-packed
 * Pauli frames through the circuit (Section 3) and XORing them against the
 * reference; detection events are XORs of measurement flips (Section 5.6).
 *
 * Conventions shared by every call:
 *   - Every function returns an int status: STIM_OK (0) or a negative
 *     STIM_E_* code. stim_last_error() gives a per-thread message for the
 *     last failure on the calling thread.
 *   - The library owns circuit handles; the caller owns every output buffer
 *     and must size it as documented.
 *   - Bit-packed arrays are little-endian within uint64 words: bit j of a row
 *     is bit (j % 64) of word (j / 64) (the LSB-first order of the paper's
 *     b8 output format, Section 5.6). Padding bits past the row's end are 0.
 *   - A flags word says whether output pointers are host or device memory and
 *     which layout they use. Device pointers must be memory of the current
 *     CUDA device. Host pointers may be pageable or pinned.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls
 *     with device outputs are asynchronous on `stream`; calls with host
 *     outputs return after the data has landed in host memory.
 *   - Calls on one handle are not thread-safe; distinct handles may be used
 *     from distinct threads.
 *   - Results depend only on (circuit text, seed, global shot index); they do
 *     not depend on layout, tile shape, batch split, shot offset or any other
 *     work running on the GPU.
 */
#ifndef STIMGB_H
#define STIMGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define STIM_OK              0
#define STIM_E_PARSE        (-1)  /* circuit text rejected (message has line) */
#define STIM_E_INVALID_ARG  (-2)  /* NULL handle, bad flags, size out of range */
#define STIM_E_OOM          (-3)  /* host or device allocation failed */
#define STIM_E_CUDA         (-4)  /* a CUDA runtime call failed */
#define STIM_E_TIMEOUT      (-5)  /* a bounded device wait ran out */
#define STIM_E_BUSY         (-6)  /* resource in use (server admission) */
#define STIM_E_UNSUPPORTED  (-7)  /* circuit exceeds a documented limit */
#define STIM_E_CAPACITY     (-8)  /* output capacity too small (the needed size is reported) */

/* ---- flags --------------------------------------------------------------- */
#define STIM_MEAS_MAJOR   0x0  /* row r = measurement/detector r; bit s = shot s */
#define STIM_SHOT_MAJOR   0x1  /* row s = shot s; bit r = measurement/detector r */
#define STIM_DEVICE       0x0  /* output pointers are device memory */
#define STIM_HOST         0x2  /* output pointers are host memory */
#define STIM_RECOMPUTE    0x4  /* stim_reference_sample, stim_reference_many: run the tableau
                                  again (ignore the handle's sample and the reference cache) */
#define STIM_ASYNC        0x8  /* stim_frame_sample(_ex): return once the work and the host
                                  copies are enqueued on the stream; see stim_frame_sample_ex */
#define STIM_EVENTS_IN_KERNEL 0x10 /* stim_frame_sample(_ex) with detection events only: compute
                                  them inside the frame kernel from a ring of the most recent
                                  measurement flips (stim_info.flip_ring_rows rows) instead of
                                  writing the measurement records and running the detector
                                  kernel; see stim_frame_sample_ex */

typedef struct stim_circuit stim_circuit;

typedef struct {
    uint32_t num_qubits;         /* max qubit target + 1 */
    uint64_t num_measurements;   /* M: targets of M, MR, MX, MY, MRX, MRY, in order */
    uint64_t num_detectors;      /* D: DETECTOR instructions, in order; detection-event
                                    outputs hold D + K rows: the detectors, then the
                                    K logical observables */
    uint64_t num_gate_targets;   /* one-qubit gate, measurement and reset targets plus CX/CZ pairs */
    uint64_t num_noise_targets;  /* X/Y/Z_ERROR, DEPOLARIZE1 targets plus DEPOLARIZE2 pairs */
    uint64_t num_instructions;   /* instruction lines after REPEAT flattening */
    uint64_t num_layers;         /* fused layers executed per shot (loops unrolled) */
    uint64_t num_program_layers; /* fused layers stored (loop bodies once) */
    uint64_t num_observables;    /* K: largest OBSERVABLE_INCLUDE index + 1 (0 without any) */
    uint64_t reference_key;      /* hash of the noiseless skeleton: circuits that differ only in
                                    noise channels, DETECTORs and OBSERVABLE_INCLUDEs share it
                                    (and their reference sample) */
    uint64_t flip_ring_rows;     /* R: rows of the ring of recent measurement flips from which
                                    the frame kernel computes detection events when only those
                                    are asked for (used when 4 R <= M and the circuit has no
                                    classically controlled ops); 0 without DETECTOR or
                                    OBSERVABLE_INCLUDE */
} stim_info;

/* Tile choice for the frame kernel; zero fields mean "let the library pick". */
typedef struct {
    uint32_t words_per_cta;    /* 64-shot words per tile: 1, 2, 4 or 8 */
    uint32_t threads;          /* threads per CTA: 32..1024, multiple of 32 */
    uint32_t frame_in_global;  /* 1: keep frames in global memory even if the tile fits shared memory */
    uint32_t cluster_size;     /* CTAs of a cluster splitting a tile's qubits: 1, 2, 4 or 8 */
} stim_tile_hint;

/*
 * stim_compile -- parse and compile circuit text (Section 5.8 line format).
 *
 * Gate set: H, S, S_DAG, X, Y, Z, SQRT_X, SQRT_X_DAG, SQRT_Y, SQRT_Y_DAG,
 * CX (alias CNOT), CZ; M, MR, R and their X- and Y-basis forms MX, MY, MRX,
 * MRY, RX, RY (random outcomes of the reference sample are the +1
 * eigenvalue); X_ERROR(p), Y_ERROR(p), Z_ERROR(p), DEPOLARIZE1(p),
 * DEPOLARIZE2(p), PAULI_CHANNEL_1(px, py, pz), PAULI_CHANNEL_2(p_IX, p_IY,
 * p_IZ, p_XI, ..., p_ZZ) (probabilities in [0, 1] summing to at most 1; the
 * first letter acts on the first target of a pair); DETECTOR rec[-k]... (optional parenthesised coordinates on
 * DETECTOR are ignored), REPEAT N { ... }, '#' comments. Broadcast targets
 * run left to right (pairs for two-qubit gates). A pair of CX may name a
 * measurement record rec[-k] as its control, a pair of CZ on either side:
 * the other target gets X (CX) or Z (CZ) in the shots whose record is 1,
 * the classically controlled Paulis a Pauli frame tracks in place of the
 * qubits (Section 3, "Tracking Corrections"). Sampling a circuit that has
 * them keeps its measurement records in device memory even when only
 * detection events are asked for. OBSERVABLE_INCLUDE(k) rec[-a]... adds the
 * records to logical observable k (0 <= k < 65536; several instructions with
 * one index accumulate): its output bit is the XOR of the flips of all the
 * records it includes, i.e. whether the shot's noise flipped the logical
 * observable, and observables follow the D detectors as rows D..D+K-1 of every
 * detection-event output (K = largest index + 1).
 *
 * text/len: the circuit (need not be NUL-terminated). *out receives a new
 * handle on success; the caller frees it with stim_free(). Compilation is
 * host-only; device memory is allocated on the current device at the first
 * sampling call. Errors: STIM_E_PARSE (unknown gate, bad target, odd target
 * count or repeated qubit pair on a two-qubit gate, p outside [0, 1], wrong
 * argument count, rec[-k] before the first measurement or k = 0, a record
 * as CX target or on both sides of a pair, unbalanced or zero REPEAT), STIM_E_UNSUPPORTED (more than 2^24 qubits, 2^28
 * flattened instructions or 2^32 measurements), STIM_E_INVALID_ARG,
 * STIM_E_OOM.
 */
int stim_compile(const char *text, size_t len, stim_circuit **out);

/* Counts of a compiled circuit. */
int stim_info_get(const stim_circuit *c, stim_info *out);

/* Shape of the frame-kernel program of a circuit for a cluster of
 * cluster_size CTAs (1, 2, 4 or 8), as the frame sampler builds it: fused
 * layers folded into merged layers of per-thread op chains, grouped into
 * segments of equal op signature (host-only, no GPU). */
typedef struct {
    uint32_t cluster_size;
    uint32_t qubits_per_cta;       /* Q = ceil(num_qubits / cluster_size) */
    uint64_t merged_layers;        /* merged layers executed per shot (loops unrolled) */
    uint64_t stored_layers;        /* merged layers stored (loop bodies once) */
    uint64_t segments, chains, ops;
    uint32_t max_chain_ops;        /* longest chain (ops one thread runs between barriers) */
    uint32_t max_cta_ops;          /* largest op range of one CTA in one merged layer */
    uint64_t deferred_ops;         /* trailing noise ops applied after their chain */
    uint64_t tails_repeating_qubit;/* chains whose deferred tail names a qubit twice
                                      (always 0 when cluster_size > 1) */
    uint64_t feedforward_not_first;/* classically controlled ops that are not the first op
                                      of their chain (always 0) */
} stim_frame_program_info;

/* Errors: STIM_E_INVALID_ARG (NULL argument, cluster_size not 1, 2, 4 or 8), STIM_E_OOM. */
int stim_frame_program_info_get(const stim_circuit *c, int cluster_size, stim_frame_program_info *out);

/* Frees the handle and its device memory (synchronizes the device first). */
void stim_free(stim_circuit *c);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len). Returns the message length. */
int stim_last_error(char *buf, size_t len);

/*
 * stim_reference_sample -- one noiseless sample from the inverse-tableau
 * simulator (Section 4, "Tracking the Tableau"), computed on the GPU.
 *
 * Gates are folded by prepending their inverse; a measurement reads the
 * Z_q column; a random measurement is resolved by appending CNOTs from a
 * pivot, a single-qubit collapse and, because the paper leaves the coin
 * open, always takes outcome 0 (an X is appended when the sign is -).
 * A reset is a measurement followed by forcing the sign to +.
 *
 * ref_bits: ceil(M/64) words; bit m = outcome of measurement m.
 * det_bits: optional (may be NULL), ceil(M/64) words; bit m = 1 when
 *   measurement m was deterministic given the earlier outcomes.
 * flags: STIM_HOST or STIM_DEVICE for both pointers, optionally
 *   STIM_RECOMPUTE to bypass the sample cached on the handle (used to time
 *   the time-to-first-sample).
 * The sample is cached on the handle and reused by stim_frame_sample.
 * Errors: STIM_E_INVALID_ARG, STIM_E_OOM, STIM_E_CUDA, STIM_E_TIMEOUT.
 */
int stim_reference_sample(stim_circuit *c, uint64_t *ref_bits, uint64_t *det_bits,
                          int flags, void *stream);

/*
 * stim_reference_many -- computes (and keeps on their handles) the reference
 * samples of k circuits at once, as stim_reference_sample would one by one.
 * Circuits whose inverse tableau (Section 4) wants at most two CTAs (up to
 * about 250 qubits) run the single-CTA tableau side by side on internal
 * streams; larger ones follow one at a time with the multi-CTA tableau.
 * Handles whose reference is already computed (or cached, see below) are
 * skipped unless flags is STIM_RECOMPUTE; a handle may appear more than once.
 * Blocks until every reference is done.
 * Errors: STIM_E_INVALID_ARG (null array or element, unknown flags),
 * STIM_E_OOM, STIM_E_CUDA, STIM_E_TIMEOUT; references finished before the
 * error stay valid.
 */
int stim_reference_many(stim_circuit *const *circuits, size_t k, int flags);

/*
 * Reference-sample cache. Reference samples are kept process-wide, keyed by
 * the circuit's noiseless skeleton (its gates, collapsing and classically
 * controlled operations with their targets and REPEAT structure, in source
 * order; noise channels, DETECTORs and OBSERVABLE_INCLUDEs do not change the
 * reference sample): a circuit compiled after another one with the same
 * skeleton -- the same experiment at another noise strength -- copies the
 * cached sample instead of running the tableau, reusing work across slight
 * variations of a circuit as the paper's conclusion (Section 7) suggests.
 * STIM_RECOMPUTE bypasses it. Entries are compared in full, not by hash.
 *
 * stim_reference_cache_set: byte budget (default 256 MiB); least recently
 *   used entries are dropped to fit; 0 turns the cache off and empties it.
 * stim_reference_cache_stats: lookups that hit and missed, entries and bytes
 *   held; any pointer may be NULL.
 * Both are thread-safe and need no GPU.
 */
int stim_reference_cache_set(size_t budget_bytes);
int stim_reference_cache_stats(uint64_t *hits, uint64_t *misses, uint64_t *entries, uint64_t *bytes);

/*
 * Tableau prefix states. A circuit with top-level REPEAT blocks has a cut
 * point before and after each; the inverse tableau there (Section 3's state,
 * with the reference bits of the measurements before it) depends only on the
 * noiseless skeleton of the source before the cut and on the qubit count. A
 * reference computation that misses the reference-sample cache and finds a
 * stored state for one of its cuts -- same qubit count, same skeleton prefix,
 * compared in full -- resumes there (the latest such cut) instead of at the
 * identity; a computation that reaches its last cut with no state stored for
 * it stores one (the tableau then runs as two launches with a device copy
 * between them). Memories that differ only after their REPEAT block, e.g. in
 * the final readout, then recompute only that part. States live in device
 * memory: 2n columns of ceil(n/64) words for each of the X and Z planes plus
 * signs, permutation and the reference words before the cut (about 200 MB at
 * 20,000 qubits). STIM_RECOMPUTE neither reads nor stores them.
 *
 * stim_prefix_cache_set: device-byte budget (default 1 GiB); least recently
 *   used states are freed to fit (after the copies out of them finish); 0
 *   turns storing and resuming off and frees every state.
 * stim_prefix_cache_stats: computations resumed from a stored state, states
 *   stored, states and device bytes held; any pointer may be NULL.
 * Both are thread-safe; they touch the GPU only to free evicted states.
 */
int stim_prefix_cache_set(size_t budget_bytes);
int stim_prefix_cache_stats(uint64_t *resumes, uint64_t *saves, uint64_t *entries, uint64_t *bytes);

/*
 * stim_debug_fail_allocations -- fault injection for tests: of the device
 * allocations the single-circuit paths make next (upload of a compiled
 * circuit, staging buffers of stim_frame_sample_ex, tableau scratch of the
 * reference sample), the first `skip` succeed and the following `count` fail
 * as if the device were out of memory, so the calls that make them return
 * STIM_E_OOM. A failed call leaves its handle usable; a later call allocates
 * afresh. count = 0 turns injection off. Process-wide, thread-safe; no GPU
 * needed to set it.
 * Errors: STIM_E_INVALID_ARG (a negative argument).
 */
int stim_debug_fail_allocations(int skip, int count);

/*
 * stim_debug_tableau_barrier -- failure-detection knob for tests (no
 * counterpart in the paper). The reference-sample kernel separates its
 * phases with a software grid barrier whose waits are bounded: a wait that
 * lasts longer than timeout_ns (0 = the default, 2 s) gives up, every CTA of
 * the tableau leaves the kernel, and stim_reference_sample returns
 * STIM_E_TIMEOUT with the handle still usable. extra_arrivals > 0 makes
 * every barrier of multi-CTA tableaus launched afterwards wait for that many
 * arrivals beyond its CTAs, which never come, so the wait runs out; 0
 * restores normal operation. Single-CTA tableaus use the CTA barrier and are
 * not affected. Applies to tableau launches prepared after the call;
 * process-wide.
 * Errors: none.
 */
int stim_debug_tableau_barrier(uint32_t extra_arrivals, uint64_t timeout_ns);

/*
 * stim_frame_sample -- bulk Pauli-frame sampling (Section 3): num_shots shots
 * with global shot indices 0..num_shots-1 under `seed`.
 *
 * meas_out: may be NULL. MEAS_MAJOR: M rows of ceil(num_shots/64) words.
 *   SHOT_MAJOR: num_shots rows of ceil(M/64) words.
 * det_out: may be NULL. Detection events (XOR of the flips of a detector's
 *   measurements, Section 5.6), then the K observable flips: with R = D + K,
 *   MEAS_MAJOR: R rows of ceil(num_shots/64) words. SHOT_MAJOR: num_shots
 *   rows of ceil(R/64) words.
 * The reference sample is computed first if the handle has none.
 * Errors: STIM_E_INVALID_ARG, STIM_E_OOM, STIM_E_CUDA, STIM_E_TIMEOUT.
 */
int stim_frame_sample(stim_circuit *c, uint64_t num_shots, uint64_t seed,
                      uint64_t *meas_out, uint64_t *det_out, int flags, void *stream);

/*
 * stim_frame_sample_ex -- as stim_frame_sample for global shot indices
 * shot_offset .. shot_offset+num_shots-1. shot_offset must be a multiple of
 * 64 (it selects 64-shot RNG words); the outputs hold the num_shots shots
 * starting at row/bit 0. hint may be NULL.
 *
 * Host outputs (STIM_HOST) are staged in device memory owned by the handle and
 * copied out on `stream`. Without STIM_ASYNC the call returns after the copy.
 * With STIM_ASYNC it returns once the kernels and copies are enqueued: the
 * host buffers must stay valid and unread until `stream` is synchronized.
 * Asynchronous calls alternate between two staging sets and run their
 * kernels in call order (each waits on the GPU for the previous asynchronous
 * call's kernels), so on two streams the copies of one call overlap the
 * kernels of the next; a call that reuses a set waits on the GPU for that
 * set's previous copies.
 * Calls on one handle must still come from one host thread at a time.
 *
 * Detection events without records (Section 5.6): when only
 * det_out is given and either STIM_EVENTS_IN_KERNEL is set or the records
 * would take more than 8 GiB, and the circuit has no classically controlled
 * ops and 4 x stim_info.flip_ring_rows <= M, the frame kernel keeps each
 * measurement's flip in a ring of flip_ring_rows rows and evaluates the
 * detectors and observables of each straight-line stretch itself: no record
 * buffer (ring: flip_ring_rows x ceil(num_shots/64) words instead of M x
 * ceil(num_shots/64)) and no detector kernel; the same bits either way.
 * With one 64-shot word per tile (the default for circuits that need thread-
 * block clusters) the ring reads are 8-byte loads from L2 on the kernel's
 * critical path, so that form is slower than the record path (the d=100
 * surface code: about 32 ms against 25 ms per 16384 shots); its gain is memory.
 */
int stim_frame_sample_ex(stim_circuit *c, uint64_t num_shots, uint64_t seed,
                         uint64_t shot_offset, uint64_t *meas_out, uint64_t *det_out,
                         int flags, const stim_tile_hint *hint, void *stream);

/*
 * stim_frame_sample_detections -- detection events of shots shot_offset ..
 * shot_offset+num_shots-1 (as stim_frame_sample_ex) as per-shot lists of the
 * fired detectors, the "hits" form of the paper's output formats (Section
 * 5.6): detectors[shot_begin[s] .. shot_begin[s+1]) are the indices of the
 * detectors that fired in shot s (0-based within the call), ascending; a
 * flipped logical observable k appears as index D + k.
 *
 * shot_begin: num_shots + 1 offsets (uint64), may be NULL.
 * detectors: uint32 detector indices, room for `capacity` entries; may be NULL
 *   (then only the count and offsets are produced).
 * count: host pointer, receives the total number of events.
 * flags: STIM_HOST (both outputs are host memory) or STIM_DEVICE. The call
 *   synchronizes `stream` (the count decides the copy size).
 * Errors: as stim_frame_sample_ex; STIM_E_CAPACITY when the events do not fit
 *   `capacity` (*count holds the number needed; the first `capacity` entries
 *   and all offsets are written).
 */
int stim_frame_sample_detections(stim_circuit *c, uint64_t num_shots, uint64_t seed, uint64_t shot_offset,
                                 uint64_t *shot_begin, uint32_t *detectors, uint64_t capacity, uint64_t *count,
                                 int flags, void *stream);

/*
 * Batched sampling: many compiled circuits in one persistent launch.
 *
 * stim_batch_create plans the work of k circuits sampling num_shots[i] shots
 * each: every circuit gets its reference sample (computed if missing) and its
 * frame program; the (circuit, 64-shot-word tile) work items are ordered most
 * expensive circuit first; one persistent kernel (clusters of CTAs when a
 * circuit's qubits need them) pulls items from an atomic counter, followed
 * by one batched detector kernel. hint may fix words_per_cta / threads /
 * cluster_size; otherwise the first stim_batch_sample times candidate tile
 * shapes on a prefix of the work list and keeps the fastest (remembered per
 * batch shape for the process, and in the file named by the environment
 * variable STIMGB_TUNE_CACHE if set). Errors: STIM_E_INVALID_ARG,
 * STIM_E_UNSUPPORTED (a circuit too wide even for 8-CTA clusters), STIM_E_OOM,
 * STIM_E_CUDA, STIM_E_TIMEOUT.
 *
 * stim_batch_sample runs the plan on `stream`: circuit i samples its
 * num_shots[i] shots with global shot indices shot_offsets[i] + 0.. (offsets
 * may be NULL = all 0; multiples of 64) under seeds[i]. meas_out[i] and
 * det_out[i] are device memory in MEAS_MAJOR layout (M or D + K rows of
 * ceil(num_shots[i]/64) words); either array or entry may be NULL. Results
 * equal stim_frame_sample_ex bit for bit. The work is captured in a CUDA
 * graph on the first call for a given set of non-NULL outputs and replayed
 * afterwards; a call waits for the plan's previous launch before reusing its
 * pinned descriptor buffer.
 */
typedef struct stim_batch stim_batch;

int stim_batch_create(stim_circuit *const *circuits, const uint64_t *num_shots, size_t k,
                      const stim_tile_hint *hint, void *stream, stim_batch **out);
int stim_batch_sample(stim_batch *b, const uint64_t *seeds, const uint64_t *shot_offsets,
                      uint64_t *const *meas_out, uint64_t *const *det_out, void *stream);
/* Tile shape chosen for the plan and its size (any pointer may be NULL). */
int stim_batch_info(const stim_batch *b, uint32_t *words_per_tile, uint32_t *threads,
                    uint32_t *cluster_size, uint32_t *ctas, uint64_t *work_items);
void stim_batch_free(stim_batch *b);

/*
 * Sampling server: continuous batching under an HBM budget.
 *
 * stim_server_create reserves hbm_budget_bytes of device memory on the
 * current device (the arena all request buffers come from) and starts one
 * dispatcher thread with `streams` CUDA streams (0 = 8). Requests queue in
 * arrival order; whenever a stream is free and the arena can hold the next
 * request's outputs and scratch, that request is admitted and launched, so
 * requests that arrive while others run start at once and overlap on the GPU.
 * Circuits stay compiled and their reference samples resident across
 * requests (a circuit without a reference sample gets one when its first
 * request is admitted; call stim_reference_sample beforehand to keep that out
 * of request latency). The caller keeps circuit handles alive until their
 * requests are released and must not sample them directly meanwhile.
 *
 * stim_server_submit: num_shots shots with global indices shot_offset + 0..
 *   (shot_offset a multiple of 64) under seed; outputs = STIM_OUT_MEAS and/or
 *   STIM_OUT_DET. Results are bit-identical to stim_frame_sample_ex.
 * stim_server_poll: STIM_OK when done, STIM_E_BUSY while queued or running,
 *   the request's error code if it failed; fills *out.
 * stim_server_wait: blocks up to timeout_ns; STIM_E_TIMEOUT if still running.
 * Result buffers (device, MEAS_MAJOR, words_per_row words per row) live in
 * the arena until stim_server_release(id); releasing frees them for queued
 * requests. stim_server_cancel removes a request that has not started.
 * stim_server_stats reports completed requests, latency percentiles (from
 * submission to completion) and arena use. stim_server_destroy finishes the
 * queued work, then frees everything.
 */
#define STIM_OUT_MEAS 0x1
#define STIM_OUT_DET  0x2

typedef struct stim_server stim_server;
typedef uint64_t stim_request_id;

typedef struct {
    int status;               /* STIM_OK, STIM_E_BUSY (not finished) or the failure code */
    uint64_t num_shots;
    uint64_t words_per_row;   /* ceil(num_shots / 64) */
    uint64_t *meas;           /* M rows, device memory (NULL if not requested) */
    uint64_t *det;            /* D + K rows, device memory (NULL if not requested) */
    double queue_s;           /* submission to admission */
    double latency_s;         /* submission to completion */
} stim_result;

typedef struct {
    uint64_t completed, failed, queued, running;
    uint64_t shots;           /* shots of completed requests */
    double gate_shots;        /* shots x gate targets of completed requests */
    size_t budget_bytes, bytes_in_use, peak_bytes_in_use;
    double p50_latency_s, p99_latency_s, max_latency_s;
    double wall_s;            /* first submission to last completion */
} stim_server_statistics;

int stim_server_create(size_t hbm_budget_bytes, int streams, stim_server **out);
int stim_server_submit(stim_server *s, stim_circuit *c, uint64_t num_shots, uint64_t seed,
                       uint64_t shot_offset, int outputs, stim_request_id *id);
int stim_server_poll(stim_server *s, stim_request_id id, stim_result *out);
int stim_server_wait(stim_server *s, stim_request_id id, uint64_t timeout_ns, stim_result *out);
int stim_server_cancel(stim_server *s, stim_request_id id);
int stim_server_release(stim_server *s, stim_request_id id);
/* Copies a finished request's outputs into caller buffers (either may be
 * NULL): flags STIM_HOST or STIM_DEVICE; MEAS_MAJOR layout. Host copies return
 * when done; device copies are asynchronous on `stream`, and a later
 * stim_server_release of the request waits for them before its buffers go
 * back to the arena. */
int stim_server_copy_result(stim_server *s, stim_request_id id, uint64_t *meas_dst, uint64_t *det_dst,
                            int flags, void *stream);
int stim_server_stats(stim_server *s, stim_server_statistics *out);
void stim_server_destroy(stim_server *s);

/*
 * stim_frame_sample_noalloc -- detection events without allocating device
 * memory. The paper has no counterpart; this is an interface addition.
 *
 * Who needs it: callers that cannot call cudaMalloc when they sample, because
 * all device memory has been handed to another allocator (a framework's
 * caching allocator, a service that reserves its memory up front), or
 * because they cannot afford the device-wide synchronization that freeing
 * device memory implies. stim_frame_sample_ex allocates a record buffer for
 * detection-event output; this call instead keeps the measurement records in
 * a fixed array of STIM_NOALLOC_SCRATCH_BYTES (32 MiB) compiled into the
 * library. Every GPU that loads the library holds that array until the
 * process exits.
 *
 * Same shots, same bits as stim_frame_sample_ex(c, num_shots, seed,
 * shot_offset, NULL, det_out, STIM_MEAS_MAJOR | STIM_DEVICE, NULL, stream).
 * det_out: device memory, D + K rows of ceil(num_shots/64) words (MEAS_MAJOR).
 * Asynchronous on `stream`.
 *
 * Preconditions and limits:
 *   - stim_reference_sample() must have run for this handle on the current
 *     device (it uploads the circuit and takes the reference sample, and
 *     does allocate); otherwise STIM_E_INVALID_ARG.
 *   - M * ceil(num_shots/64) * 8 bytes must fit the 32 MiB array; larger
 *     requests fail with STIM_E_UNSUPPORTED -- split them with shot_offset.
 *   - one 64-shot frame tile (num_qubits * 16 bytes) must fit shared memory;
 *     otherwise STIM_E_UNSUPPORTED.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls on a device share the one array and each call overwrites it
 *     before reading it; calls whose work overlaps on the same GPU (other
 *     streams, other threads) race with each other and must be serialized.
 */
#define STIM_NOALLOC_SCRATCH_BYTES (32u << 20)
int stim_frame_sample_noalloc(stim_circuit *c, uint64_t num_shots, uint64_t seed,
                              uint64_t shot_offset, uint64_t *det_out, void *stream);

/*
 * Kernel timing (measurement support; no counterpart in the paper).
 *
 * stim_profile(1) clears the statistics and starts recording a CUDA event
 * pair around every kernel the library launches, on the stream it launches
 * it on; stim_profile(0) stops recording. stim_profile_read() waits for the
 * recorded events, then fills out[k] for kernel ids k < n (STIM_KERNEL_*):
 * number of launches and summed device milliseconds. Process-wide; not
 * meant for concurrent use from several threads.
 */
#define STIM_KERNEL_FRAME      0
#define STIM_KERNEL_DETECTORS  1
#define STIM_KERNEL_TRANSPOSE  2
#define STIM_KERNEL_TABLEAU    3
#define STIM_KERNEL_COUNT      4

typedef struct {
    uint64_t launches;
    double total_ms;
} stim_kernel_stat;

int stim_profile(int enable);
int stim_profile_read(stim_kernel_stat *out, int n);

/*
 * stim_probe_smem_bandwidth -- measured shared-memory bandwidth of the current
 * device (measurement support; no counterpart in the paper), the roofline
 * denominator of the frame kernel, whose frames live in shared memory. Every
 * CTA streams 16-byte loads and stores (the frame kernel's access width) over
 * its own 64 KiB buffer (local_gbs), or over the buffer of the other CTA of a
 * 2-CTA cluster through distributed shared memory (cluster_gbs); bytes are
 * loads plus stores, timed with CUDA events (best of three after a warm-up).
 * Allocates a small device buffer; synchronizes.
 * Errors: STIM_E_INVALID_ARG (NULL argument), STIM_E_CUDA.
 */
int stim_probe_smem_bandwidth(double *local_gbs, double *cluster_gbs);

#ifdef __cplusplus
}
#endif

#endif /* STIMGB_H */
