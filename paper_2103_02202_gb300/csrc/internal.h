// internal.h -- data shared between the host compiler and the CUDA kernels.
//
// A compiled circuit is a small program of entries (fused layers and loop
// markers) over a flat array of 16-byte op records. REPEAT blocks are kept as
// loops: an op inside a loop body stores the instruction ordinal and the
// measurement index of its first iteration, and the kernels add
// iteration * stride at run time, so ordinals are those of the flattened
// circuit (the RNG keys depend on them) while the stored program stays the
// size of one loop body.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace stimgb {

// Opcodes 0..13 also appear in frame programs (4 bits there). OP_SX and the
// ones after it are gates that only the reference tableau tells apart: frame
// programs replace SQRT_X and SQRT_X_DAG (x ^= z) by H S H, S_DAG by S, SQRT_Y
// and SQRT_Y_DAG by H, and drop the Paulis X, Y, Z (they commute with every
// frame up to sign). OP_FFX and OP_FFZ are X and Z controlled by a
// measurement record ("CX rec[-k] q", "CZ rec[-k] q"): the tableau applies
// them when the reference outcome is 1, the frame where a shot's record
// differs from the reference.
enum Opcode : uint32_t {
    OP_H = 0, OP_S, OP_CX, OP_CZ,                  // Clifford gates
    OP_M, OP_MR, OP_R,                             // collapsing operations (Z basis)
    OP_XERR, OP_ZERR, OP_DEP1, OP_DEP2, OP_YERR,   // Pauli noise channels
    OP_FFX, OP_FFZ,                                // classically controlled X, Z
    OP_SX,                                         // SQRT_X (frame: x ^= z)
    OP_X, OP_Y, OP_Z, OP_SDAG, OP_SXD, OP_SY, OP_SYD,   // tableau-only gate variants
    OP_COUNT
};

inline bool op_is_gate(uint32_t o) { return o <= OP_CZ || (o >= OP_FFX && o < OP_COUNT); }
inline bool op_is_feedforward(uint32_t o) { return o == OP_FFX || o == OP_FFZ; }
inline bool op_is_collapse(uint32_t o) { return o >= OP_M && o <= OP_R; }
inline bool op_is_noise(uint32_t o) { return o >= OP_XERR && o <= OP_YERR; }
inline bool op_is_pair(uint32_t o) { return o == OP_CX || o == OP_CZ || o == OP_DEP2; }

// Frame-program opcode of a host opcode; OP_COUNT when the frame ignores it.
inline uint32_t frame_opcode(uint32_t o) {
    switch (o) {
        case OP_X: case OP_Y: case OP_Z: return OP_COUNT;
        case OP_SDAG: return OP_S;
        case OP_SXD: return OP_SX;      // expanded to H S H by the frame builder
        case OP_SY: case OP_SYD: return OP_H;
        default: return o;
    }
}

// Words of one noise table: 64 geometric gap thresholds, then 15 cumulative
// Pauli-choice thresholds of the channel and the Pauli count of a uniform
// (depolarizing) channel, 0 for other channels.
constexpr uint32_t kNoiseTableWords = 80;

constexpr uint32_t kQubitBits = 24;
constexpr uint32_t kQubitMask = (1u << kQubitBits) - 1;
constexpr uint32_t kMaxInstr = 1u << 28;       // instruction ordinals share a counter word with a 4-bit tag
constexpr int kMaxLoopDepth = 16;

// One target (or target pair) of one instruction.
//   a:     opcode << 24 | qubit a  (8-bit host opcode)
//   b:     qubit b | table << 24 (two-qubit ops, noise table in the top byte)
//          table << 24 (one-qubit noise)
//          measurement index of the first loop iteration (M, MR; the
//          controlling record of OP_FFX, OP_FFZ)
//   instr: flattened instruction ordinal of the first loop iteration
//   slot:  target index (one-qubit ops) or pair index (two-qubit ops)
struct DevOp {
    uint32_t a, b, instr, slot;
};

// Device status words written by kernels (read by the host after a sync).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_PROGRAM = 2 };

enum : uint32_t { ENT_LAYER = 0, ENT_LOOP_BEGIN = 1, ENT_LOOP_END = 2, ENT_DETS = 3 };

// One DETECTOR or OBSERVABLE_INCLUDE of a straight-line stretch of the
// program (between REPEAT boundaries): its detection-event row (detector
// index of the first loop iteration, or kObsRow | observable index) and the
// absolute measurement indices (first iteration) of its records,
// looks[look_begin .. look_begin + look_count).
struct DetItem {
    uint32_t row, look_begin, look_count, pad;
};
constexpr uint32_t kObsRow = 0x80000000u;

// Program entry (32 bytes).
//   LAYER:      ops [op_begin, op_begin + n_gate + n_noise + n_collapse), stored
//               as gates, then noise, then collapsing ops in source order.
//   LOOP_BEGIN: reps iterations of the entries up to the matching LOOP_END;
//               each iteration advances instruction ordinals by instr_stride,
//               measurement indices by meas_stride and detector indices by
//               n_noise (the loop body's DETECTOR count).
//   LOOP_END:   op_begin = index of the matching LOOP_BEGIN (strides as above).
//   DETS:       the detectors and observables of the straight-line stretch
//               that ends here: det_items [op_begin, op_begin + n_gate);
//               meas_stride = measurements made so far (first iteration).
struct ProgEntry {
    uint32_t kind;
    uint32_t op_begin;
    uint32_t n_gate, n_noise, n_collapse;
    uint32_t reps;
    uint32_t instr_stride, meas_stride;
};

struct HostProgram {
    uint32_t num_qubits = 0;
    uint64_t num_meas = 0;
    uint64_t num_det = 0;                   // detection-event rows: DETECTORs, then num_obs observables
    uint64_t num_obs = 0;                   // logical observables (largest OBSERVABLE_INCLUDE index + 1)
    uint64_t num_gate_targets = 0, num_noise_targets = 0, num_instr = 0;
    uint64_t num_layers_exec = 0;           // layer executions with loops unrolled
    uint64_t num_feedforward = 0;           // classically controlled X/Z targets (loops unrolled)
    uint64_t num_layers_stored = 0;
    uint32_t max_layer_ops = 0;
    uint32_t max_loop_depth = 0;
    std::vector<ProgEntry> prog;
    std::vector<DevOp> ops;
    std::vector<uint64_t> geo;              // [num_tables][kNoiseTableWords] noise tables
    std::vector<double> table_p;
    std::vector<uint64_t> det_ptr;          // num_det + 1 offsets into det_meas
    std::vector<uint32_t> det_meas;         // absolute measurement indices
    // the same detectors and observables as DETS entries of the program
    // (loop bodies once), for evaluation inside the frame kernel from a ring
    // of recent measurement flips; ring_len is a power of two larger than the
    // farthest a DETS entry looks back plus the measurements of one
    // straight-line stretch (0 when the program has no DETS entry)
    std::vector<DetItem> det_items;
    std::vector<uint32_t> det_looks;
    uint64_t ring_len = 0;
    // Top-level boundaries of REPEAT blocks, where the program has no open
    // loop: the tableau state there depends only on the noiseless skeleton
    // of the source before it (prefix_hash, FNV-1a like skeleton_hash) and
    // on num_qubits, so a circuit sharing that prefix may resume from it.
    struct CutPoint {
        uint32_t prog_index;     // first program entry after the boundary
        uint64_t meas;           // measurements before it
        uint64_t prefix_hash;
        uint64_t skeleton_len;   // skeleton words of that prefix
        // A cut right after a top-level REPEAT block that emitted entries:
        // the state there is also the state after loop_reps iterations of
        // any block with the same body and the same source before it, so a
        // circuit repeating that body at least as often resumes inside its
        // loop. loop_hash is prefix_hash with the repetition count (the
        // skeleton words reps_pos and reps_pos + 1) taken as zero.
        uint32_t loop_begin;     // the block's LOOP_BEGIN entry (UINT32_MAX: not such a cut)
        uint64_t loop_reps;
        uint64_t loop_meas;      // measurements per iteration
        uint64_t loop_hash;
        uint64_t reps_pos;
    };
    std::vector<CutPoint> cuts;
    // noiseless skeleton (source-order gates, collapses and classically
    // controlled ops with their targets, REPEAT structure) and its FNV-1a
    // hash: equal skeletons give equal reference samples
    std::vector<uint32_t> skeleton;
    uint64_t skeleton_hash = 0;
    // per-op-type target counts with loops unrolled (for bench accounting)
    uint64_t exec_targets[OP_COUNT] = {0};
};

// Frame-kernel program for a cluster of C CTAs that split the qubits into
// contiguous slices of Q = ceil(n / C): qubit q lives in CTA q / Q at local
// index q % Q.
//
// Consecutive layers are folded into chains: an op joins the chain of the
// previous merged layer whose first op covers all of its qubits, and runs
// right after it on the same thread. Chains of one merged layer have disjoint
// qubit footprints. A CTA owns the chains whose first op's first qubit is in
// its slice; its chains of a merged layer are grouped into segments of equal
// opcode signature (so warps run uniform code). Noise ops at the end of a
// chain (defer_from onwards) touch nothing the chain reads later, and their
// error masks commute, so the kernel may apply them after the chain; with a
// cluster they also name distinct qubits, so their hits never meet in one word. A layer
// holding a classically controlled op never folds into the open merged layer:
// the record it reads was written by another thread, and the barrier that
// ends the previous merged layer makes that write visible.
//
// Entries mirror HostProgram::prog except that folded LAYER entries are
// removed; a LAYER's op_begin indexes rank_tab, whose C + 1 values bound
// each CTA's segments in segs.
// Qubit references are (rank << 24 | local index).
// Op encoding:
//   a:     opcode << 28 | reference of qubit a
//   b:     two-qubit ops: reference of qubit b
//          M, MR, FFX, FFZ: measurement index of the first loop iteration
//          one-qubit noise: table index
//   instr: flattened instruction ordinal of the first loop iteration
//   slot:  target slot; DEPOLARIZE2 keeps its table index in bits 24..31
struct FrameSeg {
    uint32_t len;         // ops per chain
    uint32_t op_begin;    // ops step-major: step j of chain k at op_begin + j * count + k
    uint32_t count;       // chains
    uint32_t defer_from;  // chain steps >= defer_from are all noise ops (C > 1: on distinct qubits)
};

struct FrameProgram {
    int C = 1;
    uint32_t Q = 0;
    uint64_t merged_layers_exec = 0;
    uint32_t max_rank_ops = 0;          // largest op range of one CTA in one merged layer
    std::vector<ProgEntry> prog;
    std::vector<uint32_t> rank_tab;
    std::vector<FrameSeg> segs;
    std::vector<DevOp> ops;
};

void build_frame_program(const HostProgram &hp, int C, FrameProgram *out);

// Sets the calling thread's stim_last_error() message; returns code.
int report_error(int code, const std::string &msg);

// Parse + compile. Returns 0 or a STIM_E_* code with *err filled.
int compile_circuit(const char *text, size_t len, HostProgram *out, std::string *err);

// Exact geometric table of the keyed noise procedure:
//   t = round-half-even(p * 2^32), S_0 = 2^32, S_{k+1} = floor(S_k (2^32 - t) / 2^32),
//   G[k] = 2^32 - S_{k+1}.
void geometric_table(double p, uint64_t G[64]);

}  // namespace stimgb
