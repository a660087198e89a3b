// compiler.cpp -- circuit text -> device program (host side).
//
// Parses the line format of the paper's Section 5.8 (one instruction per
// line, broadcast targets, '#' comments, REPEAT N { ... }) and emits the
// program described in internal.h:
//   * every target (or target pair) becomes one 16-byte op carrying its RNG
//     key material (flattened instruction ordinal, slot) and, for M/MR, its
//     measurement index;
//   * ops of a straight-line segment are fused into layers by as-soon-as-
//     possible scheduling on qubit dependencies, so ops in one layer touch
//     disjoint qubits and commute; collapsing ops keep their relative source
//     order (the outcome-0 reference sample depends on that order);
//   * REPEAT bodies are compiled once and wrapped in LOOP entries;
//   * DETECTOR lookbacks rec[-k] are resolved to absolute measurement indices
//     in a flattened CSR list, followed by one row per logical observable
//     (all OBSERVABLE_INCLUDE(k) lookbacks of index k);
//   * a rec[-k] target in a CX (as control) or CZ pair makes a classically
//     controlled X or Z on the other target (OP_FFX, OP_FFZ), placed after
//     every collapsing op emitted before it;
//   * each distinct noise probability gets a 64-entry geometric threshold
//     table (Section 5.4's gap sampling, in exact integer form).
#include <algorithm>
#include <cctype>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>

#include "../../include/stimgb.h"
#include "internal.h"

namespace stimgb {

void geometric_table(double p, uint64_t G[64]) {
    const unsigned __int128 one = (unsigned __int128)1 << 32;
    long long t = llrint(ldexp(p, 32));     // default rounding: nearest, ties to even
    if (t < 0) t = 0;
    if (t > (1LL << 32)) t = 1LL << 32;
    unsigned __int128 survive = one;       // S_k: 2^32 * P(no error in the next k slots)
    for (int k = 0; k < 64; k++) {
        survive = (survive * (one - (unsigned __int128)t)) >> 32;
        G[k] = (uint64_t)(one - survive);
    }
}

namespace {

enum ParsedGate {
    PG_H, PG_S, PG_CX, PG_CZ, PG_M, PG_MR, PG_R, PG_XERR, PG_ZERR, PG_DEP1, PG_DEP2, PG_DET,
    PG_X, PG_Y, PG_Z, PG_SDAG, PG_SQX, PG_SQXD, PG_SQY, PG_SQYD, PG_YERR,
    PG_MX, PG_MY, PG_MRX, PG_MRY, PG_RX, PG_RY, PG_OBS, PG_PC1, PG_PC2
};

// A measurement-record target rec[-k] in a CX/CZ pair: kRecTarget | k.
constexpr uint32_t kRecTarget = 1u << 31;

struct Instr {
    int gate = 0;
    double p = 0;                    // noise probability (Pauli channels: the sum of args)
    std::vector<double> args;        // Pauli channels: the 3 or 15 probabilities
    std::vector<uint32_t> targets;   // qubits (kRecTarget | k for rec[-k] in CX/CZ), or lookbacks k for DETECTOR
    int line = 0;
};

struct Node;
struct Block {
    uint64_t reps = 1;
    std::vector<Node> items;
};
struct Node {
    std::unique_ptr<Block> block;   // non-null for REPEAT
    Instr ins;
};

struct ParseError {
    int code;
    std::string msg;
};

class Parser {
  public:
    Parser(const char *s, size_t n) : s_(s), n_(n) {}

    Block parse() {
        Block root;
        parse_into(&root, 0);
        return root;
    }

  private:
    const char *s_;
    size_t n_;
    size_t pos_ = 0;
    int line_ = 0;

    [[noreturn]] void fail(size_t col, const char *what, const std::string &extra = "") {
        char buf[96];
        snprintf(buf, sizeof buf, "line %d, column %zu: ", line_, col + 1);
        throw ParseError{STIM_E_PARSE, std::string(buf) + what + extra};
    }

    static bool space(char c) { return c == ' ' || c == '\t' || c == '\r'; }

    // Returns true if a closing brace ended the block.
    bool parse_into(Block *blk, int depth) {
        while (pos_ < n_) {
            size_t b = pos_;
            size_t e = b;
            while (e < n_ && s_[e] != '\n') e++;
            pos_ = e < n_ ? e + 1 : e;
            line_++;
            const char *ln = s_ + b;
            size_t len = e - b;
            for (size_t i = 0; i < len; i++)
                if (ln[i] == '#') { len = i; break; }
            size_t lo = 0, hi = len;
            while (lo < hi && space(ln[lo])) lo++;
            while (hi > lo && space(ln[hi - 1])) hi--;
            if (lo == hi) continue;
            if (ln[lo] == '}') {
                if (hi - lo != 1) fail(lo + 1, "unexpected text after '}'");
                if (depth == 0) fail(lo, "'}' without REPEAT");
                return true;
            }
            if (hi - lo > 6 && memcmp(ln + lo, "REPEAT", 6) == 0 && space(ln[lo + 6])) {
                size_t i = lo + 6;
                while (i < hi && space(ln[i])) i++;
                if (i >= hi || ln[i] < '0' || ln[i] > '9') fail(i, "REPEAT needs a count");
                uint64_t reps = 0;
                while (i < hi && ln[i] >= '0' && ln[i] <= '9') {
                    reps = reps * 10 + (uint64_t)(ln[i] - '0');
                    if (reps > 1000000000ull) fail(i, "REPEAT count too large");
                    i++;
                }
                while (i < hi && space(ln[i])) i++;
                if (i + 1 != hi || ln[i] != '{') fail(i, "expected '{' ending the REPEAT line");
                if (reps == 0) fail(lo, "REPEAT 0 is not allowed");
                Node nd;
                nd.block.reset(new Block);
                nd.block->reps = reps;
                int open_line = line_;
                if (!parse_into(nd.block.get(), depth + 1)) {
                    line_ = open_line;
                    fail(lo, "REPEAT block is never closed");
                }
                blk->items.push_back(std::move(nd));
                continue;
            }
            Node nd;
            parse_instruction(ln, lo, hi, &nd.ins);
            blk->items.push_back(std::move(nd));
        }
        return false;
    }

    void parse_instruction(const char *ln, size_t lo, size_t hi, Instr *ins) {
        size_t i = lo;
        while (i < hi && (isupper((unsigned char)ln[i]) || isdigit((unsigned char)ln[i]) || ln[i] == '_')) i++;
        std::string name(ln + lo, i - lo);
        static const std::map<std::string, int> kNames = {
            {"H", PG_H}, {"S", PG_S}, {"CX", PG_CX}, {"CNOT", PG_CX}, {"CZ", PG_CZ},
            {"M", PG_M}, {"MR", PG_MR}, {"R", PG_R}, {"X_ERROR", PG_XERR},
            {"Z_ERROR", PG_ZERR}, {"DEPOLARIZE1", PG_DEP1}, {"DEPOLARIZE2", PG_DEP2},
            {"DETECTOR", PG_DET}, {"X", PG_X}, {"Y", PG_Y}, {"Z", PG_Z}, {"S_DAG", PG_SDAG},
            {"SQRT_X", PG_SQX}, {"SQRT_X_DAG", PG_SQXD}, {"SQRT_Y", PG_SQY}, {"SQRT_Y_DAG", PG_SQYD},
            {"Y_ERROR", PG_YERR}, {"MX", PG_MX}, {"MY", PG_MY}, {"MRX", PG_MRX}, {"MRY", PG_MRY},
            {"RX", PG_RX}, {"RY", PG_RY}, {"OBSERVABLE_INCLUDE", PG_OBS},
            {"PAULI_CHANNEL_1", PG_PC1}, {"PAULI_CHANNEL_2", PG_PC2}};
        auto it = kNames.find(name);
        if (name.empty() || it == kNames.end()) {
            size_t j = i;
            while (j < hi && !space(ln[j]) && ln[j] != '(') j++;
            fail(lo, "unknown gate '", std::string(ln + lo, j - lo) + "'");
        }
        ins->gate = it->second;
        ins->line = line_;
        std::vector<double> args;
        if (i < hi && ln[i] == '(') {
            size_t close = i;
            while (close < hi && ln[close] != ')') close++;
            if (close >= hi) fail(i, "unterminated '('");
            size_t a = i + 1;
            while (a <= close) {
                size_t b = a;
                while (b < close && ln[b] != ',') b++;
                std::string tok(ln + a, b - a);
                char *endp = nullptr;
                errno = 0;
                double v = strtod(tok.c_str(), &endp);
                while (endp && space(*endp)) endp++;
                if (tok.empty() || endp == tok.c_str() || *endp) fail(a, "bad numeric argument");
                args.push_back(v);
                a = b + 1;
            }
            i = close + 1;
        }
        bool noise = (ins->gate >= PG_XERR && ins->gate <= PG_DEP2) || ins->gate == PG_YERR;
        if (ins->gate == PG_PC1 || ins->gate == PG_PC2) {
            const size_t want = ins->gate == PG_PC1 ? 3 : 15;
            if (args.size() != want)
                fail(lo, ins->gate == PG_PC1 ? "PAULI_CHANNEL_1 takes 3 probabilities" : "PAULI_CHANNEL_2 takes 15 probabilities");
            double total = 0;       // summed left to right
            for (double v : args) {
                if (!(v >= 0.0 && v <= 1.0)) fail(lo, "probability outside [0, 1]");
                total += v;
            }
            if (!(total <= 1.0)) fail(lo, "Pauli channel probabilities sum above 1");
            ins->p = total;
            ins->args = args;
        } else if (noise) {
            if (args.size() != 1) fail(lo, "noise channel takes exactly one probability");
            ins->p = args[0];
            if (!(ins->p >= 0.0 && ins->p <= 1.0)) fail(lo, "probability outside [0, 1]");
        } else if (ins->gate == PG_OBS) {
            if (args.size() != 1) fail(lo, "OBSERVABLE_INCLUDE takes one index");
            ins->p = args[0];
            if (!(ins->p >= 0.0 && ins->p < 65536.0) || ins->p != std::floor(ins->p))
                fail(lo, "observable index is not an integer in [0, 65535]");
        } else if (ins->gate != PG_DET && !args.empty()) {
            fail(lo, "gate takes no arguments");
        }
        if (i < hi && !space(ln[i])) fail(i, "expected a space before the targets");
        while (i < hi) {
            while (i < hi && space(ln[i])) i++;
            if (i >= hi) break;
            size_t t0 = i;
            uint64_t v = 0;
            const bool rec_target = (ins->gate == PG_CX || ins->gate == PG_CZ) && hi - i >= 6 &&
                                    memcmp(ln + i, "rec[-", 5) == 0;
            if (ins->gate == PG_DET || ins->gate == PG_OBS || rec_target) {
                if (hi - i < 6 || memcmp(ln + i, "rec[-", 5) != 0) fail(i, "expected a rec[-k] target");
                i += 5;
                if (i >= hi || !isdigit((unsigned char)ln[i])) fail(i, "expected a rec[-k] target");
                while (i < hi && isdigit((unsigned char)ln[i])) {
                    v = v * 10 + (uint64_t)(ln[i] - '0');
                    if (v > 0xFFFFFFFFull) fail(t0, "lookback too large");
                    i++;
                }
                if (i >= hi || ln[i] != ']') fail(i, "expected ']'");
                i++;
                if (v == 0) fail(t0, "rec[-0] does not name a measurement");
                if (rec_target) {
                    if (v >= kRecTarget) fail(t0, "lookback too large");
                    v |= kRecTarget;
                }
            } else {
                if (!isdigit((unsigned char)ln[i])) fail(i, "qubit targets are non-negative integers");
                while (i < hi && isdigit((unsigned char)ln[i])) {
                    v = v * 10 + (uint64_t)(ln[i] - '0');
                    if (v > kQubitMask) throw ParseError{STIM_E_UNSUPPORTED, "qubit index above 2^24 - 1"};
                    i++;
                }
            }
            if (i < hi && !space(ln[i])) fail(i, "bad target");
            ins->targets.push_back((uint32_t)v);
        }
        bool pair = ins->gate == PG_CX || ins->gate == PG_CZ || ins->gate == PG_DEP2 || ins->gate == PG_PC2;
        if (pair) {
            if (ins->targets.size() % 2) fail(lo, "two-qubit gate needs an even number of targets");
            for (size_t k = 0; k < ins->targets.size(); k += 2) {
                const uint32_t ta = ins->targets[k], tb = ins->targets[k + 1];
                if (ta == tb) fail(lo, "two-qubit gate applied to one qubit");
                if ((ta & tb) & kRecTarget) fail(lo, "a pair of two measurement records");
                if (ins->gate == PG_CX && (tb & kRecTarget)) fail(lo, "CX takes a measurement record only as control");
            }
        }
    }
};

// Opcode of an instruction; measurements and resets in the X and Y bases map
// to their Z-basis op, emitted between basis changes (basis_of).
uint32_t opcode_of(int pg) {
    switch (pg) {
        case PG_H: return OP_H;
        case PG_S: return OP_S;
        case PG_CX: return OP_CX;
        case PG_CZ: return OP_CZ;
        case PG_M: case PG_MX: case PG_MY: return OP_M;
        case PG_MR: case PG_MRX: case PG_MRY: return OP_MR;
        case PG_R: case PG_RX: case PG_RY: return OP_R;
        case PG_XERR: return OP_XERR;
        case PG_ZERR: return OP_ZERR;
        case PG_YERR: return OP_YERR;
        case PG_DEP1: case PG_PC1: return OP_DEP1;      // one-qubit Pauli channel
        case PG_PC2: return OP_DEP2;                     // two-qubit Pauli channel
        case PG_X: return OP_X;
        case PG_Y: return OP_Y;
        case PG_Z: return OP_Z;
        case PG_SDAG: return OP_SDAG;
        case PG_SQX: return OP_SX;
        case PG_SQXD: return OP_SXD;
        case PG_SQY: return OP_SY;
        case PG_SQYD: return OP_SYD;
        default: return OP_DEP2;
    }
}

// Measurement basis of a collapsing instruction: 0 Z, 1 X, 2 Y.
int basis_of(int pg) {
    if (pg == PG_MX || pg == PG_MRX || pg == PG_RX) return 1;
    if (pg == PG_MY || pg == PG_MRY || pg == PG_RY) return 2;
    return 0;
}

// Opcode of one CX/CZ pair: classically controlled X/Z when a target is a
// measurement record.
uint32_t pair_opcode(int pg, uint32_t ta, uint32_t tb) {
    if ((ta | tb) & kRecTarget) return pg == PG_CX ? OP_FFX : OP_FFZ;
    return opcode_of(pg);
}

bool records(int pg) { return pg == PG_M || pg == PG_MR || pg == PG_MX || pg == PG_MY || pg == PG_MRX || pg == PG_MRY; }

struct Counts {
    uint64_t instr = 0, meas = 0, det = 0, det_entries = 0;
    uint64_t obs = 0;                   // largest observable index + 1
    uint64_t gate_t = 0, noise_t = 0, ff_t = 0;
    uint64_t targets[OP_COUNT] = {0};
};

// Counts of a block body executed once (nested loops multiplied out).
void count_block(const Block &b, Counts *c, uint32_t *max_qubit, bool *any_qubit) {
    for (const Node &nd : b.items) {
        if (nd.block) {
            Counts inner;
            count_block(*nd.block, &inner, max_qubit, any_qubit);
            uint64_t r = nd.block->reps;
            auto mul = [&](uint64_t v) -> uint64_t {
                if (v && r > UINT64_MAX / v) throw ParseError{STIM_E_UNSUPPORTED, "circuit too large"};
                return v * r;
            };
            c->instr += mul(inner.instr);
            c->meas += mul(inner.meas);
            c->det += mul(inner.det);
            c->det_entries += mul(inner.det_entries);
            c->obs = std::max(c->obs, inner.obs);
            c->gate_t += mul(inner.gate_t);
            c->noise_t += mul(inner.noise_t);
            c->ff_t += mul(inner.ff_t);
            for (int k = 0; k < (int)OP_COUNT; k++) c->targets[k] += mul(inner.targets[k]);
            if (c->instr > kMaxInstr) throw ParseError{STIM_E_UNSUPPORTED, "more than 2^28 instructions after flattening"};
            continue;
        }
        const Instr &in = nd.ins;
        c->instr++;
        if (in.gate == PG_DET) {
            c->det++;
            c->det_entries += in.targets.size();
            continue;
        }
        if (in.gate == PG_OBS) {
            c->det_entries += in.targets.size();
            c->obs = std::max<uint64_t>(c->obs, (uint64_t)in.p + 1);
            continue;
        }
        for (uint32_t q : in.targets) {
            if (q & kRecTarget) continue;
            if (!*any_qubit || q > *max_qubit) *max_qubit = q;
            *any_qubit = true;
        }
        uint32_t op = opcode_of(in.gate);
        uint64_t slots = op_is_pair(op) ? in.targets.size() / 2 : in.targets.size();
        if (op == OP_CX || op == OP_CZ) {
            for (size_t k = 0; k < in.targets.size(); k += 2) {
                const uint32_t po = pair_opcode(in.gate, in.targets[k], in.targets[k + 1]);
                c->targets[po]++;
                if (op_is_feedforward(po)) c->ff_t++;
            }
        } else {
            c->targets[op] += slots;
        }
        if (op_is_noise(op)) c->noise_t += slots;
        else c->gate_t += slots;
        if (records(in.gate)) c->meas += in.targets.size();
    }
}

class Emitter {
  public:
    Emitter(HostProgram *hp, uint32_t n) : hp_(hp), stamp_(n, 0), last_(n, 0) {}

    // Emit the body of `b` for its first iteration, with the given starting
    // instruction ordinal, measurement index and detector index. Returns
    // layer executions.
    uint64_t emit(const Block &b, uint64_t instr, uint64_t meas, uint64_t det, uint32_t depth) {
        if (depth > hp_->max_loop_depth) hp_->max_loop_depth = depth;
        if (depth > (uint32_t)kMaxLoopDepth) throw ParseError{STIM_E_UNSUPPORTED, "REPEAT nested more than 16 deep"};
        uint64_t exec = 0;
        begin_segment();
        uint64_t seg_meas0 = meas;
        for (const Node &nd : b.items) {
            if (nd.block) {
                exec += flush();
                flush_dets(meas, meas - seg_meas0);
                Counts inner;
                uint32_t mq = 0;
                bool any = false;
                count_block(*nd.block, &inner, &mq, &any);
                size_t begin_idx = hp_->prog.size();
                ProgEntry e{};
                e.kind = ENT_LOOP_BEGIN;
                e.reps = (uint32_t)nd.block->reps;
                e.instr_stride = (uint32_t)inner.instr;
                e.meas_stride = (uint32_t)inner.meas;
                e.n_noise = (uint32_t)inner.det;        // detector stride
                if (depth == 0) cut_at(meas, (size_t)(&nd - b.items.data()));
                hp_->prog.push_back(e);
                uint64_t body = emit(*nd.block, instr, meas, det, depth + 1);
                if (hp_->prog.size() == begin_idx + 1) {
                    hp_->prog.pop_back();       // body without layers: nothing to repeat
                } else {
                    ProgEntry f = e;
                    f.kind = ENT_LOOP_END;
                    f.op_begin = (uint32_t)begin_idx;
                    hp_->prog.push_back(f);
                    hp_->prog[begin_idx].op_begin = (uint32_t)(hp_->prog.size() - 1);
                }
                exec += body * nd.block->reps;
                instr += inner.instr * nd.block->reps;
                meas += inner.meas * nd.block->reps;
                det += inner.det * nd.block->reps;
                if (depth == 0)
                    cut_at(meas, (size_t)(&nd - b.items.data()) + 1,
                           hp_->prog.size() == begin_idx ? UINT32_MAX : (uint32_t)begin_idx, nd.block->reps,
                           inner.meas);
                begin_segment();
                seg_meas0 = meas;
                continue;
            }
            const Instr &in = nd.ins;
            if (in.gate == PG_DET || in.gate == PG_OBS) {
                // record lookbacks were validated when the detectors were collected
                DetItem it{};
                it.row = in.gate == PG_DET ? (uint32_t)det++ : (kObsRow | (uint32_t)in.p);
                it.look_begin = (uint32_t)hp_->det_looks.size();
                it.look_count = (uint32_t)in.targets.size();
                for (uint32_t k : in.targets) hp_->det_looks.push_back((uint32_t)(meas - k));
                seg_dets_.push_back(it);
            } else {
                uint32_t op = opcode_of(in.gate);
                uint32_t table = 0;
                if (op_is_noise(op)) {
                    if (in.p == 0.0) {      // p = 0 channels are no-ops and draw nothing
                        instr++;
                        continue;
                    }
                    table = table_for(in);
                }
                bool pair = op_is_pair(op);
                size_t step = pair ? 2 : 1;
                const int basis = basis_of(in.gate);
                for (size_t k = 0; k < in.targets.size(); k += step) {
                    DevOp d{};
                    uint32_t qa = in.targets[k];
                    uint32_t qb = pair ? in.targets[k + 1] : qa;
                    d.instr = (uint32_t)instr;
                    d.slot = (uint32_t)(k / step);
                    if (pair && ((qa | qb) & kRecTarget)) {
                        // X or Z on the qubit target, controlled by the record
                        const uint32_t ff = pair_opcode(in.gate, qa, qb);
                        const uint32_t lookback = ((qa & kRecTarget) ? qa : qb) & ~kRecTarget;
                        const uint32_t q = (qa & kRecTarget) ? qb : qa;
                        if (lookback > meas) {
                            char buf[128];
                            snprintf(buf, sizeof buf, "line %d: rec[-%u] reaches before the first measurement",
                                     in.line, lookback);
                            throw ParseError{STIM_E_PARSE, buf};
                        }
                        d.a = (ff << 24) | q;
                        d.b = (uint32_t)(meas - lookback);
                        place(d, q, q, false, true);
                        continue;
                    }
                    d.a = (op << 24) | qa;
                    if (op == OP_M || op == OP_MR) {
                        d.b = (uint32_t)meas++;
                    } else if (pair) {
                        d.b = qb | (table << 24);
                    } else {
                        d.b = table << 24;
                    }
                    // X basis: H, op, H. Y basis: S_DAG, H, op, H, S (the basis
                    // change maps the measured Pauli to Z and back).
                    if (basis == 2) place(basis_gate(OP_SDAG, qa, d.instr), qa, qa, false);
                    if (basis != 0) place(basis_gate(OP_H, qa, d.instr), qa, qa, false);
                    place(d, qa, qb, op_is_collapse(op));
                    if (basis != 0) place(basis_gate(OP_H, qa, d.instr), qa, qa, false);
                    if (basis == 2) place(basis_gate(OP_S, qa, d.instr), qa, qa, false);
                }
            }
            instr++;
        }
        exec += flush();
        flush_dets(meas, meas - seg_meas0);
        return exec;
    }

    // Top-level cut points recorded while emitting; the caller adds the
    // prefix hashes of the items before each.
    struct Cut {
        uint32_t prog_index;     // first program entry after the cut
        uint64_t meas;           // measurements before it
        size_t items_before;     // top-level source items before it
        uint32_t loop_begin;     // after a REPEAT block: its LOOP_BEGIN entry (UINT32_MAX: none emitted)
        uint64_t loop_reps, loop_meas;
    };
    std::vector<Cut> cuts;
    void cut_at(uint64_t meas, size_t items_before, uint32_t loop_begin = UINT32_MAX, uint64_t loop_reps = 0,
                uint64_t loop_meas = 0) {
        cuts.push_back(Cut{(uint32_t)hp_->prog.size(), meas, items_before, loop_begin, loop_reps, loop_meas});
    }

    // Ring length for the DETS entries emitted (0 without any).
    uint64_t ring_len() const {
        if (!any_dets_) return 0;
        uint64_t r = 1;
        while (r <= max_det_dist_ + max_seg_meas_) r <<= 1;
        return r;
    }

  private:
    struct LayerBuild {
        std::vector<DevOp> gate, noise, collapse;
    };
    HostProgram *hp_;
    std::vector<uint32_t> stamp_;
    std::vector<uint32_t> last_;      // layer index + 1 of the last op on a qubit (this segment)
    uint32_t seg_ = 0;
    std::vector<LayerBuild> layers_;
    uint32_t last_collapse_ = 0;      // layer index + 1 of the last collapsing op
    std::map<std::vector<uint64_t>, uint32_t> tables_;
    std::vector<DetItem> seg_dets_;   // detectors and observables of the open stretch
    bool any_dets_ = false;
    uint64_t max_det_dist_ = 0;       // farthest lookback of a DETS entry from its position
    uint64_t max_seg_meas_ = 0;       // most measurements of one straight-line stretch

    // A DETS entry for the detectors and observables of the stretch that ends
    // here (meas measurements made so far, seg_meas of them in the stretch).
    void flush_dets(uint64_t meas, uint64_t seg_meas) {
        max_seg_meas_ = std::max(max_seg_meas_, seg_meas);
        if (seg_dets_.empty()) return;
        ProgEntry e{};
        e.kind = ENT_DETS;
        e.op_begin = (uint32_t)hp_->det_items.size();
        e.n_gate = (uint32_t)seg_dets_.size();
        e.meas_stride = (uint32_t)meas;
        for (const DetItem &it : seg_dets_)
            for (uint32_t k = 0; k < it.look_count; k++)
                max_det_dist_ = std::max<uint64_t>(max_det_dist_, meas - hp_->det_looks[it.look_begin + k]);
        hp_->det_items.insert(hp_->det_items.end(), seg_dets_.begin(), seg_dets_.end());
        hp_->prog.push_back(e);
        seg_dets_.clear();
        any_dets_ = true;
    }

    void begin_segment() {
        seg_++;
        layers_.clear();
        last_collapse_ = 0;
    }

    uint32_t lastq(uint32_t q) const { return stamp_[q] == seg_ ? last_[q] : 0; }

    static DevOp basis_gate(uint32_t op, uint32_t q, uint32_t instr) {
        DevOp g{};
        g.a = (op << 24) | q;
        g.instr = instr;
        return g;
    }

    // after_collapses: a classically controlled op goes after every layer
    // holding a collapsing op (its record is written there).
    void place(const DevOp &d, uint32_t qa, uint32_t qb, bool collapse, bool after_collapses = false) {
        uint32_t L = lastq(qa);
        uint32_t Lb = lastq(qb);
        if (Lb > L) L = Lb;
        // L is the first layer index after every layer touching the qubits
        if (collapse && last_collapse_ > 0 && last_collapse_ - 1 > L) L = last_collapse_ - 1;
        if (after_collapses && last_collapse_ > L) L = last_collapse_;
        if (L >= layers_.size()) layers_.resize(L + 1);
        uint32_t op = d.a >> 24;
        if (op_is_gate(op)) layers_[L].gate.push_back(d);
        else if (op_is_noise(op)) layers_[L].noise.push_back(d);
        else layers_[L].collapse.push_back(d);
        stamp_[qa] = seg_;
        last_[qa] = L + 1;
        stamp_[qb] = seg_;
        last_[qb] = L + 1;
        if (collapse) last_collapse_ = L + 1;
    }

    uint64_t flush() {
        uint64_t n = 0;
        for (LayerBuild &lb : layers_) {
            // group gates and noise by opcode to keep warps uniform; collapsing
            // ops stay in source order
            auto by_op = [](const DevOp &x, const DevOp &y) { return (x.a >> 24) < (y.a >> 24); };
            std::stable_sort(lb.gate.begin(), lb.gate.end(), by_op);
            std::stable_sort(lb.noise.begin(), lb.noise.end(), by_op);
            ProgEntry e{};
            e.kind = ENT_LAYER;
            e.op_begin = (uint32_t)hp_->ops.size();
            e.n_gate = (uint32_t)lb.gate.size();
            e.n_noise = (uint32_t)lb.noise.size();
            e.n_collapse = (uint32_t)lb.collapse.size();
            uint32_t tot = e.n_gate + e.n_noise + e.n_collapse;
            if (tot == 0) continue;
            if (tot > hp_->max_layer_ops) hp_->max_layer_ops = tot;
            hp_->ops.insert(hp_->ops.end(), lb.gate.begin(), lb.gate.end());
            hp_->ops.insert(hp_->ops.end(), lb.noise.begin(), lb.noise.end());
            hp_->ops.insert(hp_->ops.end(), lb.collapse.begin(), lb.collapse.end());
            hp_->prog.push_back(e);
            hp_->num_layers_stored++;
            n++;
        }
        layers_.clear();
        return n;
    }

    // Noise table of an instruction (kNoiseTableWords words): the 64 gap
    // thresholds of its total probability p, then 15 Pauli-choice thresholds
    // T[0..14] and T[15]. A hit's Pauli index is 1 + #{i : v >= T[i]} for a
    // fresh 32-bit draw v (1 X, 2 Y, 3 Z; pairs 4a + b):
    //   DEPOLARIZE1: T[i] = ceil((i + 1) 2^32 / 3), i < 2, so the index is 1 + floor(3v / 2^32);
    //   DEPOLARIZE2: T[i] = ceil((i + 1) 2^32 / 15), i < 14, i.e. 1 + floor(15v / 2^32);
    //   PAULI_CHANNEL_1/2 with probabilities q: T[i] = round-half-even(2^32 (q_1 + ... + q_{i+1}) / p);
    //   every other threshold 2^32. T[15]'s low half = 3 or 15 for the
    //   depolarizing channels (the kernel multiplies instead of scanning),
    //   else 0; its high half a gap estimate constant (below).
    uint32_t table_for(const Instr &in) {
        const uint64_t kind = in.gate == PG_DEP1 ? 1 : in.gate == PG_DEP2 ? 2 : in.gate == PG_PC1 ? 3
                            : in.gate == PG_PC2 ? 4 : 0;
        auto bits_of = [](double v) {
            uint64_t b;
            memcpy(&b, &v, sizeof b);
            return b;
        };
        std::vector<uint64_t> key{kind, bits_of(in.p)};
        for (double v : in.args) key.push_back(bits_of(v));
        auto it = tables_.find(key);
        if (it != tables_.end()) return it->second;
        uint32_t id = (uint32_t)hp_->table_p.size();
        if (id >= 256) throw ParseError{STIM_E_UNSUPPORTED, "more than 256 distinct noise tables"};
        hp_->table_p.push_back(in.p);
        hp_->geo.resize(hp_->geo.size() + kNoiseTableWords);
        uint64_t *G = &hp_->geo[hp_->geo.size() - kNoiseTableWords];
        geometric_table(in.p, G);
        uint64_t *T = G + 64;
        for (int i = 0; i < 15; i++) T[i] = 1ull << 32;
        T[15] = 0;
        if (kind == 1 || kind == 2) {
            const uint64_t m = kind == 1 ? 3 : 15;
            for (uint64_t i = 0; i + 1 < m; i++) T[i] = (((i + 1) << 32) + m - 1) / m;
            T[15] = m;
        } else if ((kind == 3 || kind == 4) && in.p > 0) {
            double partial = 0;
            for (size_t i = 0; i + 1 < in.args.size(); i++) {
                partial += in.args[i];
                long long t = llrint(ldexp(partial / in.p, 32));
                if (t < 0) t = 0;
                if (t > (1LL << 32)) t = 1LL << 32;
                T[i] = (uint64_t)t;
            }
        }
        // T[15]'s upper half: the float 1 / log2(1 - q) of the table's
        // per-shot probability q = t / 2^32, from which the kernel estimates
        // a gap before checking it against G (0 when q is 0 or 1)
        {
            long long t = llrint(ldexp(in.p, 32));
            if (t < 0) t = 0;
            if (t > (1LL << 32)) t = 1LL << 32;
            float inv = 0.0f;
            if (t > 0 && t < (1LL << 32)) inv = (float)(1.0 / log2(1.0 - ldexp((double)t, -32)));
            uint32_t bits;
            memcpy(&bits, &inv, sizeof bits);
            T[15] |= (uint64_t)bits << 32;
        }
        tables_[key] = id;
        return id;
    }
};

// The noiseless skeleton of a block: every instruction that acts on the
// noiseless state (gates, collapsing ops, classically controlled ops) with its
// targets, and REPEAT structure, in source order. Noise channels, DETECTOR and
// OBSERVABLE_INCLUDE do not change the reference sample, so circuits with
// equal skeletons have equal reference samples.
void skeleton_node(const Node &nd, std::vector<uint32_t> *out);

void skeleton_of(const Block &b, std::vector<uint32_t> *out) {
    for (const Node &nd : b.items) skeleton_node(nd, out);
}

// One item's part of the skeleton: a REPEAT block is bracketed by two marker
// words with its repetition count; noise channels, DETECTOR and
// OBSERVABLE_INCLUDE add nothing.
void skeleton_node(const Node &nd, std::vector<uint32_t> *out) {
    if (nd.block) {
        out->push_back(0xFFFFFFFFu);
        out->push_back((uint32_t)nd.block->reps);
        out->push_back((uint32_t)(nd.block->reps >> 32));
        skeleton_of(*nd.block, out);
        out->push_back(0xFFFFFFFEu);
        return;
    }
    const Instr &in = nd.ins;
    if (in.gate == PG_DET || in.gate == PG_OBS) return;
    if (op_is_noise(opcode_of(in.gate))) return;
    out->push_back((uint32_t)in.gate);
    out->push_back((uint32_t)in.targets.size());
    out->insert(out->end(), in.targets.begin(), in.targets.end());
}

// FNV-1a over the bytes of v, continuing from h.
uint64_t fnv_words(uint64_t h, const std::vector<uint32_t> &v, size_t begin = 0) {
    for (size_t i = begin; i < v.size(); i++)
        for (int k = 0; k < 4; k++) {
            h ^= (v[i] >> (8 * k)) & 0xFFu;
            h *= 1099511628211ull;
        }
    return h;
}

// Flattened detector list: absolute measurement index of every rec[-k].
// Observable lookbacks go to obs[k] (appended after the detectors by the caller).
void collect_detectors(const Block &b, uint64_t *meas, HostProgram *hp, std::vector<std::vector<uint32_t>> *obs) {
    for (const Node &nd : b.items) {
        if (nd.block) {
            for (uint64_t r = 0; r < nd.block->reps; r++) collect_detectors(*nd.block, meas, hp, obs);
            continue;
        }
        const Instr &in = nd.ins;
        if (records(in.gate)) {
            *meas += in.targets.size();
        } else if (in.gate == PG_DET || in.gate == PG_OBS) {
            std::vector<uint32_t> &dst = in.gate == PG_DET ? hp->det_meas : (*obs)[(size_t)in.p];
            for (uint32_t k : in.targets) {
                if (k > *meas) {
                    char buf[128];
                    snprintf(buf, sizeof buf, "line %d: rec[-%u] reaches before the first measurement", in.line, k);
                    throw ParseError{STIM_E_PARSE, buf};
                }
                dst.push_back((uint32_t)(*meas - k));
            }
            if (in.gate == PG_DET) hp->det_ptr.push_back(hp->det_meas.size());
        }
    }
}

}  // namespace

namespace {

struct Chain {
    uint32_t q0;                // first qubit of the first op (decides the owning CTA)
    std::vector<uint32_t> qs;   // footprint
    std::vector<DevOp> ops;     // global encoding (as in HostProgram::ops)
};

inline uint32_t op_q0(const DevOp &d) { return d.a & kQubitMask; }
inline uint32_t op_q1(const DevOp &d) {
    const uint32_t opc = d.a >> 24;
    return op_is_pair(opc) ? (d.b & kQubitMask) : op_q0(d);
}

// Longest chain: bounds the work one thread does between two barriers.
constexpr size_t kMaxChainOps = 12;

class FrameBuilder {
  public:
    FrameBuilder(const HostProgram &hp, int C, FrameProgram *fp) : hp_(hp), C_(C), fp_(fp), owner_(hp.num_qubits + 1, -1) {}

    // Folds the layers [first, last) (consecutive LAYER entries of hp.prog)
    // into merged layers; returns the number of merged layers emitted. A layer
    // folds into the open merged layer when none of its ops touches qubits of
    // two different chains: an op on qubits of one chain is appended to it
    // (its other qubits, untouched so far in the merged layer, join the
    // chain's footprint); an op on untouched qubits starts a new chain.
    uint32_t run(size_t first, size_t last) {
        uint32_t emitted = 0;
        for (size_t k = first; k < last; k++) {
            const ProgEntry &e = hp_.prog[k];
            const uint32_t tot = e.n_gate + e.n_noise + e.n_collapse;
            const DevOp *ops = hp_.ops.data() + e.op_begin;
            bool fold = !chains_.empty();
            std::vector<uint32_t> grow;      // ops this layer would append to each open chain
            for (uint32_t i = 0; i < tot && fold; i++) {
                if (op_is_feedforward(ops[i].a >> 24)) fold = false;       // reads a record of another thread
                if (frame_opcode(ops[i].a >> 24) == OP_COUNT) continue;     // no frame action
                const int own = chain_of(ops[i]);
                if (own == -2) {
                    fold = false;
                } else if (own >= 0) {
                    // several targets of one instruction may join one chain
                    if (grow.empty()) grow.assign(chains_.size(), 0);
                    grow[own] += frame_opcode(ops[i].a >> 24) == OP_SX ? 3u : 1u;
                    if (chains_[own].ops.size() + grow[own] > kMaxChainOps) fold = false;
                }
            }
            if (!fold && !chains_.empty()) emitted += emit();
            for (uint32_t i = 0; i < tot; i++) {
                if (frame_opcode(ops[i].a >> 24) == OP_COUNT) continue;
                const int own = chain_of(ops[i]);       // -1 after an emit
                const uint32_t q[2] = {op_q0(ops[i]), op_q1(ops[i])};
                int c = own;
                if (c < 0) {
                    c = (int)chains_.size();
                    chains_.push_back(Chain{q[0], {}, {}});
                }
                if (frame_opcode(ops[i].a >> 24) == OP_SX) {
                    // SQRT_X(_DAG) acts on frames as x ^= z, i.e. H S H
                    DevOp h = ops[i], sg = ops[i];
                    h.a = (OP_H << 24) | q[0];
                    sg.a = (OP_S << 24) | q[0];
                    chains_[c].ops.push_back(h);
                    chains_[c].ops.push_back(sg);
                    chains_[c].ops.push_back(h);
                } else {
                    chains_[c].ops.push_back(ops[i]);
                }
                for (uint32_t qq : q) {
                    if (owner_[qq] < 0) {
                        owner_[qq] = c;
                        chains_[c].qs.push_back(qq);
                    }
                }
            }
        }
        if (!chains_.empty()) emitted += emit();
        return emitted;
    }

  private:
    // Chain owning the op's qubits: -1 none, -2 two different chains.
    int chain_of(const DevOp &d) const {
        const int a = owner_[op_q0(d)], b = owner_[op_q1(d)];
        if (a >= 0 && b >= 0 && a != b) return -2;
        return a >= 0 ? a : b;
    }

    const HostProgram &hp_;
    int C_;
    FrameProgram *fp_;
    std::vector<int> owner_;       // qubit -> chain of the open merged layer
    std::vector<Chain> chains_;

    uint32_t ref(uint32_t q) const { return ((q / fp_->Q) << 24) | (q % fp_->Q); }

    DevOp encode(const DevOp &d) const {
        const uint32_t opc = d.a >> 24;
        DevOp f = d;
        f.a = (frame_opcode(opc) << 28) | ref(op_q0(d));
        if (op_is_pair(opc)) {
            f.b = ref(d.b & kQubitMask);
            if (opc == OP_DEP2) f.slot = d.slot | ((d.b >> 24) << 24);
        } else if (op_is_noise(opc)) {
            f.b = d.b >> 24;
        }
        return f;
    }

    uint32_t emit() {
        ProgEntry e{};
        e.kind = ENT_LAYER;
        e.op_begin = (uint32_t)fp_->rank_tab.size();
        uint32_t ng = 0, nn = 0, nc = 0;
        // per rank: chains sorted by opcode signature
        std::vector<std::vector<uint32_t>> by_rank((size_t)C_);
        for (uint32_t i = 0; i < chains_.size(); i++) by_rank[chains_[i].q0 / fp_->Q].push_back(i);
        for (int r = 0; r < C_; r++) {
            fp_->rank_tab.push_back((uint32_t)fp_->segs.size());
            const size_t rank_op0 = fp_->ops.size();
            auto sig_less = [&](uint32_t x, uint32_t y) {
                const auto &a = chains_[x].ops, &b = chains_[y].ops;
                if (a.size() != b.size()) return a.size() < b.size();
                for (size_t j = 0; j < a.size(); j++) {
                    const uint32_t fa = frame_opcode(a[j].a >> 24), fb = frame_opcode(b[j].a >> 24);
                    if (fa != fb) return fa < fb;
                }
                return false;
            };
            std::stable_sort(by_rank[r].begin(), by_rank[r].end(), sig_less);
            size_t i = 0;
            while (i < by_rank[r].size()) {
                size_t j = i + 1;
                while (j < by_rank[r].size() && !sig_less(by_rank[r][i], by_rank[r][j]) &&
                       !sig_less(by_rank[r][j], by_rank[r][i]))
                    j++;
                FrameSeg sg{};
                sg.len = (uint32_t)chains_[by_rank[r][i]].ops.size();
                sg.op_begin = (uint32_t)fp_->ops.size();
                sg.count = (uint32_t)(j - i);
                // first chain step from which only noise ops follow: their
                // error masks commute, so they may be applied after the chain.
                // With a cluster (C > 1) the deferred tail must also name each
                // qubit once: its hits are flushed as one warp-wide
                // red.shared::cluster.xor, which lost updates when two lanes
                // named the same address (a local red.shared.xor does not).
                uint32_t dfrom = 0;
                for (size_t k = i; k < j; k++) {
                    const auto &ops = chains_[by_rank[r][k]].ops;
                    uint32_t d = (uint32_t)ops.size();
                    std::vector<uint32_t> seen;
                    while (d > 0 && op_is_noise(ops[d - 1].a >> 24)) {
                        if (C_ > 1) {
                            const uint32_t qa = op_q0(ops[d - 1]), qb = op_q1(ops[d - 1]);
                            if (std::find(seen.begin(), seen.end(), qa) != seen.end() ||
                                std::find(seen.begin(), seen.end(), qb) != seen.end())
                                break;
                            seen.push_back(qa);
                            if (qb != qa) seen.push_back(qb);
                        }
                        d--;
                    }
                    dfrom = std::max(dfrom, d);
                }
                sg.defer_from = dfrom;
                // step-major: op s of chain k at op_begin + s * count + k, so the
                // lanes of a warp (consecutive chains) read consecutive ops
                for (uint32_t step = 0; step < sg.len; step++)
                    for (size_t k = i; k < j; k++) {
                        const DevOp &d = chains_[by_rank[r][k]].ops[step];
                        fp_->ops.push_back(encode(d));
                        const uint32_t opc = d.a >> 24;
                        if (op_is_gate(opc)) ng++;
                        else if (op_is_noise(opc)) nn++;
                        else nc++;
                    }
                fp_->segs.push_back(sg);
                i = j;
            }
            fp_->max_rank_ops = std::max<uint32_t>(fp_->max_rank_ops, (uint32_t)(fp_->ops.size() - rank_op0));
        }
        fp_->rank_tab.push_back((uint32_t)fp_->segs.size());
        e.n_gate = ng;
        e.n_noise = nn;
        e.n_collapse = nc;
        fp_->prog.push_back(e);
        for (const Chain &ch : chains_)
            for (uint32_t q : ch.qs) owner_[q] = -1;
        chains_.clear();
        return 1;
    }
};

}  // namespace

void build_frame_program(const HostProgram &hp, int C, FrameProgram *out) {
    FrameProgram fp;
    fp.C = C;
    const uint32_t n = hp.num_qubits ? hp.num_qubits : 1;
    fp.Q = (n + (uint32_t)C - 1) / (uint32_t)C;
    fp.ops.reserve(hp.ops.size());
    FrameBuilder fb(hp, C, &fp);
    // Walk the program; runs of consecutive LAYER entries are folded, loop
    // markers are copied (their cross references are rewritten).
    std::vector<size_t> open;            // indices (in fp.prog) of open LOOP_BEGINs
    std::vector<uint64_t> layer_count;   // merged layers emitted inside each open loop
    uint64_t top_layers = 0;
    size_t k = 0;
    while (k < hp.prog.size()) {
        const ProgEntry &e = hp.prog[k];
        if (e.kind == ENT_LAYER) {
            size_t j = k;
            while (j < hp.prog.size() && hp.prog[j].kind == ENT_LAYER) j++;
            const uint32_t m = fb.run(k, j);
            if (layer_count.empty()) top_layers += m;
            else layer_count.back() += m;
            k = j;
            continue;
        }
        if (e.kind == ENT_DETS) {
            fp.prog.push_back(e);       // evaluated between merged layers; indexes HostProgram::det_items
        } else if (e.kind == ENT_LOOP_BEGIN) {
            open.push_back(fp.prog.size());
            layer_count.push_back(0);
            fp.prog.push_back(e);
        } else {
            const size_t b = open.back();
            open.pop_back();
            ProgEntry f = e;
            f.op_begin = (uint32_t)b;
            fp.prog[b].op_begin = (uint32_t)fp.prog.size();
            fp.prog.push_back(f);
            const uint64_t inner = layer_count.back() * e.reps;
            layer_count.pop_back();
            if (layer_count.empty()) top_layers += inner;
            else layer_count.back() += inner;
        }
        k++;
    }
    fp.merged_layers_exec = top_layers;
    *out = std::move(fp);
}

int compile_circuit(const char *text, size_t len, HostProgram *out, std::string *err) {
    try {
        Parser ps(text, len);
        Block root = ps.parse();
        Counts c;
        uint32_t maxq = 0;
        bool any = false;
        count_block(root, &c, &maxq, &any);
        if (c.meas > 0xFFFFFFFFull) throw ParseError{STIM_E_UNSUPPORTED, "more than 2^32 - 1 measurements"};
        if (c.det_entries > (1ull << 34)) throw ParseError{STIM_E_UNSUPPORTED, "detector lists too large"};
        HostProgram hp;
        hp.num_qubits = any ? maxq + 1 : 0;
        hp.num_meas = c.meas;
        hp.num_det = c.det + c.obs;     // detection-event rows: detectors, then observables
        hp.num_obs = c.obs;
        hp.num_gate_targets = c.gate_t;
        hp.num_noise_targets = c.noise_t;
        hp.num_instr = c.instr;
        hp.num_feedforward = c.ff_t;
        for (int k = 0; k < (int)OP_COUNT; k++) hp.exec_targets[k] = c.targets[k];
        hp.det_ptr.reserve(c.det + 1);
        hp.det_ptr.push_back(0);
        hp.det_meas.reserve(c.det_entries);
        uint64_t m = 0;
        std::vector<std::vector<uint32_t>> obs((size_t)c.obs);
        collect_detectors(root, &m, &hp, &obs);
        for (const std::vector<uint32_t> &o : obs) {
            hp.det_meas.insert(hp.det_meas.end(), o.begin(), o.end());
            hp.det_ptr.push_back(hp.det_meas.size());
        }
        // skeleton item by item, with the FNV-1a hash of every prefix
        std::vector<uint64_t> prefix_hash(root.items.size() + 1);
        std::vector<size_t> prefix_len(root.items.size() + 1);
        uint64_t h = 1469598103934665603ull;
        prefix_hash[0] = h;
        prefix_len[0] = 0;
        for (size_t i = 0; i < root.items.size(); i++) {
            const size_t before = hp.skeleton.size();
            skeleton_node(root.items[i], &hp.skeleton);
            h = fnv_words(h, hp.skeleton, before);
            prefix_hash[i + 1] = h;
            prefix_len[i + 1] = hp.skeleton.size();
        }
        hp.skeleton_hash = h;
        Emitter em(&hp, hp.num_qubits ? hp.num_qubits : 1);
        hp.num_layers_exec = em.emit(root, 0, 0, 0, 0);
        hp.ring_len = em.ring_len();
        for (const Emitter::Cut &ct : em.cuts) {
            HostProgram::CutPoint cp{};
            cp.prog_index = ct.prog_index;
            cp.meas = ct.meas;
            cp.prefix_hash = prefix_hash[ct.items_before];
            cp.skeleton_len = prefix_len[ct.items_before];
            cp.loop_begin = ct.loop_begin;
            if (ct.loop_begin != UINT32_MAX) {
                // the same prefix hashed with the block's repetition count (the
                // two words after its opening marker) taken as zero
                const size_t at = prefix_len[ct.items_before - 1];
                uint64_t lh = prefix_hash[ct.items_before - 1];
                std::vector<uint32_t> part(hp.skeleton.begin() + (long)at, hp.skeleton.begin() + (long)cp.skeleton_len);
                part[1] = part[2] = 0;
                cp.loop_hash = fnv_words(lh, part);
                cp.loop_reps = ct.loop_reps;
                cp.loop_meas = ct.loop_meas;
                cp.reps_pos = at + 1;
            }
            hp.cuts.push_back(cp);
        }
        *out = std::move(hp);
        return 0;
    } catch (const ParseError &e) {
        *err = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        *err = "out of host memory while compiling";
        return STIM_E_OOM;
    }
}

}  // namespace stimgb
