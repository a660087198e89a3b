/*
 * oracle.c -- plain, slow CPU oracle for bulk stabilizer-circuit sampling.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library. It shares no source
 * with the CUDA library (its own parser, RNG, tables, tableau and frame code)
 * and it never calls into that library.
 *
 * What it computes, and where the paper defines it:
 *   - circuit text format (Section 5.8): gate lines, broadcast targets,
 *     comments, REPEAT blocks (flattened here);
 *   - Pauli products in the xz encoding and their multiplication with phase
 *     (Section 2.1); written here as a plain per-term phase rule, not the
 *     counter trick of the paper's Pauli-multiplication figure;
 *   - the inverse ("backwards") stabilizer tableau simulator (Section 4,
 *     "Tracking the Tableau"): gates are folded by prepending, measurements
 *     read the Z_q column, random measurements are resolved by appending
 *     CNOTs from a pivot, a single-qubit collapse gate and an X;
 *   - the Pauli frame simulator (Section 3, enumerated steps), one shot at a
 *     time with one byte per qubit per plane;
 *   - detectors as the XOR of measurement flips (Section 5.6); logical
 *     observables (OBSERVABLE_INCLUDE(k) rec[-a] ..., the logical errors of
 *     Section 1 made an output) the same way, accumulated per index over
 *     every instruction naming it and output after the detectors;
 *   - classically controlled Paulis (Section 3, "Tracking Corrections"):
 *     "CX rec[-k] q" applies X to q and "CZ rec[-k] q" Z when measurement
 *     record -k is 1. The tableau applies the Pauli when the reference
 *     outcome is 1; the frame applies it where the shot's record differs
 *     from the reference (the flip bit), which is the correction moved into
 *     the frame.
 *
 * Readings where the paper is silent (the same on the GPU side, defined
 * independently there):
 *   - a random measurement in the reference sample always takes outcome 0
 *     (after the collapse an X is appended on the pivot when the sign is -);
 *   - randomness is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
 *     key = (seed lo, seed hi), counter = (block, slot, tag<<28 | instr,
 *     64-shot word); tags NOISE=0, COLLAPSE=1, INIT=2;
 *   - noise masks use an exact integer geometric-gap procedure (Section 5.4's
 *     geometric sampling of gaps, made exact): t = round-half-even(p * 2^32),
 *     S_0 = 2^32, S_{k+1} = floor(S_k (2^32 - t) / 2^32), G[k] = 2^32 - S_{k+1};
 *   - DEPOLARIZE1 picks X, Y, Z uniformly; DEPOLARIZE2 one of the 15
 *     non-identity two-qubit Paulis uniformly;
 *   - PAULI_CHANNEL_1(px, py, pz) and PAULI_CHANNEL_2(p_IX, ..., p_ZZ) (the
 *     15 pair Paulis in the order IX, IY, IZ, XI, ..., ZZ) hit with the total
 *     probability p (gap sampling as above) and pick the Pauli of each hit
 *     by a fresh draw against the cumulative thresholds
 *     round-half-even(2^32 * partial sum / p).
 *
 * Parity unpinned: which Philox draw feeds which shot bit (the keying above)
 * is a convention of this implementation, not the paper's; Philox itself, the
 * geometric tables and every noise distribution are pinned, the exact bit
 * pattern of the keying only by agreement with the GPU path.
 */
#include <math.h>
#include <pthread.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Gate set                                                                  */
/* ------------------------------------------------------------------------ */
enum {
    OG_H, OG_S, OG_CX, OG_CZ, OG_M, OG_MR, OG_R,
    OG_XERR, OG_ZERR, OG_DEP1, OG_DEP2, OG_DET, OG_X,
    /* wider gate set */
    OG_Y, OG_Z, OG_SDAG, OG_SQX, OG_SQXD, OG_SQY, OG_SQYD, OG_YERR,
    OG_MX, OG_MY, OG_MRX, OG_MRY, OG_RX, OG_RY,
    OG_OBS,             /* OBSERVABLE_INCLUDE(k) rec[-a] ... */
    OG_PC1, OG_PC2      /* PAULI_CHANNEL_1(px, py, pz), PAULI_CHANNEL_2(p_IX, ..., p_ZZ) */
};

typedef struct {
    int gate;
    double p;
    uint32_t nt;
    uint32_t *t;        /* qubits, or absolute measurement indices (DETECTOR, OBSERVABLE_INCLUDE) */
    uint64_t G[64];     /* geometric table (noise ops only) */
    uint64_t C[15];     /* Pauli channels: cumulative choice thresholds */
} orc_op;

typedef struct {
    uint32_t n;         /* qubits */
    uint64_t nmeas, ndet, ngate_targets, nnoise_targets;
    uint64_t nobs;      /* observables: largest OBSERVABLE_INCLUDE index + 1 */
    size_t nops, cap;
    orc_op *ops;        /* flattened: ops[i] has instruction ordinal i */
} orc_circuit;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the SC'11 definition                                   */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { TAG_NOISE = 0, TAG_COLLAPSE = 1, TAG_INIT = 2 };

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    uint32_t j;         /* index of the next draw */
} drawer;

static void drawer_init(drawer *d, uint64_t seed, uint32_t tag, uint32_t instr,
                        uint32_t slot, uint64_t word) {
    d->key[0] = (uint32_t)seed;
    d->key[1] = (uint32_t)(seed >> 32);
    d->ctr[0] = 0;
    d->ctr[1] = slot;
    d->ctr[2] = (tag << 28) | instr;
    d->ctr[3] = (uint32_t)word;
    d->j = 0;
}

static uint32_t drawer_next(drawer *d) {
    if (d->j % 4 == 0) {
        d->ctr[0] = d->j / 4;
        orc_philox(d->ctr, d->key, d->buf);
    }
    uint32_t v = d->buf[d->j % 4];
    d->j++;
    return v;
}

/* 64 random bits with probability exactly 1/2 each: draws 0 and 1. */
static uint64_t half_mask(uint64_t seed, uint32_t tag, uint32_t instr, uint32_t slot,
                          uint64_t word) {
    drawer d;
    drawer_init(&d, seed, tag, instr, slot, word);
    uint64_t lo = drawer_next(&d);
    uint64_t hi = drawer_next(&d);
    return lo | (hi << 32);
}

uint64_t orc_half_mask(uint64_t seed, uint32_t tag, uint32_t instr, uint32_t slot,
                       uint64_t word) {
    return half_mask(seed, tag, instr, slot, word);
}

/* ------------------------------------------------------------------------ */
/* Exact geometric table                                                      */
/* ------------------------------------------------------------------------ */
void orc_geo_table(double p, uint64_t G[64]) {
    const unsigned __int128 two32 = (unsigned __int128)1 << 32;
    long long t = llrint(ldexp(p, 32));
    if (t < 0) t = 0;
    if (t > (1LL << 32)) t = 1LL << 32;
    unsigned __int128 S = two32;
    for (int k = 0; k < 64; k++) {
        S = (S * (two32 - (unsigned __int128)t)) >> 32;
        G[k] = (uint64_t)(two32 - S);
    }
}

static int gap_of(const uint64_t G[64], uint32_t u) {
    for (int k = 0; k < 64; k++)
        if ((uint64_t)u < G[k]) return k;
    return 64;
}

/* Effect of one noise op slot on the 64 shots of one word.
 * x0/z0 act on the first (or only) qubit, x1/z1 on the second. */
typedef struct { uint64_t x0, z0, x1, z1; } noise_word;

/* Pauli channels: 1 + the number of cumulative thresholds C[i] <= v, i.e.
 * the index (1 X, 2 Y, 3 Z; or 4a + b for the pair Pauli (a, b)) of the
 * probability interval that holds the draw v. */
static uint32_t channel_pick(const uint64_t C[15], int m, uint32_t v) {
    uint32_t c = 1;
    for (int i = 0; i < m - 1; i++)
        if ((uint64_t)v >= C[i]) c++;
    return c;
}

static noise_word noise_for_word(uint64_t seed, int gate, const uint64_t G[64], const uint64_t *C,
                                 uint32_t instr, uint32_t slot, uint64_t word) {
    noise_word r = {0, 0, 0, 0};
    drawer d;
    drawer_init(&d, seed, TAG_NOISE, instr, slot, word);
    int pos = -1;
    for (;;) {
        uint32_t u = drawer_next(&d);
        pos += gap_of(G, u) + 1;
        if (pos >= 64) break;
        uint64_t bit = (uint64_t)1 << pos;
        if (gate == OG_XERR) {
            r.x0 |= bit;
        } else if (gate == OG_ZERR) {
            r.z0 |= bit;
        } else if (gate == OG_YERR) {
            r.x0 |= bit;
            r.z0 |= bit;
        } else if (gate == OG_DEP1 || gate == OG_PC1) {
            uint32_t v = drawer_next(&d);
            uint32_t pa = gate == OG_DEP1 ? 1 + (uint32_t)(((uint64_t)3 * v) >> 32)   /* 1 X, 2 Y, 3 Z */
                                          : channel_pick(C, 3, v);
            if (pa == 1 || pa == 2) r.x0 |= bit;
            if (pa == 2 || pa == 3) r.z0 |= bit;
        } else { /* DEP2, PC2 */
            uint32_t v = drawer_next(&d);
            uint32_t c = gate == OG_DEP2 ? 1 + (uint32_t)(((uint64_t)15 * v) >> 32) : channel_pick(C, 15, v);
            uint32_t pa = c >> 2, pb = c & 3;                 /* 0 I, 1 X, 2 Y, 3 Z */
            if (pa == 1 || pa == 2) r.x0 |= bit;
            if (pa == 2 || pa == 3) r.z0 |= bit;
            if (pb == 1 || pb == 2) r.x1 |= bit;
            if (pb == 2 || pb == 3) r.z1 |= bit;
        }
    }
    return r;
}

/* Exposed for tests: the four masks of one (noise op, slot, word). */
void orc_noise_word(uint64_t seed, int gate, double p, uint32_t instr, uint32_t slot,
                    uint64_t word, uint64_t out[4]) {
    uint64_t G[64];
    orc_geo_table(p, G);
    noise_word r = {0, 0, 0, 0};
    if (p > 0) r = noise_for_word(seed, gate, G, NULL, instr, slot, word);
    out[0] = r.x0; out[1] = r.z0; out[2] = r.x1; out[3] = r.z1;
}

/* ------------------------------------------------------------------------ */
/* Parser (flattens REPEAT)                                                   */
/* ------------------------------------------------------------------------ */
typedef struct node node;
struct node {
    int is_block;
    uint64_t reps;
    /* leaf */
    int gate;
    double p;
    double args[15];  /* every parenthesised argument (Pauli channels) */
    int nargs;
    uint32_t nt;
    uint32_t *t;      /* qubits, or lookbacks k of rec[-k] */
    /* block */
    node *kids;
    size_t nkids, capkids;
};

typedef struct {
    const char *s;
    size_t len, pos;
    int line;
    char *err;
    size_t errlen;
} pstate;

static int perr(pstate *ps, const char *fmt, ...) {
    if (ps->err && ps->errlen) {
        int k = snprintf(ps->err, ps->errlen, "line %d: ", ps->line);
        if (k < 0) k = 0;
        if ((size_t)k < ps->errlen) {
            va_list ap;
            va_start(ap, fmt);
            vsnprintf(ps->err + k, ps->errlen - (size_t)k, fmt, ap);
            va_end(ap);
        }
    }
    return -1;
}

static node *add_kid(node *b) {
    if (b->nkids == b->capkids) {
        b->capkids = b->capkids ? 2 * b->capkids : 8;
        b->kids = (node *)realloc(b->kids, b->capkids * sizeof(node));
    }
    node *k = &b->kids[b->nkids++];
    memset(k, 0, sizeof(*k));
    return k;
}

static void free_node(node *b) {
    if (b->is_block) {
        for (size_t i = 0; i < b->nkids; i++) free_node(&b->kids[i]);
        free(b->kids);
    } else {
        free(b->t);
    }
}

static int gate_from_name(const char *w, size_t n) {
#define IS(lit) (n == strlen(lit) && strncmp(w, lit, n) == 0)
    if (IS("H")) return OG_H;
    if (IS("S")) return OG_S;
    if (IS("CX") || IS("CNOT")) return OG_CX;
    if (IS("CZ")) return OG_CZ;
    if (IS("M")) return OG_M;
    if (IS("MR")) return OG_MR;
    if (IS("R")) return OG_R;
    if (IS("X_ERROR")) return OG_XERR;
    if (IS("Z_ERROR")) return OG_ZERR;
    if (IS("DEPOLARIZE1")) return OG_DEP1;
    if (IS("DEPOLARIZE2")) return OG_DEP2;
    if (IS("DETECTOR")) return OG_DET;
    if (IS("OBSERVABLE_INCLUDE")) return OG_OBS;
    if (IS("PAULI_CHANNEL_1")) return OG_PC1;
    if (IS("PAULI_CHANNEL_2")) return OG_PC2;
    if (IS("X")) return OG_X;
    if (IS("Y")) return OG_Y;
    if (IS("Z")) return OG_Z;
    if (IS("S_DAG")) return OG_SDAG;
    if (IS("SQRT_X")) return OG_SQX;
    if (IS("SQRT_X_DAG")) return OG_SQXD;
    if (IS("SQRT_Y")) return OG_SQY;
    if (IS("SQRT_Y_DAG")) return OG_SQYD;
    if (IS("Y_ERROR")) return OG_YERR;
    if (IS("MX")) return OG_MX;
    if (IS("MY")) return OG_MY;
    if (IS("MRX")) return OG_MRX;
    if (IS("MRY")) return OG_MRY;
    if (IS("RX")) return OG_RX;
    if (IS("RY")) return OG_RY;
#undef IS
    return -1;
}

/* A CX/CZ target with this bit set is a measurement record (the control of a
 * classically controlled Pauli): lookback k while parsing, absolute index
 * after flattening. */
#define REC_FLAG 0x80000000u

static int is_noise(int g) {
    return g == OG_XERR || g == OG_ZERR || g == OG_DEP1 || g == OG_DEP2 || g == OG_YERR || g == OG_PC1 || g == OG_PC2;
}
static int is_1q_gate(int g) {
    return g == OG_H || g == OG_S || g == OG_X || g == OG_Y || g == OG_Z || g == OG_SDAG || g == OG_SQX ||
           g == OG_SQXD || g == OG_SQY || g == OG_SQYD;
}
/* Collapsing ops: basis (0 Z, 1 X, 2 Y) and kind (0 M, 1 MR, 2 R). */
static int collapse_basis(int g) {
    return (g == OG_MX || g == OG_MRX || g == OG_RX) ? 1 : (g == OG_MY || g == OG_MRY || g == OG_RY) ? 2 : 0;
}
static int collapse_kind(int g) {
    return (g == OG_M || g == OG_MX || g == OG_MY) ? 0 : (g == OG_MR || g == OG_MRX || g == OG_MRY) ? 1 : 2;
}
static int is_collapse(int g) {
    return g == OG_M || g == OG_MR || g == OG_R || g == OG_MX || g == OG_MY || g == OG_MRX || g == OG_MRY ||
           g == OG_RX || g == OG_RY;
}
static int is_pair(int g) { return g == OG_CX || g == OG_CZ || g == OG_DEP2 || g == OG_PC2; }

/* Parse one line [b, e) into node k. */
static int parse_line(pstate *ps, const char *b, const char *e, node *k) {
    const char *p = b;
    const char *w = p;
    while (p < e && (((*p >= 'A') && (*p <= 'Z')) || (*p >= '0' && *p <= '9') || *p == '_')) p++;
    int g = gate_from_name(w, (size_t)(p - w));
    if (g < 0) return perr(ps, "unknown gate '%.*s'", (int)(p - w), w);
    k->gate = g;
    k->p = 0;
    int nargs = 0;
    if (p < e && *p == '(') {
        p++;
        for (;;) {
            while (p < e && (*p == ' ' || *p == '\t')) p++;
            char *endp;
            char buf[64];
            size_t m = 0;
            while (p + m < e && p[m] != ',' && p[m] != ')' && m < sizeof(buf) - 1) { buf[m] = p[m]; m++; }
            buf[m] = 0;
            double v = strtod(buf, &endp);
            while (*endp == ' ' || *endp == '\t') endp++;
            if (endp == buf || *endp) return perr(ps, "bad argument");
            if (nargs == 0) k->p = v;
            if (nargs < 15) k->args[nargs] = v;
            nargs++;
            p += m;
            if (p < e && *p == ',') { p++; continue; }
            if (p < e && *p == ')') { p++; break; }
            return perr(ps, "unterminated argument list");
        }
    }
    k->nargs = nargs;
    if (g == OG_PC1 || g == OG_PC2) {
        /* the channel's total probability is the left-to-right sum of its arguments */
        int want = g == OG_PC1 ? 3 : 15;
        if (nargs != want) return perr(ps, "Pauli channel takes %d probabilities", want);
        double sum = 0;
        for (int i = 0; i < want; i++) {
            if (!(k->args[i] >= 0.0 && k->args[i] <= 1.0)) return perr(ps, "probability outside [0, 1]");
            sum += k->args[i];
        }
        if (!(sum <= 1.0)) return perr(ps, "Pauli channel probabilities sum above 1");
        k->p = sum;
    } else if (is_noise(g)) {
        if (nargs != 1) return perr(ps, "noise channel takes one probability");
        if (!(k->p >= 0.0 && k->p <= 1.0)) return perr(ps, "probability outside [0, 1]");
    } else if (g == OG_OBS) {
        if (nargs != 1) return perr(ps, "OBSERVABLE_INCLUDE takes one index");
        if (!(k->p >= 0.0 && k->p < 65536.0) || k->p != floor(k->p)) return perr(ps, "bad observable index");
    } else if (g != OG_DET && nargs != 0) {
        return perr(ps, "gate takes no arguments");
    }
    size_t cap = 8;
    k->t = (uint32_t *)malloc(cap * sizeof(uint32_t));
    k->nt = 0;
    for (;;) {
        while (p < e && (*p == ' ' || *p == '\t')) p++;
        if (p >= e) break;
        uint64_t v = 0;
        if ((g == OG_CX || g == OG_CZ) && e - p >= 6 && strncmp(p, "rec[-", 5) == 0) {
            /* classically controlled Pauli: the control is a measurement record */
            p += 5;
            if (p >= e || *p < '0' || *p > '9') return perr(ps, "expected rec[-k]");
            while (p < e && *p >= '0' && *p <= '9') { v = v * 10 + (uint64_t)(*p - '0'); if (v >= REC_FLAG) return perr(ps, "lookback too large"); p++; }
            if (p >= e || *p != ']') return perr(ps, "expected ]");
            p++;
            if (v == 0) return perr(ps, "rec[-0] is not a measurement");
            v |= REC_FLAG;
        } else if (g == OG_DET || g == OG_OBS) {
            if (e - p < 6 || strncmp(p, "rec[-", 5) != 0) return perr(ps, "expected rec[-k]");
            p += 5;
            if (p >= e || *p < '0' || *p > '9') return perr(ps, "expected rec[-k]");
            while (p < e && *p >= '0' && *p <= '9') { v = v * 10 + (uint64_t)(*p - '0'); if (v > 0xffffffffu) return perr(ps, "lookback too large"); p++; }
            if (p >= e || *p != ']') return perr(ps, "expected ]");
            p++;
            if (v == 0) return perr(ps, "rec[-0] is not a measurement");
        } else {
            if (*p < '0' || *p > '9') return perr(ps, "bad target");
            while (p < e && *p >= '0' && *p <= '9') { v = v * 10 + (uint64_t)(*p - '0'); if (v >= (1u << 24)) return perr(ps, "qubit index too large"); p++; }
        }
        if (p < e && *p != ' ' && *p != '\t') return perr(ps, "bad target");
        if (k->nt == cap) { cap *= 2; k->t = (uint32_t *)realloc(k->t, cap * sizeof(uint32_t)); }
        k->t[k->nt++] = (uint32_t)v;
    }
    if (is_pair(g)) {
        if (k->nt % 2) return perr(ps, "two-qubit gate needs an even number of targets");
        for (uint32_t i = 0; i < k->nt; i += 2) {
            if (k->t[i] == k->t[i + 1]) return perr(ps, "two-qubit gate on one qubit");
            if ((k->t[i] & REC_FLAG) && (k->t[i + 1] & REC_FLAG)) return perr(ps, "two measurement records in a pair");
            if (g == OG_CX && (k->t[i + 1] & REC_FLAG)) return perr(ps, "CX takes a measurement record only as control");
        }
    }
    return 0;
}

static int parse_block(pstate *ps, node *blk, int depth) {
    while (ps->pos < ps->len) {
        const char *b = ps->s + ps->pos;
        const char *nl = memchr(b, '\n', ps->len - ps->pos);
        const char *e = nl ? nl : ps->s + ps->len;
        ps->pos = (size_t)(e - ps->s) + (nl ? 1 : 0);
        ps->line++;
        const char *h = memchr(b, '#', (size_t)(e - b));
        if (h) e = h;
        while (b < e && (*b == ' ' || *b == '\t' || *b == '\r')) b++;
        while (e > b && (e[-1] == ' ' || e[-1] == '\t' || e[-1] == '\r')) e--;
        if (b == e) continue;
        if (*b == '}') {
            if (e - b != 1) return perr(ps, "junk after }");
            if (depth == 0) return perr(ps, "unmatched }");
            return 1;
        }
        if (e - b > 7 && strncmp(b, "REPEAT", 6) == 0 && (b[6] == ' ' || b[6] == '\t')) {
            const char *p = b + 6;
            while (p < e && (*p == ' ' || *p == '\t')) p++;
            uint64_t reps = 0;
            if (p >= e || *p < '0' || *p > '9') return perr(ps, "bad REPEAT count");
            while (p < e && *p >= '0' && *p <= '9') { reps = reps * 10 + (uint64_t)(*p - '0'); if (reps > 1000000000ull) return perr(ps, "REPEAT count too large"); p++; }
            while (p < e && (*p == ' ' || *p == '\t')) p++;
            if (p >= e || *p != '{' || p + 1 != e) return perr(ps, "expected { after REPEAT count");
            if (reps == 0) return perr(ps, "REPEAT 0");
            node *k = add_kid(blk);
            k->is_block = 1;
            k->reps = reps;
            int r = parse_block(ps, k, depth + 1);
            if (r < 0) return r;
            if (r == 0) return perr(ps, "unterminated REPEAT block");
            continue;
        }
        node *k = add_kid(blk);
        if (parse_line(ps, b, e, k) < 0) return -1;
    }
    return 0;
}

static orc_op *push_op(orc_circuit *c) {
    if (c->nops == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 64;
        c->ops = (orc_op *)realloc(c->ops, c->cap * sizeof(orc_op));
    }
    orc_op *o = &c->ops[c->nops++];
    memset(o, 0, sizeof(*o));
    return o;
}

/* Choice thresholds of a Pauli channel with probabilities q_1..q_m (m = 3 or
 * 15) and total p: C[i] = round-half-even(2^32 (q_1 + ... + q_{i+1}) / p)
 * for i < m - 1 (sums taken left to right in double precision), unused
 * entries 2^32. A hit takes Pauli 1 + #{i : v >= C[i]} for a fresh draw v,
 * so Pauli j has probability q_j / p up to 2^-32 rounding. */
static void pauli_channel_thresholds(const node *k, uint64_t C[15]) {
    const int m = k->gate == OG_PC1 ? 3 : 15;
    double sum = 0;
    for (int i = 0; i < 15; i++) C[i] = (uint64_t)1 << 32;
    if (!(k->p > 0)) return;
    for (int i = 0; i < m - 1; i++) {
        sum += k->args[i];
        long long t = llrint(ldexp(sum / k->p, 32));
        if (t < 0) t = 0;
        if (t > (1LL << 32)) t = 1LL << 32;
        C[i] = (uint64_t)t;
    }
}

static int flatten(pstate *ps, const node *blk, orc_circuit *c) {
    for (size_t i = 0; i < blk->nkids; i++) {
        const node *k = &blk->kids[i];
        if (k->is_block) {
            for (uint64_t r = 0; r < k->reps; r++)
                if (flatten(ps, k, c) < 0) return -1;
            continue;
        }
        if (c->nops >= (1u << 28)) return perr(ps, "too many instructions");
        orc_op *o = push_op(c);
        o->gate = k->gate;
        o->p = k->p;
        o->nt = k->nt;
        o->t = (uint32_t *)malloc((k->nt ? k->nt : 1) * sizeof(uint32_t));
        if (k->gate == OG_DET || k->gate == OG_OBS) {
            for (uint32_t j = 0; j < k->nt; j++) {
                if ((uint64_t)k->t[j] > c->nmeas) return perr(ps, "rec[-%u] reaches before the first measurement", k->t[j]);
                o->t[j] = (uint32_t)(c->nmeas - k->t[j]);
            }
            if (k->gate == OG_DET) c->ndet++;
            else if ((uint64_t)k->p + 1 > c->nobs) c->nobs = (uint64_t)k->p + 1;
        } else {
            memcpy(o->t, k->t, k->nt * sizeof(uint32_t));
            for (uint32_t j = 0; j < k->nt; j++) {
                if (k->t[j] & REC_FLAG) {      /* rec[-k] -> absolute measurement index */
                    uint32_t back = k->t[j] & ~REC_FLAG;
                    if ((uint64_t)back > c->nmeas) return perr(ps, "rec[-%u] reaches before the first measurement", back);
                    o->t[j] = REC_FLAG | (uint32_t)(c->nmeas - back);
                    continue;
                }
                if (k->t[j] + 1 > c->n) c->n = k->t[j] + 1;
            }
            uint64_t slots = is_pair(k->gate) ? k->nt / 2 : k->nt;
            if (is_noise(k->gate)) {
                c->nnoise_targets += slots;
                orc_geo_table(k->p, o->G);
                if (k->gate == OG_PC1 || k->gate == OG_PC2) pauli_channel_thresholds(k, o->C);
            } else {
                c->ngate_targets += slots;
            }
            if (is_collapse(k->gate) && collapse_kind(k->gate) != 2) c->nmeas += k->nt;
        }
    }
    return 0;
}

void orc_free(orc_circuit *c) {
    if (!c) return;
    for (size_t i = 0; i < c->nops; i++) free(c->ops[i].t);
    free(c->ops);
    free(c);
}

int orc_parse(const char *text, orc_circuit **out, char *err, size_t errlen) {
    pstate ps = {text, strlen(text), 0, 0, err, errlen};
    if (err && errlen) err[0] = 0;
    node root;
    memset(&root, 0, sizeof(root));
    root.is_block = 1;
    int r = parse_block(&ps, &root, 0);
    if (r != 0) {
        free_node(&root);
        if (r > 0) perr(&ps, "unmatched }");
        return -1;
    }
    orc_circuit *c = (orc_circuit *)calloc(1, sizeof(orc_circuit));
    if (flatten(&ps, &root, c) < 0) {
        free_node(&root);
        orc_free(c);
        return -1;
    }
    free_node(&root);
    *out = c;
    return 0;
}

/* n, M, D, gate targets, noise targets, instructions, observables */
void orc_info(const orc_circuit *c, uint64_t out[7]) {
    out[0] = c->n;
    out[1] = c->nmeas;
    out[2] = c->ndet;
    out[3] = c->ngate_targets;
    out[4] = c->nnoise_targets;
    out[5] = c->nops;
    out[6] = c->nobs;
}

/* ------------------------------------------------------------------------ */
/* Gate conjugation tables: image of each generator under G^dagger g G        */
/* ------------------------------------------------------------------------ */
/* A small Pauli on <= 2 qubits: bit 2*q of x/z for local qubit q; sign. */
typedef struct { uint8_t x, z, sign; } spauli;

/* Images of generators in order X_a, Z_a, X_b, Z_b. */
static int gate_images(int g, spauli img[4]) {
    memset(img, 0, 4 * sizeof(spauli));
    switch (g) {
    case OG_H:  /* X -> Z, Z -> X */
        img[0] = (spauli){0, 1, 0};
        img[1] = (spauli){1, 0, 0};
        return 1;
    case OG_S:  /* X -> -Y, Z -> Z */
        img[0] = (spauli){1, 1, 1};
        img[1] = (spauli){0, 1, 0};
        return 1;
    case OG_X:  /* X -> X, Z -> -Z */
        img[0] = (spauli){1, 0, 0};
        img[1] = (spauli){0, 1, 1};
        return 1;
    case OG_Y:  /* X -> -X, Z -> -Z */
        img[0] = (spauli){1, 0, 1};
        img[1] = (spauli){0, 1, 1};
        return 1;
    case OG_Z:  /* X -> -X, Z -> Z */
        img[0] = (spauli){1, 0, 1};
        img[1] = (spauli){0, 1, 0};
        return 1;
    case OG_SDAG:  /* X -> Y, Z -> Z */
        img[0] = (spauli){1, 1, 0};
        img[1] = (spauli){0, 1, 0};
        return 1;
    case OG_SQX:   /* X -> X, Z -> Y */
        img[0] = (spauli){1, 0, 0};
        img[1] = (spauli){1, 1, 0};
        return 1;
    case OG_SQXD:  /* X -> X, Z -> -Y */
        img[0] = (spauli){1, 0, 0};
        img[1] = (spauli){1, 1, 1};
        return 1;
    case OG_SQY:   /* X -> Z, Z -> -X */
        img[0] = (spauli){0, 1, 0};
        img[1] = (spauli){1, 0, 1};
        return 1;
    case OG_SQYD:  /* X -> -Z, Z -> X */
        img[0] = (spauli){0, 1, 1};
        img[1] = (spauli){1, 0, 0};
        return 1;
    case OG_CX: /* X_a -> X_a X_b, Z_a -> Z_a, X_b -> X_b, Z_b -> Z_a Z_b */
        img[0] = (spauli){1 | 2, 0, 0};
        img[1] = (spauli){0, 1, 0};
        img[2] = (spauli){2, 0, 0};
        img[3] = (spauli){0, 1 | 2, 0};
        return 2;
    case OG_CZ: /* X_a -> X_a Z_b, Z_a -> Z_a, X_b -> Z_a X_b, Z_b -> Z_b */
        img[0] = (spauli){1, 2, 0};
        img[1] = (spauli){0, 1, 0};
        img[2] = (spauli){2, 1, 0};
        img[3] = (spauli){0, 2, 0};
        return 2;
    }
    return 0;
}

/* Phase exponent (power of i) of the single-term product s(x1,z1) s(x2,z2),
 * where s(1,0)=X, s(1,1)=Y, s(0,1)=Z. Plain case table:
 * XY=iZ, YZ=iX, ZX=iY give +1; YX=-iZ, ZY=-iX, XZ=-iY give -1 (i.e. 3). */
static int term_phase(int x1, int z1, int x2, int z2) {
    int a = x1 ? (z1 ? 2 : 1) : (z1 ? 3 : 0);   /* 0 I, 1 X, 2 Y, 3 Z */
    int b = x2 ? (z2 ? 2 : 1) : (z2 ? 3 : 0);
    if (a == 0 || b == 0 || a == b) return 0;
    if ((a == 1 && b == 2) || (a == 2 && b == 3) || (a == 3 && b == 1)) return 1;
    return 3;
}

/* Conjugate a local Pauli (x, z bits on k qubits; phase as power of i) by a
 * gate: the product of the images of X_q^x Z_q^z with Y = i X Z. */
static void conj_local(const spauli img[4], int k, uint8_t x, uint8_t z,
                       uint8_t *ox, uint8_t *oz, int *ophase) {
    int ph = 0;
    uint8_t rx = 0, rz = 0;
    for (int q = 0; q < k; q++) {
        int xq = (x >> q) & 1, zq = (z >> q) & 1;
        if (xq && zq) ph += 1;    /* Y = i X Z */
        for (int which = 0; which < 2; which++) {
            int present = which == 0 ? xq : zq;
            if (!present) continue;
            const spauli *m = &img[2 * q + which];
            for (int r = 0; r < k; r++)
                ph += term_phase((rx >> r) & 1, (rz >> r) & 1, (m->x >> r) & 1, (m->z >> r) & 1);
            rx ^= m->x;
            rz ^= m->z;
            ph += 2 * m->sign;
        }
    }
    *ox = rx;
    *oz = rz;
    *ophase = ph & 3;
}

/* Exposed for tests: image of local Pauli (x, z) under gate g; returns the
 * power of i of the resulting (Hermitian-form) product. */
int orc_conj_local(int g, int x, int z, int *ox, int *oz) {
    spauli img[4];
    int k = gate_images(g, img);
    uint8_t rx, rz;
    int ph;
    conj_local(img, k, (uint8_t)x, (uint8_t)z, &rx, &rz, &ph);
    *ox = rx;
    *oz = rz;
    return ph;
}

/* ------------------------------------------------------------------------ */
/* Full Pauli strings and the inverse tableau                                 */
/* ------------------------------------------------------------------------ */
static int popc(uint64_t v) { return __builtin_popcountll(v); }

/* dst := dst * src (both Hermitian-form strings over nw words); returns the
 * power of i picked up by the term products. */
static int string_mul(uint64_t *dx, uint64_t *dz, const uint64_t *sx, const uint64_t *sz, size_t nw) {
    int plus = 0, minus = 0;
    for (size_t w = 0; w < nw; w++) {
        uint64_t x1 = dx[w], z1 = dz[w], x2 = sx[w], z2 = sz[w];
        uint64_t X1 = x1 & ~z1, Y1 = x1 & z1, Z1 = ~x1 & z1;
        uint64_t X2 = x2 & ~z2, Y2 = x2 & z2, Z2 = ~x2 & z2;
        plus += popc((X1 & Y2) | (Y1 & Z2) | (Z1 & X2));
        minus += popc((Y1 & X2) | (Z1 & Y2) | (X1 & Z2));
        dx[w] = x1 ^ x2;
        dz[w] = z1 ^ z2;
    }
    return ((plus - minus) % 4 + 4) % 4;
}

int orc_string_mul(size_t nw, uint64_t *dx, uint64_t *dz, const uint64_t *sx, const uint64_t *sz) {
    return string_mul(dx, dz, sx, sz, nw);
}

/* The tableau is stored column-major (column c = the n-term image of its
 * generator) while gates are folded, and row-major (row r = term r of every
 * column) during bursts of random measurements, as the paper's Section 5.1
 * describes: prepending is a column operation, the appends of the random-
 * measurement elimination are row operations. */
typedef struct {
    uint32_t n;
    size_t nw;         /* words per column (n rows) */
    size_t cw;         /* words per row (2n columns) */
    int rows;          /* 1 while the data lives in rx / rz / rs */
    uint64_t *x;       /* [2n][nw]: column 2q = image of X_q, 2q+1 = image of Z_q */
    uint64_t *z;
    uint8_t *sign;     /* [2n] */
    uint64_t *rx;      /* [n][cw] */
    uint64_t *rz;
    uint64_t *rs;      /* [cw] sign bits */
} tableau;

#define TX(T, c) ((T)->x + (size_t)(c) * (T)->nw)
#define TZ(T, c) ((T)->z + (size_t)(c) * (T)->nw)
#define RX(T, r) ((T)->rx + (size_t)(r) * (T)->cw)
#define RZ(T, r) ((T)->rz + (size_t)(r) * (T)->cw)
#define GETB(a, q) ((int)(((a)[(q) >> 6] >> ((q) & 63)) & 1))
#define FLIPB(a, q) ((a)[(q) >> 6] ^= (uint64_t)1 << ((q) & 63))
#define SETB(a, q, v) ((a)[(q) >> 6] = ((a)[(q) >> 6] & ~((uint64_t)1 << ((q) & 63))) | ((uint64_t)(v) << ((q) & 63)))

static int tableau_init(tableau *T, uint32_t n) {
    T->n = n;
    T->nw = (n + 63) / 64;
    if (T->nw == 0) T->nw = 1;
    T->cw = (2 * (size_t)n + 63) / 64;
    if (T->cw == 0) T->cw = 1;
    T->rows = 0;
    size_t words = (size_t)2 * n * T->nw;
    size_t rwords = (size_t)n * T->cw;
    T->x = (uint64_t *)calloc(words ? words : 1, sizeof(uint64_t));
    T->z = (uint64_t *)calloc(words ? words : 1, sizeof(uint64_t));
    T->sign = (uint8_t *)calloc(2 * (size_t)n + 1, 1);
    T->rx = (uint64_t *)calloc(rwords ? rwords : 1, sizeof(uint64_t));
    T->rz = (uint64_t *)calloc(rwords ? rwords : 1, sizeof(uint64_t));
    T->rs = (uint64_t *)calloc(T->cw, sizeof(uint64_t));
    if (!T->x || !T->z || !T->sign || !T->rx || !T->rz || !T->rs) return -1;
    for (uint32_t q = 0; q < n; q++) {
        FLIPB(TX(T, 2 * q), q);
        FLIPB(TZ(T, 2 * q + 1), q);
    }
    return 0;
}

static void tableau_free(tableau *T) {
    free(T->x);
    free(T->z);
    free(T->sign);
    free(T->rx);
    free(T->rz);
    free(T->rs);
}

static void to_rows(tableau *T) {
    if (T->rows) return;
    memset(T->rx, 0, (size_t)T->n * T->cw * sizeof(uint64_t));
    memset(T->rz, 0, (size_t)T->n * T->cw * sizeof(uint64_t));
    memset(T->rs, 0, T->cw * sizeof(uint64_t));
    for (uint32_t c = 0; c < 2 * T->n; c++) {
        for (size_t w = 0; w < T->nw; w++) {
            uint64_t v = TX(T, c)[w];
            while (v) { FLIPB(RX(T, w * 64 + (size_t)__builtin_ctzll(v)), c); v &= v - 1; }
            v = TZ(T, c)[w];
            while (v) { FLIPB(RZ(T, w * 64 + (size_t)__builtin_ctzll(v)), c); v &= v - 1; }
        }
        if (T->sign[c]) FLIPB(T->rs, c);
    }
    T->rows = 1;
}

static void to_cols(tableau *T) {
    if (!T->rows) return;
    memset(T->x, 0, (size_t)2 * T->n * T->nw * sizeof(uint64_t));
    memset(T->z, 0, (size_t)2 * T->n * T->nw * sizeof(uint64_t));
    for (uint32_t r = 0; r < T->n; r++) {
        for (size_t w = 0; w < T->cw; w++) {
            uint64_t v = RX(T, r)[w];
            while (v) { FLIPB(TX(T, w * 64 + (size_t)__builtin_ctzll(v)), r); v &= v - 1; }
            v = RZ(T, r)[w];
            while (v) { FLIPB(TZ(T, w * 64 + (size_t)__builtin_ctzll(v)), r); v &= v - 1; }
        }
    }
    for (uint32_t c = 0; c < 2 * T->n; c++) T->sign[c] = (uint8_t)GETB(T->rs, c);
    T->rows = 0;
}


static void set_sign(tableau *T, uint32_t c, int v) {
    if (T->rows) SETB(T->rs, c, v);
    else T->sign[c] = (uint8_t)v;
}

/* Prepend (fold) gate g on qubits q[0..k): new column for generator h is
 * T(g^dagger h g), built as a product of old columns. */
static void tableau_prepend(tableau *T, int g, const uint32_t *q, uint64_t *tmpx, uint64_t *tmpz,
                            uint8_t *tmps) {
    spauli img[4];
    int k = gate_images(g, img);
    size_t nw = T->nw;
    to_cols(T);
    for (int h = 0; h < 2 * k; h++) {
        uint64_t *ox = tmpx + (size_t)h * nw, *oz = tmpz + (size_t)h * nw;
        memset(ox, 0, nw * sizeof(uint64_t));
        memset(oz, 0, nw * sizeof(uint64_t));
        int ph = 2 * img[h].sign;
        for (int j = 0; j < k; j++) {
            int xj = (img[h].x >> j) & 1, zj = (img[h].z >> j) & 1;
            if (xj && zj) ph += 1;       /* Y = i X Z */
            if (xj) {
                uint32_t c = 2 * q[j];
                ph += string_mul(ox, oz, TX(T, c), TZ(T, c), nw) + 2 * T->sign[c];
            }
            if (zj) {
                uint32_t c = 2 * q[j] + 1;
                ph += string_mul(ox, oz, TX(T, c), TZ(T, c), nw) + 2 * T->sign[c];
            }
        }
        ph &= 3;
        if (ph & 1) { fprintf(stderr, "oracle: non-Hermitian prepend result\n"); abort(); }
        tmps[h] = (uint8_t)(ph >> 1);
    }
    for (int h = 0; h < 2 * k; h++) {
        uint32_t c = 2 * q[h >> 1] + (h & 1);
        memcpy(TX(T, c), tmpx + (size_t)h * nw, nw * sizeof(uint64_t));
        memcpy(TZ(T, c), tmpz + (size_t)h * nw, nw * sizeof(uint64_t));
        T->sign[c] = tmps[h];
    }
}

/* Appending gate g on start-of-time qubits conjugates every column P into
 * g^dagger P g. In row-major form that is word-wide logic across columns on
 * the gate's rows; the four rules below are checked against the generic
 * conjugation (conj_local, itself pinned against matrices) by
 * check_row_rules() before every reference sample.
 *   CX(p->k): s ^= x_p z_k (x_k ^ z_p ^ 1); x_k ^= x_p; z_p ^= z_k
 *   H(p):     s ^= x_p z_p; swap(x_p, z_p)
 *   S(p):     s ^= x_p ~z_p; z_p ^= x_p
 *   X(p):     s ^= z_p                                                   */
static void row_cx(tableau *T, uint32_t p, uint32_t k) {
    uint64_t *xp = RX(T, p), *zp = RZ(T, p), *xk = RX(T, k), *zk = RZ(T, k);
    for (size_t w = 0; w < T->cw; w++) {
        T->rs[w] ^= xp[w] & zk[w] & ~(xk[w] ^ zp[w]);
        xk[w] ^= xp[w];
        zp[w] ^= zk[w];
    }
}

static void row_1q(tableau *T, int g, uint32_t p) {
    uint64_t *xp = RX(T, p), *zp = RZ(T, p);
    for (size_t w = 0; w < T->cw; w++) {
        uint64_t x = xp[w], z = zp[w];
        if (g == OG_H) { T->rs[w] ^= x & z; xp[w] = z; zp[w] = x; }
        else if (g == OG_S) { T->rs[w] ^= x & ~z; zp[w] = z ^ x; }
        else { T->rs[w] ^= z; }   /* OG_X */
    }
}

static void check_row_rules(void) {
    static int checked = 0;
    if (checked) return;
    for (int g = 0; g < 3; g++) {
        int gate = g == 0 ? OG_H : g == 1 ? OG_S : OG_X;
        spauli img[4];
        gate_images(gate, img);
        for (int bits = 0; bits < 4; bits++) {
            tableau T;
            tableau_init(&T, 1);
            to_rows(&T);
            T.rx[0] = (uint64_t)(bits & 1);
            T.rz[0] = (uint64_t)(bits >> 1);
            T.rs[0] = 0;
            row_1q(&T, gate, 0);
            uint8_t ox, oz;
            int ph;
            conj_local(img, 1, (uint8_t)(bits & 1), (uint8_t)(bits >> 1), &ox, &oz, &ph);
            if ((T.rx[0] & 1) != ox || (T.rz[0] & 1) != oz || (int)(T.rs[0] & 1) != ph / 2) {
                fprintf(stderr, "oracle: row rule mismatch for gate %d\n", gate);
                abort();
            }
            tableau_free(&T);
        }
    }
    spauli img[4];
    gate_images(OG_CX, img);
    for (int bits = 0; bits < 16; bits++) {
        tableau T;
        tableau_init(&T, 2);
        to_rows(&T);
        /* rows 0 (control) and 1 (target), one column (bit 0 of each word) */
        T.rx[0] = (uint64_t)(bits & 1);
        T.rz[0] = (uint64_t)((bits >> 1) & 1);
        T.rx[T.cw] = (uint64_t)((bits >> 2) & 1);
        T.rz[T.cw] = (uint64_t)((bits >> 3) & 1);
        T.rs[0] = 0;
        row_cx(&T, 0, 1);
        uint8_t ox, oz;
        int ph;
        conj_local(img, 2, (uint8_t)((bits & 1) | (((bits >> 2) & 1) << 1)),
                   (uint8_t)(((bits >> 1) & 1) | (((bits >> 3) & 1) << 1)), &ox, &oz, &ph);
        uint8_t gx = (uint8_t)((T.rx[0] & 1) | ((T.rx[T.cw] & 1) << 1));
        uint8_t gz = (uint8_t)((T.rz[0] & 1) | ((T.rz[T.cw] & 1) << 1));
        if (gx != ox || gz != oz || (int)(T.rs[0] & 1) != ph / 2) {
            fprintf(stderr, "oracle: row rule mismatch for CX\n");
            abort();
        }
        tableau_free(&T);
    }
    checked = 1;
}

/* Measure Z_q; returns the outcome, sets *det to 1 if it was deterministic. */
static int tableau_measure(tableau *T, uint32_t q, int *det) {
    uint32_t cz = 2 * q + 1;
    if (!T->rows) {
        const uint64_t *mx = TX(T, cz);
        int any = 0;
        for (size_t w = 0; w < T->nw; w++) any |= mx[w] != 0;
        if (!any) {
            *det = 1;
            return T->sign[cz];
        }
        to_rows(T);     /* a random measurement: switch to rows for the elimination */
    }
    int64_t pivot = -1;
    for (uint32_t r = 0; r < T->n && pivot < 0; r++)
        if (GETB(RX(T, r), cz)) pivot = r;
    if (pivot < 0) {
        *det = 1;
        return GETB(T->rs, cz);
    }
    *det = 0;
    uint32_t p = (uint32_t)pivot;
    for (uint32_t k = p + 1; k < T->n; k++)
        if (GETB(RX(T, k), cz)) row_cx(T, p, k);          /* CNOT pivot -> k */
    if (GETB(RZ(T, p), cz)) row_1q(T, OG_S, p);           /* Y on the pivot: S maps it to X */
    row_1q(T, OG_H, p);                                   /* X on the pivot -> Z */
    if (GETB(T->rs, cz)) row_1q(T, OG_X, p);              /* outcome 0 */
    return GETB(T->rs, cz);
}

/* Reference sample: outcome of every measurement (outcome 0 when random),
 * plus a flag telling whether it was deterministic. */
int orc_reference(const orc_circuit *c, uint8_t *ref, uint8_t *detflag) {
    tableau T;
    check_row_rules();
    if (tableau_init(&T, c->n) < 0) return -1;
    size_t nw = T.nw;
    uint64_t *tmpx = (uint64_t *)malloc(4 * nw * sizeof(uint64_t));
    uint64_t *tmpz = (uint64_t *)malloc(4 * nw * sizeof(uint64_t));
    uint8_t tmps[4];
    uint64_t m = 0;
    for (size_t i = 0; i < c->nops; i++) {
        const orc_op *o = &c->ops[i];
        if (is_1q_gate(o->gate)) {
            for (uint32_t j = 0; j < o->nt; j++) tableau_prepend(&T, o->gate, &o->t[j], tmpx, tmpz, tmps);
            continue;
        }
        if (is_collapse(o->gate)) {
            /* X and Y bases: the basis change (H; or S_DAG then H) that maps the
             * measured observable to Z, the Z-basis op, then its inverse */
            const int basis = collapse_basis(o->gate), kind = collapse_kind(o->gate);
            for (uint32_t j = 0; j < o->nt; j++) {
                const uint32_t *q = &o->t[j];
                if (basis == 2) tableau_prepend(&T, OG_SDAG, q, tmpx, tmpz, tmps);
                if (basis != 0) tableau_prepend(&T, OG_H, q, tmpx, tmpz, tmps);
                int det;
                int r = tableau_measure(&T, *q, &det);
                if (kind != 2) {
                    ref[m] = (uint8_t)r;
                    if (detflag) detflag[m] = (uint8_t)det;
                    m++;
                }
                if (kind != 0) set_sign(&T, 2 * *q + 1, 0);   /* force the +1 eigenstate */
                if (basis != 0) tableau_prepend(&T, OG_H, q, tmpx, tmpz, tmps);
                if (basis == 2) tableau_prepend(&T, OG_S, q, tmpx, tmpz, tmps);
            }
            continue;
        }
        switch (o->gate) {
        case OG_CX: case OG_CZ:
            for (uint32_t j = 0; j < o->nt; j += 2) {
                const uint32_t a = o->t[j], b = o->t[j + 1];
                if ((a | b) & REC_FLAG) {
                    /* classically controlled X (CX) or Z (CZ) on the qubit,
                     * applied when the reference recorded a 1 */
                    const uint32_t rec = (a & REC_FLAG) ? a : b, q = (a & REC_FLAG) ? b : a;
                    if (ref[rec & ~REC_FLAG]) tableau_prepend(&T, o->gate == OG_CX ? OG_X : OG_Z, &q, tmpx, tmpz, tmps);
                    continue;
                }
                tableau_prepend(&T, o->gate, &o->t[j], tmpx, tmpz, tmps);
            }
            break;
        default:
            break;   /* noise and detectors do not touch the noiseless sample */
        }
    }
    free(tmpx);
    free(tmpz);
    tableau_free(&T);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-shot Pauli frame simulation                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    const orc_circuit *c;
    const uint8_t *ref;
    uint64_t seed, shot_offset;
    const uint64_t *shots;
    size_t begin, end;
    uint8_t *meas;     /* [nshots][M] */
    uint8_t *dets;     /* [nshots][D] */
} frame_job;

static void *frame_worker(void *arg) {
    frame_job *jb = (frame_job *)arg;
    const orc_circuit *c = jb->c;
    uint8_t *x = (uint8_t *)calloc(c->n + 1, 1);
    uint8_t *z = (uint8_t *)calloc(c->n + 1, 1);
    uint8_t *flip = (uint8_t *)calloc(c->nmeas + 1, 1);
    spauli img1[OG_RY + 1][4], imgCX[4], imgCZ[4];
    for (int g = 0; g <= OG_RY; g++)
        if (is_1q_gate(g)) gate_images(g, img1[g]);
    gate_images(OG_CX, imgCX);
    gate_images(OG_CZ, imgCZ);
    for (size_t si = jb->begin; si < jb->end; si++) {
        uint64_t shot = jb->shot_offset + jb->shots[si];
        uint64_t word = shot / 64;
        int b = (int)(shot % 64);
        uint8_t *mrow = jb->meas ? jb->meas + si * c->nmeas : NULL;
        /* detection-event row: D detectors, then the observables */
        uint8_t *drow = jb->dets ? jb->dets + si * (c->ndet + c->nobs) : NULL;
        if (drow) memset(drow + c->ndet, 0, c->nobs);
        /* Step 2: every qubit starts as I or Z with probability 1/2. */
        for (uint32_t q = 0; q < c->n; q++) {
            x[q] = 0;
            z[q] = (uint8_t)((half_mask(jb->seed, TAG_INIT, 0, q, word) >> b) & 1);
        }
        uint64_t m = 0, dk = 0;
        for (size_t i = 0; i < c->nops; i++) {
            const orc_op *o = &c->ops[i];
            uint32_t instr = (uint32_t)i;
            if (is_1q_gate(o->gate)) {
                for (uint32_t j = 0; j < o->nt; j++) {
                    uint32_t q = o->t[j];
                    uint8_t rx, rz;
                    int ph;
                    conj_local(img1[o->gate], 1, x[q], z[q], &rx, &rz, &ph);
                    x[q] = rx;
                    z[q] = rz;
                }
                continue;
            }
            switch (o->gate) {
            case OG_CX: case OG_CZ: {
                const spauli *img = o->gate == OG_CX ? imgCX : imgCZ;
                for (uint32_t j = 0; j < o->nt; j += 2) {
                    uint32_t a = o->t[j], bq = o->t[j + 1];
                    if ((a | bq) & REC_FLAG) {
                        /* the frame gains the Pauli exactly when the record
                         * differs from the reference (its flip) */
                        const uint32_t rec = (a & REC_FLAG) ? a : bq, q = (a & REC_FLAG) ? bq : a;
                        const uint8_t f = flip[rec & ~REC_FLAG];
                        if (o->gate == OG_CX) x[q] ^= f;
                        else z[q] ^= f;
                        continue;
                    }
                    uint8_t rx, rz;
                    int ph;
                    conj_local(img, 2, (uint8_t)(x[a] | (x[bq] << 1)), (uint8_t)(z[a] | (z[bq] << 1)), &rx, &rz, &ph);
                    x[a] = rx & 1; x[bq] = (rx >> 1) & 1;
                    z[a] = rz & 1; z[bq] = (rz >> 1) & 1;
                }
                break;
            }
            case OG_M: case OG_MR: case OG_R:
            case OG_MX: case OG_MY: case OG_MRX: case OG_MRY: case OG_RX: case OG_RY: {
                const int basis = collapse_basis(o->gate), kind = collapse_kind(o->gate);
                for (uint32_t j = 0; j < o->nt; j++) {
                    uint32_t q = o->t[j];
                    uint8_t coin = (uint8_t)((half_mask(jb->seed, TAG_COLLAPSE, instr, j, word) >> b) & 1);
                    uint8_t rx, rz;
                    int ph;
                    if (basis == 2) { conj_local(img1[OG_SDAG], 1, x[q], z[q], &rx, &rz, &ph); x[q] = rx; z[q] = rz; }
                    if (basis != 0) { conj_local(img1[OG_H], 1, x[q], z[q], &rx, &rz, &ph); x[q] = rx; z[q] = rz; }
                    if (kind != 2) {
                        flip[m] = x[q];
                        if (mrow) mrow[m] = (uint8_t)(jb->ref[m] ^ x[q]);
                        m++;
                    }
                    if (kind == 0) {
                        z[q] ^= coin;
                    } else {
                        x[q] = 0;
                        z[q] = coin;
                    }
                    if (basis != 0) { conj_local(img1[OG_H], 1, x[q], z[q], &rx, &rz, &ph); x[q] = rx; z[q] = rz; }
                    if (basis == 2) { conj_local(img1[OG_S], 1, x[q], z[q], &rx, &rz, &ph); x[q] = rx; z[q] = rz; }
                }
                break;
            }
            case OG_XERR: case OG_ZERR: case OG_YERR: case OG_DEP1: case OG_DEP2: case OG_PC1: case OG_PC2: {
                if (o->p <= 0) break;
                int pair = is_pair(o->gate);
                for (uint32_t j = 0; j < o->nt; j += pair ? 2 : 1) {
                    uint32_t slot = pair ? j / 2 : j;
                    noise_word nwd = noise_for_word(jb->seed, o->gate, o->G, o->C, instr, slot, word);
                    uint32_t a = o->t[j];
                    x[a] ^= (uint8_t)((nwd.x0 >> b) & 1);
                    z[a] ^= (uint8_t)((nwd.z0 >> b) & 1);
                    if (pair) {
                        uint32_t bq = o->t[j + 1];
                        x[bq] ^= (uint8_t)((nwd.x1 >> b) & 1);
                        z[bq] ^= (uint8_t)((nwd.z1 >> b) & 1);
                    }
                }
                break;
            }
            case OG_DET: {
                uint8_t v = 0;
                for (uint32_t j = 0; j < o->nt; j++) v ^= flip[o->t[j]];
                if (drow) drow[dk] = v;
                dk++;
                break;
            }
            case OG_OBS: {      /* an observable is the XOR of the flips of every record it includes */
                uint8_t v = 0;
                for (uint32_t j = 0; j < o->nt; j++) v ^= flip[o->t[j]];
                if (drow) drow[c->ndet + (uint64_t)o->p] ^= v;
                break;
            }
            }
        }
    }
    free(x);
    free(z);
    free(flip);
    return NULL;
}

/* Sample the listed shots (global shot index = shot_offset + shots[i]).
 * meas: [nshots][M] record bytes (0/1), dets: [nshots][D]; either may be NULL. */
int orc_frame_shots(const orc_circuit *c, const uint8_t *ref, uint64_t seed, uint64_t shot_offset,
                    const uint64_t *shots, size_t nshots, uint8_t *meas, uint8_t *dets, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if ((size_t)nthreads > nshots) nthreads = nshots ? (int)nshots : 1;
    pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
    frame_job *jobs = (frame_job *)malloc((size_t)nthreads * sizeof(frame_job));
    for (int t = 0; t < nthreads; t++) {
        frame_job j = {c, ref, seed, shot_offset, shots,
                       nshots * (size_t)t / (size_t)nthreads, nshots * (size_t)(t + 1) / (size_t)nthreads,
                       meas, dets};
        jobs[t] = j;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, frame_worker, &jobs[t]);
    frame_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th);
    free(jobs);
    return 0;
}

/* Exposed for tests: conjugate a local Pauli (x, z bits over k <= 2 qubits)
 * by a gate given as the images of its generators (X_a, Z_a, X_b, Z_b; each
 * as x bits, z bits, sign). Returns the power of i. */
int orc_conj_custom(int k, const int *img_x, const int *img_z, const int *img_sign,
                    int x, int z, int *ox, int *oz) {
    spauli img[4];
    memset(img, 0, sizeof(img));
    for (int h = 0; h < 2 * k; h++) {
        img[h].x = (uint8_t)img_x[h];
        img[h].z = (uint8_t)img_z[h];
        img[h].sign = (uint8_t)img_sign[h];
    }
    uint8_t rx, rz;
    int ph;
    conj_local(img, k, (uint8_t)x, (uint8_t)z, &rx, &rz, &ph);
    *ox = rx;
    *oz = rz;
    return ph;
}
