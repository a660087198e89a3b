// tableau.cu -- noiseless reference sample by inverse-tableau simulation
// (Section 4 of the paper, "Tracking the Tableau").
//
// The tableau T tracks the inverse of the circuit so far: logical column 2q
// holds the start-of-time image of X_q, column 2q+1 that of Z_q, each as an
// n-term Pauli string (x words, z words) with a sign. Columns are stored
// column-major ([column][nw] words per plane) behind a permutation, so an H
// (which swaps the X_q and Z_q columns) is a swap of two permutation entries.
//
// Folding a gate prepends its inverse: new column(g) = T(G^dagger g G),
//   S:  X_a <- -i X_a Z_a          S_DAG: X_a <- +i X_a Z_a
//   SQRT_X: Z_a <- -i Z_a X_a      SQRT_X_DAG: Z_a <- +i Z_a X_a
//   CX: X_c <- X_c X_t,  Z_t <- Z_t Z_c
//   CZ: X_a <- X_a Z_b,  X_b <- X_b Z_a
//   X, Y, Z negate the anticommuting columns; SQRT_Y(_DAG) swap the two
//   columns (like H) and negate one of them.
// each a column product (one warp per product) whose phase is the sum, over
// qubit positions, of the +-i factors of the single-qubit products (popcounts
// of the +i and -i position masks, warp-reduced).
//
// A measurement of Z_q is deterministic when column Z_q has no X/Y term; the
// outcome is its sign. Otherwise a pivot p (lowest X/Y row) is chosen, CNOTs
// p -> k are appended for every other X/Y row k, then S (if the pivot term is
// Y) and H turn the pivot term into Z, and -- because the paper leaves the coin
// open -- an X is appended on the pivot when the sign is -, so the outcome is
// always 0. Appends act on rows of every column; the sign update of the CNOT
// chain uses the closed form
//   flips = popcount(z & (z_p ? x : ~x) & K) + C(popcount(z & K), 2)  (mod 2).
// A reset is a measurement followed by forcing the sign of column Z_q to +.
//
// Work inside a layer is spread over the whole grid; a bounded software grid
// barrier (cooperative launch, so all CTAs are resident) separates phases.
// Collapsing ops of a layer are first checked in parallel; outcomes before the
// first random one are written in parallel; from there a leader warp walks
// the ops in source order and every random one costs two grid barriers.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace stimgb {

namespace {

constexpr uint32_t kListLimit = 16;                     // CNOT targets handled by list, else by mask

// Barrier over the a.nblk CTAs of one tableau (the whole grid, or one
// circuit's CTA range of a batched launch). A wait gives up after
// a.bar_timeout_ns: it sets the circuit's abort flag and DEV_TIMEOUT, every
// CTA then leaves the kernel at its next barrier, and the host reports
// STIM_E_TIMEOUT. (a.bar_extra > 0, a test knob, makes the barrier wait for
// arrivals that never come.)
__device__ __forceinline__ bool tab_barrier(const TabArgs &a) {
    if (a.nblk == 1) {
        __syncthreads();
        return true;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &a.ctl->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&a.ctl->bar_count, 1u);
        if (arrived == a.nblk + a.bar_extra - 1) {
            atomicExch(&a.ctl->bar_count, 0u);
            __threadfence();
            atomicAdd(&a.ctl->bar_gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (*gen == g) {
                if (*(volatile int *)&a.ctl->abort) break;
                __nanosleep(64);
                if (globaltimer_ns() - t0 > a.bar_timeout_ns) {
                    atomicExch(&a.ctl->abort, 1);
                    atomicExch(a.status, DEV_TIMEOUT);
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int *)&a.ctl->abort == 0;
}

// Tableau accesses. With several CTAs the data is shared through L2 (cache-
// global loads and stores, ordered by the grid barrier); a single CTA (L1)
// keeps it in its own L1, ordered by __syncthreads.
template <bool L1>
__device__ __forceinline__ uint32_t ld_u32(const uint32_t *p) {
    if constexpr (L1) return *p;
    else return __ldcg(p);
}
template <bool L1>
__device__ __forceinline__ uint64_t ld_u64(const uint64_t *p) {
    if constexpr (L1) return *p;
    else return __ldcg(p);
}
template <bool L1, class T>
__device__ __forceinline__ void st_tab(T *p, T v) {
    if constexpr (L1) *p = v;
    else __stcg(p, v);
}

// dst column := dst * src (logical columns); extra = additional power of i.
//
// Phase of a product of two Pauli strings (Section 2, xz encoding): per qubit
// position the single-qubit product P1 P2 contributes i^g, with g = +1 for the
// cyclic pairs XY, YZ, ZX, g = -1 (i^3) for YX, ZY, XZ, and g = 0 when the two
// commute. Each lane classifies its words into X-only, Y and Z-only masks for
// both factors, forms the +i and -i position masks and adds their popcounts
// into one integer exponent (mod 4), which the warp then sums.
template <bool L1>
__device__ void column_product(const TabArgs &a, uint32_t dst, uint32_t src, uint32_t extra, uint32_t lane) {
    const uint32_t pd = ld_u32<L1>(a.perm + dst), ps = ld_u32<L1>(a.perm + src);
    uint64_t *dx = a.tx + (uint64_t)pd * a.nw, *dz = a.tz + (uint64_t)pd * a.nw;
    const uint64_t *sx = a.tx + (uint64_t)ps * a.nw, *sz = a.tz + (uint64_t)ps * a.nw;
    uint32_t ph = 0;      // this lane's exponent of i
    for (uint32_t w = lane; w < a.nw; w += 32) {
        const uint64_t ax = ld_u64<L1>(dx + w), az = ld_u64<L1>(dz + w);
        const uint64_t bx = ld_u64<L1>(sx + w), bz = ld_u64<L1>(sz + w);
        const uint64_t a_x = ax & ~az, a_y = ax & az, a_z = az & ~ax;    // left factor: X, Y, Z
        const uint64_t b_x = bx & ~bz, b_y = bx & bz, b_z = bz & ~bx;    // right factor: X, Y, Z
        const uint64_t up = (a_x & b_y) | (a_y & b_z) | (a_z & b_x);    // XY = iZ, YZ = iX, ZX = iY
        const uint64_t dn = (a_y & b_x) | (a_z & b_y) | (a_x & b_z);    // YX = -iZ, ZY = -iX, XZ = -iY
        ph += (uint32_t)__popcll(up) + 3u * (uint32_t)__popcll(dn);
        st_tab<L1>(dx + w, ax ^ bx);
        st_tab<L1>(dz + w, az ^ bz);
    }
    for (int d = 16; d > 0; d >>= 1) ph += __shfl_xor_sync(0xffffffffu, ph, d);
    if (lane == 0) {
        const uint32_t tot = (ph + extra + 2u * ld_u32<L1>(a.sign + pd) + 2u * ld_u32<L1>(a.sign + ps)) & 3u;
        st_tab<L1>(a.sign + pd, tot >> 1);   // tot is even: the product of the images is Hermitian
    }
}

__device__ __forceinline__ void write_outcome(const TabArgs &a, uint32_t opc, uint32_t m, uint32_t bit,
                                              uint32_t det) {
    if (opc == OP_R) return;
    const unsigned long long b = 1ull << (m & 63);
    if (bit) atomicOr((unsigned long long *)(a.ref + (m >> 6)), b);
    if (det) atomicOr((unsigned long long *)(a.detflag + (m >> 6)), b);
}

// Leader warp: walk collapsing ops from j in source order. Deterministic ones
// are resolved here; at the first random one the elimination data is
// published for the grid. Returns nothing; results go to a.ctl.
template <bool L1>
__device__ void leader_walk(const TabArgs &a, const DevOp *cops, uint32_t nc, uint32_t j, uint32_t meas_off,
                            uint32_t lane) {
    for (; j < nc; j++) {
        const DevOp op = cops[j];
        const uint32_t opc = op.a >> 24, q = op.a & kQubitMask;
        const uint32_t pz = ld_u32<L1>(a.perm + 2 * q + 1);
        const uint64_t *x = a.tx + (uint64_t)pz * a.nw, *z = a.tz + (uint64_t)pz * a.nw;
        int64_t pivot = -1;
        for (uint32_t base = 0; base < a.nw && pivot < 0; base += 32) {
            const uint32_t w = base + lane;
            const uint64_t v = w < a.nw ? ld_u64<L1>(x + w) : 0;
            const uint32_t bal = __ballot_sync(0xffffffffu, v != 0);
            if (bal) {
                const uint32_t src = __ffs(bal) - 1;
                const uint64_t vv = __shfl_sync(0xffffffffu, v, src);
                pivot = (int64_t)(base + src) * 64 + (__ffsll((long long)vv) - 1);
            }
        }
        if (pivot < 0) {
            if (lane == 0) {
                const uint32_t s = ld_u32<L1>(a.sign + pz);
                write_outcome(a, opc, op.b + meas_off, s, 1);
                if (opc != OP_M) st_tab<L1>(a.sign + pz, 0u);
            }
            __syncwarp();
            continue;
        }
        const uint32_t p = (uint32_t)pivot;
        const uint32_t pw = p >> 6;
        const uint64_t pb = 1ull << (p & 63);
        uint32_t cnt = 0, m = 0;
        for (uint32_t base = 0; base < a.nw; base += 32) {
            const uint32_t w = base + lane;
            uint64_t xv = w < a.nw ? ld_u64<L1>(x + w) : 0;
            const uint64_t zv = w < a.nw ? ld_u64<L1>(z + w) : 0;
            if (w == pw) xv &= ~pb;
            if (w < a.nw) st_tab<L1>(a.kmask + w, xv);
            const uint32_t c = __popcll(xv);
            uint32_t incl = c;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += t;
            }
            uint32_t off = cnt + incl - c;
            uint64_t rest = xv;
            while (rest) {
                const uint32_t bpos = __ffsll((long long)rest) - 1;
                st_tab<L1>(a.klist + off, w * 64 + bpos);
                off++;
                rest &= rest - 1;
            }
            cnt += __shfl_sync(0xffffffffu, incl, 31);
            uint32_t mz = __popcll(xv & zv);
            for (int d = 16; d > 0; d >>= 1) mz += __shfl_xor_sync(0xffffffffu, mz, d);
            m += mz;
        }
        if (lane == 0) {
            const uint32_t zp = (uint32_t)((ld_u64<L1>(z + pw) & pb) != 0);
            // column Z_q after the CNOT chain: sign flips floor(m/2) (z_p = 0) or ceil(m/2) (z_p = 1)
            const uint32_t flips = zp ? ((m + 1) >> 1) : (m >> 1);
            const uint32_t s_new = ld_u32<L1>(a.sign + pz) ^ (flips & 1u);
            a.ctl->pivot = p;
            a.ctl->nk = cnt;
            a.ctl->pivot_is_y = zp ^ (m & 1u);
            a.ctl->fix_x = s_new;                 // outcome 0: append X on the pivot if the sign is -
            a.ctl->use_mask = cnt > kListLimit ? 1u : 0u;
            a.ctl->next_j = j;
            a.ctl->has_random = 1u;
            a.ctl->nk_sum += cnt;
            a.ctl->nk_cnt += 1u;
            // outcome 0 and not deterministic: nothing to set in ref / detflag
        }
        __syncwarp();
        return;
    }
    if (lane == 0) {
        a.ctl->next_j = nc;
        a.ctl->has_random = 0u;
    }
    __syncwarp();
}

// Pivot collapse on bits (xp, zp) of one column: optional S, then H, then X fix.
__device__ __forceinline__ void pivot_ops(uint32_t &xp, uint32_t &zp, uint32_t &s, uint32_t py, uint32_t fx) {
    if (py) {            // S: X -> -Y, Y -> X
        s ^= xp & (zp ^ 1u);
        zp ^= xp;
    }
    s ^= xp & zp;        // H: Y -> -Y, X <-> Z
    const uint32_t t = xp;
    xp = zp;
    zp = t;
    if (fx) s ^= zp;     // X: Z -> -Z, Y -> -Y
}

template <bool L1>
__device__ __forceinline__ void set_bit(uint64_t *w, uint64_t b, uint32_t v) {
    const uint64_t old = ld_u64<L1>(w);
    st_tab<L1>(w, v ? (old | b) : (old & ~b));
}

// Apply the random measurement's appends to every column (list form: one thread per column).
template <bool L1>
__device__ void column_pass_list(const TabArgs &a, uint32_t p, uint32_t nk, uint32_t py, uint32_t fx,
                                 uint32_t gtid, uint32_t nthreads) {
    const uint32_t pw = p >> 6;
    const uint64_t pb = 1ull << (p & 63);
    for (uint32_t c = gtid; c < 2 * a.n; c += nthreads) {
        uint64_t *x = a.tx + (uint64_t)c * a.nw, *z = a.tz + (uint64_t)c * a.nw;
        uint32_t xp = (ld_u64<L1>(x + pw) & pb) != 0;
        uint32_t zp = (ld_u64<L1>(z + pw) & pb) != 0;
        uint32_t s = ld_u32<L1>(a.sign + c);
        for (uint32_t t = 0; t < nk; t++) {
            const uint32_t k = ld_u32<L1>(a.klist + t);
            const uint64_t kb = 1ull << (k & 63);
            const uint32_t zk = (ld_u64<L1>(z + (k >> 6)) & kb) != 0;
            if (xp) {
                const uint64_t xw = ld_u64<L1>(x + (k >> 6));
                const uint32_t xk = (xw & kb) != 0;
                s ^= zk & (xk ^ zp ^ 1u);
                st_tab<L1>(x + (k >> 6), xw ^ kb);
            }
            zp ^= zk;
        }
        pivot_ops(xp, zp, s, py, fx);
        set_bit<L1>(x + pw, pb, xp);
        set_bit<L1>(z + pw, pb, zp);
        st_tab<L1>(a.sign + c, s);
    }
}

// Mask form: one warp per column, word-parallel.
template <bool L1>
__device__ void column_pass_mask(const TabArgs &a, uint32_t p, uint32_t py, uint32_t fx, uint32_t gwarp,
                                 uint32_t nwarps, uint32_t lane) {
    const uint32_t pw = p >> 6;
    const uint64_t pb = 1ull << (p & 63);
    for (uint32_t c = gwarp; c < 2 * a.n; c += nwarps) {
        uint64_t *x = a.tx + (uint64_t)c * a.nw, *z = a.tz + (uint64_t)c * a.nw;
        const uint32_t xp = (ld_u64<L1>(x + pw) & pb) != 0;
        const uint32_t zp = (ld_u64<L1>(z + pw) & pb) != 0;
        uint32_t cnt_a = 0, cnt_b = 0;
        for (uint32_t w = lane; w < a.nw; w += 32) {
            const uint64_t kw = ld_u64<L1>(a.kmask + w);
            const uint64_t zw = ld_u64<L1>(z + w);
            cnt_b += __popcll(zw & kw);
            if (xp) {
                const uint64_t xw = ld_u64<L1>(x + w);
                cnt_a += __popcll(zw & (zp ? xw : ~xw) & kw);
                st_tab<L1>(x + w, xw ^ kw);
            }
        }
        for (int d = 16; d > 0; d >>= 1) {
            cnt_a += __shfl_xor_sync(0xffffffffu, cnt_a, d);
            cnt_b += __shfl_xor_sync(0xffffffffu, cnt_b, d);
        }
        __syncwarp();
        if (lane == 0) {
            uint32_t s = ld_u32<L1>(a.sign + c);
            if (xp) {
                const uint64_t pairs = (uint64_t)cnt_b * (cnt_b - (cnt_b > 0 ? 1u : 0u)) / 2;
                s ^= (uint32_t)((cnt_a + pairs) & 1u);
            }
            uint32_t xn = xp, zn = zp ^ (cnt_b & 1u);
            pivot_ops(xn, zn, s, py, fx);
            set_bit<L1>(x + pw, pb, xn);
            set_bit<L1>(z + pw, pb, zn);
            st_tab<L1>(a.sign + c, s);
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// Bursts of random measurements in row-major form (Section 5's data layout:
// the tableau is transposed while random measurements are resolved). Appending
// a CNOT p -> k to the tableau touches every column at rows p and k; with
// columns stored contiguously that is a pass over all 2n columns, with rows
// stored contiguously it is a few words of rows p and k. A layer with many
// random measurements, in a circuit whose random measurements have had few
// enough CNOT targets for one CTA (the mean target count times the row
// length, below), is transposed to rows by the whole grid, walked by CTA 0
// (one measurement at a time, CTA barriers only), and transposed back.
// ---------------------------------------------------------------------------
constexpr uint32_t kTableauMaxThreads = 512;   // the kernels' launch bound
constexpr uint32_t kBurstMinRandom = 16;    // random measurements in the layer
// one CTA's fan-out of a random measurement touches (targets x row words)
// words; measured: bursts win up to about 16k (random circuits of 1000
// qubits: 1.5x) and lose at 63k (2000 qubits: 1.7x slower)
constexpr uint32_t kBurstMaxRowWords = 32768;
// the other CTAs wait out a burst at one bounded barrier wait: cap its length
constexpr uint32_t kBurstMaxOps = 20000;
constexpr uint32_t kFanBatch = 4;           // fan-out targets loaded together
constexpr uint32_t kBurstCluster = 8;       // CTAs of the cluster that walks a burst
constexpr uint32_t kBurstClusterMinQubits = 16384;

// rows <- columns: word cw of row k holds bit k of physical columns 64cw .. 64cw + 63.
__device__ void to_rows(const TabArgs &a, uint32_t gtid, uint32_t nthreads) {
    const uint64_t total = (uint64_t)a.n * a.nw2;
    for (uint64_t i = gtid; i < total; i += nthreads) {
        const uint32_t k = (uint32_t)(i % a.n), cw = (uint32_t)(i / a.n);   // consecutive threads: consecutive rows
        const uint32_t kw = k >> 6, kb = k & 63;
        uint64_t vx = 0, vz = 0;
        for (uint32_t j = 0; j < 64; j++) {
            const uint32_t c = 64 * cw + j;
            if (c >= 2 * a.n) break;
            vx |= ((__ldcg(a.tx + (uint64_t)c * a.nw + kw) >> kb) & 1ull) << j;
            vz |= ((__ldcg(a.tz + (uint64_t)c * a.nw + kw) >> kb) & 1ull) << j;
        }
        __stcg(a.rx + (uint64_t)k * a.nw2 + cw, vx);
        __stcg(a.rz + (uint64_t)k * a.nw2 + cw, vz);
    }
    for (uint32_t cw = gtid; cw < a.nw2; cw += nthreads) {
        uint64_t v = 0;
        for (uint32_t j = 0; j < 64 && 64 * cw + j < 2 * a.n; j++)
            v |= (uint64_t)(__ldcg(a.sign + 64 * cw + j) & 1u) << j;
        __stcg(a.rsign + cw, v);
    }
}

// columns <- rows: word w of column c holds bit c of rows 64w .. 64w + 63.
__device__ void to_cols(const TabArgs &a, uint32_t gtid, uint32_t nthreads) {
    const uint64_t total = (uint64_t)2 * a.n * a.nw;
    for (uint64_t i = gtid; i < total; i += nthreads) {
        const uint32_t c = (uint32_t)(i % (2 * a.n)), w = (uint32_t)(i / (2 * a.n));
        const uint32_t cw = c >> 6, cb = c & 63;
        uint64_t vx = 0, vz = 0;
        for (uint32_t j = 0; j < 64; j++) {
            const uint32_t k = 64 * w + j;
            if (k >= a.n) break;
            vx |= ((__ldcg(a.rx + (uint64_t)k * a.nw2 + cw) >> cb) & 1ull) << j;
            vz |= ((__ldcg(a.rz + (uint64_t)k * a.nw2 + cw) >> cb) & 1ull) << j;
        }
        __stcg(a.tx + (uint64_t)c * a.nw + w, vx);
        __stcg(a.tz + (uint64_t)c * a.nw + w, vz);
    }
    for (uint32_t c = gtid; c < 2 * a.n; c += nthreads)
        __stcg(a.sign + c, (uint32_t)((__ldcg(a.rsign + (c >> 6)) >> (c & 63)) & 1ull));
}


// The collapsing ops j .. nc - 1 of a layer in row-major form, by one CTA in
// source order (the same results as the leader walk plus column passes):
// a measurement of Z_q reads column pc = perm(Z_q); rows with an X/Y bit there
// are found; none: deterministic, the outcome is the column's sign (a reset
// then clears it); else the lowest such row p is the pivot, the CNOT fan-out
// p -> k over the other rows k updates x_k ^= x_p, z_p ^= XOR of z_k and every
// column's sign by the closed form of the column pass, and the pivot collapse
// (S if the pivot term is Y, H, X when the sign is -) makes the outcome 0.
// The burst's CTAs work as one: with a cluster (bclu > 1) its barrier and the
// scalars of CTA rank 0 reached through distributed shared memory; alone,
// the CTA barrier and its own shared memory.
template <bool CLU>
__device__ __forceinline__ void bw_sync() {
    if (CLU) asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    else __syncthreads();
}
__device__ __forceinline__ uint32_t cl_map(uint32_t sa, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(sa), "r"(rank));
    return r;
}
__device__ __forceinline__ uint32_t cl_ld32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t cl_ld64(uint32_t a) {
    uint64_t v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void cl_st32(uint32_t a, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_min32(uint32_t a, uint32_t v) {
    asm volatile("red.shared::cluster.min.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t cl_add32(uint32_t a, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared::cluster.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v) : "memory");
    return old;
}

// The burst walk's shared state (one copy per CTA for both forms below).
__shared__ uint32_t s_ctl[4];                           // pivot, count, pivot term is Y, its sign is -
__shared__ uint64_t s_part[3][kTableauMaxThreads];     // per-thread chunk sums of the fan-out

// CLU: walked by a cluster of bclu CTAs (rank: this CTA's in it), else by one CTA.
template <bool CLU>
__device__ void burst_walk(const TabArgs &a, const DevOp *cops, uint32_t nc, uint32_t j, uint32_t meas_off,
                           uint32_t rank, uint32_t bclu) {
    const uint32_t CL = CLU ? bclu : 1u, B = blockDim.x * CL, tid = (CLU ? rank * blockDim.x : 0u) + threadIdx.x;
    // rank 0's scalars (own shared memory without a cluster)
    const uint32_t ctl0 = CLU ? cl_map(smem_addr(s_ctl), 0) : smem_addr(s_ctl);
    auto ld_ctl = [&](uint32_t i) { return CLU ? cl_ld32(ctl0 + 4 * i) : s_ctl[i]; };
    auto st_ctl = [&](uint32_t i, uint32_t v) {
        if (CLU) cl_st32(ctl0 + 4 * i, v);
        else s_ctl[i] = v;
    };
    for (; j < nc; j++) {
        const DevOp op = cops[j];
        const uint32_t opc = op.a >> 24, q = op.a & kQubitMask;
        const uint32_t pc = __ldcg(a.perm + 2 * q + 1);
        const uint32_t cwp = pc >> 6;
        const uint64_t bitp = 1ull << (pc & 63);
        if (tid == 0) {
            st_ctl(0, a.n);
            st_ctl(1, 0u);
        }
        bw_sync<CLU>();
        for (uint32_t k = tid; k < a.n; k += B) {
            if (__ldcg(a.rx + (uint64_t)k * a.nw2 + cwp) & bitp) {
                uint32_t slot;
                if (CLU) {
                    cl_min32(ctl0, k);
                    slot = cl_add32(ctl0 + 4, 1u);
                } else {
                    atomicMin(&s_ctl[0], k);
                    slot = atomicAdd(&s_ctl[1], 1u);
                }
                __stcg(a.klist + slot, k);
            }
        }
        bw_sync<CLU>();
        const uint32_t p = ld_ctl(0), cnt = ld_ctl(1);
        if (cnt == 0) {     // deterministic: the outcome is the sign of column Z_q
            if (tid == 0) {
                const uint64_t sw = __ldcg(a.rsign + cwp);
                write_outcome(a, opc, op.b + meas_off, (uint32_t)((sw & bitp) != 0), 1);
                if (opc != OP_M) __stcg(a.rsign + cwp, sw & ~bitp);
            }
            bw_sync<CLU>();
            continue;
        }
        if (tid == 0) {
            a.ctl->nk_sum += cnt - 1;
            a.ctl->nk_cnt += 1;
        }
        // CNOT fan-out p -> k, k in K \ {p}, word by word over the columns:
        // x_k ^= x_p for every k; z_p ^= XOR of the z_k; the sign of each
        // column picks up x_p times the parity of the Y and Z terms the
        // products meet (apar) plus the second bit of the count of z_k bits
        // (b1 b0: that count mod 4). Both are sums over k, so a row narrower
        // than the burst's threads splits the targets into CH chunks per
        // word, each thread summing its chunk, and the chunk sums are added
        // per word.
        // Targets are taken kFanBatch at a time so that their row loads are
        // in flight together.
        const uint32_t WP = a.nw2 < B ? a.nw2 : B;      // words handled side by side
        const uint32_t CH = B / WP;                     // target chunks per word
        const uint32_t chunk = tid / WP, wl = tid % WP;
        const uint32_t per = (cnt + CH - 1) / CH;
        const uint32_t t0 = chunk * per < cnt ? chunk * per : cnt;
        const uint32_t t1 = t0 + per < cnt ? t0 + per : cnt;
        if (chunk < CH) {
            for (uint32_t w = wl; w < a.nw2; w += WP) {
                const uint64_t xp = __ldcg(a.rx + (uint64_t)p * a.nw2 + w);
                uint64_t zp = __ldcg(a.rz + (uint64_t)p * a.nw2 + w);
                uint64_t apar = 0, b0 = 0, b1 = 0;
                uint32_t t = t0;
                for (; t + kFanBatch <= t1; t += kFanBatch) {
                    uint32_t k[kFanBatch];
                    uint64_t xk[kFanBatch], zk[kFanBatch];
#pragma unroll
                    for (int i = 0; i < (int)kFanBatch; i++) k[i] = __ldcg(a.klist + t + i);
#pragma unroll
                    for (int i = 0; i < (int)kFanBatch; i++) {
                        xk[i] = __ldcg(a.rx + (uint64_t)k[i] * a.nw2 + w);
                        zk[i] = __ldcg(a.rz + (uint64_t)k[i] * a.nw2 + w);
                    }
#pragma unroll
                    for (int i = 0; i < (int)kFanBatch; i++) {
                        if (k[i] == p) continue;
                        apar ^= zk[i] & ~(zp ^ xk[i]);
                        b1 ^= b0 & zk[i];
                        b0 ^= zk[i];
                        __stcg(a.rx + (uint64_t)k[i] * a.nw2 + w, xk[i] ^ xp);
                    }
                }
                for (; t < t1; t++) {
                    const uint32_t k = __ldcg(a.klist + t);
                    if (k == p) continue;
                    const uint64_t xk = __ldcg(a.rx + (uint64_t)k * a.nw2 + w);
                    const uint64_t zk = __ldcg(a.rz + (uint64_t)k * a.nw2 + w);
                    apar ^= zk & ~(zp ^ xk);
                    b1 ^= b0 & zk;
                    b0 ^= zk;
                    __stcg(a.rx + (uint64_t)k * a.nw2 + w, xk ^ xp);
                }
                if (CH > 1) {       // one word per thread: hand the chunk sums to chunk 0
                    s_part[0][threadIdx.x] = apar;
                    s_part[1][threadIdx.x] = b0;
                    s_part[2][threadIdx.x] = b1;
                    break;
                }
                const uint64_t s = __ldcg(a.rsign + w) ^ (xp & (apar ^ b1));
                zp ^= b0;
                __stcg(a.rz + (uint64_t)p * a.nw2 + w, zp);
                __stcg(a.rsign + w, s);
                if (w == cwp) {
                    st_ctl(2, (uint32_t)((zp & bitp) != 0));     // the pivot term of Z_q is Y
                    st_ctl(3, (uint32_t)((s & bitp) != 0));      // its sign is -
                }
            }
        }
        if (CH > 1) {
            bw_sync<CLU>();
            if (chunk == 0) {
                // the chunk sums of thread o sit in CTA o / blockDim.x of the burst
                auto part = [&](uint32_t i, uint32_t o) -> uint64_t {
                    if (!CLU) return s_part[i][o];
                    return cl_ld64(cl_map(smem_addr(&s_part[i][o % blockDim.x]), o / blockDim.x));
                };
                const uint32_t w = wl;
                uint64_t apar = part(0, w), b0 = part(1, w), b1 = part(2, w);
                for (uint32_t c = 1; c < CH; c++) {
                    const uint32_t o = c * WP + w;
                    const uint64_t c0 = part(1, o), c1 = part(2, o);
                    apar ^= part(0, o);
                    b1 ^= c1 ^ (b0 & c0);       // (b1 b0) += (c1 c0) mod 4
                    b0 ^= c0;
                }
                const uint64_t xp = __ldcg(a.rx + (uint64_t)p * a.nw2 + w);
                const uint64_t zp = __ldcg(a.rz + (uint64_t)p * a.nw2 + w) ^ b0;
                const uint64_t s = __ldcg(a.rsign + w) ^ (xp & (apar ^ b1));
                __stcg(a.rz + (uint64_t)p * a.nw2 + w, zp);
                __stcg(a.rsign + w, s);
                if (w == cwp) {
                    st_ctl(2, (uint32_t)((zp & bitp) != 0));
                    st_ctl(3, (uint32_t)((s & bitp) != 0));
                }
            }
        }
        bw_sync<CLU>();
        const bool py = ld_ctl(2) != 0, fx = ld_ctl(3) != 0;
        for (uint32_t w = tid; w < a.nw2; w += B) {      // pivot collapse on row p
            uint64_t xp = __ldcg(a.rx + (uint64_t)p * a.nw2 + w);
            uint64_t zp = __ldcg(a.rz + (uint64_t)p * a.nw2 + w);
            uint64_t s = __ldcg(a.rsign + w);
            if (py) {        // S: X -> -Y, Y -> X
                s ^= xp & ~zp;
                zp ^= xp;
            }
            s ^= xp & zp;    // H: Y -> -Y, X <-> Z
            const uint64_t t = xp;
            xp = zp;
            zp = t;
            if (fx) s ^= zp; // X: Z -> -Z, Y -> -Y
            __stcg(a.rx + (uint64_t)p * a.nw2 + w, xp);
            __stcg(a.rz + (uint64_t)p * a.nw2 + w, zp);
            __stcg(a.rsign + w, s);
        }
        bw_sync<CLU>();
        // a random outcome is 0: nothing to write (reference and flags start cleared)
    }
}

}  // namespace

__global__ void tableau_init_kernel(TabArgs a) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += gridDim.x * blockDim.x) {
        a.tx[(uint64_t)(2 * q) * a.nw + (q >> 6)] = 1ull << (q & 63);
        a.tz[(uint64_t)(2 * q + 1) * a.nw + (q >> 6)] = 1ull << (q & 63);
        a.perm[2 * q] = 2 * q;
        a.perm[2 * q + 1] = 2 * q + 1;
    }
}

// The inverse-tableau walk of one circuit by CTA bid of its a.nblk CTAs.
// CLU: the launch may be a cluster launch whose cluster 0 (a.bclu CTAs) walks
// the bursts together (the batched kernel's circuits never are).
template <bool L1, bool CLU = false>
__device__ __forceinline__ void tableau_body(const TabArgs &a, uint32_t bid) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    const uint32_t gwarp = bid * wpb + (threadIdx.x >> 5);
    const uint32_t nwarps = a.nblk * wpb;
    const uint32_t gtid = bid * blockDim.x + threadIdx.x;
    const uint32_t nthreads = a.nblk * blockDim.x;
    const bool leader = bid == 0 && threadIdx.x < 32;
    __shared__ uint32_t s_first, s_nrand;

    uint32_t meas_off = 0;
    uint32_t loop_pc[kMaxLoopDepth];
    uint32_t loop_iter[kMaxLoopDepth];
    int sp = 0;
    uint32_t pc = a.pc_begin;
    const uint32_t pc_end = a.pc_end < a.nprog ? a.pc_end : a.nprog;
    // a computation resumed inside a loop enters it at iteration iter_begin
    uint32_t enter_iter = a.iter_begin;
    if (enter_iter && (pc >= pc_end || a.prog[pc].kind != ENT_LOOP_BEGIN)) {
        if (gtid == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
        return;
    }
    while (pc < pc_end) {
        const ProgEntry e = a.prog[pc];
        if (e.kind == ENT_LOOP_BEGIN) {
            if (sp >= kMaxLoopDepth || enter_iter >= (e.reps > 0 ? e.reps : 1u)) {
                if (gtid == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return;
            }
            loop_pc[sp] = pc;
            loop_iter[sp] = enter_iter;
            meas_off += enter_iter * e.meas_stride;
            enter_iter = 0;
            sp++;
            pc++;
            continue;
        }
        if (e.kind == ENT_DETS) {       // detectors do not act on the tableau
            pc++;
            continue;
        }
        if (e.kind == ENT_LOOP_END) {
            if (sp <= 0) {
                if (gtid == 0) atomicExch(a.status, DEV_BAD_PROGRAM);
                return;
            }
            const uint32_t it = ++loop_iter[sp - 1];
            if (it < e.reps) {
                meas_off += e.meas_stride;
                pc = loop_pc[sp - 1] + 1;
            } else {
                meas_off -= e.meas_stride * (e.reps - 1);
                sp--;
                pc++;
            }
            continue;
        }
        pc++;
        const DevOp *ops = a.ops + e.op_begin;
        if (e.n_gate) {
            for (uint32_t t = gwarp; t < 2 * e.n_gate; t += nwarps) {
                const DevOp op = ops[t >> 1];
                const uint32_t k = t & 1, opc = op.a >> 24;
                const uint32_t qa = op.a & kQubitMask, qb = op.b & kQubitMask;
                switch (opc) {
                    case OP_H:
                        if (k == 0 && lane == 0) {
                            const uint32_t u = ld_u32<L1>(a.perm + 2 * qa), v = ld_u32<L1>(a.perm + 2 * qa + 1);
                            st_tab<L1>(a.perm + 2 * qa, v);
                            st_tab<L1>(a.perm + 2 * qa + 1, u);
                        }
                        break;
                    case OP_S:
                        if (k == 0) column_product<L1>(a, 2 * qa, 2 * qa + 1, 3u, lane);
                        break;
                    case OP_CX:
                        if (k == 0) column_product<L1>(a, 2 * qa, 2 * qb, 0u, lane);
                        else column_product<L1>(a, 2 * qb + 1, 2 * qa + 1, 0u, lane);
                        break;
                    case OP_CZ:
                        if (k == 0) column_product<L1>(a, 2 * qa, 2 * qb + 1, 0u, lane);
                        else column_product<L1>(a, 2 * qb, 2 * qa + 1, 0u, lane);
                        break;
                    case OP_SDAG:   // X_a <- +i X_a Z_a
                        if (k == 0) column_product<L1>(a, 2 * qa, 2 * qa + 1, 1u, lane);
                        break;
                    case OP_SX:     // Z_a <- Y_a = -i Z_a X_a
                        if (k == 0) column_product<L1>(a, 2 * qa + 1, 2 * qa, 3u, lane);
                        break;
                    case OP_SXD:    // Z_a <- -Y_a = +i Z_a X_a
                        if (k == 0) column_product<L1>(a, 2 * qa + 1, 2 * qa, 1u, lane);
                        break;
                    case OP_X:      // Z_a <- -Z_a
                    case OP_Y:      // X_a <- -X_a, Z_a <- -Z_a
                    case OP_Z:      // X_a <- -X_a
                        if (k == 0 && lane == 0) {
                            if (opc != OP_X) {
                                const uint32_t c = ld_u32<L1>(a.perm + 2 * qa);
                                st_tab<L1>(a.sign + c, ld_u32<L1>(a.sign + c) ^ 1u);
                            }
                            if (opc != OP_Z) {
                                const uint32_t c = ld_u32<L1>(a.perm + 2 * qa + 1);
                                st_tab<L1>(a.sign + c, ld_u32<L1>(a.sign + c) ^ 1u);
                            }
                        }
                        break;
                    case OP_FFX:    // X_a (Z_a <- -Z_a) when the reference outcome of the record is 1
                    case OP_FFZ:    // Z_a (X_a <- -X_a) likewise
                        if (k == 0 && lane == 0) {
                            const uint32_t m = op.b + meas_off;
                            if ((ld_u64<L1>(a.ref + (m >> 6)) >> (m & 63)) & 1ull) {
                                const uint32_t c = ld_u32<L1>(a.perm + 2 * qa + (opc == OP_FFX ? 1u : 0u));
                                st_tab<L1>(a.sign + c, ld_u32<L1>(a.sign + c) ^ 1u);
                            }
                        }
                        break;
                    case OP_SY:     // X_a <- Z_a, Z_a <- -X_a: swap, then negate the new Z column
                    case OP_SYD:    // X_a <- -Z_a, Z_a <- X_a: swap, then negate the new X column
                        if (k == 0 && lane == 0) {
                            const uint32_t u = ld_u32<L1>(a.perm + 2 * qa), v = ld_u32<L1>(a.perm + 2 * qa + 1);
                            st_tab<L1>(a.perm + 2 * qa, v);
                            st_tab<L1>(a.perm + 2 * qa + 1, u);
                            const uint32_t c = opc == OP_SY ? u : v;
                            st_tab<L1>(a.sign + c, ld_u32<L1>(a.sign + c) ^ 1u);
                        }
                        break;
                    default:
                        break;
                }
            }
            if (!tab_barrier(a)) return;
        }
        if (e.n_collapse == 0) continue;
        const DevOp *cops = ops + e.n_gate + e.n_noise;
        const uint32_t nc = e.n_collapse;
        // (A) which collapsing ops are random, checked in parallel
        for (uint32_t j = gwarp; j < nc; j += nwarps) {
            const uint32_t q = cops[j].a & kQubitMask;
            const uint64_t *x = a.tx + (uint64_t)ld_u32<L1>(a.perm + 2 * q + 1) * a.nw;
            uint32_t any = 0;
            for (uint32_t w = lane; w < a.nw; w += 32) any |= ld_u64<L1>(x + w) != 0;
            any = __any_sync(0xffffffffu, any);
            if (lane == 0) st_tab<L1>(a.rnd + j, any);
        }
        if (!tab_barrier(a)) return;
        // (B) first random op; everything before it is deterministic and independent
        if (threadIdx.x == 0) {
            s_first = nc;
            s_nrand = 0;
        }
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < nc; j += blockDim.x)
            if (ld_u32<L1>(a.rnd + j)) {
                atomicMin(&s_first, j);
                atomicAdd(&s_nrand, 1u);
            }
        __syncthreads();
        const uint32_t first = s_first;
        // row-major burst for this layer's random measurements: the same
        // choice in every CTA (the statistics last changed before the barrier above)
        bool burst = false, wide = false;
        // the burst cluster, taken only when the launch really is a cluster
        // launch of that size (a launch that lost its cluster shape walks its
        // bursts on CTA 0); crank: this CTA's rank in cluster 0, else bclu
        uint32_t bclu = 1, crank = 0;
        if constexpr (CLU) {
            if (a.bclu > 1) {
                uint32_t ncta, cx;
                asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(ncta));
                asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(cx));
                asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
                if (ncta == a.bclu && gridDim.x % a.bclu == 0) bclu = a.bclu;
                if (cx != 0) crank = bclu;
            }
        }
        if (!L1 && a.rx != nullptr && s_nrand >= kBurstMinRandom && nc - s_first <= kBurstMaxOps) {
            const uint32_t kc = ld_u32<L1>(&a.ctl->nk_cnt), ks = ld_u32<L1>(&a.ctl->nk_sum);
            // fan-out words of the random measurements so far, against what one
            // CTA (or, in a cluster launch, the burst cluster) takes
            const uint64_t work = (uint64_t)ks * a.nw2, one = (uint64_t)kBurstMaxRowWords * kc;
            const bool clu = CLU && bclu > 1;
            burst = kc >= 4 && (work <= one || (clu && work <= one * bclu));
            wide = clu && (a.n >= kBurstClusterMinQubits || work > one);
        }
        for (uint32_t j = gtid; j < first; j += nthreads) {
            const DevOp op = cops[j];
            const uint32_t opc = op.a >> 24, q = op.a & kQubitMask;
            const uint32_t pz = ld_u32<L1>(a.perm + 2 * q + 1);
            write_outcome(a, opc, op.b + meas_off, ld_u32<L1>(a.sign + pz), 1);
            if (opc != OP_M) st_tab<L1>(a.sign + pz, 0u);
        }
        if (!tab_barrier(a)) return;
        if (first >= nc) continue;
        if (burst) {
            to_rows(a, gtid, nthreads);
            if (!tab_barrier(a)) return;
            if (wide) {
                if (crank < bclu) burst_walk<true>(a, cops, nc, first, meas_off, crank, bclu);
            } else if (bid == 0) {
                burst_walk<false>(a, cops, nc, first, meas_off, 0u, 1u);
            }
            if (!tab_barrier(a)) return;
            to_cols(a, gtid, nthreads);
            if (!tab_barrier(a)) return;
            continue;
        }
        // (C) sequential from the first random op
        uint32_t j = first;
        for (;;) {
            if (leader) leader_walk<L1>(a, cops, nc, j, meas_off, lane);
            if (!tab_barrier(a)) return;
            if (!ld_u32<L1>(&a.ctl->has_random)) break;
            j = ld_u32<L1>(&a.ctl->next_j);
            const uint32_t p = ld_u32<L1>(&a.ctl->pivot), nk = ld_u32<L1>(&a.ctl->nk);
            const uint32_t py = ld_u32<L1>(&a.ctl->pivot_is_y), fx = ld_u32<L1>(&a.ctl->fix_x);
            if (ld_u32<L1>(&a.ctl->use_mask)) column_pass_mask<L1>(a, p, py, fx, gwarp, nwarps, lane);
            else column_pass_list<L1>(a, p, nk, py, fx, gtid, nthreads);
            if (!tab_barrier(a)) return;
            j++;
        }
    }
}

template <bool L1>
__global__ void __launch_bounds__(kTableauMaxThreads) tableau_kernel(TabArgs a) {
    tableau_body<L1, !L1>(a, blockIdx.x);
}

// Several circuits in one cooperative launch: CTA b works for circuit
// job_of[b] as its CTA b - first[job_of[b]]; each circuit's CTAs meet only at
// that circuit's barrier.
__global__ void __launch_bounds__(kTableauMaxThreads) tableau_batch_kernel(const TabArgs *jobs, const uint32_t *job_of,
                                                            const uint32_t *first) {
    const uint32_t j = job_of[blockIdx.x];
    tableau_body<false>(jobs[j], blockIdx.x - first[j]);     // arguments read in place (global, cached)
}

cudaError_t launch_tableau_init(const TabArgs &a, cudaStream_t stream) {
    const uint32_t threads = 256;
    uint32_t blocks = (a.n + threads - 1) / threads;
    if (blocks == 0) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    tableau_init_kernel<<<blocks, threads, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tableau_batch(const TabArgs *jobs, const uint32_t *job_of, const uint32_t *first, uint32_t blocks,
                                 uint32_t threads, cudaStream_t stream) {
    const TabArgs *j = jobs;
    const uint32_t *o = job_of, *f = first;
    void *params[] = {(void *)&j, (void *)&o, (void *)&f};
    return cudaLaunchCooperativeKernel((const void *)tableau_batch_kernel, dim3(blocks), dim3(threads), params, 0,
                                       stream);
}

int tableau_batch_max_blocks(uint32_t threads, int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tableau_batch_kernel, (int)threads, 0) != cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    const int b = per_sm * sms;
    return b > 0 ? b : 1;
}

int tableau_max_blocks(uint32_t threads, int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tableau_kernel<false>, (int)threads, 0) !=
        cudaSuccess)
        return 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 1;
    const int b = per_sm * sms;
    return b > 0 ? b : 1;
}

cudaError_t launch_tableau(const TabArgs &a, uint32_t blocks, uint32_t threads, cudaStream_t stream) {
    TabArgs args = a;
    args.nblk = blocks;
    args.bclu = 1;
    void *params[] = {&args};
    if (blocks == 1)    // one CTA: the tableau stays in its L1, no grid barrier
        return cudaLaunchCooperativeKernel((const void *)tableau_kernel<true>, dim3(1), dim3(threads), params, 0,
                                           stream);
    // a large circuit with a row-major copy is launched as clusters of
    // kBurstCluster CTAs (still cooperative: every CTA co-resident), so that
    // cluster 0 walks its bursts with kBurstCluster times the threads. A
    // cluster barrier costs far more than a CTA barrier, and a burst takes
    // four per random measurement, so this pays only where each random
    // measurement's row scan is long: from kBurstClusterMinQubits qubits
    // (surface code d=100, 20k qubits: reference 0.31 -> 0.18 s; Bacon-Shor
    // d=60, 10.7k qubits: 3.9 -> 4.5 s, and worse for smaller circuits).
    if (a.rx != nullptr && blocks >= 2 * kBurstCluster) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kBurstCluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cfg.blockDim = dim3(threads);
        cfg.stream = stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(blocks - blocks % kBurstCluster);     // the query wants whole clusters
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, tableau_kernel<false>, &cfg) == cudaSuccess && clusters >= 2) {
            uint32_t b = blocks < (uint32_t)clusters * kBurstCluster ? blocks : (uint32_t)clusters * kBurstCluster;
            b -= b % kBurstCluster;
            args.nblk = b;
            args.bclu = kBurstCluster;
            cfg.gridDim = dim3(b);
            cfg.numAttrs = 2;
            if (cudaLaunchKernelEx(&cfg, tableau_kernel<false>, args) == cudaSuccess) return cudaSuccess;
        }
        cudaGetLastError();     // not launched: the plain cooperative grid below
        args.nblk = blocks;
        args.bclu = 1;
    }
    return cudaLaunchCooperativeKernel((const void *)tableau_kernel<false>, dim3(blocks), dim3(threads), params, 0,
                                       stream);
}

}  // namespace stimgb
