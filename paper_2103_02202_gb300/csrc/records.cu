// records.cu -- detection events and record layout conversion.
//
// Detection events (Section 5.6 of the paper): a detector is a set of
// measurements whose XOR is deterministic without noise; its event bit is the
// XOR of the measurements' flips, i.e. of (record ^ reference) over its set.
//
// Layout conversion: measurement-major rows (one row per measurement, bit s =
// shot s) become shot-major rows (one row per shot, bit m = measurement m,
// the LSB-first order of the b8 format of Section 5.6). One warp transposes a
// 64 x 64 bit block: lane l holds block rows l and l + 32; a 32-bit-distance
// swap inside the lane and five shuffle-xor stages exchange the off-diagonal
// sub-blocks.
#include <cuda_runtime.h>

#include "device.cuh"
#include "kernels.h"

namespace stimgb {

// One warp per detector row (warps stride over detectors): the detector's
// measurement list and reference bits are warp-uniform loads, and the lanes
// sweep the row's 64-shot words two at a time with 16-byte loads when the
// record rows are 16-byte aligned.
__global__ void __launch_bounds__(256) detector_kernel(const uint64_t *__restrict__ rec, uint64_t rec_stride,
                                                       const uint64_t *__restrict__ det_ptr,
                                                       const uint32_t *__restrict__ det_meas,
                                                       const uint64_t *__restrict__ ref, uint64_t ndet,
                                                       uint64_t nwords, uint64_t last_mask,
                                                       uint64_t *__restrict__ det, uint64_t det_stride) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const bool pairs = (rec_stride % 2 == 0) && (det_stride % 2 == 0) &&
                       ((reinterpret_cast<uintptr_t>(rec) | reinterpret_cast<uintptr_t>(det)) % 16 == 0);
    for (uint64_t k = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < ndet; k += warps) {
        const uint64_t b = __ldg(det_ptr + k), e = __ldg(det_ptr + k + 1);
        uint64_t *out = det + k * det_stride;
        if (pairs) {
            for (uint64_t w = 2 * lane; w < nwords; w += 64) {
                uint64_t v0 = 0, v1 = 0;
                for (uint64_t t = b; t < e; t++) {
                    const uint32_t m = __ldg(det_meas + t);
                    const uint64_t refm = 0ull - ((__ldg(ref + (m >> 6)) >> (m & 63)) & 1ull);
                    const ulonglong2 r = __ldg(reinterpret_cast<const ulonglong2 *>(rec + (uint64_t)m * rec_stride + w));
                    v0 ^= r.x ^ refm;
                    v1 ^= r.y ^ refm;
                }
                if (w == nwords - 1) v0 &= last_mask;
                if (w + 1 == nwords - 1) v1 &= last_mask;
                if (w + 1 < nwords) {
                    *reinterpret_cast<ulonglong2 *>(out + w) = make_ulonglong2(v0, v1);
                } else {
                    out[w] = v0;
                }
            }
        } else {
            for (uint64_t w = lane; w < nwords; w += 32) {
                uint64_t v = 0;
                for (uint64_t t = b; t < e; t++) {
                    const uint32_t m = __ldg(det_meas + t);
                    const uint64_t refm = 0ull - ((__ldg(ref + (m >> 6)) >> (m & 63)) & 1ull);
                    v ^= __ldg(rec + (uint64_t)m * rec_stride + w) ^ refm;
                }
                if (w == nwords - 1) v &= last_mask;
                out[w] = v;
            }
        }
    }
}

__device__ __forceinline__ void transpose64_warp(uint64_t &a0, uint64_t &a1, uint32_t lane) {
    // stage 32: rows r and r + 32 live in the same lane
    {
        const uint64_t m = 0x00000000FFFFFFFFull;
        const uint64_t t = ((a0 >> 32) ^ a1) & m;
        a1 ^= t;
        a0 ^= t << 32;
    }
    const uint64_t masks[5] = {0x0000FFFF0000FFFFull, 0x00FF00FF00FF00FFull, 0x0F0F0F0F0F0F0F0Full,
                               0x3333333333333333ull, 0x5555555555555555ull};
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int j = 16 >> s;
        const uint64_t m = masks[s];
        const uint64_t p0 = __shfl_xor_sync(0xffffffffu, a0, j);
        const uint64_t p1 = __shfl_xor_sync(0xffffffffu, a1, j);
        if ((lane & j) == 0) {      // this lane holds the upper row r, partner row r + j
            a0 ^= (((a0 >> j) ^ p0) & m) << j;
            a1 ^= (((a1 >> j) ^ p1) & m) << j;
        } else {                    // this lane holds row r + j, partner row r
            a0 ^= ((p0 >> j) ^ a0) & m;
            a1 ^= ((p1 >> j) ^ a1) & m;
        }
    }
}

// One warp per 64 x 64 block; a CTA's warps take consecutive row blocks of the
// same column block so that each output row receives a contiguous run.
__global__ void __launch_bounds__(256) transpose_kernel(const uint64_t *__restrict__ in, uint64_t rows,
                                                        uint64_t in_stride, uint64_t cols,
                                                        uint64_t *__restrict__ out, uint64_t out_stride) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x >> 5;
    const uint64_t row_blocks = (rows + 63) / 64;
    const uint64_t col_blocks = (cols + 63) / 64;
    const uint64_t rb_groups = (row_blocks + wpb - 1) / wpb;
    const uint64_t total = rb_groups * col_blocks;
    for (uint64_t g = blockIdx.x; g < total; g += gridDim.x) {
        const uint64_t cb = g / rb_groups;
        const uint64_t rb = (g % rb_groups) * wpb + (threadIdx.x >> 5);
        if (rb >= row_blocks) continue;
        const uint64_t r0 = rb * 64 + lane, r1 = r0 + 32;
        uint64_t a0 = r0 < rows ? __ldg(in + r0 * in_stride + cb) : 0;
        uint64_t a1 = r1 < rows ? __ldg(in + r1 * in_stride + cb) : 0;
        transpose64_warp(a0, a1, lane);
        const uint64_t c0 = cb * 64 + lane, c1 = c0 + 32;
        if (c0 < cols) out[c0 * out_stride + rb] = a0;
        if (c1 < cols) out[c1 * out_stride + rb] = a1;
    }
}

// ---- per-shot lists of fired detectors (CSR) from shot-major event rows ----

// counts[s] = number of set bits of row s (one warp per row).
__global__ void __launch_bounds__(256) hits_count_kernel(const uint64_t *__restrict__ rows, uint64_t nrows,
                                                         uint64_t stride, uint32_t *__restrict__ counts) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += warps) {
        const uint64_t *row = rows + r * stride;
        uint32_t c = 0;
        for (uint64_t w = lane; w < stride; w += 32) c += __popcll(__ldg(row + w));
        for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
        if (lane == 0) counts[r] = c;
    }
}

// Inclusive scan of counts inside blocks of 1024: part[s], block totals tot[b].
__global__ void __launch_bounds__(1024) hits_scan_kernel(const uint32_t *__restrict__ counts, uint64_t n,
                                                         uint64_t *__restrict__ part, uint64_t *__restrict__ tot) {
    __shared__ uint64_t warp_sum[32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t i = (uint64_t)blockIdx.x * 1024 + threadIdx.x;
    uint64_t v = i < n ? counts[i] : 0;
    for (int d = 1; d < 32; d <<= 1) {
        const uint64_t u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    if (lane == 31) warp_sum[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = warp_sum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= (uint32_t)d) w += u;
        }
        warp_sum[lane] = w;     // inclusive over warps
    }
    __syncthreads();
    if (warp > 0) v += warp_sum[warp - 1];
    if (i < n) part[i] = v;
    if (threadIdx.x == 1023) tot[blockIdx.x] = v;
}

// Exclusive scan of the block totals, in place (one thread: a few thousand
// blocks at most per call), then begin[0] = 0 and begin[s + 1] = part[s] +
// the exclusive total of s's block.
__global__ void hits_block_offsets_kernel(uint64_t *tot, uint64_t nblocks) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    uint64_t run = 0;
    for (uint64_t b = 0; b < nblocks; b++) {
        const uint64_t t = tot[b];
        tot[b] = run;
        run += t;
    }
}

__global__ void hits_begin_kernel(const uint64_t *__restrict__ part, const uint64_t *__restrict__ off, uint64_t n,
                                  uint64_t *__restrict__ begin) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (uint64_t)gridDim.x * blockDim.x)
        begin[i] = i == 0 ? 0 : part[i - 1] + off[(i - 1) / 1024];
}

// Writes the fired columns of row r at begin[r]... (one warp per row; lanes
// take 32 consecutive words, a warp prefix sum of their popcounts places each
// lane's bits). Entries at or beyond `capacity` are not written.
__global__ void __launch_bounds__(256) hits_write_kernel(const uint64_t *__restrict__ rows, uint64_t nrows,
                                                         uint64_t stride, const uint64_t *__restrict__ begin,
                                                         uint32_t *__restrict__ out, uint64_t capacity) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t r = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nrows; r += warps) {
        const uint64_t *row = rows + r * stride;
        uint64_t base = begin[r];
        for (uint64_t w0 = 0; w0 < stride; w0 += 32) {
            const uint64_t w = w0 + lane;
            uint64_t bits = w < stride ? __ldg(row + w) : 0;
            const uint32_t c = __popcll(bits);
            uint32_t incl = c;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= (uint32_t)d) incl += u;
            }
            uint64_t pos = base + incl - c;
            while (bits) {
                const uint32_t b = (uint32_t)__ffsll((long long)bits) - 1u;
                bits &= bits - 1;
                if (pos < capacity) out[pos] = (uint32_t)(w * 64 + b);
                pos++;
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

static uint32_t grid_for(uint64_t items, uint32_t threads) {
    uint64_t g = (items + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535ull * 32) g = 65535ull * 32;
    return (uint32_t)g;
}

cudaError_t launch_detectors(const uint64_t *rec, uint64_t rec_stride, const uint64_t *det_ptr,
                             const uint32_t *det_meas, const uint64_t *ref, uint64_t ndet, uint64_t nwords,
                             uint64_t last_mask, uint64_t *det, uint64_t det_stride, cudaStream_t stream) {
    if (ndet == 0 || nwords == 0) return cudaSuccess;
    const uint32_t threads = 256;
    detector_kernel<<<grid_for(ndet, threads / 32), threads, 0, stream>>>(rec, rec_stride, det_ptr, det_meas, ref,
                                                                         ndet, nwords, last_mask, det, det_stride);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const uint64_t *in, uint64_t rows, uint64_t in_stride, uint64_t cols,
                             uint64_t *out, uint64_t out_stride, cudaStream_t stream) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const uint32_t threads = 256;
    const uint64_t row_blocks = (rows + 63) / 64, col_blocks = (cols + 63) / 64;
    const uint64_t groups = ((row_blocks + 7) / 8) * col_blocks;
    uint64_t grid = groups < 1 ? 1 : groups;
    if (grid > 1u << 20) grid = 1u << 20;
    transpose_kernel<<<(uint32_t)grid, threads, 0, stream>>>(in, rows, in_stride, cols, out, out_stride);
    return cudaGetLastError();
}

cudaError_t launch_hits(const uint64_t *rows, uint64_t nrows, uint64_t stride, uint32_t *counts, uint64_t *part,
                        uint64_t *tot, uint64_t *begin, cudaStream_t stream) {
    if (nrows == 0) {
        return cudaMemsetAsync(begin, 0, sizeof(uint64_t), stream);
    }
    const uint32_t warps_per_block = 8;
    const uint32_t grid = grid_for(nrows, warps_per_block);
    hits_count_kernel<<<grid, 32 * warps_per_block, 0, stream>>>(rows, nrows, stride, counts);
    const uint64_t nblocks = (nrows + 1023) / 1024;
    hits_scan_kernel<<<(uint32_t)nblocks, 1024, 0, stream>>>(counts, nrows, part, tot);
    hits_block_offsets_kernel<<<1, 1, 0, stream>>>(tot, nblocks);
    hits_begin_kernel<<<grid_for(nrows + 1, 256), 256, 0, stream>>>(part, tot, nrows, begin);
    return cudaGetLastError();
}

cudaError_t launch_hits_write(const uint64_t *rows, uint64_t nrows, uint64_t stride, const uint64_t *begin,
                              uint32_t *out, uint64_t capacity, cudaStream_t stream) {
    if (nrows == 0) return cudaSuccess;
    const uint32_t warps_per_block = 8;
    hits_write_kernel<<<grid_for(nrows, warps_per_block), 32 * warps_per_block, 0, stream>>>(rows, nrows, stride,
                                                                                           begin, out, capacity);
    return cudaGetLastError();
}

}  // namespace stimgb
