// sph_blocksort.cuh -- stable radix sort of one index range by one thread block (the
// crowded cells of the grid order: their particles are put in id order here instead of
// being ranked one by one by counting, which is quadratic in the cell's occupancy).
#pragma once

#include <stdint.h>

namespace sph {

constexpr int kLargeThreads = 1024;

// Stable sort of the pairs (key[t], val[t]), t in [b, e), by the 32-bit key, by the calling
// block of kLargeThreads threads (every thread must call it).  Four counting-sort passes
// of 8 bits, least significant first; each pass takes the histogram of the range and its
// exclusive scan, then walks the range in tiles of one element per thread, in order,
// placing each element after the same-digit elements of earlier tiles, of earlier warps
// of its tile and of earlier lanes of its warp (stable).  Passes alternate between
// (key, val) and (key2, val2), so after the fourth the result is back in (key, val).
__device__ __forceinline__ void block_sort_segment(uint32_t *key, uint32_t *val, uint32_t *key2, uint32_t *val2,
                                                   uint32_t b, uint32_t e)
{
    constexpr int kWarps = kLargeThreads / 32;
    __shared__ uint32_t s_base[256];              // next position of each digit
    __shared__ uint32_t s_tile[256];              // the tile's count of each digit
    __shared__ uint16_t s_cnt[kWarps][256];       // per warp and digit: count, then prefix
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t *ks = key, *vs = val, *kd = key2, *vd = val2;
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 8 * pass;
        for (int d = tid; d < 256; d += kLargeThreads) s_base[d] = 0u;
        __syncthreads();
        for (uint32_t t = b + (uint32_t)tid; t < e; t += kLargeThreads) atomicAdd(&s_base[(ks[t] >> sh) & 255u], 1u);
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 256 counts, 8 per lane, offset by the range start
            uint32_t c[8], sum = 0u;
#pragma unroll
            for (int q = 0; q < 8; ++q) { c[q] = s_base[8 * lane + q]; sum += c[q]; }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            uint32_t run = b + incl - sum;
#pragma unroll
            for (int q = 0; q < 8; ++q) { s_base[8 * lane + q] = run; run += c[q]; }
        }
        __syncthreads();
        for (uint32_t t0 = b; t0 < e; t0 += kLargeThreads) {
            const uint32_t t = t0 + (uint32_t)tid;
            const bool ok = t < e;
            const uint32_t k = ok ? ks[t] : 0u, v = ok ? vs[t] : 0u;
            const uint32_t d = ok ? (k >> sh) & 255u : 256u;   // 256: past the range
            for (int q = tid; q < kWarps * 256; q += kLargeThreads) s_cnt[q >> 8][q & 255] = 0;
            __syncthreads();
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const unsigned before = peers & ((1u << lane) - 1u);
            if (ok && before == 0u) s_cnt[warp][d] = (uint16_t)__popc(peers);
            __syncthreads();
            if (tid < 256) {   // counts -> exclusive prefix over the warps, and the tile's total
                uint32_t run = 0u;
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t cw = s_cnt[w][tid];
                    s_cnt[w][tid] = (uint16_t)run;
                    run += cw;
                }
                s_tile[tid] = run;
            }
            __syncthreads();
            if (ok) {
                const uint32_t pos = s_base[d] + s_cnt[warp][d] + (uint32_t)__popc(before);
                kd[pos] = k;
                vd[pos] = v;
            }
            __syncthreads();
            if (tid < 256) s_base[tid] += s_tile[tid];
            __syncthreads();
        }
        uint32_t *tk = ks; ks = kd; kd = tk;
        uint32_t *tv = vs; vs = vd; vd = tv;
        __syncthreads();
    }
}

}  // namespace sph
