// radix.cuh -- stable LSD radix sort of 64-bit keys with 32-bit values, one
// 8-bit digit per pass (digit histograms per tile, an exclusive scan of them,
// a stable scatter).  Used by the banding step (band keys) and the
// prefix-filter candidate generator (index entries and candidate pairs).
#pragma once

#include "common.cuh"
#include "scan.cuh"

namespace blsh_radix {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSortThreads = 256;
constexpr int kSortPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortPerThread;   // 4096 items per CTA
constexpr int kWarps = kSortThreads / 32;

// ---- stable LSD radix sort, one 8-bit digit per pass ----------------------

static __global__ void __launch_bounds__(kSortThreads) digit_hist_kernel(const unsigned long long *keys, long long n,
                                                                  int shift, uint32_t *hist, int tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortPerThread; ++i) {
        const long long p = base + (long long)i * kSortThreads + threadIdx.x;
        if (p < n) atomicAdd(&h[(keys[p] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Scatter with stable ranks: warp w handles the contiguous items
// [w*512, (w+1)*512) of the tile, 32 at a time; lanes holding the same digit
// are ranked with __match_any_sync, running counts per (warp, digit) live in
// shared memory, and warps are then offset by the counts of lower warps.
static __global__ void __launch_bounds__(kSortThreads) digit_scatter_kernel(const unsigned long long *keys_in,
                                                                     const uint32_t *vals_in, long long n,
                                                                     int shift, const uint32_t *offsets, int tiles,
                                                                     unsigned long long *keys_out,
                                                                     uint32_t *vals_out) {
    __shared__ uint32_t cnt[kWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const long long base = (long long)blockIdx.x * kSortTile + (long long)w * (kSortTile / kWarps);
    unsigned long long k[kSortPerThread];
    uint32_t v[kSortPerThread], rank[kSortPerThread];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const long long p = base + r * 32 + lane;
        const bool ok = p < n;
        k[r] = ok ? keys_in[p] : 0ull;
        v[r] = ok ? vals_in[p] : 0u;
        const uint32_t d = ok ? (uint32_t)((k[r] >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t before = ok ? cnt[w][d] : 0u;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0) cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps, per digit
    for (int d = threadIdx.x; d < 256; d += kSortThreads) {
        uint32_t s = 0;
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = cnt[ww][d];
            cnt[ww][d] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const long long p = base + r * 32 + lane;
        if (p < n) {
            const uint32_t d = (uint32_t)((k[r] >> shift) & 255u);
            const long long dst = (long long)offsets[(size_t)d * tiles + blockIdx.x] + cnt[w][d] + rank[r];
            keys_out[dst] = k[r];
            vals_out[dst] = v[r];
        }
    }
}


// Entries of hist (256 per tile) and of the scan's partial sums that sort()
// needs for n items.
inline long long hist_entries(long long n) { return 256 * ((n + kSortTile - 1) / kSortTile); }
inline long long partial_entries(long long n) { return blsh_scan::tiles_for(hist_entries(n)) + 1; }

// Sorts keys[0][0..n) (and vals[0] alongside) by their bits
// first_bit .. first_bit + key_bits - 1, stably (items equal there keep their
// order), ping-ponging between buffers 0 and 1; *cur receives the index of
// the buffer that holds the result.  hist: hist_entries(n) uint32; partial:
// partial_entries(n) uint32; grand: one uint32 (device).
inline int sort(blsh_ctx *ctx, unsigned long long *keys[2], uint32_t *vals[2], long long n, int key_bits,
                uint32_t *hist, uint32_t *partial, uint32_t *grand, cudaStream_t s, int *cur_out,
                int first_bit = 0) {
    const int passes = (key_bits + 7) / 8;
    const long long tiles = (n + kSortTile - 1) / kSortTile;
    int cur = 0;
    for (int pass = 0; pass < passes && n > 0; ++pass) {
        const int shift = first_bit + 8 * pass;
        blsh_time_start(ctx, s);
        digit_hist_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(keys[cur], n, shift, hist, (int)tiles);
        BLSH_LAUNCHED(ctx, "digit_hist_kernel");
        blsh_time_start(ctx, s);
        BLSH_CUDA(ctx, blsh_scan::exclusive_scan<uint32_t>(hist, hist, 256 * tiles, partial, grand, s));
        ctx->launches.fetch_add(3, std::memory_order_relaxed);
        blsh_time_stop(ctx, "exclusive scan (3 launches)");
        blsh_time_start(ctx, s);
        digit_scatter_kernel<<<(unsigned)tiles, kSortThreads, 0, s>>>(keys[cur], vals[cur], n, shift, hist,
                                                                      (int)tiles, keys[cur ^ 1], vals[cur ^ 1]);
        BLSH_LAUNCHED(ctx, "digit_scatter_kernel");
        cur ^= 1;
    }
    *cur_out = cur;
    return BLSH_OK;
}

}  // namespace blsh_radix
