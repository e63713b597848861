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
static_assert(kSortThreads == 256, "digit_scatter_kernel gives each of the 256 digits one thread");

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

// Scatter with stable ranks, through shared memory.  Warp w ranks the
// contiguous items [w*512, (w+1)*512) of the tile, 32 at a time: lanes
// holding the same digit are ranked with __match_any_sync and running counts
// per (warp, digit) live in shared memory; only the digits and ranks stay in
// registers.  The warps' counts are then offset by those of lower warps, the
// tile's digit totals scanned, and every item placed in shared memory in
// digit order (its tile items re-read, from L2); finally consecutive threads
// write consecutive positions, so each digit's run of the tile goes out in
// coalesced stores.  Equal digits keep the tile's order (warp, then round,
// then lane), so the sort is stable.
constexpr size_t kScatterSmem = (size_t)kSortTile * (sizeof(unsigned long long) + sizeof(uint32_t)) +
                                (size_t)kWarps * 256 * sizeof(uint32_t) + 256 * sizeof(uint32_t);
static __global__ void __launch_bounds__(kSortThreads) digit_scatter_kernel(const unsigned long long *keys_in,
                                                                     const uint32_t *vals_in, long long n,
                                                                     int shift, const uint32_t *offsets, int tiles,
                                                                     unsigned long long *keys_out,
                                                                     uint32_t *vals_out) {
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long *s_key = reinterpret_cast<unsigned long long *>(sm);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(s_key + kSortTile);
    uint32_t(*cnt)[256] = reinterpret_cast<uint32_t(*)[256]>(s_val + kSortTile);
    uint32_t *s_start = reinterpret_cast<uint32_t *>(cnt + kWarps);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) cnt[w][d] = 0;
    __syncwarp();
    const long long tile0 = (long long)blockIdx.x * kSortTile;
    const long long base = tile0 + (long long)w * (kSortTile / kWarps);
    uint32_t dig[kSortPerThread], rank[kSortPerThread];
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const long long p = base + r * 32 + lane;
        const bool ok = p < n;
        const uint32_t d = ok ? (uint32_t)((keys_in[p] >> shift) & 255u) : 256u;
        dig[r] = d;
        const unsigned peers = __match_any_sync(kFull, d);
        const uint32_t before = ok ? cnt[w][d] : 0u;
        rank[r] = before + __popc(peers & lt);
        __syncwarp();
        if (ok && (peers & lt) == 0) cnt[w][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then the tile's digit totals scanned
    uint32_t total = 0;
    {
        const int d = threadIdx.x;   // kSortThreads == 256: one digit per thread
        for (int ww = 0; ww < kWarps; ++ww) {
            const uint32_t c = cnt[ww][d];
            cnt[ww][d] = total;
            total += c;
        }
    }
    const uint32_t start = blsh_scan::block_exclusive<uint32_t>(total, nullptr);
    s_start[threadIdx.x] = start;
    __syncthreads();
    // the tile in digit order in shared memory
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const long long p = base + r * 32 + lane;
        if (p < n) {
            const uint32_t pos = s_start[dig[r]] + cnt[w][dig[r]] + rank[r];
            s_key[pos] = keys_in[p];
            s_val[pos] = vals_in[p];
        }
    }
    __syncthreads();
    const int tn = (int)(n - tile0 < kSortTile ? n - tile0 : kSortTile);
    for (int i = threadIdx.x; i < tn; i += kSortThreads) {
        const unsigned long long k = s_key[i];
        const uint32_t d = (uint32_t)((k >> shift) & 255u);
        const long long dst = (long long)offsets[(size_t)d * tiles + blockIdx.x] + (i - (int)s_start[d]);
        keys_out[dst] = k;
        vals_out[dst] = s_val[i];
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
    BLSH_CUDA(ctx, cudaFuncSetAttribute(digit_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kScatterSmem));
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
        digit_scatter_kernel<<<(unsigned)tiles, kSortThreads, kScatterSmem, s>>>(
            keys[cur], vals[cur], n, shift, hist, (int)tiles, keys[cur ^ 1], vals[cur ^ 1]);
        BLSH_LAUNCHED(ctx, "digit_scatter_kernel");
        cur ^= 1;
    }
    *cur_out = cur;
    return BLSH_OK;
}

}  // namespace blsh_radix
