// compact.cu -- the output set O of Algorithms 1 and 2: a stable compaction
// of the retained pair indices.
//
// A fixed grid of C CTAs splits [0, P) into C contiguous ranges (starting
// at multiples of 16 statuses, read 16 at a time).  Pass 1
// counts the kept items of each range; pass 2 gives each CTA the sum of the
// counts of the ranges before it and writes its range's indices in order,
// one tile at a time with a block-wide prefix sum.  The count array (C
// entries) lives in the context's scratch area.
#include "common.cuh"
#include "scan.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 16;
constexpr int kTile = kThreads * kPer;

__device__ __forceinline__ bool kept(uint8_t st, uint32_t mask) { return st < 32 && ((mask >> st) & 1u); }

__device__ __forceinline__ long long resolve_p(long long P, const long long *P_dev) {
    if (!P_dev) return P;
    const long long pd = *P_dev;
    return pd < 0 ? 0 : (pd < P ? pd : P);
}

// CTA b owns [lo, hi): P * b / C rounded down to a multiple of 16, so that
// with a 16-byte aligned status array every thread reads its 16 statuses
// with one 16-byte load.
__device__ __forceinline__ void cta_range(long long P, long long &lo, long long &hi) {
    lo = (P * blockIdx.x / gridDim.x) & ~15ll;
    hi = blockIdx.x + 1 == gridDim.x ? P : (P * (blockIdx.x + 1) / gridDim.x) & ~15ll;
}

// Bit i of the result: status q0 + i is kept (q0 + i < hi).
__device__ __forceinline__ uint32_t kept16(const uint8_t *status, long long q0, long long hi, uint32_t mask,
                                           bool vec) {
    uint32_t bits = 0;
    if (vec && q0 + 16 <= hi) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(status + q0));
        for (uint32_t m = mask; m; m &= m - 1) bits |= blsh_eq16(v, (uint32_t)(__ffs(m) - 1));   // each kept status
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (q0 + i < hi) bits |= (uint32_t)kept(status[q0 + i], mask) << i;
    }
    return bits;
}

__global__ void __launch_bounds__(kThreads) compact_count(const uint8_t *status, long long P_cap,
                                                          const long long *P_dev, uint32_t mask, bool vec,
                                                          blsh_dev_scratch *scratch) {
    const long long P = resolve_p(P_cap, P_dev);
    long long lo, hi;
    cta_range(P, lo, hi);
    long long c = 0;
#pragma unroll 4
    for (long long q0 = lo + 16ll * threadIdx.x; q0 < hi; q0 += 16ll * kThreads)
        c += __popc(kept16(status, q0, hi, mask, vec));
    long long total;
    blsh_scan::block_exclusive<long long>(c, &total);
    if (threadIdx.x == 0) scratch->cta_counts[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kThreads) compact_write(const uint8_t *status, long long P_cap,
                                                          const long long *P_dev, uint32_t mask, bool vec,
                                                          int64_t *out, long long cap, long long *n_out,
                                                          blsh_dev_scratch *scratch) {
    __shared__ long long s_base;
    const long long P = resolve_p(P_cap, P_dev);
    long long lo, hi;
    cta_range(P, lo, hi);
    long long before = 0;
    for (int c = threadIdx.x; c < (int)blockIdx.x; c += kThreads) before += scratch->cta_counts[c];
    long long tot;
    blsh_scan::block_exclusive<long long>(before, &tot);
    if (threadIdx.x == 0) s_base = tot;
    __syncthreads();
    long long base = s_base;
    // kBatch tiles at a time: their loads are issued together, then each
    // tile gets its block-wide prefix sum and writes its indices in order
    constexpr int kBatch = 8;
    for (long long t0 = lo; t0 < hi; t0 += (long long)kBatch * kTile) {
        uint32_t bits[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const long long q0 = t0 + (long long)u * kTile + (long long)threadIdx.x * kPer;
            bits[u] = q0 < hi ? kept16(status, q0, hi, mask, vec) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            if (t0 + (long long)u * kTile >= hi) break;      // uniform across the CTA
            const long long q0 = t0 + (long long)u * kTile + (long long)threadIdx.x * kPer;
            long long tile_total;
            long long o = base + blsh_scan::block_exclusive<long long>((long long)__popc(bits[u]), &tile_total);
            for (uint32_t b = bits[u]; b; b &= b - 1) {
                if (o < cap) out[o] = q0 + __ffs(b) - 1;
                ++o;
            }
            base += tile_total;
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
        *n_out = base;
        if (base > cap) blsh_dev_error(scratch, BLSH_ETRUNC, 1, (unsigned long long)(base - cap));
    }
}

}  // namespace

extern "C" int blsh_compact(blsh_ctx *ctx, const uint8_t *status, int64_t P, const int64_t *P_dev,
                            uint32_t keep_mask, int64_t *out_idx, int64_t cap, int64_t *n_out, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!n_out || (P > 0 && !status) || (cap > 0 && !out_idx))
        return blsh_fail(ctx, BLSH_EINVAL, "status and n_out required");
    if (P < 0 || cap < 0) return blsh_fail(ctx, BLSH_EINVAL, "bad P or cap");
    if (!blsh_aligned(out_idx, 8) || !blsh_aligned(n_out, 8) || !blsh_aligned(P_dev, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    long long ctas = (P + kTile - 1) / kTile;
    const long long most = (long long)ctx->sm_count * 4 < BLSH_COMPACT_MAX_CTAS ? (long long)ctx->sm_count * 4
                                                                                 : BLSH_COMPACT_MAX_CTAS;
    if (ctas > most) ctas = most;
    if (ctas < 1) ctas = 1;
    const bool vec = blsh_aligned(status, 16);
    blsh_time_start(ctx, s);
    compact_count<<<(unsigned)ctas, kThreads, 0, s>>>(status, P, (const long long *)P_dev, keep_mask, vec,
                                                      ctx->scratch);
    BLSH_LAUNCHED(ctx, "compact_count");
    blsh_time_start(ctx, s);
    compact_write<<<(unsigned)ctas, kThreads, 0, s>>>(status, P, (const long long *)P_dev, keep_mask, vec, out_idx,
                                                      cap, (long long *)n_out, ctx->scratch);
    BLSH_LAUNCHED(ctx, "compact_write");
    return BLSH_OK;
}
