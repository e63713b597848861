// allpairs.cu -- candidate generation by prefix filtering: the AllPairs
// method (Bayardo, Ma and Srikant, "Scaling up all pairs similarity search",
// WWW 2007), which Section 5.1 pairs with BayesLSH as the other source of
// candidates besides LSH.
//
//   1. feature statistics: document frequency df_f and the largest |weight|
//      maxabs_f of every feature (atomics over the nonzeros);
//   2. every row's indexed features.  Walking the row in the global order
//      (decreasing df, then increasing id), a running bound grows by
//      w_e = rn(|x_e| maxabs_f 2^48) (cosine; an exact integer sum, so the
//      order of the additions does not matter) or by 1 (sets); a feature is
//      indexed once the bound including it reaches the row's threshold
//      (cosine: ceil((t - 1e-9) 2^48); sets: ceil(t |x| - 1e-9)).  The
//      unindexed prefix then cannot lift a similarity to t, so every pair that
//      reaches t shares an indexed feature of its first row.  Rows of up to
//      32 elements: a warp, lane = element, each lane's bound the sum over the
//      elements that precede or equal it (shuffles); up to 4096: a CTA sorts
//      (order key, position) in shared memory and scans; longer rows index
//      every feature;
//   3. the inverted index: a key (feature, row) per indexed nonzero (padding
//      for the others), radix-sorted, so that a feature's list holds its rows
//      in increasing order, and each feature's list bounds from a scan of the
//      per-feature counts;
//   4. candidates: for every row y and feature f of y, the rows x < y of f's
//      list (a prefix of it, found by binary search) give the keys
//      (x << 32) | y: a count pass, an exclusive scan, a write pass (a warp
//      writes each prefix with coalesced stores);
//   5. the keys are radix-sorted, and the distinct ones are written as pairs
//      (x, y) in increasing order.
#include "common.cuh"
#include "radix.cuh"
#include "scan.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kShortRow = 32;
constexpr int kLongRow = 4096;
constexpr double kTwo48 = 281474976710656.0;
constexpr long long kTermCap = 1ll << 50;

struct ApArgs {
    const int64_t *indptr;
    const uint32_t *indices;
    const float *values;    // NULL for sets
    long long N, dim;
    int cosine;
    double t;
    long long thr;          // cosine threshold in units of 2^-48
    uint32_t *df, *maxabs;  // [dim]: document frequency, largest |weight| (float bits)
    uint8_t *indexed;       // [nnz]
    blsh_dev_scratch *scratch;
};

// rn(|x| maxabs 2^48), capped (the cap lies far above any threshold, so it
// changes no decision and keeps the sums of a row below 2^63)
__device__ __forceinline__ long long ap_weight(const ApArgs &A, long long e, uint32_t f) {
    if (!A.cosine) return 1;
    const double p = __dmul_rn(__dmul_rn((double)fabsf(__ldg(A.values + e)), (double)__uint_as_float(A.maxabs[f])),
                               kTwo48);
    const long long w = __double2ll_rn(p);
    return w > kTermCap ? kTermCap : w;
}

// Threshold of a row of n elements: the bound value from which features are
// indexed (sets: ceil(t n - 1e-9) elements, formed in FP64 exactly as the
// oracle forms it).
__device__ __forceinline__ long long ap_threshold(const ApArgs &A, long long n) {
    if (A.cosine) return A.thr;
    return (long long)ceil(__dadd_rn(__dmul_rn(A.t, (double)n), -1e-9));
}

// Order key: decreasing df, then increasing id (ascending key order).
__device__ __forceinline__ unsigned long long ap_key(const ApArgs &A, uint32_t f) {
    return ((unsigned long long)(0xffffffffu - A.df[f]) << 32) | f;
}

__global__ void __launch_bounds__(256) ap_stats_kernel(ApArgs A, long long nnz) {
    unsigned long long bad = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (long long)gridDim.x * blockDim.x) {
        const uint32_t f = __ldg(A.indices + e);
        if (f >= A.dim) { ++bad; continue; }
        atomicAdd(&A.df[f], 1u);
        if (A.cosine) atomicMax(&A.maxabs[f], __float_as_uint(fabsf(__ldg(A.values + e))));
    }
    if (bad) blsh_dev_error(A.scratch, BLSH_ERANGE, 0, bad);
}

// Rows of up to kShortRow elements (one warp per row, lane = element) and
// rows longer than kLongRow (every feature indexed); the rows in between are
// left to ap_prefix_cta_kernel.
__global__ void __launch_bounds__(256) ap_prefix_warp_kernel(ApArgs A) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < A.N; row += nw) {
        const long long s = __ldg(A.indptr + row), n = __ldg(A.indptr + row + 1) - s;
        if (n > kLongRow) {
            for (long long i = lane; i < n; i += 32) A.indexed[s + i] = 1;
            continue;
        }
        if (n == 0 || n > kShortRow) continue;
        uint32_t f = 0;
        unsigned long long key = ~0ull;
        long long w = 0;
        if (lane < n) {
            f = __ldg(A.indices + s + lane);
            if (f < A.dim) {
                key = ap_key(A, f);
                w = ap_weight(A, s + lane, f);
            }
        }
        // bound including this element: the weights of the elements that
        // precede it in the global order, and its own
        long long b = 0;
        for (int j = 0; j < n; ++j) {
            const unsigned long long kj = __shfl_sync(kFull, key, j);
            const long long wj = __shfl_sync(kFull, w, j);
            if (kj <= key) b += wj;
        }
        if (lane < n) A.indexed[s + lane] = b >= ap_threshold(A, n);
    }
}

// Rows of kShortRow+1 .. kLongRow elements, one CTA per row: (key, position)
// sorted in shared memory (bitonic), the weights scanned in that order.
constexpr int kCtaThreads = 256;
__global__ void __launch_bounds__(kCtaThreads) ap_prefix_cta_kernel(ApArgs A) {
    __shared__ unsigned long long s_key[kLongRow];
    __shared__ uint16_t s_pos[kLongRow];
    __shared__ long long s_part[kCtaThreads / 32];
    for (long long row = blockIdx.x; row < A.N; row += gridDim.x) {
        const long long s = __ldg(A.indptr + row), n = __ldg(A.indptr + row + 1) - s;
        if (n <= kShortRow || n > kLongRow) continue;
        int m = 1;
        while (m < n) m <<= 1;
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
            unsigned long long k = ~0ull;
            if (i < n) {
                const uint32_t f = __ldg(A.indices + s + i);
                if (f < A.dim) k = ap_key(A, f);
            }
            s_key[i] = k;
            s_pos[i] = (uint16_t)i;
        }
        __syncthreads();
        for (int size = 2; size <= m; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = threadIdx.x; i < m; i += blockDim.x) {
                    const int p = i ^ stride;
                    if (p > i) {
                        const bool up = (i & size) == 0;
                        const unsigned long long a = s_key[i], b = s_key[p];
                        if ((a > b) == up) {
                            s_key[i] = b;
                            s_key[p] = a;
                            const uint16_t t = s_pos[i];
                            s_pos[i] = s_pos[p];
                            s_pos[p] = t;
                        }
                    }
                }
                __syncthreads();
            }
        // inclusive scan of the weights in sorted order, kCtaThreads at a time
        const long long thr = ap_threshold(A, n);
        long long carry = 0;
        for (int c0 = 0; c0 < n; c0 += blockDim.x) {
            const int i = c0 + threadIdx.x;
            long long w = 0;
            int pos = 0;
            if (i < n) {
                pos = s_pos[i];
                const uint32_t f = __ldg(A.indices + s + pos);
                w = f < A.dim ? ap_weight(A, s + pos, f) : 0;
            }
            long long x = w;
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_part[wid] = x;
            __syncthreads();
            long long before = carry;
            for (int q = 0; q < wid; ++q) before += s_part[q];
            long long total = carry;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) total += s_part[q];
            if (i < n) A.indexed[s + pos] = before + x >= thr;
            __syncthreads();
            carry = total;
        }
    }
}

// Index keys: (feature << xbits) | row for indexed nonzeros, the padding key
// (all ones) for the others; per-feature counts of indexed nonzeros.
__global__ void __launch_bounds__(256) ap_index_keys_kernel(ApArgs A, int xbits, unsigned long long *keys,
                                                            unsigned long long *fcnt) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < A.N; row += nw) {
        const long long s = __ldg(A.indptr + row), e = __ldg(A.indptr + row + 1);
        for (long long i = s + lane; i < e; i += 32) {
            const uint32_t f = __ldg(A.indices + i);
            unsigned long long k = ~0ull;
            if (f < A.dim && A.indexed[i]) {
                k = ((unsigned long long)f << xbits) | (unsigned long long)row;
                atomicAdd(fcnt + f, 1ull);
            }
            keys[i] = k;
        }
    }
}

// First position in the sorted list L[0..n) (row ids in the low xbits of the
// keys) whose row is >= y.
__device__ __forceinline__ long long ap_lower(const unsigned long long *L, long long n, uint32_t y,
                                              unsigned long long xmask) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((uint32_t)(__ldg(L + mid) & xmask) < y) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Count pass (WRITE = false): ycnt[y] = sum over the features f of row y of
// the number of rows x < y in f's list.  Write pass: the keys (x << 32) | y at
// offsets ycnt[y] (after the scan), at most cap of them.
template <bool WRITE>
__global__ void __launch_bounds__(256) ap_emit_kernel(ApArgs A, const unsigned long long *ikeys,
                                                      const unsigned long long *fstart, unsigned long long xmask,
                                                      unsigned long long *ycnt, unsigned long long *out,
                                                      long long cap) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long y = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; y < A.N; y += nw) {
        const long long s = __ldg(A.indptr + y), e = __ldg(A.indptr + y + 1);
        unsigned long long base = WRITE ? ycnt[y] : 0ull;
        unsigned long long total = 0;
        for (long long c0 = s; c0 < e; c0 += 32) {
            long long lo = 0, cnt = 0;
            if (c0 + lane < e) {
                const uint32_t f = __ldg(A.indices + c0 + lane);
                if (f < A.dim) {
                    lo = (long long)fstart[f];
                    cnt = ap_lower(ikeys + lo, (long long)(fstart[f + 1] - fstart[f]), (uint32_t)y, xmask);
                }
            }
            if (!WRITE) {
                total += (unsigned long long)cnt;
                continue;
            }
            // offsets of this chunk's prefixes, then each written by the whole warp
            long long incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            const long long excl = incl - cnt;
            for (int l = 0; l < 32; ++l) {
                const long long n_l = __shfl_sync(kFull, cnt, l);
                if (n_l == 0) continue;
                const long long lo_l = __shfl_sync(kFull, lo, l);
                const unsigned long long o_l = base + (unsigned long long)__shfl_sync(kFull, excl, l);
                for (long long i = lane; i < n_l; i += 32) {
                    const unsigned long long x = __ldg(ikeys + lo_l + i) & xmask;
                    if (o_l + (unsigned long long)i < (unsigned long long)cap)
                        out[o_l + i] = (x << 32) | (unsigned long long)y;
                }
            }
            base += (unsigned long long)__shfl_sync(kFull, incl, 31);
        }
        if (!WRITE) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(kFull, total, o);
            if (lane == 0) ycnt[y] = total;
        }
    }
}

// Keys from the total (device) up to cap get the padding key (sorted last).
__global__ void __launch_bounds__(256) ap_pad_kernel(unsigned long long *keys, const unsigned long long *total,
                                                     long long cap) {
    const long long n = (long long)*total;
    for (long long i = (n < 0 ? 0 : n) + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cap;
         i += (long long)gridDim.x * blockDim.x)
        keys[i] = ~0ull;
}

// Distinct-key marks: mark[i] = 1 where key i is not padding and differs
// from key i-1.
__global__ void __launch_bounds__(256) ap_mark_kernel(const unsigned long long *keys, long long n, uint32_t *mark) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        mark[i] = k != ~0ull && (i == 0 || keys[i - 1] != k);
    }
}

// The distinct keys as pairs, at their scanned positions (at most cap).
__global__ void __launch_bounds__(256) ap_write_kernel(const unsigned long long *keys, const uint32_t *mark,
                                                       const uint32_t *pos, long long n, uint32_t *pairs, long long cap) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        const long long p = pos[i];
        if (p < cap) {
            pairs[2 * p] = (uint32_t)(keys[i] >> 32);
            pairs[2 * p + 1] = (uint32_t)keys[i];
        }
    }
}

// n_pairs = the number of distinct keys; truncation and an undersized key
// buffer are reported on the device.
__global__ void ap_finish_kernel(const uint32_t *mark_total, const unsigned long long *dup_total, long long dup_cap,
                                 long long cap, int64_t *n_pairs, int64_t *n_dups, blsh_dev_scratch *scratch) {
    const long long dups = (long long)*dup_total;
    if (n_dups) *n_dups = dups;
    if (dups > dup_cap) {   // the key buffer was too small: no pairs
        *n_pairs = 0;
        blsh_dev_error(scratch, BLSH_ETRUNC, 1, (unsigned long long)(dups - dup_cap));
        return;
    }
    const long long n = (long long)*mark_total;
    *n_pairs = n;
    if (n > cap) blsh_dev_error(scratch, BLSH_ETRUNC, 1, (unsigned long long)(n - cap));
}

// Count-only calls: n_dups and n_pairs = 0 (the pairs are not formed).
__global__ void ap_count_only_kernel(const unsigned long long *dup_total, int64_t *n_pairs, int64_t *n_dups) {
    if (n_dups) *n_dups = (long long)*dup_total;
    *n_pairs = 0;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct ApLayout {
    size_t df, maxabs, indexed, ik0, ik1, iv0, iv1, fcnt, ycnt, k0, k1, v0, v1, mark, pos, hist, partial, grand,
        total;
};

ApLayout ap_layout(long long N, long long nnz, long long dim, long long max_dups) {
    const long long big = nnz > max_dups ? nnz : max_dups;
    const long long scan_n = (N + 1 > dim + 1 ? N + 1 : dim + 1) > big ? (N + 1 > dim + 1 ? N + 1 : dim + 1) : big;
    ApLayout L;
    size_t o = 0;
    L.df = o; o = up256(o + dim * 4);
    L.maxabs = o; o = up256(o + dim * 4);
    L.indexed = o; o = up256(o + nnz);
    L.ik0 = o; o = up256(o + nnz * 8);
    L.ik1 = o; o = up256(o + nnz * 8);
    L.iv0 = o; o = up256(o + nnz * 4);
    L.iv1 = o; o = up256(o + nnz * 4);
    L.fcnt = o; o = up256(o + (dim + 1) * 8);
    L.ycnt = o; o = up256(o + (N + 1) * 8);
    L.k0 = o; o = up256(o + max_dups * 8);
    L.k1 = o; o = up256(o + max_dups * 8);
    L.v0 = o; o = up256(o + max_dups * 4);
    L.v1 = o; o = up256(o + max_dups * 4);
    L.mark = o; o = up256(o + max_dups * 4);
    L.pos = o; o = up256(o + max_dups * 4);
    L.hist = o; o = up256(o + blsh_radix::hist_entries(big) * 4);
    const long long part = blsh_radix::partial_entries(big) + blsh_scan::tiles_for(scan_n) + 2;
    L.partial = o; o = up256(o + part * 8);
    L.grand = o; o = up256(o + 64);
    L.total = o;
    return L;
}

int bits_for(long long v) {
    int b = 1;
    while (b < 63 && (1ll << b) <= v) ++b;
    return b;
}

}  // namespace

extern "C" int blsh_allpairs_workspace(int64_t N, int64_t nnz, int64_t dim, int64_t max_dups, size_t *bytes) {
    if (!bytes || N < 0 || nnz < 0 || dim <= 0 || max_dups < 0) return BLSH_EINVAL;
    *bytes = ap_layout(N, nnz, dim, max_dups).total;
    return BLSH_OK;
}

extern "C" int blsh_allpairs_candidates(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                        const float *values, int64_t N, int64_t nnz, int64_t dim, double t,
                                        int32_t kind,
                                        int64_t max_dups, uint32_t *pairs, int64_t cap, int64_t *n_pairs,
                                        int64_t *n_dups, void *workspace, size_t workspace_bytes, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !n_pairs || (N > 0 && !indices) || (cap > 0 && !pairs))
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices and n_pairs are required");
    if (kind != BLSH_JACCARD && kind != BLSH_COSINE) return blsh_fail(ctx, BLSH_EINVAL, "bad kind");
    if ((kind == BLSH_COSINE) != (values != nullptr))
        return blsh_fail(ctx, BLSH_EINVAL, "values must be given for cosine rows and only for them");
    if (!(t > 0 && t < 1)) return blsh_fail(ctx, BLSH_EINVAL, "t must lie in (0, 1)");
    if (N < 0 || N >= (1ll << 32) || dim <= 0 || dim > (1ll << 32) || cap < 0 || max_dups < 0 || max_dups >= (1ll << 32))
        return blsh_fail(ctx, BLSH_EINVAL, "bad N, dim, cap or max_dups");
    if (!blsh_aligned(indptr, 8) || !blsh_aligned(n_pairs, 8) || !blsh_aligned(n_dups, 8) ||
        !blsh_aligned(workspace, 256) || !blsh_aligned(pairs, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    if (N < 2) {
        BLSH_CUDA(ctx, cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s));
        if (n_dups) BLSH_CUDA(ctx, cudaMemsetAsync(n_dups, 0, sizeof(int64_t), s));
        return BLSH_OK;
    }
    if (nnz < 0 || nnz >= (1ll << 32)) return blsh_fail(ctx, BLSH_EINVAL, "nnz must lie in [0, 2^32)");
    const long long dcap = cap > 0 ? max_dups : 0;   // a count-only call needs no key buffers
    const ApLayout L = ap_layout(N, nnz, dim, dcap);
    if (!workspace || workspace_bytes < L.total) return blsh_fail(ctx, BLSH_ETRUNC, "workspace needs %zu bytes", L.total);
    char *ws = (char *)workspace;
    ApArgs A;
    A.indptr = indptr;
    A.indices = indices;
    A.values = values;
    A.N = N;
    A.dim = dim;
    A.cosine = kind == BLSH_COSINE;
    A.t = t;
    A.thr = (long long)ceil((t - 1e-9) * kTwo48);
    A.df = (uint32_t *)(ws + L.df);
    A.maxabs = (uint32_t *)(ws + L.maxabs);
    A.indexed = (uint8_t *)(ws + L.indexed);
    A.scratch = ctx->scratch;
    unsigned long long *fcnt = (unsigned long long *)(ws + L.fcnt);
    unsigned long long *ycnt = (unsigned long long *)(ws + L.ycnt);
    uint32_t *hist = (uint32_t *)(ws + L.hist);
    unsigned long long *partial64 = (unsigned long long *)(ws + L.partial);
    unsigned long long *grand64 = (unsigned long long *)(ws + L.grand);
    uint32_t *grand32 = (uint32_t *)(ws + L.grand + 16);
    unsigned long long *dup_total = (unsigned long long *)(ws + L.grand + 32);
    const int sms = ctx->sm_count;
    auto grid_for = [&](long long items, long long per_block) {
        const long long b = (items + per_block - 1) / per_block, cap_b = (long long)sms * 16;
        return (unsigned)(b < 1 ? 1 : (b < cap_b ? b : cap_b));
    };

    // 1. statistics
    BLSH_CUDA(ctx, cudaMemsetAsync(A.df, 0, L.indexed - L.df, s));   // df and maxabs
    blsh_time_start(ctx, s);
    ap_stats_kernel<<<grid_for(nnz, 256), 256, 0, s>>>(A, nnz);
    BLSH_LAUNCHED(ctx, "ap_stats_kernel");
    // 2. indexed features
    blsh_time_start(ctx, s);
    ap_prefix_warp_kernel<<<grid_for(N, 8), 256, 0, s>>>(A);
    BLSH_LAUNCHED(ctx, "ap_prefix_warp_kernel");
    blsh_time_start(ctx, s);
    ap_prefix_cta_kernel<<<(unsigned)sms * 4, kCtaThreads, 0, s>>>(A);
    BLSH_LAUNCHED(ctx, "ap_prefix_cta_kernel");
    // 3. the inverted index
    const int xbits = bits_for(N);
    const int key_bits = xbits + bits_for(dim);
    unsigned long long *ik[2] = {(unsigned long long *)(ws + L.ik0), (unsigned long long *)(ws + L.ik1)};
    uint32_t *iv[2] = {(uint32_t *)(ws + L.iv0), (uint32_t *)(ws + L.iv1)};
    BLSH_CUDA(ctx, cudaMemsetAsync(fcnt, 0, (dim + 1) * 8, s));
    blsh_time_start(ctx, s);
    ap_index_keys_kernel<<<grid_for(N, 8), 256, 0, s>>>(A, xbits, ik[0], fcnt);
    BLSH_LAUNCHED(ctx, "ap_index_keys_kernel");
    int cur = 0;
    {
        // the padding key (all ones) sorts after every real key in key_bits bits
        const int rc = blsh_radix::sort(ctx, ik, iv, nnz, 64 > key_bits ? key_bits + 1 : 64, hist,
                                        (uint32_t *)partial64, grand32, s, &cur);
        if (rc) return rc;
    }
    // feature list starts: exclusive scan of the per-feature counts (dim + 1 entries)
    blsh_time_start(ctx, s);
    BLSH_CUDA(ctx, blsh_scan::exclusive_scan<unsigned long long>(fcnt, fcnt, dim + 1, partial64, grand64, s));
    ctx->launches.fetch_add(3, std::memory_order_relaxed);
    blsh_time_stop(ctx, "exclusive scan (3 launches)");
    const unsigned long long xmask = (1ull << xbits) - 1ull;
    // 4. candidate keys: count, scan, write
    blsh_time_start(ctx, s);
    ap_emit_kernel<false><<<grid_for(N, 8), 256, 0, s>>>(A, ik[cur], fcnt, xmask, ycnt, nullptr, 0);
    BLSH_LAUNCHED(ctx, "ap_emit_kernel (count pass)");
    BLSH_CUDA(ctx, cudaMemsetAsync(ycnt + N, 0, 8, s));
    blsh_time_start(ctx, s);
    BLSH_CUDA(ctx, blsh_scan::exclusive_scan<unsigned long long>(ycnt, ycnt, N + 1, partial64, dup_total, s));
    ctx->launches.fetch_add(3, std::memory_order_relaxed);
    blsh_time_stop(ctx, "exclusive scan (3 launches)");
    if (cap == 0 || max_dups == 0) {
        ap_count_only_kernel<<<1, 1, 0, s>>>(dup_total, n_pairs, n_dups);
        BLSH_LAUNCHED(ctx, "ap_count_only_kernel");
        return BLSH_OK;
    }
    unsigned long long *ck[2] = {(unsigned long long *)(ws + L.k0), (unsigned long long *)(ws + L.k1)};
    uint32_t *cv[2] = {(uint32_t *)(ws + L.v0), (uint32_t *)(ws + L.v1)};
    blsh_time_start(ctx, s);
    ap_emit_kernel<true><<<grid_for(N, 8), 256, 0, s>>>(A, ik[cur], fcnt, xmask, ycnt, ck[0], max_dups);
    BLSH_LAUNCHED(ctx, "ap_emit_kernel (write pass)");
    blsh_time_start(ctx, s);
    ap_pad_kernel<<<grid_for(max_dups, 256), 256, 0, s>>>(ck[0], dup_total, max_dups);
    BLSH_LAUNCHED(ctx, "ap_pad_kernel");
    // 5. sort, keep the distinct keys
    int kc = 0;
    {
        // keys (x << 32) | y: the write pass leaves them grouped by y in
        // increasing order, so a stable sort by x alone (bits 32 .. 32 + xbits,
        // one more bit for the padding key) orders them by (x, y)
        const int kbits = xbits + 1 < 32 ? xbits + 1 : 32;
        const int rc = blsh_radix::sort(ctx, ck, cv, max_dups, kbits, hist, (uint32_t *)partial64, grand32, s, &kc,
                                        32);
        if (rc) return rc;
    }
    uint32_t *mark = (uint32_t *)(ws + L.mark), *pos = (uint32_t *)(ws + L.pos);
    blsh_time_start(ctx, s);
    ap_mark_kernel<<<grid_for(max_dups, 256), 256, 0, s>>>(ck[kc], max_dups, mark);
    BLSH_LAUNCHED(ctx, "ap_mark_kernel");
    blsh_time_start(ctx, s);
    BLSH_CUDA(ctx, blsh_scan::exclusive_scan<uint32_t>(mark, pos, max_dups, (uint32_t *)partial64, grand32, s));
    ctx->launches.fetch_add(3, std::memory_order_relaxed);
    blsh_time_stop(ctx, "exclusive scan (3 launches)");
    blsh_time_start(ctx, s);
    ap_write_kernel<<<grid_for(max_dups, 256), 256, 0, s>>>(ck[kc], mark, pos, max_dups, pairs, cap);
    BLSH_LAUNCHED(ctx, "ap_write_kernel");
    ap_finish_kernel<<<1, 1, 0, s>>>(grand32, dup_total, max_dups, cap, n_pairs, n_dups, ctx->scratch);
    BLSH_LAUNCHED(ctx, "ap_finish_kernel");
    return BLSH_OK;
}
