// hashing.cu -- the signature producers: minhash (Section 4.1, "LSH family")
// and sign random projections of sparse rows (Section 4.2, "LSH family").
#include <type_traits>

#include "common.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kP31 = 0x7fffffffu;   // 2^31 - 1

// (a x + b) mod (2^31 - 1) for a, b < 2^31 - 1 and any 32-bit x, exactly:
// v < 2^63, and 2^31 = 1 (mod p) lets a fold of the high bits onto the low
// 31 bits bring v below 2^32 + 2^31, a second fold (in 32 bits) below
// 2^31 + 2, then one conditional subtraction.
__device__ __forceinline__ uint32_t mod_mersenne31(uint32_t a, uint32_t b, uint32_t x) {
    const unsigned long long v = (unsigned long long)a * x + b;
    const unsigned long long r = (v & kP31) + (v >> 31);
    const uint32_t h = ((uint32_t)r & kP31) + (uint32_t)(r >> 31);
    return h >= kP31 ? h - kP31 : h;
}

// One warp per set; lane l owns hashes l, l+32, ..., l+32(HPL-1) of the
// current tile of 32*HPL hashes and keeps their running minima in
// registers.  The set's elements are read 32 at a time (coalesced) and
// broadcast with shuffles.  Sets longer than kBigSet are left to
// minhash_big_kernel.
constexpr long long kBigSet = 2048;

constexpr long long kBigChunk = 4096;   // elements of a long set per CTA task

template <int HPL>
__global__ void __launch_bounds__(256) minhash_kernel(const int64_t *__restrict__ indptr,
                                                      const uint32_t *__restrict__ indices, long long N,
                                                      int n_hashes, const uint32_t *__restrict__ A,
                                                      const uint32_t *__restrict__ B, uint32_t *__restrict__ sig,
                                                      blsh_dev_scratch *scratch, uint2 *__restrict__ big) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < N; i += warps) {
        const long long s = __ldg(indptr + i), e = __ldg(indptr + i + 1);
        if (e - s > kBigSet) {
            // a long set: its row starts at the identity of min, the chunks of
            // minhash_big_kernel lower it; queued unless the queue is full
            for (int k = lane; k < n_hashes; k += 32) sig[(size_t)i * n_hashes + k] = 0xffffffffu;
            unsigned long long slot = 0;
            if (lane == 0) slot = atomicAdd(&scratch->work3, 1ull);
            slot = __shfl_sync(kFull, slot, 0);
            if (slot < BLSH_RECHECK_CAP) {
                if (lane == 0) big[slot] = make_uint2((uint32_t)i, (uint32_t)((e - s + kBigChunk - 1) / kBigChunk));
                continue;
            }
        }
        for (int t0 = 0; t0 < n_hashes; t0 += 32 * HPL) {
            uint32_t a[HPL], b[HPL], mn[HPL];
#pragma unroll
            for (int u = 0; u < HPL; ++u) {
                a[u] = __ldg(A + t0 + 32 * u + lane);
                b[u] = __ldg(B + t0 + 32 * u + lane);
                mn[u] = 0xffffffffu;
            }
            for (long long e0 = s; e0 < e; e0 += 32) {
                const uint32_t mine = e0 + lane < e ? __ldg(indices + e0 + lane) : 0u;
                const int cnt = (int)min(32ll, e - e0);
                for (int l = 0; l < cnt; ++l) {
                    const uint32_t x = __shfl_sync(kFull, mine, l);
#pragma unroll
                    for (int u = 0; u < HPL; ++u) mn[u] = min(mn[u], mod_mersenne31(a[u], b[u], x));
                }
            }
#pragma unroll
            for (int u = 0; u < HPL; ++u) sig[(size_t)i * n_hashes + t0 + 32 * u + lane] = mn[u];
        }
    }
}

// Sets longer than kBigSet, queued by minhash_kernel as (set, chunks of
// kBigChunk elements).  Every CTA walks the queue and takes the chunks of
// each set that fall to it (chunk c of queue entry q goes to CTA
// (c + 7919 q) mod gridDim), so one set with thousands of elements is
// hashed by many SMs.  In a chunk, warp w takes every 32nd block of 32
// elements; the warps' minima meet in shared memory, and the chunk's minima
// in the set's row in global memory (atomicMin: the minimum does not depend
// on the order).
template <int HPL>
__global__ void __launch_bounds__(1024) minhash_big_kernel(const int64_t *__restrict__ indptr,
                                                           const uint32_t *__restrict__ indices, int n_hashes,
                                                           const uint32_t *__restrict__ A,
                                                           const uint32_t *__restrict__ B,
                                                           uint32_t *__restrict__ sig, const blsh_dev_scratch *scratch,
                                                           const uint2 *__restrict__ big) {
    __shared__ uint32_t smin[32 * HPL];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const unsigned long long total = scratch->work3;
    const unsigned long long nq = total < BLSH_RECHECK_CAP ? total : BLSH_RECHECK_CAP;
    const unsigned G = gridDim.x;
    for (unsigned long long qi = 0; qi < nq; ++qi) {
        const uint2 ent = big[qi];
        const long long i = ent.x;
        const unsigned chunks = ent.y;
        const unsigned first = (unsigned)((blockIdx.x + (unsigned long long)G * chunks - (qi * 7919ull) % G) % G);
        for (unsigned c = first; c < chunks; c += G) {
            const long long s0 = __ldg(indptr + i) + (long long)c * kBigChunk;
            const long long e1 = __ldg(indptr + i + 1);
            const long long e = e1 < s0 + kBigChunk ? e1 : s0 + kBigChunk;
            for (int t0 = 0; t0 < n_hashes; t0 += 32 * HPL) {
                __syncthreads();
                for (int k = threadIdx.x; k < 32 * HPL; k += blockDim.x) smin[k] = 0xffffffffu;
                __syncthreads();
                uint32_t a[HPL], b[HPL], mn[HPL];
#pragma unroll
                for (int u = 0; u < HPL; ++u) {
                    a[u] = __ldg(A + t0 + 32 * u + lane);
                    b[u] = __ldg(B + t0 + 32 * u + lane);
                    mn[u] = 0xffffffffu;
                }
                for (long long e0 = s0 + 32ll * warp; e0 < e; e0 += 32ll * nwarps) {
                    const uint32_t mine = e0 + lane < e ? __ldg(indices + e0 + lane) : 0u;
                    const int cnt = (int)min(32ll, e - e0);
                    for (int l = 0; l < cnt; ++l) {
                        const uint32_t x = __shfl_sync(kFull, mine, l);
#pragma unroll
                        for (int u = 0; u < HPL; ++u) mn[u] = min(mn[u], mod_mersenne31(a[u], b[u], x));
                    }
                }
#pragma unroll
                for (int u = 0; u < HPL; ++u) atomicMin(&smin[32 * u + lane], mn[u]);
                __syncthreads();
                for (int k = threadIdx.x; k < 32 * HPL; k += blockDim.x)
                    atomicMin(&sig[(size_t)i * n_hashes + t0 + k], smin[k]);
            }
        }
    }
}

// Sign random projections of sparse rows.  One CTA per row (grid-stride);
// thread t owns bits t, t+T, ..., so that the threads of a warp read 128
// contiguous bytes of a row of R and a warp ballot of one of its bits forms
// one signature word.  Sums are FP32 with fused multiply-adds in row order;
// next to each sum the thread keeps sum |v r|.  Recursive summation of n
// exact products has error at most (n-1) u sum|v r| (u = 2^-24); a sum whose
// magnitude exceeds 1.25 n u sum|v r| + n 2^-149 has the sign of the exact
// sum (and of the FP64 row-order sum, whose error is 2^29 times smaller).
// Otherwise the thread recomputes the sum in FP64 in row order, which
// reproduces that FP64 sum bit for bit (products of floats are exact in FP64,
// so one rounding per addition with or without fusion).
// Entry (i) of R as FP64: a float, or a two-byte code q read back as
// q 2^-12 - 8 (Section 4.3), which is exact in FP64 (and in FP32).
__device__ __forceinline__ double r_fp64(const float *R, size_t i) { return (double)__ldg(R + i); }
__device__ __forceinline__ double r_fp64(const uint16_t *R, size_t i) {
    return (double)__ldg(R + i) * (1.0 / 4096.0) - 8.0;
}
__device__ __forceinline__ float r_fp32(const float *R, size_t i) { return __ldg(R + i); }
__device__ __forceinline__ float r_fp32(const uint16_t *R, size_t i) {
    return __fmaf_rn((float)__ldg(R + i), 1.0f / 4096.0f, -8.0f);
}

constexpr int kSrpMaxPerThread = 16;
constexpr int kSrpLooseRow = 256;   // rows up to this length use the 2^15 sum|v| magnitude bound (two-byte codes)
constexpr int kSrpBatch = 8;
constexpr int kSrpGrab = 8;         // (row, piece) items a CTA of srp_sparse4_kernel takes per grab
constexpr int kSrpChunk = 256;

template <typename RT>
__global__ void __launch_bounds__(256) srp_sparse_kernel(const int64_t *__restrict__ indptr,
                                                         const uint32_t *__restrict__ indices,
                                                         const float *__restrict__ values, long long N,
                                                         const RT *__restrict__ R, long long dim, int bits,
                                                         int per_thread,
                                                         uint32_t *__restrict__ sig, blsh_dev_scratch *scratch) {
    __shared__ uint32_t s_idx[kSrpChunk];
    __shared__ float s_val[kSrpChunk];
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int words = bits >> 5;
    unsigned long long rechecked = 0, zeros = 0;
    for (long long row = blockIdx.x; row < N; row += gridDim.x) {
        const long long s = __ldg(indptr + row), e = __ldg(indptr + row + 1);
        float acc[kSrpMaxPerThread], mag[kSrpMaxPerThread];
#pragma unroll
        for (int u = 0; u < kSrpMaxPerThread; ++u) acc[u] = mag[u] = 0.0f;
        for (long long c0 = s; c0 < e; c0 += kSrpChunk) {
            const int cnt = (int)min((long long)kSrpChunk, e - c0);
            __syncthreads();
            for (int i = t; i < cnt; i += T) {
                uint32_t ix = __ldg(indices + c0 + i);
                float v = __ldg(values + c0 + i);
                if (ix >= dim) {   // malformed row: record it, contribute nothing
                    blsh_dev_error(scratch, BLSH_ERANGE, 0, 1ull);
                    ix = 0;
                    v = 0.0f;
                }
                s_idx[i] = ix;
                s_val[i] = v;
            }
            __syncthreads();
            for (int i = 0; i < cnt; ++i) {
                const float v = s_val[i];
                const RT *Rrow = R + (size_t)s_idx[i] * bits + t;
#pragma unroll
                for (int u = 0; u < kSrpMaxPerThread; ++u) {
                    if (u < per_thread) {
                        const float r = r_fp32(Rrow, (size_t)u * T);
                        acc[u] = __fmaf_rn(v, r, acc[u]);
                        mag[u] = __fmaf_rn(fabsf(v), fabsf(r), mag[u]);
                    }
                }
            }
        }
        const float n = (float)(int)(e - s < (1ll << 30) ? e - s : (1ll << 30));   // 32-bit conversion
        const bool long_row = n * 5.9604644775390625e-8f > 0.05f;   // the 1.25 slack needs n u <= 0.05
        const int w = t >> 5;
#pragma unroll
        for (int u = 0; u < kSrpMaxPerThread; ++u) {
            if (u < per_thread) {
                const float bound = 1.25f * n * 5.9604644775390625e-8f * mag[u] + n * 1.4e-45f;
                bool bit;
                if (!long_row && fabsf(acc[u]) > bound) {
                    bit = acc[u] >= 0.0f;
                } else {
                    double d = 0.0;
                    for (long long k = s; k < e; ++k) {
                        const uint32_t ix = __ldg(indices + k);
                        if (ix < dim) d += (double)__ldg(values + k) * r_fp64(R, (size_t)ix * bits + t + u * T);
                    }
                    bit = d >= 0.0;
                    ++rechecked;
                    zeros += d == 0.0;
                }
                const unsigned word = __ballot_sync(kFull, bit);
                if ((t & 31) == 0) sig[(size_t)row * words + w + u * (T >> 5)] = word;
            }
        }
    }
    if (rechecked) atomicAdd(&scratch->counters[2], rechecked);
    if (zeros) atomicAdd(&scratch->counters[3], zeros);
}


// The FP64 row-order sum of row [s, e) against column j of R, as the oracle
// forms it (rare: only signs the FP32 bound cannot decide).  Kept out of line
// so the hot accumulation loop keeps its registers.
template <typename RT>
__device__ __noinline__ double srp_recheck_fp64(const uint32_t *__restrict__ indices,
                                                const float *__restrict__ values, long long s, long long e,
                                                const RT *__restrict__ R, long long dim, int bits, int j) {
    double d = 0.0;
    for (long long k = s; k < e; ++k) {
        const uint32_t ix = __ldg(indices + k);
        if (ix < dim) d += (double)__ldg(values + k) * r_fp64(R, (size_t)ix * bits + j);
    }
    return d;
}

// Paired FP32 arithmetic (two lanes of a 64-bit register per instruction,
// each an IEEE single-precision operation rounded to nearest): the two-byte
// projection's decode, sum and magnitude for two columns at a time.
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long p, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// The two codes of a 32-bit word as the pair (2^23 + low code, 2^23 + high
// code): each code's bits placed under the exponent of 2^23.
__device__ __forceinline__ unsigned long long f2_codes(uint32_t w) {
    return f2_pack(__int_as_float((int)__byte_perm(w, 0x4b00u, 0x5410)),
                   __int_as_float((int)__byte_perm(w, 0x4b00u, 0x5432)));
}

// The same computation when bits is a multiple of 128: thread t owns the
// groups of four columns t, t+T, ... of each row of R (bits 4t..4t+3,
// 4(t+T).., ...), so every load moves 16 bytes (float R) or 8 bytes (RT =
// uint16_t: the two-byte codes of Section 4.3) and a warp reads 512 or 256
// contiguous bytes.  A row's indices and values are read 32 at a time, one
// per lane (coalesced), and reach the other lanes by shuffles; the gathers
// of several nonzeros are issued together, so a long row is not a chain of
// dependent loads, and no barrier is needed.  Every column keeps its sum and
// the sum of the products' magnitudes for the error bound.  The sum is formed
// in blocks of 32 nonzeros (a block's FMA chain, then the block added to the
// total), so a column's result carries at most min(n, 32) + ceil(n / 32)
// roundings in any chain rather than n: a long row leaves far fewer signs to
// the FP64 recheck.  The four bits of
// a group form a nibble; eight lanes OR their nibbles into one signature
// word with shuffles.  CTAs take (row, piece of 4 V T columns) items from a
// counter, kSrpGrab at a time (a fixed share per CTA when there are few).
template <int V, typename RT>
__global__ void __launch_bounds__(256) srp_sparse4_kernel(const int64_t *__restrict__ indptr,
                                                          const uint32_t *__restrict__ indices,
                                                          const float *__restrict__ values, long long N,
                                                          const RT *__restrict__ R, long long dim, int bits,
                                                          int col_first, int pieces,
                                                          const uint8_t *__restrict__ row_mask,
                                                          uint32_t *__restrict__ sig, blsh_dev_scratch *scratch,
                                                          uint2 *__restrict__ queue, int grab) {
    // columns col_first .. col_first + pieces 4 V T - 1 of the signatures of
    // the rows row_mask selects (all rows when it is NULL); a CTA works on
    // one (row, piece of 4 V T columns) at a time, so that a few selected
    // rows still spread over many CTAs
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int words = bits >> 5;
    unsigned long long rechecked = 0, zeros = 0, bad = 0;
    // items are handed out `grab` at a time from a counter: row lengths
    // follow a power law (a single row can hold more work than a thousand
    // average ones), and a fixed share per CTA left most of the GPU idle
    // while the CTAs that drew the longest rows finished
    // (grab == 0: a fixed share per CTA, items blockIdx.x, blockIdx.x +
    // gridDim.x, ...: few items per CTA, where a counter would cost more
    // than it balances)
    __shared__ unsigned long long s_next;
    const long long items = N * pieces;
    long long next_static = blockIdx.x;
    for (;;) {
        long long g0, g1;
        if (grab > 0) {
            __syncthreads();                               // every thread has read the previous grab
            if (threadIdx.x == 0) s_next = atomicAdd(&scratch->hash_work, (unsigned long long)grab);
            __syncthreads();
            g0 = (long long)s_next;
            g1 = g0 + grab < items ? g0 + grab : items;
        } else {
            g0 = next_static;
            g1 = g0 + 1;
            next_static += gridDim.x;
        }
        if (g0 >= items) break;
        for (long long item = g0; item < g1; ++item) {
            const long long row = pieces == 1 ? item : item / pieces;   // (a 64-bit division is a long call)
            const int col0 = col_first + (int)(item - row * pieces) * 4 * V * T;
            if (row_mask && !row_mask[row]) continue;
            const long long s = __ldg(indptr + row), e = __ldg(indptr + row + 1);
            constexpr bool Q16 = sizeof(RT) == 2;
            float acc[4 * V], mag[4 * V], tot[4 * V];
#pragma unroll
            for (int u = 0; u < 4 * V; ++u) acc[u] = mag[u] = tot[u] = 0.0f;
            // two-byte codes: the same sums kept as pairs of columns (one 64-bit
            // register each) for the paired instructions, unpacked once per row
            unsigned long long acc2[2 * V], mag2[2 * V], tot2[2 * V];
#pragma unroll
            for (int u = 0; u < 2 * V; ++u) acc2[u] = mag2[u] = tot2[u] = 0ull;
            // Rows of at most kSrpLooseRow nonzeros (two-byte codes): the
            // magnitude bound 2^15 sum|v_i| (every decoded code has |q - 2^15| <=
            // 2^15) instead of each column's sum|v_i| |q_ij - 2^15|; about ten
            // times looser, but the blocked sums keep short rows' bounds small,
            // and it saves two paired FMAs and four masks per nonzero
            const bool loose = Q16 && e - s <= kSrpLooseRow;
            float sav = 0.0f;
            // the row's nonzeros 32 at a time: lane l of every warp loads entry
            // l (coalesced), then the gathers of kSrpBatch / V entries are issued
            // together (their indices come by shuffle), so that a long row is not
            // a chain of dependent loads
            constexpr int NB = kSrpBatch / V > 0 ? kSrpBatch / V : 1;
            for (long long k0 = s; k0 < e; k0 += 32) {
                const int cnt = e - k0 < 32 ? (int)(e - k0) : 32;
                uint32_t my_ix = 0;
                float my_v = 0.0f;
                if (lane < cnt) {
                    my_ix = __ldg(indices + k0 + lane);
                    my_v = __ldg(values + k0 + lane);
                    if (my_ix >= dim) {   // malformed entry: counted once, contributes nothing
                        bad += t < 32;
                        my_ix = 0;
                        my_v = 0.0f;
                    }
                }
                if constexpr (Q16) {
                    // the decoded value of code q is (q - 2^15) 2^-12: (2^23 + q) - (2^23 + 2^15),
                    // exact, with the sums kept in units of 2^-12
                    const unsigned long long off2 = f2_pack(-8421376.0f, -8421376.0f);
                    auto chunk = [&](auto with_mag) {
                        constexpr bool kMag = decltype(with_mag)::value;
                        for (int u0 = 0; u0 < cnt; u0 += NB) {
                            uint2 qb[NB][V];
                            float vb[NB];
#pragma unroll
                            for (int b = 0; b < NB; ++b) {
                                const uint32_t ix = __shfl_sync(kFull, my_ix, (u0 + b) & 31);
                                vb[b] = __shfl_sync(kFull, my_v, (u0 + b) & 31);   // 0 past the row's end
                                const uint2 *Rrow = reinterpret_cast<const uint2 *>(R + (size_t)ix * bits + col0) + t;
#pragma unroll
                                for (int g = 0; g < V; ++g) qb[b][g] = __ldg(Rrow + g * T);
                            }
#pragma unroll
                            for (int b = 0; b < NB; ++b) {
                                const unsigned long long v2 = f2_pack(vb[b], vb[b]);
                                const unsigned long long av2 = f2_pack(fabsf(vb[b]), fabsf(vb[b]));
                                if (!kMag) sav += fabsf(vb[b]);
#pragma unroll
                                for (int g = 0; g < V; ++g) {
                                    const unsigned long long d01 = f2_add(f2_codes(qb[b][g].x), off2);
                                    const unsigned long long d23 = f2_add(f2_codes(qb[b][g].y), off2);
                                    acc2[2 * g] = f2_fma(v2, d01, acc2[2 * g]);
                                    acc2[2 * g + 1] = f2_fma(v2, d23, acc2[2 * g + 1]);
                                    if (kMag) {
                                        mag2[2 * g] = f2_fma(av2, d01 & 0x7fffffff7fffffffull, mag2[2 * g]);
                                        mag2[2 * g + 1] = f2_fma(av2, d23 & 0x7fffffff7fffffffull, mag2[2 * g + 1]);
                                    }
                                }
                            }
                        }
                    };
                    if (loose) chunk(std::false_type{});
                    else chunk(std::true_type{});
                    // the block of (at most) 32 nonzeros into the total
#pragma unroll
                    for (int u = 0; u < 2 * V; ++u) {
                        tot2[u] = f2_add(tot2[u], acc2[u]);
                        acc2[u] = 0ull;
                    }
                } else {   // float R: 16-byte loads of four columns
                    for (int u0 = 0; u0 < cnt; u0 += NB) {
                        float4 r[NB][V];
                        float vb[NB];
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            const uint32_t ix = __shfl_sync(kFull, my_ix, (u0 + b) & 31);
                            vb[b] = __shfl_sync(kFull, my_v, (u0 + b) & 31);   // 0 past the row's end
                            const float4 *Rrow = reinterpret_cast<const float4 *>(R + (size_t)ix * bits + col0) + t;
#pragma unroll
                            for (int g = 0; g < V; ++g) r[b][g] = __ldg(Rrow + g * T);
                        }
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            const float v = vb[b], av = fabsf(v);
#pragma unroll
                            for (int g = 0; g < V; ++g) {
                                acc[4 * g + 0] = __fmaf_rn(v, r[b][g].x, acc[4 * g + 0]);
                                acc[4 * g + 1] = __fmaf_rn(v, r[b][g].y, acc[4 * g + 1]);
                                acc[4 * g + 2] = __fmaf_rn(v, r[b][g].z, acc[4 * g + 2]);
                                acc[4 * g + 3] = __fmaf_rn(v, r[b][g].w, acc[4 * g + 3]);
                                mag[4 * g + 0] = __fmaf_rn(av, fabsf(r[b][g].x), mag[4 * g + 0]);
                                mag[4 * g + 1] = __fmaf_rn(av, fabsf(r[b][g].y), mag[4 * g + 1]);
                                mag[4 * g + 2] = __fmaf_rn(av, fabsf(r[b][g].z), mag[4 * g + 2]);
                                mag[4 * g + 3] = __fmaf_rn(av, fabsf(r[b][g].w), mag[4 * g + 3]);
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4 * V; ++u) {
                        tot[u] = __fadd_rn(tot[u], acc[u]);
                        acc[u] = 0.0f;
                    }
                }
            }
            if constexpr (sizeof(RT) == 2) {
#pragma unroll
                for (int u = 0; u < 2 * V; ++u) {
                    f2_unpack(tot2[u], tot[2 * u], tot[2 * u + 1]);
                    f2_unpack(mag2[u], mag[2 * u], mag[2 * u + 1]);
                }
                if (loose) {
#pragma unroll
                    for (int u = 0; u < 4 * V; ++u) mag[u] = 32768.0f * sav;
                }
            }
            // the row length through a 32-bit integer (a 64-bit conversion would run
            // on the narrow FP64 pipe); rows past 2^30 count as 2^30, which is long
            const int len = (int)(e - s < (1ll << 30) ? e - s : (1ll << 30));
            const float n = (float)len;
            const bool long_row = n * 5.9604644775390625e-8f > 0.05f;   // the 1.25 slack needs n u <= 0.05
            // Roundings in a column's sum: a block's chain (at most 32 FMAs, error
            // <= gamma_32 of its magnitudes) and the chain of block totals (at
            // most ceil(n / 32) - 1 adds), so |sum - exact| <= (gamma_32 +
            // gamma_nb + gamma_32 gamma_nb) sum|p|, below 1.12 (min(n, 32) + nb) u
            // mag when n u <= 0.05 (mag, the computed sum of magnitudes, is within
            // gamma_n of sum|p|); each rounding near underflow adds at most 2^-150,
            // and there are at most 2n of them.
            const float kround = fminf(n, 32.0f) + (float)((len + 31) >> 5);
#pragma unroll
            for (int g = 0; g < V; ++g) {
                uint32_t nib = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int u = 4 * g + c;
                    const float bound = 1.25f * kround * 5.9604644775390625e-8f * mag[u] + n * 1.4e-45f;
                    bool bit;
                    if (!long_row && fabsf(tot[u]) > bound) {
                        bit = tot[u] >= 0.0f;
                    } else {
                        // undecided: queue it for srp_recheck_kernel (bit left 0 here),
                        // or recompute in line if the queue is full
                        const uint32_t j = col0 + 4 * (t + g * T) + c;
                        const unsigned long long slot = atomicAdd(&scratch->recheck_count, 1ull);
                        if (slot < BLSH_RECHECK_CAP) {
                            queue[slot] = make_uint2((uint32_t)row, j);
                            bit = false;
                        } else {
                            const double d = srp_recheck_fp64<RT>(indices, values, s, e, R, dim, bits, j);
                            bit = d >= 0.0;
                            ++rechecked;
                            zeros += d == 0.0;
                        }
                    }
                    nib |= (uint32_t)bit << c;
                }
                uint32_t word = nib << (4 * (lane & 7));
                word |= __shfl_xor_sync(kFull, word, 1);
                word |= __shfl_xor_sync(kFull, word, 2);
                word |= __shfl_xor_sync(kFull, word, 4);
                if ((lane & 7) == 0) sig[(size_t)row * words + (col0 >> 5) + ((t + g * T) >> 3)] = word;
            }
        }
    }
    if (bad) blsh_dev_error(scratch, BLSH_ERANGE, 0, bad);
    if (rechecked) atomicAdd(&scratch->counters[2], rechecked);
    if (zeros) atomicAdd(&scratch->counters[3], zeros);
}

// The queued signs: one warp per (row, bit).  The lanes form the row's exact
// FP64 products (coalesced reads of the row, gathers of R) and sum them in
// parallel, together with their magnitudes: that sum errs by at most
// (n/32 + 5) u sum|p| (u = 2^-53), the oracle's row-order sum by at most
// (n - 1) u sum|p|, so a parallel sum larger than 1.25 (2n + 8) u sum|p| has
// the sign of the exact sum and of the oracle's.  Only the rest (exact zeros
// and ties within that bound) are summed in row order, one product at a
// time, which is the oracle's sum bit for bit.  A nonnegative sum sets the
// bit (the word was written with it clear).
template <typename RT>
__global__ void __launch_bounds__(256) srp_recheck_kernel(const uint2 *__restrict__ queue,
                                                          const int64_t *__restrict__ indptr,
                                                          const uint32_t *__restrict__ indices,
                                                          const float *__restrict__ values,
                                                          const RT *__restrict__ R, long long dim, int bits,
                                                          uint32_t *__restrict__ sig, blsh_dev_scratch *scratch) {
    const unsigned long long total = scratch->recheck_count;
    const unsigned long long n = total < BLSH_RECHECK_CAP ? total : BLSH_RECHECK_CAP;
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    unsigned long long done = 0, zeros = 0;
    for (unsigned long long it = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n;
         it += warps) {
        const uint2 rj = queue[it];
        const long long s = __ldg(indptr + rj.x), e = __ldg(indptr + rj.x + 1);
        // lane l sums entries l, l + 32, ... in that order; four of its
        // gathers are in flight at a time (a product of 0 for entries past
        // the row leaves the sums unchanged)
        double ps = 0.0, qs = 0.0;
        for (long long k0 = s + lane; k0 < e; k0 += 128) {
            double p[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long k = k0 + 32 * u;
                p[u] = 0.0;
                if (k < e) {
                    const uint32_t ix = __ldg(indices + k);
                    if (ix < dim) p[u] = (double)__ldg(values + k) * r_fp64(R, (size_t)ix * bits + rj.y);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ps += p[u];
                qs += fabs(p[u]);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ps += __shfl_xor_sync(kFull, ps, o);
            qs += __shfl_xor_sync(kFull, qs, o);
        }
        const double len = (double)(e - s);
        bool bit = ps >= 0.0;
        if (!(fabs(ps) > 1.25 * (2.0 * len + 8.0) * 1.1102230246251565e-16 * qs + (2.0 * len + 8.0) * 5e-324)) {
            // row order: lanes load 32 products at a time, every lane adds them in order
            double d = 0.0;
            for (long long c0 = s; c0 < e; c0 += 32) {
                double p = 0.0;
                if (c0 + lane < e) {
                    const uint32_t ix = __ldg(indices + c0 + lane);
                    if (ix < dim) p = (double)__ldg(values + c0 + lane) * r_fp64(R, (size_t)ix * bits + rj.y);
                }
                const int cnt = (int)min(32ll, e - c0);
                for (int l = 0; l < cnt; ++l) d += __shfl_sync(kFull, p, l);
            }
            bit = d >= 0.0;
            zeros += lane == 0 && d == 0.0;
        }
        if (lane == 0) {
            if (bit) atomicOr(sig + (size_t)rj.x * (bits >> 5) + (rj.y >> 5), 1u << (rj.y & 31));
            ++done;
        }
    }
    if (lane == 0 && done) atomicAdd(&scratch->counters[2], done);
    if (lane == 0 && zeros) atomicAdd(&scratch->counters[3], zeros);
}

// Sign random projections with R stored in two bytes per entry (Section 4.3,
// "Cheaper storage of hash functions").  Thread t owns the groups of 8 bits
// t, t+T, ...: one 16-byte load brings the 8 codes of a group for a nonzero.

// Two-byte codes of Gaussian samples (Section 4.3): q = floor((x + 8) 2^12),
// formed as floor(x 2^12) + 2^15 (exact in FP32).  Codes outside [0, 65535]
// (x < -8 or x >= 8) and NaN are clamped (NaN to 0) and reported.
__global__ void __launch_bounds__(256) quantize_gaussian_kernel(const float *__restrict__ x, long long n,
                                                                uint16_t *__restrict__ q, blsh_dev_scratch *scratch) {
    unsigned long long outside = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float c = floorf(__ldg(x + i) * 4096.0f) + 32768.0f;
        if (!(c >= 0.0f)) {
            c = 0.0f;
            ++outside;
        } else if (c > 65535.0f) {
            c = 65535.0f;
            ++outside;
        }
        q[i] = (uint16_t)c;
    }
    if (outside) blsh_dev_error(scratch, BLSH_ENUMERIC, -1, outside);
}

// SplitMix64 (Steele, Lea and Flood 2014) read as a counter-based
// generator: output k of the stream `seed` is the finaliser of
// seed + (k + 1) * 0x9E3779B97F4A7C15.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k) {
    unsigned long long z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Eight codes per thread (one 16-byte store): entry c = t * bits + j sums
// the twelve 16-bit pieces of outputs 3c .. 3c+2 (Irwin-Hall, mean 393210,
// standard deviation 65536 to 1e-10) and encodes x = (S - 393210) / 2^16 as
// floor((x + 8) 2^16 / 16) = floor((S - 393210) / 16) + 32768.
__global__ void __launch_bounds__(256) gaussian_codes_kernel(unsigned long long seed, long long groups,
                                                             uint16_t *__restrict__ codes) {
    for (long long gidx = (long long)blockIdx.x * blockDim.x + threadIdx.x; gidx < groups;
         gidx += (long long)gridDim.x * blockDim.x) {
        uint32_t packed[4];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const unsigned long long c = (unsigned long long)gidx * 8ull + (unsigned long long)e;
            int S = 0;
#pragma unroll
            for (int w = 0; w < 3; ++w) {
                const unsigned long long o = splitmix64_at(seed, 3ull * c + (unsigned long long)w);
                S += (int)(o & 0xFFFFull) + (int)((o >> 16) & 0xFFFFull) + (int)((o >> 32) & 0xFFFFull) +
                     (int)(o >> 48);
            }
            const int code = ((S - 393210) >> 4) + 32768;   // arithmetic shift: floor division by 16
            if (e & 1) packed[e >> 1] |= (uint32_t)code << 16;
            else packed[e >> 1] = (uint32_t)code;
        }
        reinterpret_cast<uint4 *>(codes)[gidx] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    }
}

// Dense rows X [N][d] against R [d][bits], the same FP32 sums with the same
// error bound and FP64 recheck (coordinates in order 0..d-1).  One CTA per
// row; the row is staged in shared memory.
__global__ void __launch_bounds__(256) srp_dense_simt_kernel(const float *__restrict__ X, long long N, int d,
                                                             const float *__restrict__ R, int bits, int per_thread,
                                                             uint32_t *__restrict__ sig, blsh_dev_scratch *scratch) {
    extern __shared__ float xs[];
    const int T = blockDim.x;
    const int t = threadIdx.x;
    const int words = bits >> 5;
    unsigned long long rechecked = 0, zeros = 0;
    for (long long row = blockIdx.x; row < N; row += gridDim.x) {
        __syncthreads();
        for (int c = t; c < d; c += T) xs[c] = __ldg(X + (size_t)row * d + c);
        __syncthreads();
        float acc[kSrpMaxPerThread], mag[kSrpMaxPerThread];
#pragma unroll
        for (int u = 0; u < kSrpMaxPerThread; ++u) acc[u] = mag[u] = 0.0f;
        for (int c = 0; c < d; ++c) {
            const float v = xs[c];
            const float *Rrow = R + (size_t)c * bits + t;
#pragma unroll
            for (int u = 0; u < kSrpMaxPerThread; ++u) {
                if (u < per_thread) {
                    const float r = __ldg(Rrow + u * T);
                    acc[u] = __fmaf_rn(v, r, acc[u]);
                    mag[u] = __fmaf_rn(fabsf(v), fabsf(r), mag[u]);
                }
            }
        }
        const float n = (float)d;
        const int w = t >> 5;
#pragma unroll
        for (int u = 0; u < kSrpMaxPerThread; ++u) {
            if (u < per_thread) {
                const float bound = 1.25f * n * 5.9604644775390625e-8f * mag[u] + n * 1.4e-45f;
                bool bit;
                if (fabsf(acc[u]) > bound) {
                    bit = acc[u] >= 0.0f;
                } else {
                    double dd = 0.0;
                    for (int c = 0; c < d; ++c) dd += (double)xs[c] * (double)__ldg(R + (size_t)c * bits + t + u * T);
                    bit = dd >= 0.0;
                    ++rechecked;
                    zeros += dd == 0.0;
                }
                const unsigned word = __ballot_sync(kFull, bit);
                if ((t & 31) == 0) sig[(size_t)row * words + w + u * (T >> 5)] = word;
            }
        }
    }
    if (rechecked) atomicAdd(&scratch->counters[2], rechecked);
    if (zeros) atomicAdd(&scratch->counters[3], zeros);
}

// Columns [col0, col0 + ncols) of the sparse projection (multiples of 128)
// for the rows row_mask selects, on the 16-byte path (R float or two-byte
// codes); -1 when that path does not take the shape.
template <typename RT>
int srp_sparse_cols(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                    const RT *R, int64_t dim, int bits, int col0, int ncols, const uint8_t *row_mask,
                    uint32_t *sig, cudaStream_t s) {
    // selected rows (usually few): pieces of 512 columns, one per CTA; all
    // rows: the whole range per CTA.  T4 = 32 wt threads, V = groups / T4
    // groups of four columns per thread: for two-byte codes the fewest warps
    // that give every thread at most two groups (each nonzero's shuffles and
    // address then serve eight columns: measured faster, e.g. one warp per
    // row for 256 columns), otherwise the largest divisor of groups/32 up to 8
    const int piece = row_mask && ncols % 512 == 0 ? 512 : ncols;
    const int pieces = ncols / piece;
    const int groups = piece / 4;
    int wt = 0;
    if (sizeof(RT) == 2)
        for (int c = 1; c <= 8 && !wt; ++c)
            if ((groups / 32) % c == 0 && groups / (32 * c) <= 2) wt = c;
    if (!wt) {
        wt = 8;
        while ((groups / 32) % wt) --wt;
    }
    const int T4 = 32 * wt, V = groups / T4;
    if (V < 1 || V > 4) return -1;
    // many small CTAs (rows have very different lengths): 32 per SM measured best
    const long long cap = (long long)ctx->sm_count * 32;
    const unsigned grid = (unsigned)(N * pieces < cap ? N * pieces : cap);
    // items from a counter where each CTA has many of them (at least 256;
    // otherwise a fixed share per CTA): kSrpGrab per grab, eight times as
    // many when a row mask selects the rows (most items of a grab are then
    // skipped at once)
    const int grab = N * pieces >= 256ll * grid ? (row_mask ? 8 * kSrpGrab : kSrpGrab) : 0;
    BLSH_CUDA(ctx, cudaMemsetAsync(&ctx->scratch->recheck_count, 0, sizeof(unsigned long long), s));
    BLSH_CUDA(ctx, cudaMemsetAsync(&ctx->scratch->hash_work, 0, sizeof(unsigned long long), s));
    uint2 *q = ctx->recheck_queue;
    blsh_dev_scratch *scr = ctx->scratch;
    const char *name = sizeof(RT) == 2 ? "srp_sparse4_kernel (two-byte codes)" : "srp_sparse4_kernel";
    blsh_time_start(ctx, s);
    switch (V) {
    case 1: srp_sparse4_kernel<1, RT><<<grid, T4, 0, s>>>(indptr, indices, values, N, R, dim, bits, col0, pieces, row_mask, sig, scr, q, grab); break;
    case 2: srp_sparse4_kernel<2, RT><<<grid, T4, 0, s>>>(indptr, indices, values, N, R, dim, bits, col0, pieces, row_mask, sig, scr, q, grab); break;
    case 3: srp_sparse4_kernel<3, RT><<<grid, T4, 0, s>>>(indptr, indices, values, N, R, dim, bits, col0, pieces, row_mask, sig, scr, q, grab); break;
    default: srp_sparse4_kernel<4, RT><<<grid, T4, 0, s>>>(indptr, indices, values, N, R, dim, bits, col0, pieces, row_mask, sig, scr, q, grab); break;
    }
    BLSH_LAUNCHED(ctx, name);
    blsh_time_start(ctx, s);
    srp_recheck_kernel<RT><<<ctx->sm_count * 4, 256, 0, s>>>(q, indptr, indices, values, R, dim, bits, sig, scr);
    BLSH_LAUNCHED(ctx, "srp_recheck_kernel");
    return BLSH_OK;
}

// Column ranges the kernel cannot take in one launch (col_count / 128 with no
// divisor in 1..8 that leaves at most 4 groups per thread) are split: the
// largest piece it can take first, and so on (128 columns always can).
template <typename RT>
int srp_sparse_range(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                     const RT *R, int64_t dim, int bits, int col_begin, int col_count, const uint8_t *row_mask,
                     uint32_t *sig, cudaStream_t s) {
    for (int c0 = col_begin, left = col_count; left > 0;) {
        int rc = -1, piece = left;
        for (; piece > 0; piece -= 128) {
            rc = srp_sparse_cols<RT>(ctx, indptr, indices, values, N, R, dim, bits, c0, piece, row_mask, sig, s);
            if (rc != -1) break;
        }
        if (rc != BLSH_OK) return rc == -1 ? blsh_fail(ctx, BLSH_EINVAL, "no launch shape") : rc;
        c0 += piece;
        left -= piece;
    }
    return BLSH_OK;
}

int srp_threads(int bits, int *per_thread) {
    const int words = bits / 32;
    int wt = 8;
    while (words % wt) --wt;
    *per_thread = bits / (32 * wt);
    return 32 * wt;
}

}  // namespace

// minhash_kernel over every set, then minhash_big_kernel over the long sets
// the first one queued.
template <int WV>
int minhash_launch(blsh_ctx *ctx, cudaStream_t s, unsigned grid, unsigned big_grid, const int64_t *indptr,
                   const uint32_t *indices, int64_t N, int n_hashes, const uint32_t *a, const uint32_t *b,
                   uint32_t *sig, uint2 *big) {
    blsh_dev_scratch *scr = ctx->scratch;
    blsh_time_start(ctx, s);
    minhash_kernel<WV><<<grid, 256, 0, s>>>(indptr, indices, N, n_hashes, a, b, sig, scr, big);
    BLSH_LAUNCHED(ctx, "minhash_kernel");
    blsh_time_start(ctx, s);
    minhash_big_kernel<WV><<<big_grid, 1024, 0, s>>>(indptr, indices, n_hashes, a, b, sig, scr, big);
    BLSH_LAUNCHED(ctx, "minhash_big_kernel");
    return BLSH_OK;
}

extern "C" int blsh_minhash(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, int64_t N,
                            int32_t n_hashes, const uint32_t *a, const uint32_t *b, uint32_t *sig, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !indices || !a || !b || !sig)
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices, a, b and sig are required");
    if (N < 0 || n_hashes <= 0 || n_hashes % 32)
        return blsh_fail(ctx, BLSH_EINVAL, "n_hashes must be a positive multiple of 32");
    if (!blsh_aligned(indptr, 8)) return blsh_fail(ctx, BLSH_EINVAL, "misaligned indptr");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long blocks_needed = (N + 7) / 8;
    const long long cap = (long long)ctx->sm_count * 8;
    const unsigned grid = (unsigned)(blocks_needed < cap ? blocks_needed : cap);
    const int words = n_hashes / 32;
    const unsigned big_grid = (unsigned)ctx->sm_count * 2;
    // long sets go to minhash_big_kernel through the context's work queue
    uint2 *big = ctx->recheck_queue;
    BLSH_CUDA(ctx, cudaMemsetAsync(&ctx->scratch->work3, 0, sizeof(unsigned long long), s));
    const int wv = words % 8 == 0 ? 8 : words % 4 == 0 ? 4 : words % 2 == 0 ? 2 : 1;
    switch (wv) {
    case 8: return minhash_launch<8>(ctx, s, grid, big_grid, indptr, indices, N, n_hashes, a, b, sig, big);
    case 4: return minhash_launch<4>(ctx, s, grid, big_grid, indptr, indices, N, n_hashes, a, b, sig, big);
    case 2: return minhash_launch<2>(ctx, s, grid, big_grid, indptr, indices, N, n_hashes, a, b, sig, big);
    default: return minhash_launch<1>(ctx, s, grid, big_grid, indptr, indices, N, n_hashes, a, b, sig, big);
    }
}

extern "C" int blsh_srp_sparse(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *values,
                               int64_t N, const float *R, int64_t dim, int32_t bits, uint32_t *sig, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !indices || !values || !R || !sig)
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices, values, R and sig are required");
    if (N < 0 || N >= (1ll << 32) || dim <= 0 || bits <= 0 || bits % 32 || bits > 4096)
        return blsh_fail(ctx, BLSH_EINVAL, "bits must be a positive multiple of 32, at most 4096; N < 2^32");
    if (!blsh_aligned(indptr, 8)) return blsh_fail(ctx, BLSH_EINVAL, "misaligned indptr");
    if (N == 0) return BLSH_OK;
    // threads = 32 * (largest divisor of bits/32 that is at most 8)
    const int words = bits / 32;
    int wt = 8;
    while (words % wt) --wt;
    const int T = 32 * wt;
    const int per_thread = bits / T;
    if (per_thread > kSrpMaxPerThread) return blsh_fail(ctx, BLSH_EINVAL, "bits/32 needs a divisor in 2..8");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    // many small CTAs (rows have very different lengths): 32 per SM measured best
    const long long cap = (long long)ctx->sm_count * 32;
    const unsigned grid = (unsigned)(N < cap ? N : cap);
    if (bits % 128 == 0 && blsh_aligned(R, 16)) {
        const int rc = srp_sparse_cols<float>(ctx, indptr, indices, values, N, R, dim, bits, 0, bits, nullptr, sig, s);
        if (rc != -1) return rc;
    }
    blsh_time_start(ctx, s);
    srp_sparse_kernel<float><<<grid, T, 0, s>>>(indptr, indices, values, N, R, dim, bits, per_thread, sig, ctx->scratch);
    BLSH_LAUNCHED(ctx, "srp_sparse_kernel");
    return BLSH_OK;
}

int blsh_srp_dense_simt(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                        uint32_t *sig, cudaStream_t s) {
    int per_thread = 0;
    const int T = srp_threads(bits, &per_thread);
    if (per_thread > kSrpMaxPerThread) return blsh_fail(ctx, BLSH_EINVAL, "bits/32 needs a divisor in 2..8");
    const size_t smem = sizeof(float) * (size_t)d;
    if (smem > 48 * 1024) {
        if (smem > ctx->smem_optin) return blsh_fail(ctx, BLSH_EINVAL, "d too large");
        BLSH_CUDA(ctx, cudaFuncSetAttribute(srp_dense_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
    }
    const long long cap = (long long)ctx->sm_count * 16;
    const unsigned grid = (unsigned)(N < cap ? N : cap);
    blsh_time_start(ctx, s);
    srp_dense_simt_kernel<<<grid, T, smem, s>>>(X, N, d, R, bits, per_thread, sig, ctx->scratch);
    BLSH_LAUNCHED(ctx, "srp_dense_simt_kernel");
    return BLSH_OK;
}

extern "C" int blsh_quantize_gaussian(blsh_ctx *ctx, const float *x, int64_t n, uint16_t *q, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (n < 0 || (n > 0 && (!x || !q))) return blsh_fail(ctx, BLSH_EINVAL, "x and q are required");
    if (n == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long blocks = (n + 255) / 256;
    const long long cap = (long long)ctx->sm_count * 16;
    blsh_time_start(ctx, s);
    quantize_gaussian_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(x, n, q, ctx->scratch);
    BLSH_LAUNCHED(ctx, "quantize_gaussian_kernel");
    return BLSH_OK;
}

extern "C" int blsh_gaussian_codes(blsh_ctx *ctx, uint64_t seed, int64_t dim, int32_t bits, uint16_t *codes,
                                   void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (dim < 0 || bits <= 0 || bits % 8 || (dim > 0 && !codes))
        return blsh_fail(ctx, BLSH_EINVAL, "bits must be a positive multiple of 8; codes are required");
    if (!blsh_aligned(codes, 16)) return blsh_fail(ctx, BLSH_EINVAL, "codes must be 16-byte aligned");
    if (dim == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long groups = dim * (long long)(bits / 8);
    const long long blocks = (groups + 255) / 256;
    const long long cap = (long long)ctx->sm_count * 32;
    blsh_time_start(ctx, s);
    gaussian_codes_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>((unsigned long long)seed, groups,
                                                                                  codes);
    BLSH_LAUNCHED(ctx, "gaussian_codes_kernel");
    return BLSH_OK;
}

extern "C" int blsh_srp_sparse_cols(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                    const float *values, int64_t N, const float *R, int64_t dim, int32_t bits,
                                    int32_t col_begin, int32_t col_count, const uint8_t *row_mask, uint32_t *sig,
                                    void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !indices || !values || !R || !sig)
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices, values, R and sig are required");
    if (N < 0 || N >= (1ll << 32) || dim <= 0 || bits <= 0 || bits % 128 || bits > 4096 || col_begin < 0 ||
        col_count <= 0 || col_begin % 128 || col_count % 128 || col_begin + col_count > bits)
        return blsh_fail(ctx, BLSH_EINVAL, "bits, col_begin and col_count must be multiples of 128 within bits");
    if (!blsh_aligned(indptr, 8) || !blsh_aligned(R, 16)) return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    return srp_sparse_range<float>(ctx, indptr, indices, values, N, R, dim, bits, col_begin, col_count, row_mask,
                                   sig, blsh_stream(stream));
}

extern "C" int blsh_srp_sparse_q16_cols(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                        const float *values, int64_t N, const uint16_t *Rq, int64_t dim,
                                        int32_t bits, int32_t col_begin, int32_t col_count,
                                        const uint8_t *row_mask, uint32_t *sig, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !indices || !values || !Rq || !sig)
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices, values, Rq and sig are required");
    if (N < 0 || N >= (1ll << 32) || dim <= 0 || bits <= 0 || bits % 128 || bits > 4096 || col_begin < 0 ||
        col_count <= 0 || col_begin % 128 || col_count % 128 || col_begin + col_count > bits)
        return blsh_fail(ctx, BLSH_EINVAL, "bits, col_begin and col_count must be multiples of 128 within bits");
    if (!blsh_aligned(indptr, 8) || !blsh_aligned(Rq, 8)) return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    return srp_sparse_range<uint16_t>(ctx, indptr, indices, values, N, Rq, dim, bits, col_begin, col_count, row_mask,
                                      sig, blsh_stream(stream));
}

extern "C" int blsh_srp_sparse_q16(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                   const float *values, int64_t N, const uint16_t *Rq, int64_t dim, int32_t bits,
                                   uint32_t *sig, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!indptr || !indices || !values || !Rq || !sig)
        return blsh_fail(ctx, BLSH_EINVAL, "indptr, indices, values, Rq and sig are required");
    if (N < 0 || N >= (1ll << 32) || dim <= 0 || bits <= 0 || bits % 32 || bits > 4096)
        return blsh_fail(ctx, BLSH_EINVAL, "bits must be a positive multiple of 32, at most 4096; N < 2^32");
    if (!blsh_aligned(indptr, 8) || !blsh_aligned(Rq, 2)) return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long cap = (long long)ctx->sm_count * 32;
    const unsigned grid = (unsigned)(N < cap ? N : cap);
    if (bits % 128 == 0 && blsh_aligned(Rq, 8))   // 8-byte loads of four codes
        return srp_sparse_range<uint16_t>(ctx, indptr, indices, values, N, Rq, dim, bits, 0, bits, nullptr, sig, s);
    int per_thread;
    const int T = srp_threads(bits, &per_thread);
    if (per_thread > kSrpMaxPerThread) return blsh_fail(ctx, BLSH_EINVAL, "bits/32 needs a divisor in 2..8");
    blsh_time_start(ctx, s);
    srp_sparse_kernel<uint16_t><<<grid, T, 0, s>>>(indptr, indices, values, N, Rq, dim, bits, per_thread, sig,
                                                   ctx->scratch);
    BLSH_LAUNCHED(ctx, "srp_sparse_kernel");
    return BLSH_OK;
}
