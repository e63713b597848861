// band.cu -- LSH banding candidate generation (Section 2, "Candidate
// generation via LSH"): objects whose `rows` hashes agree on a whole band
// become a candidate pair.
//
// The paper's hashtables are replaced by a sort:
//   1. every (band b, object i) gets a sort key: the band index in the top
//      bits, below it the band's hashes themselves (cosine: the `rows` sign
//      bits, exact) or a 64-bit hash of them (Jaccard);
//   2. an LSD radix sort (8-bit digits, stable) groups equal keys, objects in
//      increasing order inside a group;
//   3. for each sorted position p, the pairs (p, q > p) inside its group are
//      counted, then written at offsets from a prefix sum.  A pair is written
//      only for the first band in which it collides, so every distinct pair
//      appears once.  To find that band cheaply every object also gets a row
//      of its band keys in band order: cosine keys packed as bytes, 16-bit
//      or 32-bit lanes (by `rows`), compared four / two / one band at a time
//      with a SWAR zero-lane test on the XOR of two rows; Jaccard 64-bit band
//      hashes, confirmed by comparing the hashes themselves, so a hash
//      collision never merges buckets.  The count pass records which pairs
//      it keeps (one bit per tested pair, in the workspace's keep record),
//      and the write pass writes those pairs without testing them again.
#include "common.cuh"
#include "radix.cuh"
#include "scan.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
using blsh_radix::kSortTile;

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// `rows` sign bits starting at bit `start` of a row (bit j in word j/32).
__device__ __forceinline__ uint32_t bit_field(const uint32_t *row, int start, int rows) {
    const int w = start >> 5, o = start & 31;
    unsigned long long two = __ldg(row + w);
    if (o + rows > 32) two |= (unsigned long long)__ldg(row + w + 1) << 32;
    const unsigned long long mask = rows == 32 ? 0xffffffffull : ((1ull << rows) - 1);
    return (uint32_t)((two >> o) & mask);
}

__device__ __forceinline__ unsigned long long band_hash(const uint32_t *row, int start, int rows) {
    unsigned long long h = 0x243f6a8885a308d3ull;
    for (int r = 0; r < rows; ++r) h = mix64(h ^ (__ldg(row + start + r) + 0x9e3779b97f4a7c15ull * (r + 1)));
    return h;
}

struct BandArgs {
    const uint32_t *sig;
    long long N;
    int W, kind, rows, bands, band_bits, key_shift;
    unsigned long long *bk;   // Jaccard: [N][bands] band hashes
    uint32_t *ck;             // cosine: [N][ck_words] band keys packed in lanes of ck_lane bytes
    int ck_lane, ck_words;
    int vec16;                // rows of sig start 16-byte aligned
    int exact_classes;        // Jaccard: class ids in ck (4-byte lanes), 32-bit sort keys, no bk
};

// Lane width (bytes) of packed cosine band keys, and 32-bit words per row
// (rounded up to a multiple of 4 words so rows are 16-byte aligned).
__host__ __device__ inline int cos_lane_bytes(int rows) { return rows <= 8 ? 1 : (rows <= 16 ? 2 : 4); }
__host__ __device__ inline int cos_row_words(int rows, int bands) {
    const int words = (bands * cos_lane_bytes(rows) + 3) / 4;
    return (words + 3) & ~3;
}

__global__ void band_keys_kernel(BandArgs A, unsigned long long *keys, uint32_t *vals) {
    const long long n = A.N * A.bands;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < n;
         it += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(it / A.N);
        const long long i = it - (long long)b * A.N;
        const uint32_t *row = A.sig + (size_t)i * A.W;
        unsigned long long key;
        if (A.kind == BLSH_COSINE) {
            const uint32_t f = bit_field(row, b * A.rows, A.rows);
            key = ((unsigned long long)b << A.rows) | f;
            unsigned char *kr = reinterpret_cast<unsigned char *>(A.ck + (size_t)i * A.ck_words);
            if (A.ck_lane == 1) kr[b] = (unsigned char)f;
            else if (A.ck_lane == 2) reinterpret_cast<uint16_t *>(kr)[b] = (uint16_t)f;
            else reinterpret_cast<uint32_t *>(kr)[b] = f;
        } else {
            const unsigned long long h = band_hash(row, b * A.rows, A.rows);
            if (A.exact_classes) {
                // 32-bit key: the band, then the top bits of its hash (equal
                // keys are sorted together; the class ids split collisions)
                key = ((unsigned long long)b << (32 - A.band_bits)) | (h >> (32 + A.band_bits));
            } else {
                A.bk[(size_t)i * A.bands + b] = h;
                key = A.band_bits == 0 ? h : (((unsigned long long)b << A.key_shift) | (h >> A.band_bits));
            }
        }
        keys[it] = key;
        vals[it] = (uint32_t)i;
    }
}

// ---- pair emission -----------------------------------------------------------

__device__ __forceinline__ bool same_band(const BandArgs &A, uint32_t x, uint32_t y, int b) {
    const uint32_t *rx = A.sig + (size_t)x * A.W, *ry = A.sig + (size_t)y * A.W;
    if (A.kind == BLSH_COSINE) return bit_field(rx, b * A.rows, A.rows) == bit_field(ry, b * A.rows, A.rows);
    const int start = b * A.rows;
    if (A.vec16 && (A.rows & 3) == 0 && (start & 3) == 0) {   // whole 16-byte groups
        const uint4 *vx = reinterpret_cast<const uint4 *>(rx + start), *vy = reinterpret_cast<const uint4 *>(ry + start);
        for (int r = 0; r < (A.rows >> 2); ++r) {
            const uint4 u = __ldg(vx + r), v = __ldg(vy + r);
            if (u.x != v.x || u.y != v.y || u.z != v.z || u.w != v.w) return false;
        }
        return true;
    }
    for (int r = 0; r < A.rows; ++r)
        if (__ldg(rx + start + r) != __ldg(ry + start + r)) return false;
    return true;
}

// Jaccard: the pair (x, y) met in band b is emitted iff b is the first band
// whose keys agree in full.  The 64-bit band hashes find the candidate bands
// (equal keys have equal hashes); a hash match is confirmed on the keys
// themselves before it decides anything.
__device__ __forceinline__ bool emit_here_jaccard(const BandArgs &A, uint32_t x, uint32_t y, int b) {
    const unsigned long long *bx = A.bk + (size_t)x * A.bands, *by = A.bk + (size_t)y * A.bands;
    for (int c = 0; c <= b; ++c)
        if (__ldg(bx + c) == __ldg(by + c) && same_band(A, x, y, c)) return c == b;
    return false;   // band b's hashes or keys differ: only a truncated-hash collision put them together
}

// Nonzero iff some lane of v (lanes of 1, 2 or 4 bytes) is zero.  The
// borrow of the subtraction can also flag a lane above a zero lane, never a
// lane below the lowest zero lane, so "any zero lane among the low lanes" is
// exact once the lanes above are masked off.
__device__ __forceinline__ uint32_t zero_lanes(uint32_t v, int lane) {
    if (lane == 1) return (v - 0x01010101u) & ~v & 0x80808080u;
    if (lane == 2) return (v - 0x00010001u) & ~v & 0x80008000u;
    return v == 0u ? 0x80000000u : 0u;
}

// Does any band c < b of x and y agree?  Cosine: packed key rows.
__device__ __forceinline__ bool earlier_band_cos(const BandArgs &A, uint32_t x, uint32_t y, int b) {
    const uint32_t *kx = A.ck + (size_t)x * A.ck_words, *ky = A.ck + (size_t)y * A.ck_words;
    const int per_word = 4 / A.ck_lane;
    const int full = b / per_word, rest = b % per_word;
    for (int w = 0; w < full; ++w)
        if (zero_lanes(__ldg(kx + w) ^ __ldg(ky + w), A.ck_lane)) return true;
    if (rest) {
        const uint32_t keep = (1u << (8 * A.ck_lane * rest)) - 1u;   // the low `rest` lanes
        if (zero_lanes(__ldg(kx + full) ^ __ldg(ky + full), A.ck_lane) & keep) return true;
    }
    return false;
}

// The pair (x, y) met in band b is emitted iff its band-b keys agree in full
// and no earlier band has them agree.
__device__ __forceinline__ bool emit_here(const BandArgs &A, uint32_t x, uint32_t y, int b) {
    if (A.kind == BLSH_COSINE) return !earlier_band_cos(A, x, y, b);
    return emit_here_jaccard(A, x, y, b);
}

// Cosine rows of packed band keys are at most kCkRegWords words long when
// they fit the register fast path below (64 one-byte bands, 32 two-byte
// bands or 16 four-byte bands).
constexpr int kCkRegWords = 16;

// Cosine emission with x's packed keys held in registers: a pair (x, y) of
// band b is checked against bands < b with 16-byte loads of y's key row only.
__device__ __forceinline__ bool earlier_band_cos_reg(const BandArgs &A, const uint4 (&kx)[kCkRegWords / 4],
                                                     uint32_t y, int b) {
    const uint4 *ky = reinterpret_cast<const uint4 *>(A.ck + (size_t)y * A.ck_words);
    const int per_word = 4 / A.ck_lane;
    const int need = (b + per_word - 1) / per_word;   // words holding bands 0..b-1
#pragma unroll
    for (int w4 = 0; w4 < kCkRegWords / 4; ++w4) {
        if (4 * w4 < need) {
            const uint4 yv = __ldg(ky + w4);
            const uint32_t z[4] = {kx[w4].x ^ yv.x, kx[w4].y ^ yv.y, kx[w4].z ^ yv.z, kx[w4].w ^ yv.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int w = 4 * w4 + c;
                if (w < need) {
                    const int lanes = (w + 1) * per_word <= b ? per_word : b - w * per_word;
                    const uint32_t keep = lanes == per_word ? 0xffffffffu : (1u << (8 * A.ck_lane * lanes)) - 1u;
                    if (zero_lanes(z[c], A.ck_lane) & keep) return true;
                }
            }
        }
    }
    return false;
}

template <bool WRITE>
__global__ void emit_kernel(BandArgs A, const unsigned long long *keys, const uint32_t *vals, long long n,
                            unsigned long long *counts, uint32_t *pairs, long long cap) {
    // Lanes of a warp take 32 consecutive sorted positions.  A position whose
    // bucket continues for at most 32 more entries walks them alone; longer
    // ones are walked afterwards by the whole warp, 32 partners per step, so
    // a bucket of thousands of objects is not a serial chain of loads.
    const bool reg_path = A.kind == BLSH_COSINE && A.ck_words <= kCkRegWords;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long pb = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); pb < n; pb += stride) {
        const long long p = pb + lane;
        const bool live = p < n;
        unsigned long long key = 0;
        uint32_t x = 0;
        int b = 0;
        bool longrun = false;
        unsigned long long c = 0, out = 0;
        if (live) {
            key = keys[p];
            x = vals[p];
            b = A.kind == BLSH_COSINE ? (int)(key >> A.rows) : (A.band_bits == 0 ? 0 : (int)(key >> A.key_shift));
            out = WRITE ? counts[p] : 0;
            longrun = p + 33 < n && keys[p + 33] == key;
        }
        if (live && !longrun) {
            if (reg_path) {
                uint4 kx[kCkRegWords / 4];
                const uint4 *kxp = reinterpret_cast<const uint4 *>(A.ck + (size_t)x * A.ck_words);
#pragma unroll
                for (int w4 = 0; w4 < kCkRegWords / 4; ++w4)
                    kx[w4] = 4 * w4 < A.ck_words ? __ldg(kxp + w4) : make_uint4(0u, 0u, 0u, 0u);
                for (long long q = p + 1; q < n && keys[q] == key; ++q) {
                    const uint32_t y = vals[q];
                    if (!earlier_band_cos_reg(A, kx, y, b)) {
                        if (WRITE) {
                            const long long o = (long long)(out + c);
                            if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(x, y);
                        }
                        ++c;
                    }
                }
            } else {
                for (long long q = p + 1; q < n && keys[q] == key; ++q) {
                    const uint32_t y = vals[q];
                    if (emit_here(A, x, y, b)) {
                        if (WRITE) {
                            const long long o = (long long)(out + c);
                            if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(x, y);
                        }
                        ++c;
                    }
                }
            }
        }
        // the warp walks the long buckets of its lanes, one position at a time
        unsigned pending = __ballot_sync(kFull, longrun);
        while (pending) {
            const int l = __ffs(pending) - 1;
            pending &= pending - 1;
            const long long pl = __shfl_sync(kFull, p, l);
            const unsigned long long kl = __shfl_sync(kFull, key, l);
            const uint32_t xl = __shfl_sync(kFull, x, l);
            const int bl = __shfl_sync(kFull, b, l);
            const unsigned long long ol = __shfl_sync(kFull, out, l);
            unsigned long long cl = 0;
            for (long long q0 = pl + 1;; q0 += 32) {
                const long long q = q0 + lane;
                const bool in = q < n && keys[q] == kl;
                bool ok = false;
                uint32_t y = 0;
                if (in) {
                    y = vals[q];
                    ok = emit_here(A, xl, y, bl);
                }
                const unsigned m = __ballot_sync(kFull, ok);
                if (WRITE && ok) {
                    const long long o = (long long)(ol + cl + __popc(m & lt));
                    if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(xl, y);
                }
                cl += __popc(m);
                if (__ballot_sync(kFull, in) != kFull) break;   // the bucket ended in this step
            }
            if (lane == l) c = cl;
        }
        if (!WRITE && live) counts[p] = c;
    }
}

constexpr int kEmitWinMax = 768;
constexpr int kStageWords = 32;          // key rows of up to 128 bytes take this path

// Staged key rows are cws = (ck_words / 4) | 1 16-byte words apart: an odd
// stride, so lanes reading different rows hit different banks.
__host__ __device__ inline int stage_stride(int ck_words) { return (ck_words >> 2) | 1; }

// emit_warp_kernel: one warp's part of shared memory (16-byte aligned) for a
// window of `win` positions (key rows, keys, ids), the rows and ids of 32
// partners past the window and 32 words of kept bits, and the largest window
// (a multiple of 32) that fits the warp's budget.
__host__ __device__ inline size_t emit_warp_region(int ck_words, int win) {
    const int kw4 = ck_words <= 16 ? 4 : 8;
    const size_t b = (size_t)win * (stage_stride(ck_words) * 16 + 8 + 4) + 32 * 16 * kw4 + 2 * 32 * 4;
    return (b + 15) & ~(size_t)15;
}
// (two CTAs of eight warps per SM; three for the count pass over key rows
// of at most 64 bytes, whose smaller window measured faster there -- the
// window only decides which partners are staged, not which pairs are
// emitted, so the two passes may differ)
inline size_t emit_warp_budget(int ck_words, bool count_pass) {
    return ck_words <= 16 ? (count_pass ? 9 * 1024 : 13 * 1024) : 14 * 1024;
}
inline int emit_warp_ctas(int ck_words, bool count_pass) { return ck_words <= 16 && count_pass ? 3 : 2; }
int emit_warp_win(int ck_words, bool count_pass) {
    int w = 32;
    while (w < kEmitWinMax && emit_warp_region(ck_words, w + 32) <= emit_warp_budget(ck_words, count_pass)) w += 32;
    return w;
}

// First position q >= from with q == n or keys[q] != key, given
// keys[from - 1] == key: galloping, then a binary search.
__device__ long long run_end_global(const unsigned long long *keys, long long n, long long from,
                                    unsigned long long key) {
    long long lo = from, step = 1;
    while (lo < n && keys[lo] == key) {
        const long long probe = lo + step;
        if (probe >= n || keys[probe] != key) {
            long long hi = probe < n ? probe : n;
            ++lo;
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (keys[mid] == key) lo = mid + 1; else hi = mid;
            }
            return lo;
        }
        lo = probe;
        step <<= 1;
    }
    return lo;
}

// How a pair's key rows are compared at band b: the words of chunks below
// nf4 (16-byte chunks) hold earlier bands only and are tested without a mask,
// three operations a word: z = x ^ y, then (z - one) & ~z is OR-ed into t,
// whose lane high bits show a zero lane (an agreeing band) once t is masked
// with `high` at the end.  Chunk nf4 is the tail: word q of it is tested
// under tm[q] (all lanes when the whole word is earlier bands, the low lanes
// of pmask for the word holding band b's own lane, nothing past it).  For
// Jaccard class ids word r of the tail (band b) must match.
struct EmitCmp {
    int nf4, r;
    uint32_t tm[4];
};

__device__ __forceinline__ EmitCmp emit_cmp(int full, uint32_t pmask, uint32_t high) {
    EmitCmp c;
    c.nf4 = full >> 2;
    c.r = full & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) c.tm[q] = q < c.r ? high : (q == c.r ? pmask : 0u);
    return c;
}

// True when the pair (x, y) is emitted at band b: no earlier band agrees
// (and, for Jaccard class ids, band b itself agrees).  xrow and yrow are the
// two key rows (registers or shared memory); NW4 bounds the chunks read.
template <int NW4, int K0 = 0, typename XR, typename YR>
__device__ __forceinline__ bool emit_test(const XR &xrow, const YR &yrow, const EmitCmp &c, bool jac, uint32_t one,
                                          uint32_t high) {
    // the unmasked words in four independent chains (one per word of a
    // chunk), joined and masked with `high` at the end; the tail under tm
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, tt = 0, zr = 0;
#pragma unroll
    for (int k = K0; k < NW4; ++k) {
        if (k <= c.nf4) {
            const uint4 xv = xrow[k], yv = yrow[k];
            const uint32_t z0 = xv.x ^ yv.x, z1 = xv.y ^ yv.y, z2 = xv.z ^ yv.z, z3 = xv.w ^ yv.w;
            if (k < c.nf4) {
                t0 |= (z0 - one) & ~z0;
                t1 |= (z1 - one) & ~z1;
                t2 |= (z2 - one) & ~z2;
                t3 |= (z3 - one) & ~z3;
            } else {
                tt = ((z0 - one) & ~z0 & c.tm[0]) | ((z1 - one) & ~z1 & c.tm[1]) | ((z2 - one) & ~z2 & c.tm[2]) |
                     ((z3 - one) & ~z3 & c.tm[3]);
                if (jac) zr = c.r == 0 ? z0 : c.r == 1 ? z1 : c.r == 2 ? z2 : z3;
            }
        }
    }
    return ((((t0 | t1) | (t2 | t3)) & high) | tt) == 0 && (!jac || zr == 0);
}

// Rows of at most four 16-byte chunks (KW4 <= 4), walk form: the lane's
// plan as one poison word per key-row word, p[w] nonzero in every lane of a
// band >= b (0 below, `one` past band b's word).  (x ^ y) | p can be zero
// only in a lane of an earlier band, so a word's test is three operations
// without masks or branches; a borrow into a poisoned lane comes only from a
// zero lane below it, which is a hit already.
template <int NW4>
__device__ __forceinline__ bool emit_test_poison(const uint4 *kx, const uint4 *yrow, const uint32_t *p, bool jac,
                                                 int eqw, uint32_t one, uint32_t high) {
    uint32_t t0 = 0, t1 = 0, t2 = 0, t3 = 0, zr = 1;
#pragma unroll
    for (int k = 0; k < NW4; ++k) {
        const uint4 yv = yrow[k];
        const uint32_t z0 = (kx[k].x ^ yv.x) | p[4 * k + 0], z1 = (kx[k].y ^ yv.y) | p[4 * k + 1];
        const uint32_t z2 = (kx[k].z ^ yv.z) | p[4 * k + 2], z3 = (kx[k].w ^ yv.w) | p[4 * k + 3];
        t0 |= (z0 - one) & ~z0;
        t1 |= (z1 - one) & ~z1;
        t2 |= (z2 - one) & ~z2;
        t3 |= (z3 - one) & ~z3;
        if (jac) {   // class id word b (not poisoned by the Jaccard plan) must match
            const uint32_t e0 = kx[k].x ^ yv.x, e1 = kx[k].y ^ yv.y, e2 = kx[k].z ^ yv.z, e3 = kx[k].w ^ yv.w;
            zr = eqw == 4 * k ? e0 : eqw == 4 * k + 1 ? e1 : eqw == 4 * k + 2 ? e2 : eqw == 4 * k + 3 ? e3 : zr;
        }
    }
    return (((t0 | t1) | (t2 | t3)) & high) == 0 && (!jac || zr == 0);
}

// The poison words of a lane at band b (see emit_test_poison): bands 0..b-1
// are `full` whole words and the low `rest` lanes of word `full`.
template <int NW>
__device__ __forceinline__ void emit_poison(uint32_t *p, int full, int rest, int lane_bits, uint32_t one) {
    const uint32_t partial = rest ? one & ~((1u << (lane_bits * rest)) - 1u) : one;
#pragma unroll
    for (int w = 0; w < NW; ++w) p[w] = w < full ? 0u : (w == full ? partial : one);
}

template <int NW4, bool WRITE, bool PZ>
__device__ __forceinline__ bool emit_step(const uint4 *yrow, uint32_t y, unsigned j, bool live, int i,
                                          long long p0, long long end, uint32_t x, const uint4 *kx,
                                          const EmitCmp &cmp, const uint32_t *pz, int eqw, bool jac, uint32_t one,
                                          uint32_t high, unsigned long long out, unsigned long long &cnt,
                                          uint32_t *pairs, long long cap) {
    // the test for every lane (no branch around it), then the lane's range
    bool pass;
    if constexpr (PZ) pass = emit_test_poison<NW4>(kx, yrow, pz, jac, eqw, one, high);
    else pass = emit_test<NW4>(kx, yrow, cmp, jac, one, high);
    const bool ok = pass && live && (int)j > i && p0 + (long long)j < end;
    if (WRITE && ok) {
        const long long o = (long long)(out + cnt);
        if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(x, y);
    }
    cnt += ok;
    return ok;
}

// Position of set bit number k (from 0, lowest first) of m; k < popc(m).
__device__ __forceinline__ int nth_set_bit(uint32_t m, unsigned k) {
    int pos = 0;
#pragma unroll
    for (int w = 16; w > 0; w >>= 1) {
        const unsigned c = (unsigned)__popc(m & ((1u << w) - 1u));
        if (k >= c) {
            k -= c;
            m >>= w;
            pos += w;
        }
    }
    return pos;
}

// The walk of one warp over partners [jmin, jmax) (tile-relative), NW4
// 16-byte words of key rows compared per pair (cmp: the lane's plan for
// its band).  Partners inside the window come from the stage; partners past
// it (long buckets) are fetched 32 at a time into the warp's own buffer, one
// row per lane, so that their loads overlap.  With a keep record (rec, count
// pass) each lane also stores which partners it keeps: bit t of word
// rec[32 w + lane] is partner jmin + 32 w + t.
template <int NW4, bool WRITE, bool PZ>
__device__ __forceinline__ void emit_walk(const BandArgs &A, const uint4 *s_ck, const uint32_t *s_val,
                                          uint4 *w_rows, uint32_t *w_ids, uint32_t *s_und, const uint32_t *vals,
                                          long long p0,
                                          int win, int stride, unsigned jmin, unsigned jmax, bool live, int i,
                                          long long end, uint32_t x, const uint4 *kx, const EmitCmp &cmp,
                                          const uint32_t *pz, int eqw, bool jac, uint32_t one, uint32_t high,
                                          unsigned long long out, unsigned long long &cnt, uint32_t *pairs,
                                          long long cap, uint32_t *rec) {
    const unsigned wend = jmax < (unsigned)win ? jmax : (unsigned)win;
    const int lane = threadIdx.x & 31;
    // the lane's record word being filled (index ridx) and its bits
    unsigned ridx = 0;
    uint32_t racc = 0;
    // partners g0 .. g0 + n - 1 (relative to jmin, n <= 32) with the kept ones in `keep`
    auto rec_put = [&](unsigned g0, unsigned n, uint32_t keep) {
        const unsigned w = g0 >> 5, sh = g0 & 31;
        if (w != ridx) {
            rec[(size_t)ridx * 32 + lane] = racc;
            racc = 0;
            ridx = w;
        }
        racc |= keep << sh;
        if (sh + n > 32) {
            rec[(size_t)ridx * 32 + lane] = racc;
            ++ridx;
            racc = keep >> (32 - sh);
        }
    };
    if constexpr (!PZ && NW4 >= 2) {
        // Long key rows: partners in batches of 32.  Each (lane, partner) is
        // first tested on the first 16-byte chunk only (bands 0..7 of 16-bit
        // keys), which settles nearly every pair that agrees in an earlier
        // band; the rest (noted in `und`) are finished by their own lane at
        // the end of the batch, and the batch's pairs are then counted, or
        // written in partner order.
        const bool more = cmp.nf4 >= 2 || (cmp.nf4 == 1 && (jac || (cmp.tm[0] | cmp.tm[1] | cmp.tm[2] | cmp.tm[3])));
        // the lane's partners: jlo <= j < jhi (none for an idle lane)
        const unsigned jlo = (unsigned)i + 1u, jhi = live ? (unsigned)(end - p0) : 0u;
        const bool whole = cmp.nf4 >= 1;
        const uint32_t m0 = whole ? high : cmp.tm[0], m1 = whole ? high : cmp.tm[1];
        const uint32_t m2 = whole ? high : cmp.tm[2], m3 = whole ? high : cmp.tm[3];
        const bool need_zr = !whole && jac;     // band b's own class id, in the first chunk
        auto batch = [&](unsigned j0, unsigned n, const uint4 *rows, int rstride, const uint32_t *ids) {
            // bit u: no earlier band of the first chunk agrees (hz), band b's
            // class id agrees (zm, Jaccard in the first chunk only)
            uint32_t hz = 0, zm = 0;
            for (unsigned u = 0; u < n; ++u) {
                const uint4 yv = rows[(size_t)u * rstride];
                const uint32_t z0 = kx[0].x ^ yv.x, z1 = kx[0].y ^ yv.y, z2 = kx[0].z ^ yv.z, z3 = kx[0].w ^ yv.w;
                const uint32_t h = ((z0 - one) & ~z0 & m0) | ((z1 - one) & ~z1 & m1) | ((z2 - one) & ~z2 & m2) |
                                   ((z3 - one) & ~z3 & m3);
                hz |= (uint32_t)(h == 0) << u;
                if (need_zr) {
                    const uint32_t zr = cmp.r == 0 ? z0 : cmp.r == 1 ? z1 : cmp.r == 2 ? z2 : z3;
                    zm |= (uint32_t)(zr == 0) << u;
                }
            }
            // partners j0 + u inside [jlo, jhi)
            const unsigned lo = jlo > j0 ? (jlo - j0 < 32u ? jlo - j0 : 32u) : 0u;
            const unsigned hi = jhi > j0 ? (jhi - j0 < n ? jhi - j0 : n) : 0u;
            const uint32_t below_hi = hi >= 32u ? ~0u : (1u << hi) - 1u;
            const uint32_t below_lo = lo >= 32u ? ~0u : (1u << lo) - 1u;
            hz &= below_hi & ~below_lo;
            uint32_t keep = 0, und = 0;
            if (whole && more) und = hz;
            else keep = need_zr ? hz & zm : hz;
            // The undecided (lane, partner) tests.  Where they are uneven
            // (the lane with the most has over 1.25 times the rounds of 32
            // that the warp's total takes, plus one) they are spread evenly
            // over the warp: numbered lane by
            // lane, test t goes to lane t mod 32, which reads both key rows
            // from shared memory and sets the kept bit in the owner's word of
            // s_und.  Otherwise every lane finishes its own.
            const unsigned nu = (unsigned)__popc(und);
            unsigned incl = nu;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned v = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += v;
            }
            const unsigned off = incl - nu, total = __shfl_sync(kFull, incl, 31);
            const unsigned most = __reduce_max_sync(kFull, nu);
            const unsigned rounds = (total + 31) / 32;
            if (most > rounds + rounds / 4 + 1) {
                s_und[lane] = 0;
                __syncwarp();
                const int my_full = 4 * cmp.nf4 + cmp.r;
                const uint32_t my_pm = cmp.r == 0 ? cmp.tm[0] : cmp.r == 1 ? cmp.tm[1] : cmp.r == 2 ? cmp.tm[2] : cmp.tm[3];
                for (unsigned t0 = 0; t0 < total; t0 += 32) {
                    const unsigned t = t0 + lane;
                    int o = 0;                            // the last lane whose first test is <= t
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const unsigned oc = __shfl_sync(kFull, off, o + step);
                        if (oc <= t) o += step;
                    }
                    const unsigned k = t - __shfl_sync(kFull, off, o);
                    const uint32_t um = __shfl_sync(kFull, und, o);
                    const int full_o = __shfl_sync(kFull, my_full, o);
                    const uint32_t pm_o = __shfl_sync(kFull, my_pm, o);
                    if (t < total) {
                        const int u = nth_set_bit(um, k);
                        const uint4 *xr = s_ck + (size_t)o * stride;   // position o of the chunk
                        if (emit_test<NW4, 1>(xr, rows + (size_t)u * rstride, emit_cmp(full_o, pm_o, high), jac, one,
                                              high))
                            atomicOr(&s_und[o], 1u << u);
                    }
                }
                __syncwarp();
                keep |= s_und[lane];
                __syncwarp();
            } else {
                for (uint32_t b = und; b; b &= b - 1) {
                    const int u = __ffs(b) - 1;
                    if (emit_test<NW4, 1>(kx, rows + (size_t)u * rstride, cmp, jac, one, high)) keep |= 1u << u;
                }
            }
            if (!WRITE && rec) rec_put(j0 - jmin, n, keep);
            if (WRITE) {
                for (uint32_t b = keep; b; b &= b - 1) {
                    const long long o = (long long)(out + cnt);
                    if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(x, ids[__ffs(b) - 1]);
                    ++cnt;
                }
            } else {
                cnt += __popc(keep);
            }
        };
        // one call site for both kinds of batch (the code is large): partners
        // inside the window from the stage, past it fetched into the warp's
        // buffer (whole key rows: cw4 chunks, at most NW4)
        const int cw4 = A.ck_words >> 2;
        for (unsigned j0 = jmin; j0 < jmax;) {
            const uint4 *rows;
            int rstride;
            const uint32_t *ids;
            unsigned n;
            if (j0 < wend) {
                n = wend - j0 < 32u ? wend - j0 : 32u;
                rows = s_ck + (size_t)j0 * stride;
                rstride = stride;
                ids = s_val + j0;
            } else {
                n = jmax - j0 < 32u ? jmax - j0 : 32u;
                __syncwarp();
                if (j0 + lane < jmax) {
                    const uint32_t yv = __ldg(vals + p0 + j0 + lane);
                    w_ids[lane] = yv;
                    const uint4 *g = reinterpret_cast<const uint4 *>(A.ck + (size_t)yv * A.ck_words);
#pragma unroll
                    for (int c = 0; c < NW4; ++c)
                        if (c < cw4) w_rows[lane * NW4 + c] = __ldg(g + c);
                }
                __syncwarp();
                rows = w_rows;
                rstride = NW4;
                ids = w_ids;
            }
            batch(j0, n, rows, rstride, ids);
            j0 += n;
        }
        if (!WRITE && rec && jmax > jmin) rec[(size_t)ridx * 32 + lane] = racc;   // the last word
    } else {
        // one kept bit per step into the lane's record word
        auto rec_bit = [&](unsigned j, bool ok) {
            const unsigned g = j - jmin;
            racc |= (uint32_t)ok << (g & 31);
            if ((g & 31) == 31) {
                rec[(size_t)(g >> 5) * 32 + lane] = racc;
                racc = 0;
            }
        };
        for (unsigned j = jmin; j < wend; ++j) {
            const bool ok = emit_step<NW4, WRITE, PZ>(s_ck + (size_t)j * stride, s_val[j], j, live, i, p0, end, x, kx,
                                                      cmp, pz, eqw, jac, one, high, out, cnt, pairs, cap);
            if (!WRITE && rec) rec_bit(j, ok);
        }
        for (unsigned j0 = jmin > (unsigned)win ? jmin : (unsigned)win; j0 < jmax; j0 += 32) {
            __syncwarp();
            if (j0 + lane < jmax) {
                const uint32_t yv = __ldg(vals + p0 + j0 + lane);
                w_ids[lane] = yv;
                const uint4 *g = reinterpret_cast<const uint4 *>(A.ck + (size_t)yv * A.ck_words);
#pragma unroll
                for (int c = 0; c < NW4; ++c) w_rows[lane * NW4 + c] = __ldg(g + c);
            }
            __syncwarp();
            const unsigned n = jmax - j0 < 32u ? jmax - j0 : 32u;
            for (unsigned u = 0; u < n; ++u) {
                const bool ok = emit_step<NW4, WRITE, PZ>(w_rows + u * NW4, w_ids[u], j0 + u, live, i, p0, end, x, kx,
                                                          cmp, pz, eqw, jac, one, high, out, cnt, pairs, cap);
                if (!WRITE && rec) rec_bit(j0 + u, ok);
            }
        }
        // the last, partly filled word (a full one was stored by rec_bit)
        if (!WRITE && rec && jmax > jmin && ((jmax - jmin) & 31)) rec[(size_t)((jmax - jmin) >> 5) * 32 + lane] = racc;
    }
}

// The write pass of a walk the count pass recorded: lane l's partners are the
// set bits of rec[32 w + l] (partner jmin + 32 w + t for bit t), written in
// partner order from its offset `out`; no key rows are read.
__device__ __forceinline__ void emit_replay_walk(const uint32_t *rec, unsigned words, unsigned jmin,
                                                 const uint32_t *s_val, const uint32_t *vals, long long p0, int win,
                                                 uint32_t x, unsigned long long out, uint32_t *pairs, long long cap) {
    const int lane = threadIdx.x & 31;
    unsigned long long cnt = 0;
    for (unsigned w = 0; w < words; ++w) {
        for (uint32_t bits = rec[(size_t)w * 32 + lane]; bits; bits &= bits - 1) {
            const unsigned j = jmin + 32 * w + (unsigned)(__ffs(bits) - 1);
            const uint32_t y = (int)j < win ? s_val[j] : __ldg(vals + p0 + j);
            const long long o = (long long)(out + cnt);
            if (o < cap) reinterpret_cast<uint2 *>(pairs)[o] = make_uint2(x, y);
            ++cnt;
        }
    }
}

// The flat walk for warps whose buckets are small: the pairs (i, j) of the
// warp's 32 positions are numbered in order (position, then partner) and
// lane l takes pairs l, l + 32, ...; the owner of pair t is found by a
// binary search of the lanes' exclusive prefix of partner counts.  Every
// lane reads both rows from the stage.  A kept pair's slot is its owner's
// output offset plus the kept pairs of that owner before it: those of
// earlier steps (acc[owner], kept in shared memory) and those of lower lanes
// in this step (lanes of one owner are contiguous).  All partners are
// staged (the caller checks).  With a keep record (rec), the count pass
// stores each step's ballot of kept pairs as one word and the write pass
// takes its pairs from those words instead of testing them again.
template <int NW4, bool WRITE>
__device__ __forceinline__ void emit_flat(const BandArgs &A, const uint4 *s_ck, const uint32_t *s_val,
                                          const unsigned long long *s_key, uint32_t *acc, int cws, int warp,
                                          bool live, int i, long long end, long long p0, unsigned long long out,
                                          uint32_t one, uint32_t high, int per_word, uint32_t *pairs,
                                          long long cap, uint32_t *rec) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned mine = live ? (unsigned)(end - p0 - i - 1) : 0u;
    unsigned incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const unsigned off = incl - mine;
    const unsigned total = __shfl_sync(kFull, incl, 31);
    acc[lane] = 0;
    __syncwarp();
    for (unsigned t0 = 0; t0 < total; t0 += 32) {
        const unsigned t = t0 + lane;
        const bool valid = t < total;
        int o = 0;                                        // the last lane whose prefix is <= t
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const unsigned oc = __shfl_sync(kFull, off, o + step);
            if (oc <= t) o += step;
        }
        const unsigned off_o = __shfl_sync(kFull, off, o);
        const unsigned long long out_o = __shfl_sync(kFull, out, o);
        const int io = warp * 32 + o;
        const int j = io + 1 + (int)(t - off_o);
        bool ok = false;
        uint32_t x = 0, y = 0;
        if (valid) {
            if (WRITE && rec) {
                ok = (rec[t0 >> 5] >> lane) & 1u;
            } else {
                const unsigned long long key = s_key[io];
                const int b = A.exact_classes ? (A.band_bits == 0 ? 0 : (int)(key >> (32 - A.band_bits)))
                                              : (int)(key >> A.rows);
                const int full = b / per_word, rest = b % per_word;
                const uint32_t pmask = rest ? ((1u << (8 * A.ck_lane * rest)) - 1u) & high : 0u;
                const uint4 *xr = s_ck + (size_t)io * cws, *yr = s_ck + (size_t)j * cws;
                ok = emit_test<NW4>(xr, yr, emit_cmp(full, pmask, high), A.exact_classes != 0, one, high);
            }
            x = s_val[io];
            y = s_val[j];
        }
        const unsigned okm = __ballot_sync(kFull, ok);
        if (!WRITE && rec && lane == 0) rec[t0 >> 5] = okm;
        const unsigned seg = __match_any_sync(kFull, valid ? o : 32 + lane);
        if (WRITE && ok) {
            const long long slot = (long long)(out_o + acc[o] + __popc(okm & seg & lt));
            if (slot < cap) reinterpret_cast<uint2 *>(pairs)[slot] = make_uint2(x, y);
        }
        __syncwarp();
        if (valid && (seg >> lane) == 1u) acc[o] += __popc(okm & seg);   // the segment's highest lane
        __syncwarp();
    }
}

// Emission staged in shared memory, with warps as independent workers.  A
// warp takes the next chunk of 32 sorted positions from a counter and
// stages its own window (the chunk and the positions after it: keys, object
// ids and the objects' key rows) in its own part of shared memory; no
// barrier ties it to the other warps, so a warp with long buckets holds up
// no one.  Lane l owns position l of the chunk (its object x, band b and key
// row in registers) and finds the end of its bucket by a binary search of
// the staged keys (continued in global memory when the bucket runs past the
// window).  Where buckets are long the warp walks the partners j of its 32
// positions in order: each step reads one staged key row (the same address
// for every lane: a broadcast) and every lane tests its own pair (x, y_j) on
// the bands before its b.  Where they are short it numbers the pairs and
// gives each lane one (emit_flat).  Pairs of position i are counted, or
// written, in partner order, the order emit_kernel uses.
//
// Keep record: the count pass stores which pairs it keeps, one bit per
// tested pair, so that the write pass only writes them.  A chunk takes its
// words (emit_flat: one per step; the walk: 32 per 32 partners) from a
// counter in the record area rec[0, rec_cap); rec_off[chunk] is its first
// word times 2 plus 1 if it went flat, or ~0 where the area was full (the
// write pass then tests that chunk's pairs again).  With rec == NULL
// nothing is recorded.
template <bool WRITE, int KW4>
__global__ void __launch_bounds__(256, (KW4 <= 4 && !WRITE) ? 3 : 2) emit_warp_kernel(BandArgs A, const unsigned long long *keys,
                                                             const uint32_t *vals, long long n,
                                                             unsigned long long *counts, uint32_t *pairs,
                                                             long long cap, int win_cap,
                                                             unsigned long long *next_chunk, uint32_t *rec,
                                                             unsigned long long *rec_off,
                                                             unsigned long long rec_cap,
                                                             unsigned long long *rec_next) {
    extern __shared__ uint4 s_all[];
    const int cw4 = A.ck_words >> 2, cws = stage_stride(A.ck_words);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the warp's region: [win_cap][cws] key rows, [32][KW4] partner rows,
    // keys [win_cap], object ids [win_cap], ids or counts [32], kept bits [32]
    const size_t region = emit_warp_region(A.ck_words, win_cap);
    uint4 *s_ck = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(s_all) + warp * region);
    uint4 *w_rows = s_ck + (size_t)win_cap * cws;
    unsigned long long *s_key = reinterpret_cast<unsigned long long *>(w_rows + 32 * KW4);
    uint32_t *s_val = reinterpret_cast<uint32_t *>(s_key + win_cap);
    uint32_t *w_ids = s_val + win_cap;
    uint32_t *s_und = w_ids + 32;
    const uint32_t one = A.ck_lane == 1 ? 0x01010101u : (A.ck_lane == 2 ? 0x00010001u : 1u);
    const uint32_t high = one << (8 * A.ck_lane - 1);
    const int per_word = 4 / A.ck_lane;
    const long long chunks = (n + 31) >> 5;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(next_chunk, 1ull);
        c = __shfl_sync(kFull, c, 0);
        if ((long long)c >= chunks) break;
        const long long p0 = (long long)c << 5;
        int win = (int)(n - p0 < win_cap ? n - p0 : win_cap);
        // write pass: a recorded chunk needs no key rows and no tests
        const unsigned long long ro = WRITE && rec ? rec_off[c] : ~0ull;
        const bool replay = ro != ~0ull;
        __syncwarp();                                     // the previous chunk is done with the stage
        // keys first; ids and key rows only as far as the chunk's buckets
        // reach inside the window (all of it if one runs past it)
        for (int k = lane; k < win; k += 32) s_key[k] = keys[p0 + k];
        __syncwarp();
        {
            int lo = lane + 1, hi = win;
            if (lane < win) {
                const unsigned long long kl = s_key[lane];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (s_key[mid] == kl) lo = mid + 1; else hi = mid;
                }
            } else {
                lo = 0;
            }
            win = (int)__reduce_max_sync(kFull, (unsigned)lo);
        }
        for (int k = lane; k < win; k += 32) {
            const uint32_t v = vals[p0 + k];
            s_val[k] = v;
            if (!replay) {
                const uint4 *src = reinterpret_cast<const uint4 *>(A.ck + (size_t)v * A.ck_words);
                for (int q = 0; q < cw4; ++q) s_ck[(size_t)k * cws + q] = __ldg(src + q);
            }
        }
        __syncwarp();
        const int tile = win < 32 ? win : 32;
        const int i = lane;
        const bool live = i < tile;
        unsigned long long key = 0;
        uint32_t x = 0;
        int b = 0;
        long long end = p0;
        uint4 kx[KW4];                                    // KW4 >= cw4
#pragma unroll
        for (int c = 0; c < KW4; ++c) kx[c] = make_uint4(0u, 0u, 0u, 0u);
        if (live) {
            key = s_key[i];
            x = s_val[i];
            b = A.exact_classes ? (A.band_bits == 0 ? 0 : (int)(key >> (32 - A.band_bits))) : (int)(key >> A.rows);
            int lo = i + 1, hi = win;                     // first staged position past the bucket
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_key[mid] == key) lo = mid + 1; else hi = mid;
            }
            end = p0 + lo;
            if (lo == win && end < n) end = run_end_global(keys, n, end, key);
            if (!replay) {
#pragma unroll
                for (int c = 0; c < KW4; ++c)
                    if (c < cw4) kx[c] = s_ck[(size_t)i * cws + c];
            }
        }
        const int full = b / per_word, rest = b % per_word;   // bands 0..b-1: `full` words and `rest` lanes
        const uint32_t pmask = rest ? ((1u << (8 * A.ck_lane * rest)) - 1u) & high : 0u;
        // Jaccard class ids: word b must match too (a key collision is not a bucket)
        const int need = A.exact_classes ? b + 1 : full + (rest ? 1 : 0);
        const int nw4 = (__reduce_max_sync(kFull, (unsigned)(live ? need : 0)) + 3) >> 2;
        const unsigned jmin = 1u;
        const unsigned jmax = __reduce_max_sync(kFull, live ? (unsigned)(end - p0) : 0u);
        const unsigned long long out = WRITE && live ? counts[p0 + i] : 0;
        unsigned long long cnt = 0;
        // small buckets: number the pairs and give each lane one (the walk
        // below would spend a step per partner position on mostly idle lanes)
        const unsigned pairs_w = __reduce_add_sync(kFull, live ? (unsigned)(end - p0 - i - 1) : 0u);
        const bool flat = replay ? (ro & 1ull) != 0
                                 : jmax <= (unsigned)win && 5ull * ((pairs_w + 31) / 32) < 2ull * (jmax - jmin);
        uint32_t *crec = nullptr;                         // this chunk's record words
        if (replay) {
            crec = rec + (ro >> 1);
        } else if (!WRITE && rec) {
            const unsigned long long words =
                flat ? (pairs_w + 31) / 32 : (jmax > jmin ? 32ull * ((jmax - jmin + 31) / 32) : 0ull);
            unsigned long long off = 0;
            if (lane == 0) {
                off = atomicAdd(rec_next, words);
                rec_off[c] = off + words <= rec_cap ? off << 1 | (flat ? 1ull : 0ull) : ~0ull;
            }
            off = __shfl_sync(kFull, off, 0);
            if (off + words <= rec_cap) crec = rec + off;
        }
        if (replay && !flat) {
            emit_replay_walk(crec, jmax > jmin ? (jmax - jmin + 31) / 32 : 0u, jmin, s_val, vals, p0, win, x, out,
                             pairs, cap);
            continue;
        }
        if (flat) {
#define BLSH_FLAT(NW) emit_flat<NW, WRITE>(A, s_ck, s_val, s_key, w_ids, cws, 0, live, i, end, p0, out, one, high, \
                                           per_word, pairs, cap, crec)
            if constexpr (KW4 <= 4) {
                switch (nw4) {
                case 0: BLSH_FLAT(0); break;
                case 1: BLSH_FLAT(1); break;
                case 2: BLSH_FLAT(2); break;
                case 3: BLSH_FLAT(3); break;
                default: BLSH_FLAT(4); break;
                }
            } else {
                switch (nw4) {
                case 0: BLSH_FLAT(0); break;
                case 1: case 2: BLSH_FLAT(2); break;
                case 3: case 4: BLSH_FLAT(4); break;
                case 5: case 6: BLSH_FLAT(6); break;
                default: BLSH_FLAT(8); break;
                }
            }
#undef BLSH_FLAT
            if (!WRITE && live) counts[p0 + i] = w_ids[lane];
            continue;
        }
        const EmitCmp cmp = emit_cmp(full, pmask, high);
        const bool jac = A.exact_classes != 0;
        const int eqw = jac ? b : -1;
        // rows of at most four chunks: the plan as poison words (see emit_test_poison)
        constexpr bool kPZ = KW4 <= 4;
        uint32_t pz[kPZ ? 16 : 1];
        if constexpr (kPZ) emit_poison<16>(pz, full, rest, 8 * A.ck_lane, one);
#define BLSH_WALK(NW) emit_walk<NW, WRITE, kPZ>(A, s_ck, s_val, w_rows, w_ids, s_und, vals, p0, win, cws, jmin, jmax, live, \
                                                i, end, x, kx, cmp, pz, eqw, jac, one, high, out, cnt, pairs, cap, crec)
        if constexpr (KW4 <= 4) {
            switch (nw4) {
            case 0: BLSH_WALK(0); break;
            case 1: BLSH_WALK(1); break;
            case 2: BLSH_WALK(2); break;
            case 3: BLSH_WALK(3); break;
            default: BLSH_WALK(4); break;
            }
        } else {
            // rows of 5-8 chunks: the walk reads chunk 0 of every pair and
            // the rest only for the few pairs it leaves undecided, so one
            // form (NW4 = 8, chunks past the plan skipped) serves every band
            if (nw4 == 0) BLSH_WALK(0);
            else BLSH_WALK(8);
        }
#undef BLSH_WALK
        if (!WRITE && live) counts[p0 + i] = cnt;
    }
}

// First position of the run of `key` that contains p (keys[p] == key):
// galloping backwards, then a binary search.
__device__ long long run_start_global(const unsigned long long *keys, long long p, unsigned long long key) {
    long long hi = p, step = 1;                           // keys[hi] == key
    for (;;) {
        const long long probe = hi - step;
        if (probe < 0 || keys[probe] != key) {
            long long lo = probe < 0 ? 0 : probe + 1;     // the start is in [lo, hi]
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (keys[mid] == key) hi = mid; else lo = mid + 1;
            }
            return lo;
        }
        hi = probe;
        step <<= 1;
    }
}

// Jaccard class ids: for sorted position p (object v, band b) the id is the
// first position of its run whose band-b hashes equal v's, so two objects
// share an id in band b iff they agree on the whole band.  Almost always
// that is the run's first position; a hash collision inside a run is split
// off by comparing the hashes themselves.
__global__ void __launch_bounds__(256) class_id_kernel(BandArgs A, const unsigned long long *keys,
                                                       const uint32_t *vals, long long n) {
    const int shift = 32 - A.band_bits;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[p];
        const uint32_t v = vals[p];
        const int b = A.band_bits == 0 ? 0 : (int)(key >> shift);
        long long cid = p;
        if (p > 0 && keys[p - 1] == key) {
            const long long h = run_start_global(keys, p, key);
            if (same_band(A, v, vals[h], b)) {
                cid = h;
            } else {
                for (long long q = h + 1; q < p; ++q)
                    if (same_band(A, v, vals[q], b)) { cid = q; break; }
            }
        }
        A.ck[(size_t)v * A.ck_words + b] = (uint32_t)cid;
    }
}

__global__ void check_cap_kernel(const long long *n_pairs, long long cap, blsh_dev_scratch *scratch) {
    if (*n_pairs > cap) blsh_dev_error(scratch, BLSH_ETRUNC, 1, (unsigned long long)(*n_pairs - cap));
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t keys0, keys1, vals0, vals1, bk, ck, counts, hist, partial, grand, rec_off, rec, total;
};

// The emission's keep record (emit_warp_kernel): 16 words per position by
// default; bytes a caller's workspace has beyond rec go to it.
constexpr size_t kRecBytesPerPos = 64;

// Jaccard class-id rows: one 32-bit id per band, rounded to 16 bytes.
int jac_row_words(int bands) { return (bands + 3) & ~3; }

Layout layout(long long N, int kind, int rows, int bands) {
    const long long n = N * bands;
    const long long tiles = (n + kSortTile - 1) / kSortTile;
    const long long hist_n = 256 * tiles;
    const long long part = blsh_scan::tiles_for(hist_n > n ? hist_n : n) + 1;
    Layout L;
    size_t o = 0;
    L.keys0 = o; o = up256(o + n * 8);
    L.keys1 = o; o = up256(o + n * 8);
    L.vals0 = o; o = up256(o + n * 4);
    L.vals1 = o; o = up256(o + n * 4);
    const bool classes = kind == BLSH_JACCARD && jac_row_words(bands) <= kStageWords;
    L.bk = o; o = up256(o + (kind == BLSH_JACCARD && !classes ? n * 8 : 0));
    L.ck = o; o = up256(o + (kind == BLSH_COSINE ? (size_t)N * cos_row_words(rows, bands) * 4
                                                  : (classes ? (size_t)N * jac_row_words(bands) * 4 : 0)));
    L.counts = o; o = up256(o + n * 8);
    L.hist = o; o = up256(o + hist_n * 4);
    L.partial = o; o = up256(o + part * 8);
    L.grand = o; o = up256(o + 16);
    L.rec_off = o; o = up256(o + ((n + 31) / 32) * 8);
    L.rec = o;
    L.total = o + (size_t)n * kRecBytesPerPos;
    return L;
}

int band_bits_for(int bands) {
    int b = 0;
    while ((1 << b) < bands) ++b;
    return b;
}

}  // namespace

extern "C" int blsh_lsh_candidates_workspace(int64_t N, int32_t kind, int32_t rows, int32_t bands, size_t *bytes) {
    if (!bytes || N < 0 || bands <= 0 || rows <= 0) return BLSH_EINVAL;
    if (kind != BLSH_JACCARD && kind != BLSH_COSINE) return BLSH_EINVAL;
    *bytes = layout(N, kind, rows, bands).total;
    return BLSH_OK;
}

extern "C" int blsh_lsh_candidates(blsh_ctx *ctx, const uint32_t *sig, int64_t N, int32_t sig_words, int32_t kind,
                                   int32_t rows, int32_t bands, uint32_t *pairs, int64_t cap, int64_t *n_pairs,
                                   void *workspace, size_t workspace_bytes, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!sig || !n_pairs || (cap > 0 && !pairs)) return blsh_fail(ctx, BLSH_EINVAL, "sig and n_pairs are required");
    if (kind != BLSH_JACCARD && kind != BLSH_COSINE) return blsh_fail(ctx, BLSH_EINVAL, "bad kind");
    if (N < 0 || N > (1ll << 32) || rows <= 0 || bands <= 0 || cap < 0)
        return blsh_fail(ctx, BLSH_EINVAL, "bad N, rows, bands or cap");
    if (kind == BLSH_COSINE && (rows > 32 || (long long)rows * bands > 32ll * sig_words))
        return blsh_fail(ctx, BLSH_EINVAL, "cosine bands need rows <= 32 and rows*bands <= 32*sig_words bits");
    if (kind == BLSH_JACCARD && (long long)rows * bands > sig_words)
        return blsh_fail(ctx, BLSH_EINVAL, "rows*bands exceeds the signature length");
    const int band_bits = band_bits_for(bands);
    if (kind == BLSH_COSINE && band_bits + rows > 64) return blsh_fail(ctx, BLSH_EINVAL, "too many bands");
    if ((long long)N * bands >= (1ll << 32)) return blsh_fail(ctx, BLSH_EINVAL, "N * bands must be < 2^32");
    if (!blsh_aligned(n_pairs, 8) || !blsh_aligned(workspace, 256) || !blsh_aligned(pairs, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    const Layout L = layout(N, kind, rows, bands);
    if (!workspace || workspace_bytes < L.rec)
        return blsh_fail(ctx, BLSH_ETRUNC, "workspace needs %zu bytes", L.rec);
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long n = N * bands;
    if (n == 0 || N < 2) {
        BLSH_CUDA(ctx, cudaMemsetAsync(n_pairs, 0, sizeof(int64_t), s));
        return BLSH_OK;
    }
    char *ws = (char *)workspace;
    unsigned long long *keys[2] = {(unsigned long long *)(ws + L.keys0), (unsigned long long *)(ws + L.keys1)};
    uint32_t *vals[2] = {(uint32_t *)(ws + L.vals0), (uint32_t *)(ws + L.vals1)};
    unsigned long long *counts = (unsigned long long *)(ws + L.counts);
    uint32_t *hist = (uint32_t *)(ws + L.hist);

    BandArgs A;
    A.sig = sig;
    A.N = N;
    A.W = sig_words;
    A.kind = kind;
    A.rows = rows;
    A.bands = bands;
    A.band_bits = band_bits;
    A.key_shift = 64 - band_bits;
    A.exact_classes = kind == BLSH_JACCARD && jac_row_words(bands) <= kStageWords;
    A.bk = kind == BLSH_JACCARD && !A.exact_classes ? (unsigned long long *)(ws + L.bk) : nullptr;
    A.ck = kind == BLSH_COSINE || A.exact_classes ? (uint32_t *)(ws + L.ck) : nullptr;
    A.ck_lane = A.exact_classes ? 4 : cos_lane_bytes(rows);
    A.vec16 = blsh_aligned(sig, 16) && sig_words % 4 == 0;
    A.ck_words = A.exact_classes ? jac_row_words(bands) : cos_row_words(rows, bands);
    if (kind == BLSH_COSINE)   // pad lanes past the last band stay zero
        BLSH_CUDA(ctx, cudaMemsetAsync(A.ck, 0, (size_t)N * A.ck_words * 4, s));

    const unsigned grid = (unsigned)((n + 255) / 256 < 65535ll * 16 ? (n + 255) / 256 : 65535ll * 16);
    blsh_time_start(ctx, s);
    band_keys_kernel<<<grid, 256, 0, s>>>(A, keys[0], vals[0]);
    BLSH_LAUNCHED(ctx, "band_keys_kernel");

    const int key_bits = kind == BLSH_COSINE ? band_bits + rows : (A.exact_classes ? 32 : 64);
    int cur = 0;
    {
        const int rc = blsh_radix::sort(ctx, keys, vals, n, key_bits, hist, (uint32_t *)(ws + L.partial),
                                        (uint32_t *)(ws + L.grand), s, &cur);
        if (rc) return rc;
    }
    if (A.exact_classes) {
        blsh_time_start(ctx, s);
        class_id_kernel<<<grid, 256, 0, s>>>(A, keys[cur], vals[cur], n);
        BLSH_LAUNCHED(ctx, "class_id_kernel");
    }
    const bool staged = (kind == BLSH_COSINE || A.exact_classes) && A.ck_words <= kStageWords;
    // per pass: the window, its shared memory and the grid (CTAs per SM)
    const int win_c = staged ? emit_warp_win(A.ck_words, true) : 0;
    const int win_w = staged ? emit_warp_win(A.ck_words, false) : 0;
    const size_t smem_c = staged ? 8 * emit_warp_region(A.ck_words, win_c) : 0;
    const size_t smem_w = staged ? 8 * emit_warp_region(A.ck_words, win_w) : 0;
    const unsigned egrid_c = (unsigned)(ctx->sm_count * emit_warp_ctas(A.ck_words, true));
    const unsigned egrid_w = (unsigned)(ctx->sm_count * emit_warp_ctas(A.ck_words, false));
    // the two chunk counters (count pass, write pass) and the record's
    unsigned long long *next_chunk = &ctx->scratch->band_work[0];
    BLSH_CUDA(ctx, cudaMemsetAsync(next_chunk, 0, 3 * sizeof(unsigned long long), s));
    // the keep record: the workspace past L.rec, in 4-byte words
    const unsigned long long rec_cap = (workspace_bytes - L.rec) / 4;
    uint32_t *rec = staged && rec_cap > 0 ? (uint32_t *)(ws + L.rec) : nullptr;
    unsigned long long *rec_off = (unsigned long long *)(ws + L.rec_off);
    unsigned long long *rec_next = &ctx->scratch->band_work[2];
    if (staged) {
        if (A.ck_words <= 16) {
            BLSH_CUDA(ctx, cudaFuncSetAttribute(emit_warp_kernel<false, 4>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            BLSH_CUDA(ctx, cudaFuncSetAttribute(emit_warp_kernel<true, 4>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
            blsh_time_start(ctx, s);
            emit_warp_kernel<false, 4><<<egrid_c, 256, smem_c, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap,
                                                                    win_c, next_chunk, rec, rec_off, rec_cap,
                                                                    rec_next);
        } else {
            BLSH_CUDA(ctx, cudaFuncSetAttribute(emit_warp_kernel<false, 8>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c));
            BLSH_CUDA(ctx, cudaFuncSetAttribute(emit_warp_kernel<true, 8>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_w));
            blsh_time_start(ctx, s);
            emit_warp_kernel<false, 8><<<egrid_c, 256, smem_c, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap,
                                                                    win_c, next_chunk, rec, rec_off, rec_cap,
                                                                    rec_next);
        }
    } else {
        blsh_time_start(ctx, s);
        emit_kernel<false><<<grid, 256, 0, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap);
    }
    BLSH_LAUNCHED(ctx, staged ? "emit_warp_kernel (count pass)" : "emit_kernel (count pass)");
    blsh_time_start(ctx, s);
    BLSH_CUDA(ctx, blsh_scan::exclusive_scan<unsigned long long>(counts, counts, n,
                                                                 (unsigned long long *)(ws + L.partial),
                                                                 (unsigned long long *)n_pairs, s));
    ctx->launches.fetch_add(3, std::memory_order_relaxed);
    blsh_time_stop(ctx, "exclusive scan (3 launches)");
    blsh_time_start(ctx, s);
    if (staged && A.ck_words <= 16)
        emit_warp_kernel<true, 4><<<egrid_w, 256, smem_w, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap,
                                                               win_w, next_chunk + 1, rec, rec_off, rec_cap, rec_next);
    else if (staged)
        emit_warp_kernel<true, 8><<<egrid_w, 256, smem_w, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap,
                                                               win_w, next_chunk + 1, rec, rec_off, rec_cap, rec_next);
    else
        emit_kernel<true><<<grid, 256, 0, s>>>(A, keys[cur], vals[cur], n, counts, pairs, cap);
    BLSH_LAUNCHED(ctx, staged ? "emit_warp_kernel (write pass)" : "emit_kernel (write pass)");
    blsh_time_start(ctx, s);
    check_cap_kernel<<<1, 1, 0, s>>>((const long long *)n_pairs, cap, ctx->scratch);
    BLSH_LAUNCHED(ctx, "check_cap_kernel");
    return BLSH_OK;
}
