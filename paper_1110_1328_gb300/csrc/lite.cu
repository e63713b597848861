// lite.cu -- Algorithm 2 (BayesLSH-Lite).
//
// Pass 1 is the verification kernel of verify.cu in its Lite form: the
// pruning loop over at most h hashes, no concentration test; an unpruned
// pair is marked as a survivor in its status byte.  Pass 2 (this file) gives
// every survivor its exact similarity: the survivors are collected into a
// queue (one atomic per tile of 512 statuses) and warps take them in
// grid-stride order, so the many survivors of one bucket of near-duplicates
// spread over the GPU; a warp computes a survivor's similarity
// cooperatively by intersecting the two sorted index lists (each lane
// binary-searches elements of the shorter row in the longer one, staged in
// shared memory when it is short).  Survivors beyond the queue's capacity
// are found by a scan of the statuses in tiles handed out by a counter.
//
//   Jaccard: s = |A n B| / |A u B|, one FP64 division.
//   Cosine:  s = D / sqrt(Nx * Ny) with D = sum over common indices of
//            rn(x_i * y_i * 2^60), Nx = sum rn(x_i^2 * 2^60), Ny likewise,
//            each term the exact product of two floats rounded to an
//            integer (formed with integer arithmetic) and added in int64, so
//            the sums do not depend on the order the lanes add them in.
// A pair is kept iff s > t.
#include "verify.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;

struct LiteArgs {
    const uint2 *pairs;
    long long P;
    const long long *P_dev;
    const int64_t *indptr;
    const uint32_t *indices;
    const float *values;
    double t;
    uint8_t *status;
    double *sim;
    blsh_dev_scratch *scratch;
    int vec;                  // status is 16-byte aligned
    const long long *norm2;   // cosine: each row's sum of fixed_term(v, v), or NULL (formed per pair)
};

constexpr int kLiteGrab = 16;   // tiles of 512 statuses per grab (this pass sees only survivors the queue missed)

// rn(u v 2^60) for two floats, by integer arithmetic: u = mu 2^eu and
// v = mv 2^ev with 24-bit integer mantissas, so u v 2^60 = mu mv 2^(eu+ev+60)
// and the 48-bit product is shifted with round-half-to-even (symmetric, as
// the FP64 conversion rounds).  The same value as the FP64 expression
// rn((double)u * (double)v * 2^60) (the product of two floats is exact in
// FP64).  Products of |u v| >= 2^2 (outside rows of squared norm below 4)
// are shifted up as far as they fit and otherwise saturate to the int64
// limit of their sign, as that conversion does; non-finite inputs saturate
// by sign.  All integer arithmetic: the FP64 pipe is narrow on this part,
// and a branch to FP64 code here was executed (predicated) for every term.
__device__ __forceinline__ long long fixed_term(float u, float v) {
    const uint32_t bu = __float_as_uint(u), bv = __float_as_uint(v);
    int eu = (int)((bu >> 23) & 0xffu), ev = (int)((bv >> 23) & 0xffu);
    uint32_t mu = bu & 0x7fffffu, mv = bv & 0x7fffffu;
    if (eu) mu |= 0x800000u; else eu = 1;   // subnormals: exponent 1 - 150
    if (ev) mv |= 0x800000u; else ev = 1;
    const unsigned long long prod = (unsigned long long)mu * mv;   // < 2^48
    const int sh = eu + ev - 300 + 60;                               // u v 2^60 = prod 2^sh
    unsigned long long r;
    if (sh >= 0) {
        if (sh > 15 && (sh >= 63 || (prod >> (63 - sh)) != 0))   // at least 2^63 in magnitude
            return ((bu ^ bv) >> 31) ? (long long)0x8000000000000000ull : 0x7fffffffffffffffll;
        r = prod << sh;
    } else if (-sh > 48) {
        r = 0;                                                       // below half of 2^0
    } else {
        const int k = -sh;
        const unsigned long long q = prod >> k, rem = prod & ((1ull << k) - 1ull), half = 1ull << (k - 1);
        r = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);
    }
    return ((bu ^ bv) >> 31) ? -(long long)r : (long long)r;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// First position in L[0..n) holding a value >= v (L in global or shared
// memory).
__device__ __forceinline__ long long lower_bound(const uint32_t *L, long long n, uint32_t v) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (L[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

constexpr int kLiteStage = 512;   // longer-row elements a warp stages in shared memory

// The sums of one survivor's exact similarity (the whole warp): rows
// x = [ax, ax+na) and y = [ay, ay+nb) of the CSR; D_out = the intersection
// size (sets) or D (cosine), and for cosine without have_norms the two
// squared norms.  The shorter row's elements are spread over the lanes and each
// is looked up in the longer row by binary search: with the longer row held
// one element per lane (at most 32 elements: the search steps are shuffles),
// staged in the warp's shared memory (at most kLiteStage), or read from
// global memory.  No search touches global memory unless the longer row has
// more than kLiteStage elements.
template <bool COSINE>
__device__ __forceinline__ void lite_exact_one(const LiteArgs &A, long long ax, long long na, long long ay,
                                               long long nb, bool have_norms, uint32_t *w_idx, float *w_val,
                                               long long &D_out, long long &Nx_out, long long &Ny_out) {
    const int lane = threadIdx.x & 31;
    // the shorter row S, the longer row L (the sums below do not depend on
    // which row is which)
    long long s0 = ax, ns = na, l0 = ay, nl = nb;
    if (nb < na) { s0 = ay; ns = nb; l0 = ax; nl = na; }
    long long inter = 0, D = 0, Ns = 0, Nl = 0;
    if (nl <= 32) {
        // lane e holds element e of both rows
        uint32_t si = 0, li = 0;
        float sv = 0.0f, lv = 0.0f;
        if (lane < ns) {
            si = __ldg(A.indices + s0 + lane);
            if (COSINE) sv = __ldg(A.values + s0 + lane);
        }
        if (lane < nl) {
            li = __ldg(A.indices + l0 + lane);
            if (COSINE) lv = __ldg(A.values + l0 + lane);
        }
        // first position p of L with L[p] >= si: at most 32 candidates, so six
        // halvings of [lo, hi) settle every lane
        int lo = 0, hi = (int)nl;
#pragma unroll
        for (int it = 0; it < 6; ++it) {
            const int mid = (lo + hi) >> 1;
            const uint32_t v = __shfl_sync(kFull, li, mid & 31);
            if (lo < hi) {
                if (v < si) lo = mid + 1;
                else hi = mid;
            }
        }
        const uint32_t at = __shfl_sync(kFull, li, lo & 31);
        const bool hit = lane < ns && lo < nl && at == si;
        if (!COSINE) {
            inter = __popc(__ballot_sync(kFull, hit));
        } else {
            const float atv = __shfl_sync(kFull, lv, lo & 31);
            D = hit ? fixed_term(sv, atv) : 0;
            if (!have_norms) {
                Ns = lane < ns ? fixed_term(sv, sv) : 0;
                Nl = lane < nl ? fixed_term(lv, lv) : 0;
            }
        }
    } else {
        const uint32_t *Lidx = A.indices + l0;
        const float *Lval = COSINE ? A.values + l0 : nullptr;
        __syncwarp();                                      // the previous survivor is done with the stage
        if (nl <= kLiteStage) {
            for (long long i = lane; i < nl; i += 32) {
                w_idx[i] = __ldg(A.indices + l0 + i);
                if (COSINE) {
                    const float v = __ldg(A.values + l0 + i);
                    w_val[i] = v;
                    if (!have_norms) Nl += fixed_term(v, v);
                }
            }
            __syncwarp();
            Lidx = w_idx;
            if (COSINE) Lval = w_val;
        } else if (COSINE && !have_norms) {
#pragma unroll 4
            for (long long i = lane; i < nl; i += 32) {
                const float v = __ldg(A.values + l0 + i);
                Nl += fixed_term(v, v);
            }
        }
#pragma unroll 2
        for (long long i = lane; i < ns; i += 32) {
            const uint32_t v = __ldg(A.indices + s0 + i);
            const long long pos = lower_bound(Lidx, nl, v);
            const bool hit = pos < nl && Lidx[pos] == v;
            if (!COSINE) {
                inter += hit;
            } else {
                const float sv = __ldg(A.values + s0 + i);
                if (hit) D += fixed_term(sv, Lval[pos]);
                if (!have_norms) Ns += fixed_term(sv, sv);
            }
        }
    }
    // the warp's sums (the same in every lane): the intersection size, or D
    // and the two squared norms (which row is which does not matter: the
    // similarity uses their product)
    if (!COSINE) {
        D_out = nl > 32 ? warp_sum(inter) : inter;
    } else {
        D_out = warp_sum(D);
        if (!have_norms) {
            Nx_out = warp_sum(Ns);
            Ny_out = warp_sum(Nl);
        }
    }
}

// The sums of up to 32 / W survivors at once, each in its own W-lane
// segment of the warp (W = 8 or 16), for survivors whose two rows have at
// most W elements each: the register path of lite_exact_one with the
// shuffles, the search and the sums kept inside the segment.  sel holds the
// lanes whose survivors are to be formed; lane i's survivor rows are
// [ax, ex) and [ay, ey) in lane i.  Segment k takes the k-th survivor left
// in sel; each survivor's lane receives its sums.
template <bool COSINE, int W>
__device__ __forceinline__ void lite_segments(const LiteArgs &A, unsigned sel, long long ax, long long ex,
                                              long long ay, long long ey, bool have_norms, long long &myD,
                                              long long &myNx, long long &myNy) {
    constexpr int S = 32 / W;
    const int lane = threadIdx.x & 31;
    const int e = lane & (W - 1), seg = lane / W;
    const unsigned lt = (1u << lane) - 1u;
    while (sel) {
        // the first S survivors left: segment seg takes the seg-th of them
        unsigned taken = sel, rest = sel;
#pragma unroll
        for (int k = 0; k < S; ++k) rest &= rest - 1;
        taken &= ~rest;
        unsigned m = taken;
        for (int k = 0; k < seg && m; ++k) m &= m - 1;
        const int pick = m ? __ffs(m) - 1 : -1;
        const int src = pick < 0 ? 0 : pick;
        const long long a0 = __shfl_sync(kFull, ax, src), a1 = __shfl_sync(kFull, ex, src);
        const long long b0 = __shfl_sync(kFull, ay, src), b1 = __shfl_sync(kFull, ey, src);
        long long s0 = a0, ns = a1 - a0, l0 = b0, nl = b1 - b0;
        if (nl < ns) { s0 = b0; ns = b1 - b0; l0 = a0; nl = a1 - a0; }
        if (pick < 0) ns = nl = 0;
        uint32_t si = 0, li = 0;
        float sv = 0.0f, lv = 0.0f;
        if (e < ns) {
            si = __ldg(A.indices + s0 + e);
            if (COSINE) sv = __ldg(A.values + s0 + e);
        }
        if (e < nl) {
            li = __ldg(A.indices + l0 + e);
            if (COSINE) lv = __ldg(A.values + l0 + e);
        }
        // first position p of L with L[p] >= si, among 0..nl (nl <= W)
        int lo = 0, hi = (int)nl;
#pragma unroll
        for (int it = 0; (1 << it) <= W; ++it) {
            const int mid = (lo + hi) >> 1;
            const uint32_t v = __shfl_sync(kFull, li, mid & (W - 1), W);
            if (lo < hi) {
                if (v < si) lo = mid + 1;
                else hi = mid;
            }
        }
        const uint32_t at = __shfl_sync(kFull, li, lo & (W - 1), W);
        const bool hit = e < ns && lo < nl && at == si;
        long long D = 0, Ns = 0, Nl = 0;
        if (!COSINE) {
            const unsigned segmask = (W == 32 ? kFull : ((1u << W) - 1u)) << (seg * W);
            D = __popc(__ballot_sync(kFull, hit) & segmask);
        } else {
            const float atv = __shfl_sync(kFull, lv, lo & (W - 1), W);
            D = hit ? fixed_term(sv, atv) : 0;
            if (!have_norms) {
                Ns = e < ns ? fixed_term(sv, sv) : 0;
                Nl = e < nl ? fixed_term(lv, lv) : 0;
            }
#pragma unroll
            for (int o = W / 2; o > 0; o >>= 1) {
                D += __shfl_xor_sync(kFull, D, o);
                if (!have_norms) {
                    Ns += __shfl_xor_sync(kFull, Ns, o);
                    Nl += __shfl_xor_sync(kFull, Nl, o);
                }
            }
        }
        // survivor i's sums from the first lane of its segment
        const int from = W * __popc(taken & lt);
        const long long gD = __shfl_sync(kFull, D, from & 31);
        const long long gNs = __shfl_sync(kFull, Ns, from & 31), gNl = __shfl_sync(kFull, Nl, from & 31);
        if ((taken >> lane) & 1u) {
            myD = gD;
            if (COSINE && !have_norms) {
                myNx = gNs;
                myNy = gNl;
            }
        }
        sel = rest;
    }
}

// The similarity from the sums (one lane per survivor: FP64 is a narrow
// pipe on this part, so the division and square root run once per survivor
// rather than once per lane of a warp-wide computation).
template <bool COSINE>
__device__ __forceinline__ double lite_similarity(long long D, long long Nx, long long Ny, long long na,
                                                  long long nb) {
    if (!COSINE) {
        const long long uni = na + nb - D;
        return uni == 0 ? 0.0 : __ddiv_rn((double)D, (double)uni);
    }
    if (Nx == 0 || Ny == 0) return 0.0;
    return __ddiv_rn(__ll2double_rn(D), __dsqrt_rn(__dmul_rn(__ll2double_rn(Nx), __ll2double_rn(Ny))));
}

// Up to 32 survivors, survivor my_q of lane l (-1: none): their pairs, row
// bounds and (when formed) squared norms are loaded by all lanes at once, so
// those dependent loads overlap across the batch; then the warp forms the
// survivors' sums one after the other, and finally every lane turns its own
// survivor's sums into the similarity and writes it with the verdict.
template <bool COSINE>
__device__ __forceinline__ void lite_batch(const LiteArgs &A, long long my_q, bool have_norms, uint32_t *w_idx,
                                           float *w_val) {
    long long ax = 0, ex = 0, ay = 0, ey = 0, nx = 0, ny = 0;
    if (my_q >= 0) {
        const uint2 pr = __ldg(A.pairs + my_q);
        ax = __ldg(A.indptr + pr.x);
        ex = __ldg(A.indptr + pr.x + 1);
        ay = __ldg(A.indptr + pr.y);
        ey = __ldg(A.indptr + pr.y + 1);
        if (have_norms) {
            nx = __ldg(A.norm2 + pr.x);
            ny = __ldg(A.norm2 + pr.y);
        }
    }
    const int lane = threadIdx.x & 31;
    // lane i keeps survivor i's sums
    long long myD = 0, myNx = nx, myNy = ny;
    // survivors whose rows are short share the warp: four at a time when
    // both rows have at most 8 elements, two when at most 16 (a group too
    // small to fill the segments joins the next wider one)
    unsigned todo = __ballot_sync(kFull, my_q >= 0);
    {
        const long long longest = ex - ax > ey - ay ? ex - ax : ey - ay;
        unsigned s8 = __ballot_sync(kFull, my_q >= 0 && longest <= 8);
        unsigned s16 = __ballot_sync(kFull, my_q >= 0 && longest <= 16) & ~s8;
        if (__popc(s8) < 3) {
            s16 |= s8;
            s8 = 0u;
        }
        if (__popc(s16) < 2) s16 = 0u;
        if (s8) lite_segments<COSINE, 8>(A, s8, ax, ex, ay, ey, have_norms, myD, myNx, myNy);
        if (s16) lite_segments<COSINE, 16>(A, s16, ax, ex, ay, ey, have_norms, myD, myNx, myNy);
        todo &= ~(s8 | s16);
    }
    for (; todo; todo &= todo - 1) {
        const int i = __ffs(todo) - 1;
        const long long a0 = __shfl_sync(kFull, ax, i), a1 = __shfl_sync(kFull, ex, i);
        const long long b0 = __shfl_sync(kFull, ay, i), b1 = __shfl_sync(kFull, ey, i);
        long long D = 0, Nx = 0, Ny = 0;
        lite_exact_one<COSINE>(A, a0, a1 - a0, b0, b1 - b0, have_norms, w_idx, w_val, D, Nx, Ny);
        if (lane == i) {
            myD = D;
            if (!have_norms) {
                myNx = Nx;
                myNy = Ny;
            }
        }
    }
    if (my_q >= 0) {
        const double s = lite_similarity<COSINE>(myD, myNx, myNy, ex - ax, ey - ay);
        A.sim[my_q] = s;
        A.status[my_q] = s > A.t ? BLSH_LITE_ACCEPT : BLSH_LITE_REJECT;
    }
}

// Each row's sum of fixed_term(v, v) (the squared norm of the exact cosine,
// an integer: independent of the order of the terms).  One warp per group of
// 32 consecutive rows: lane l holds the end of row l of the group, the warp
// reads the group's nonzeros 32 at a time (four such reads in flight), finds
// each element's row by a binary search of the lanes' row ends (shuffles),
// sums the terms of each row's run of lanes by a segmented scan, and the
// run's last lane adds the run's sum into the row's 64-bit sum in shared
// memory (one adding lane per row and read, so no two lanes collide).  Formed
// only when there are more survivors than half the rows (the collection pass
// has counted them); otherwise each survivor forms its two norms itself,
// which is less work.
__global__ void __launch_bounds__(256) row_norm2_kernel(const int64_t *__restrict__ indptr,
                                                        const float *__restrict__ values, long long N,
                                                        long long *__restrict__ norm2,
                                                        blsh_dev_scratch *scratch) {
    const bool form = scratch->work3 * 2ull > (unsigned long long)N;
    if (blockIdx.x == 0 && threadIdx.x == 0) scratch->norm2_valid = form ? 1u : 0u;
    if (!form) return;
    __shared__ unsigned long long part[8][32];
    const int lane = threadIdx.x & 31;
    unsigned long long *sum = part[threadIdx.x >> 5];
    const long long groups = (N + 31) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < groups; g += nwarps) {
        const long long r0 = g << 5;
        const int nr = (int)(N - r0 < 32 ? N - r0 : 32);
        const long long s = __ldg(indptr + r0);
        // lanes past the last row repeat its end (the ends stay nondecreasing)
        const long long end = __ldg(indptr + r0 + (lane < nr ? lane + 1 : nr));
        const long long e = __shfl_sync(kFull, end, 31);
        sum[lane] = 0ull;
        __syncwarp();
        for (long long c = s; c < e; c += 128) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = c + 32 * u + lane;
                v[u] = i < e ? __ldg(values + i) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const long long i = c + 32 * u + lane;
                if (c + 32 * u >= e) break;                 // warp-uniform
                int row = 0;                                // rows of the group ending at or before i
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (__shfl_sync(kFull, end, row + step - 1) <= i) row += step;
                unsigned long long term = i < e ? (unsigned long long)fixed_term(v[u], v[u]) : 0ull;
                // inclusive sums over the lanes of the same row (rows are
                // nondecreasing across the lanes)
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long tv = __shfl_up_sync(kFull, term, o);
                    const int tr = __shfl_up_sync(kFull, row, o);
                    if (lane >= o && tr == row) term += tv;
                }
                const int next_row = __shfl_down_sync(kFull, row, 1);
                if (i < e && (lane == 31 || i + 1 == e || next_row != row)) sum[row] += term;
                __syncwarp();
            }
        }
        __syncwarp();
        if (lane < nr) norm2[r0 + lane] = (long long)sum[lane];
        __syncwarp();
    }
}

template <bool COSINE>
__global__ void __launch_bounds__(256) lite_exact_kernel(const LiteArgs A) {
    long long P = A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // per warp: the longer row's indices and values, when it has at most
    // kLiteStage elements (binary searches then run in shared memory), and
    // the survivors of the current tile (offsets within it)
    extern __shared__ uint32_t lite_smem[];
    uint32_t *w_idx = lite_smem + warp * 2 * kLiteStage;
    float *w_val = reinterpret_cast<float *>(w_idx + kLiteStage);
    uint16_t *w_list = reinterpret_cast<uint16_t *>(lite_smem + (blockDim.x >> 5) * 2 * kLiteStage) + warp * 512;
    const bool have_norms = COSINE && A.norm2 && A.scratch->norm2_valid;
    // A warp takes kLiteGrab tiles of 512 statuses per grab of the work
    // counter; a lane reads 16 statuses with one 16-byte load; the tile's
    // survivors are listed in shared memory and computed 32 at a time.
    for (;;) {
        unsigned long long grab = 0;
        if (lane == 0) grab = atomicAdd(&A.scratch->work2, 1ull);
        grab = __shfl_sync(kFull, grab, 0);
        const long long g0 = (long long)grab * kLiteGrab * 512;
        if (g0 >= P) break;
        for (int tt = 0; tt < kLiteGrab; ++tt) {
            const long long q0 = g0 + 512ll * tt;
            if (q0 >= P) break;
            const long long qs = q0 + 16ll * lane;
            uint32_t surv = 0;
            if (A.vec && qs + 16 <= P) {
                surv = blsh_eq16(__ldg(reinterpret_cast<const uint4 *>(A.status + qs)), BLSH_LITE_SURVIVOR);
            } else {
                for (int i = 0; i < 16; ++i)
                    if (qs + i < P && A.status[qs + i] == BLSH_LITE_SURVIVOR) surv |= 1u << i;
            }
            const int c = __popc(surv);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            if (total == 0) continue;
            __syncwarp();                                  // the previous tile's list has been read
            int slot = incl - c;
            for (uint32_t b = surv; b; b &= b - 1) w_list[slot++] = (uint16_t)(16 * lane + __ffs(b) - 1);
            __syncwarp();
            for (int b0 = 0; b0 < total; b0 += 32) {
                const long long q = b0 + lane < total ? q0 + w_list[b0 + lane] : -1;
                lite_batch<COSINE>(A, q, have_norms, w_idx, w_val);
            }
        }
    }
}

// Survivors into a queue (the context's survivor queue, BLSH_LITE_QUEUE_CAP
// entries): warps scan groups of four 512-status tiles in grid-stride order
// and append their survivors' indices with one atomic per group.  Survivors
// beyond the queue are left for lite_exact_kernel.
__global__ void __launch_bounds__(256) lite_collect_kernel(const LiteArgs A, unsigned long long *queue) {
    long long P = A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // four tiles of 512 statuses per warp at a time: their 16-byte loads are
    // in flight together, and one atomic reserves queue slots for all four
    for (long long q0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 2048; q0 < P;
         q0 += nwarps * 2048) {
        uint32_t surv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long qs = q0 + 512ll * t + 16ll * lane;
            surv[t] = 0;
            if (A.vec && qs + 16 <= P) {
                surv[t] = blsh_eq16(__ldg(reinterpret_cast<const uint4 *>(A.status + qs)), BLSH_LITE_SURVIVOR);
            } else {
                for (int i = 0; i < 16; ++i)
                    if (qs + i < P && A.status[qs + i] == BLSH_LITE_SURVIVOR) surv[t] |= 1u << i;
            }
        }
        const unsigned c = __popc(surv[0]) + __popc(surv[1]) + __popc(surv[2]) + __popc(surv[3]);
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const unsigned total = __shfl_sync(kFull, incl, 31);
        if (total == 0) continue;
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(&A.scratch->work3, (unsigned long long)total);
        base = __shfl_sync(kFull, base, 31);
        unsigned long long slot = base + incl - c;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long qs = q0 + 512ll * t + 16ll * lane;
            for (uint32_t b = surv[t]; b; b &= b - 1, ++slot)
                if (slot < BLSH_LITE_QUEUE_CAP) queue[slot] = (unsigned long long)(qs + __ffs(b) - 1);
        }
    }
}

// The queued survivors, one per warp at a time in grid-stride order: the
// survivors of one dense tile (a bucket of near-duplicates) spread over many
// warps.
template <bool COSINE>
__global__ void __launch_bounds__(256) lite_queue_kernel(const LiteArgs A, const unsigned long long *queue) {
    const unsigned long long total = A.scratch->work3;
    const unsigned long long n = total < BLSH_LITE_QUEUE_CAP ? total : BLSH_LITE_QUEUE_CAP;
    extern __shared__ uint32_t lite_smem[];
    const int lane = threadIdx.x & 31;
    uint32_t *w_idx = lite_smem + (threadIdx.x >> 5) * 2 * kLiteStage;
    float *w_val = reinterpret_cast<float *>(w_idx + kLiteStage);
    const bool have_norms = COSINE && A.norm2 && A.scratch->norm2_valid;
    // bs consecutive queue entries per warp at a time (one per lane): 32, or
    // fewer when the survivors are too few to give every warp a full batch
    // (a warp computes its batch's survivors one after the other)
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long bs = (n + nwarps - 1) / nwarps;
    bs = bs < 1 ? 1 : (bs > 32 ? 32 : bs);
    for (unsigned long long base = (((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * bs; base < n;
         base += nwarps * bs) {
        const long long q = lane < bs && base + lane < n ? (long long)queue[base + lane] : -1;
        lite_batch<COSINE>(A, q, have_norms, w_idx, w_val);
    }
}

int lite_exact_pass(blsh_ctx *ctx, const uint2 *pairs, int64_t P, const long long *P_dev, int64_t N,
                    const int64_t *indptr, const uint32_t *indices, const float *values, double t, uint8_t *status,
                    double *sim, cudaStream_t s);

}  // namespace

extern "C" int blsh_verify_lite(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                                const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                                const int64_t *indptr, const uint32_t *indices, const float *values,
                                uint8_t *status, uint16_t *n_used, double *sim, void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    const blsh_params &p = tab->p;
    if (tab->device != ctx->device) return blsh_fail(ctx, BLSH_EINVAL, "tables built on another device");
    if (p.h <= 0) return blsh_fail(ctx, BLSH_EINVAL, "the tables were built with h = 0");
    if (!sig || !indptr || (P > 0 && (!pairs || !status || !sim || !indices)))
        return blsh_fail(ctx, BLSH_EINVAL, "pairs, sig, status, sim, indptr and indices are required");
    if ((p.kind == BLSH_COSINE) != (values != nullptr))
        return blsh_fail(ctx, BLSH_EINVAL, "values must be given for cosine rows and only for them");
    if (P < 0 || N < 0 || N > (1ll << 32)) return blsh_fail(ctx, BLSH_EINVAL, "bad P or N");
    const int need = p.kind == BLSH_JACCARD ? p.h : (p.h + 31) / 32;
    if (sig_words < need || sig_words % 4)
        return blsh_fail(ctx, BLSH_EINVAL, "sig_words must be a multiple of 4 covering h hashes");
    if (!blsh_aligned(sig, 16) || !blsh_aligned(pairs, 8) || !blsh_aligned(sim, 8) || !blsh_aligned(indptr, 8) ||
        !blsh_aligned(n_used, 2) || !blsh_aligned(P_dev, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    VerifyArgs A;
    A.pairs = reinterpret_cast<const uint2 *>(pairs);
    A.P = P;
    A.P_dev = reinterpret_cast<const long long *>(P_dev);
    A.sig = sig;
    A.N = N;
    A.W = sig_words;
    A.k = p.k;
    A.chunk_words = p.kind == BLSH_JACCARD ? p.k : p.k / 32;
    A.levels = p.h / p.k;
    A.lite = 1;
    A.conc_words = tab->conc_words;
    A.est_stride = p.n_max + 1;
    A.min_matches = tab->min_matches;
    A.conc_bits = tab->conc_bits;
    A.conc_lo = tab->conc_lo;
    A.conc_upper = tab->conc_upper ? 1 : 0;
    A.est_tab = tab->est;
    A.status = status;
    A.n_used = n_used;
    A.m_out = nullptr;
    A.est_out = nullptr;
    A.sim_out = sim;
    A.stop_hist = nullptr;
    A.scratch = ctx->scratch;
    A.lite_levels = 0;
    A.lstatus = nullptr;
    A.ln_used = nullptr;
    A.lsim = nullptr;
    A.cap_levels = A.levels;
    A.need = nullptr;
    const blsh_plan plan = blsh_plan_for(ctx, tab);
    A.grab = (plan.grab + 31) / 32 * 32;
    int rc = blsh_launch_verify(ctx, A, plan, s);
    if (rc) return rc;
    if (P == 0) return BLSH_OK;
    return lite_exact_pass(ctx, A.pairs, P, A.P_dev, N, indptr, indices, values, p.t, status, sim, s);
}

namespace {

// Pass 2 of Algorithm 2: the exact similarity of every survivor.
int lite_exact_pass(blsh_ctx *ctx, const uint2 *pairs, int64_t P, const long long *P_dev, int64_t N,
                    const int64_t *indptr, const uint32_t *indices, const float *values, double t, uint8_t *status,
                    double *sim, cudaStream_t s) {
    LiteArgs L;
    L.pairs = pairs;
    L.P = P;
    L.P_dev = P_dev;
    L.indptr = indptr;
    L.indices = indices;
    L.values = values;
    L.t = t;
    L.status = status;
    L.sim = sim;
    L.scratch = ctx->scratch;
    L.vec = blsh_aligned(status, 16);
    L.norm2 = nullptr;
    // the rows' squared norms once per call, in the buffer blsh_ctx_reserve
    // allocated; with more rows than were reserved each survivor forms its
    // two sums itself (no allocation here: this is a hot call)
    if (values && N > 0 && ctx->norm2_cap >= N) L.norm2 = (const long long *)ctx->norm2;
    // survivors: queued (balanced over warps), then any beyond the queue in place
    BLSH_CUDA(ctx, cudaMemsetAsync(&ctx->scratch->work2, 0, 2 * sizeof(unsigned long long), s));   // work2, work3
    unsigned long long *queue = ctx->lite_queue;
    blsh_time_start(ctx, s);
    lite_collect_kernel<<<ctx->sm_count * 8, 256, 0, s>>>(L, queue);
    BLSH_LAUNCHED(ctx, "lite_collect_kernel");
    if (L.norm2) {
        const long long blocks = (N + 255) / 256, cap = (long long)ctx->sm_count * 8;   // 32 rows per warp
        blsh_time_start(ctx, s);
        row_norm2_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(
            indptr, values, N, const_cast<long long *>(L.norm2), ctx->scratch);
        BLSH_LAUNCHED(ctx, "row_norm2_kernel");
    }
    int occ = 0;
    // per warp of the CTA's 8: the staging area (4 KB) and a tile's survivor list (1 KB)
    const size_t smem = 8 * (2 * kLiteStage * sizeof(uint32_t) + 512 * sizeof(uint16_t));
    if (values) {
        BLSH_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lite_queue_kernel<true>, 256, smem));
        blsh_time_start(ctx, s);
        lite_queue_kernel<true><<<(occ > 0 ? occ : 1) * ctx->sm_count, 256, smem, s>>>(L, queue);
        BLSH_LAUNCHED(ctx, "lite_queue_kernel");
        blsh_time_start(ctx, s);
        lite_exact_kernel<true><<<(occ > 0 ? occ : 1) * ctx->sm_count, 256, smem, s>>>(L);
        BLSH_LAUNCHED(ctx, "lite_exact_kernel");
    } else {
        BLSH_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lite_queue_kernel<false>, 256, smem));
        blsh_time_start(ctx, s);
        lite_queue_kernel<false><<<(occ > 0 ? occ : 1) * ctx->sm_count, 256, smem, s>>>(L, queue);
        BLSH_LAUNCHED(ctx, "lite_queue_kernel");
        blsh_time_start(ctx, s);
        lite_exact_kernel<false><<<(occ > 0 ? occ : 1) * ctx->sm_count, 256, smem, s>>>(L);
        BLSH_LAUNCHED(ctx, "lite_exact_kernel");
    }
    return BLSH_OK;
}

}  // namespace

namespace {

int verify_both(blsh_ctx *ctx, const blsh_tables *tab, int32_t hash_limit, const uint32_t *pairs, int64_t P,
                const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words, uint8_t *status,
                uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist, const int64_t *indptr,
                const uint32_t *indices, const float *values, uint8_t *lite_status, uint16_t *lite_n_used,
                double *sim, uint8_t *need, void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    const blsh_params &p = tab->p;
    if (tab->device != ctx->device) return blsh_fail(ctx, BLSH_EINVAL, "tables built on another device");
    if (p.h <= 0) return blsh_fail(ctx, BLSH_EINVAL, "the tables were built with h = 0");
    if (hash_limit % p.k || hash_limit < p.h || hash_limit > p.n_max)
        return blsh_fail(ctx, BLSH_EINVAL, "hash_limit must be a multiple of k in [h, n_max]");
    if (hash_limit < p.n_max && !need) return blsh_fail(ctx, BLSH_EINVAL, "need is required below n_max");
    if (!indptr || (P > 0 && (!lite_status || !sim || !indices)))
        return blsh_fail(ctx, BLSH_EINVAL, "lite_status, sim, indptr and indices are required");
    if ((p.kind == BLSH_COSINE) != (values != nullptr))
        return blsh_fail(ctx, BLSH_EINVAL, "values must be given for cosine rows and only for them");
    if (!blsh_aligned(sim, 8) || !blsh_aligned(indptr, 8) || !blsh_aligned(lite_n_used, 2))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    VerifyArgs A;
    int rc = blsh_make_verify_args(ctx, tab, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est,
                                   stop_hist, A);
    if (rc) return rc;
    A.lite_levels = p.h / p.k;
    A.lstatus = lite_status;
    A.ln_used = lite_n_used;
    A.lsim = sim;
    A.cap_levels = hash_limit / p.k;
    A.need = need;
    const blsh_plan plan = blsh_plan_for(ctx, tab);
    A.grab = (plan.grab + 31) / 32 * 32;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    if (stop_hist) BLSH_CUDA(ctx, cudaMemsetAsync(stop_hist, 0, sizeof(uint64_t) * tab->levels, s));
    rc = blsh_launch_verify(ctx, A, plan, s);
    if (rc) return rc;
    if (P == 0) return BLSH_OK;
    return lite_exact_pass(ctx, A.pairs, P, A.P_dev, N, indptr, indices, values, p.t, lite_status, sim, s);
}

}  // namespace

extern "C" int blsh_verify_both(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                                const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                                uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                                const int64_t *indptr, const uint32_t *indices, const float *values,
                                uint8_t *lite_status, uint16_t *lite_n_used, double *sim, void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    return verify_both(ctx, tab, tab->p.n_max, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est,
                       stop_hist, indptr, indices, values, lite_status, lite_n_used, sim, nullptr, stream);
}

extern "C" int blsh_verify_both_capped(blsh_ctx *ctx, const blsh_tables *tab, int32_t hash_limit,
                                       const uint32_t *pairs, int64_t P, const int64_t *P_dev, const uint32_t *sig,
                                       int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used, uint16_t *m,
                                       float *est, uint64_t *stop_hist, const int64_t *indptr,
                                       const uint32_t *indices, const float *values, uint8_t *lite_status,
                                       uint16_t *lite_n_used, double *sim, uint8_t *need, void *stream) {
    return verify_both(ctx, tab, hash_limit, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est, stop_hist,
                       indptr, indices, values, lite_status, lite_n_used, sim, need, stream);
}
