// verify.cu -- Algorithm 1 (BayesLSH) verification kernel, its launch plans
// and the autotuner.
//
// One pair is owned by a group of G lanes.  A step loads, per lane, U uint4
// (4 words) from each of the two signature rows, so a group moves 16*U*G
// bytes per row per step with coalesced 16-byte loads:
//   - Jaccard: a chunk is k uint32 minhashes; agreements are counted per
//     word and summed across the group with xor-shuffles; a chunk takes
//     k / (4 U G) steps.
//   - Cosine: a chunk is k/32 words of sign bits; one lane owns a pair
//     (G = 1) and one uint4 holds 4*32/k chunks, agreements = 32 - popc(x^y)
//     per word.
// After every chunk the tables (minMatches and the concentration bitmap of
// Section 4.3, staged in shared memory) decide: prune, accept, or go on.
//
// Two launch forms:
//   PLAIN      -- one group per pair, grid covers all pairs; a warp lives as
//                 long as its slowest pair.  For cosine with k = 32 it runs
//                 in two passes: every pair's first four chunks, then the
//                 pairs still open (verify_tile_kernel does both, tile by
//                 tile; verify_first_kernel then verify_kernel's OPEN form
//                 where the outputs take no packed stores).
//   PERSISTENT -- one wave of CTAs; each warp takes `grab` pairs at a time
//                 from an atomic counter and hands a new pair to a group as
//                 soon as its pair stops (pairs stop after very different
//                 chunk counts: most after the first chunk).
#include <type_traits>
#include <vector>

#include "verify.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) { return __ldg(reinterpret_cast<const uint4 *>(p)); }

// Status of a pair Algorithm 1 leaves open after its first four chunks in
// the two-pass form (verify_tile_kernel, or verify_first_kernel then
// verify_kernel with OPEN); internal to one call (every such pair is
// finished, and its status overwritten, before the call returns).  It differs
// from every other status, BLSH_LITE_SURVIVOR (254) included: a Lite
// survivor is decided, not open.
constexpr uint8_t kOpenStatus = 252;
static_assert(kOpenStatus != BLSH_LITE_SURVIVOR && kOpenStatus != BLSH_NEEDS_HASHES && kOpenStatus != BLSH_BAD_PAIR,
              "the open status must differ from every other status");

// Parked pairs per warp (FAST plain form): at most 31 waiting plus the 32 of
// a step.
constexpr int kDefer = 64;
// Byte offset of the parked-pair area in the dynamic shared memory, after the
// three per-level arrays (8-byte aligned).
__host__ __device__ __forceinline__ size_t defer_offset(int levels) {
    return ((size_t)levels * 3 * sizeof(int32_t) + 7) & ~(size_t)7;
}

template <int KIND, int G, int U, bool PERSIST, bool PLANE, bool FAST = false, bool OPEN = false>
__global__ void __launch_bounds__(512) verify_kernel(const VerifyArgs A) {
    // minMatches is staged in shared memory; the concentration bitmap (up to
    // tens of KB, consulted only by pairs that pass the pruning test) is
    // read through L1.
    extern __shared__ __align__(16) unsigned char smem[];
    int32_t *s_mm = reinterpret_cast<int32_t *>(smem);
    unsigned *s_hist = reinterpret_cast<unsigned *>(s_mm + A.levels);
    int32_t *s_clo = reinterpret_cast<int32_t *>(s_hist + A.levels);   // FAST: the concentration thresholds
    // FAST, plain form: each warp's parked pairs (index, pair, agreements)
    long long *s_defq = reinterpret_cast<long long *>(smem + defer_offset(A.levels));
    uint2 *s_defp = reinterpret_cast<uint2 *>(s_defq + (blockDim.x >> 5) * kDefer);
    int *s_defm = reinterpret_cast<int *>(s_defp + (blockDim.x >> 5) * kDefer);
    for (int i = threadIdx.x; i < A.levels; i += blockDim.x) {
        s_mm[i] = A.min_matches[i];
        s_hist[i] = 0;
        if (FAST) s_clo[i] = A.conc_lo[i];
    }
    __syncthreads();
    // FAST: the thresholds of levels 0..3 in registers for every pair's
    // first step (j = 0 for all lanes there)
    int mm0[4], clo0[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        mm0[i] = FAST && i < A.levels ? s_mm[i] : 0;
        clo0[i] = FAST && i < A.levels ? s_clo[i] : 0;
    }

    long long P = A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const int lane = threadIdx.x & 31;
    const int g = lane % G;      // lane within its group
    const int grp = lane / G;    // group within the warp
    constexpr int kWordsPerStep = 4 * U * G;
    const int steps_per_chunk = KIND == BLSH_JACCARD ? A.chunk_words / kWordsPerStep : 1;

    bool active = false, a1 = false, al = false;   // a pair is active while either algorithm is undecided
    long long q = 0;
    uint2 cur_pair = make_uint2(0u, 0u);
    const uint32_t *rx = nullptr, *ry = nullptr;
    int m = 0, j = 0, w = 0, acc = 0, sub = 0;

    auto finish = [&](int st) {
        if (g == 0) {
            A.status[q] = (uint8_t)st;
            if (A.n_used) A.n_used[q] = (uint16_t)((j + 1) * A.k);
            if (A.m_out) A.m_out[q] = (uint16_t)m;
            // the estimate is an output only for pairs that are kept (Algorithm 1);
            // a pruned pair's entry is left as it was
            if (A.est_out && st != BLSH_PRUNED) A.est_out[q] = __ldg(A.est_tab + (size_t)j * A.est_stride + m);
            atomicAdd(&s_hist[j], 1u);
        }
        a1 = false;
        active = al;
    };
    // Algorithm 1 cannot go on without the hashes not yet computed
    auto finish_capped = [&]() {
        if (g == 0) {
            A.status[q] = BLSH_NEEDS_HASHES;
            if (A.n_used) A.n_used[q] = (uint16_t)((j + 1) * A.k);
            if (A.m_out) A.m_out[q] = (uint16_t)m;
            A.need[cur_pair.x] = 1;
            A.need[cur_pair.y] = 1;
        }
        a1 = false;
        active = al;
    };
    // Algorithm 2's verdict when both run in one pass
    auto finish_lite = [&](int st) {
        if (g == 0) {
            A.lstatus[q] = (uint8_t)st;
            if (A.ln_used) A.ln_used[q] = (uint16_t)((j + 1) * A.k);
        }
        al = false;
        active = a1;
    };
    // Chunk j has just been completed with m agreements in n = (j+1) k hashes.
    auto decide = [&]() {
        const bool pruned = m < s_mm[j];                           // Pr[S >= t | M] < eps
        if (a1) {
            if (pruned) {
                finish(BLSH_PRUNED);
            } else if (!A.lite && ((__ldg(A.conc_bits + j * A.conc_words + (m >> 5)) >> (m & 31)) & 1u)) {
                finish(BLSH_ACCEPT);                               // concentrated
            } else if (j + 1 == A.levels) {
                finish(A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX);
            } else if (j + 1 == A.cap_levels) {
                finish_capped();
            }
        }
        if (al) {                                                  // Algorithm 2: the same test, h hashes
            if (pruned) finish_lite(BLSH_PRUNED);
            else if (j + 1 == A.lite_levels) finish_lite(BLSH_LITE_SURVIVOR);
        }
        if (active) ++j;
    };
    auto start_pair = [&](long long qq, unsigned px, unsigned py) {
        q = qq;
        const uint2 pr = make_uint2(px, py);
        if ((long long)pr.x >= A.N || (long long)pr.y >= A.N) {
            if (g == 0) {
                A.status[q] = BLSH_BAD_PAIR;
                if (A.n_used) A.n_used[q] = 0;
                if (A.m_out) A.m_out[q] = 0;
                if (A.lite_levels) {
                    A.lstatus[q] = BLSH_BAD_PAIR;
                    if (A.ln_used) A.ln_used[q] = 0;
                }
                blsh_dev_error(A.scratch, BLSH_ERANGE, 0, 1ull);
            }
            active = a1 = al = false;
            return;
        }
        cur_pair = pr;
        rx = A.sig + (size_t)pr.x * A.W;
        ry = A.sig + (size_t)pr.y * A.W;
        m = 0; j = 0; w = 0; acc = 0; sub = 0;
        active = a1 = true;
        al = A.lite_levels > 0;
    };
    // One step for every group of the warp (all lanes execute it, so the
    // group reductions may use full-warp shuffles).
    // (first: std::true_type for a pair's first step, whose four words come
    // from the plane and whose levels are 0..3)
    auto step = [&](auto first) {
        [[maybe_unused]] constexpr bool kFirst = decltype(first)::value;
        if constexpr (KIND == BLSH_JACCARD) {
            int c = 0;
            if (active) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int off = w + 4 * (u * G + g);
                    const uint4 a = ldg4(rx + off), b = ldg4(ry + off);
                    c += (a.x == b.x) + (a.y == b.y) + (a.z == b.z) + (a.w == b.w);
                }
            }
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
            if (active) {
                w += kWordsPerStep;
                acc += c;
                if (++sub == steps_per_chunk) {
                    m += acc;
                    acc = 0;
                    sub = 0;
                    decide();
                }
            }
        } else {
            int hj = -1;   // the chunk this lane's pair stopped at in this step (for the histogram)
            if (active) {
                // The step's four words (from the rows, or from the plane) are counted and
                // every completed chunk is tested, recording where each
                // algorithm stops and why; the outputs of a stop are written
                // once, after the words.
                int st1 = -1, j1 = 0, m1 = 0, stl = -1, jl = 0;
                auto words = [&](uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, int i0, int i1) {
                    const uint32_t x[4] = {x0, x1, x2, x3};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (i < i0 || i >= i1 || !active) continue;
                        acc += 32 - __popc(x[i]);
                        if (++sub < A.chunk_words) continue;
                        m += acc;
                        acc = 0;
                        sub = 0;
                        const bool pruned = m < s_mm[j];
                        if (a1) {
                            int st = -1;
                            if (pruned) st = BLSH_PRUNED;
                            else if (!A.lite && ((__ldg(A.conc_bits + j * A.conc_words + (m >> 5)) >> (m & 31)) & 1u))
                                st = BLSH_ACCEPT;
                            else if (j + 1 == A.levels) st = A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX;
                            else if (j + 1 == A.cap_levels) st = BLSH_NEEDS_HASHES;
                            if (st >= 0) {
                                st1 = st;
                                j1 = j;
                                m1 = m;
                                a1 = false;
                            }
                        }
                        if (al) {
                            if (pruned || j + 1 == A.lite_levels) {
                                stl = pruned ? BLSH_PRUNED : BLSH_LITE_SURVIVOR;
                                jl = j;
                                al = false;
                            }
                        }
                        active = a1 || al;
                        if (active) ++j;
                    }
                };
                // k = 32 with upper-range concentration sets: the step's four
                // chunks are tested together, without branches, and the first
                // chunk at which each algorithm stops is found by bit scans (the
                // tests and their order are those of the chunk-by-chunk loop)
                auto fast = [&](uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3) {
                    if (kFirst) j = 0, m = 0;
                    const int c0 = m + 32 - __popc(x0), c1 = c0 + 32 - __popc(x1);
                    const int c2 = c1 + 32 - __popc(x2), c3 = c2 + 32 - __popc(x3);
                    // m after chunk i of the four (selected without a dynamic index,
                    // which would put an array in local memory)
                    auto m_at = [&](int i) { return i == 0 ? c0 : i == 1 ? c1 : i == 2 ? c2 : c3; };
                    unsigned valid = 0, prune = 0, conc = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int jj = j + i;
                        if (jj < A.levels) {
                            valid |= 1u << i;
                            prune |= (unsigned)(m_at(i) < (kFirst ? mm0[i] : s_mm[jj])) << i;
                            conc |= (unsigned)(m_at(i) >= (kFirst ? clo0[i] : s_clo[jj])) << i;
                        }
                    }
                    // the bit of the chunk after which a level limit is reached
                    auto at = [&](int lim) { const int d = lim - 1 - j; return d >= 0 && d < 4 ? 1u << d : 0u; };
                    const unsigned last = at(A.levels), cap = at(A.cap_levels), lite_last = at(A.lite_levels);
                    if (a1) {
                        const unsigned s1 = (prune | (A.lite ? 0u : conc) | last | cap) & valid;
                        if (s1) {
                            const int i = __ffs(s1) - 1;
                            const unsigned b = 1u << i;
                            st1 = (prune & b) ? BLSH_PRUNED
                                  : (!A.lite && (conc & b)) ? BLSH_ACCEPT
                                  : (last & b) ? (A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX)
                                               : BLSH_NEEDS_HASHES;
                            j1 = j + i;
                            m1 = m_at(i);
                            a1 = false;
                        }
                    }
                    if (al) {
                        const unsigned sl = (prune | lite_last) & valid;
                        if (sl) {
                            const int i = __ffs(sl) - 1;
                            stl = (prune >> i) & 1u ? BLSH_PRUNED : BLSH_LITE_SURVIVOR;
                            jl = j + i;
                            al = false;
                        }
                    }
                    active = a1 || al;
                    if (active) {   // all four chunks passed: none was the last level
                        m = c3;
                        j += 4;
                    }
                };
                uint4 a, b;
                if (PLANE && (kFirst || w == 0)) {   // the first four words from the plane (L2-resident)
                    a = __ldg(A.plane + cur_pair.x);
                    b = __ldg(A.plane + cur_pair.y);
                } else {
                    a = ldg4(rx + w);
                    b = ldg4(ry + w);
                }
                if constexpr (FAST) fast(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w);
                else words(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w, 0, 4);
                w += 4;
                if (st1 >= 0 && g == 0) {
                    A.status[q] = (uint8_t)st1;
                    if (A.n_used) A.n_used[q] = (uint16_t)((j1 + 1) * A.k);
                    if (A.m_out) A.m_out[q] = (uint16_t)m1;
                    if (st1 == BLSH_NEEDS_HASHES) {   // Algorithm 1 needs hashes not yet computed
                        A.need[cur_pair.x] = 1;
                        A.need[cur_pair.y] = 1;
                    } else {
                        // the estimate is an output only for pairs that are kept
                        if (A.est_out && st1 != BLSH_PRUNED)
                            A.est_out[q] = __ldg(A.est_tab + (size_t)j1 * A.est_stride + m1);
                        hj = j1;
                    }
                }
                if (stl >= 0 && g == 0) {
                    A.lstatus[q] = (uint8_t)stl;
                    if (A.ln_used) A.ln_used[q] = (uint16_t)((jl + 1) * A.k);
                }
            }
            // the stop histogram: the stops at levels 0..3 (most pairs) by
            // one ballot per level, lane c adding level c's count (four
            // different addresses: one atomic instruction, no collision);
            // later levels one atomic per lane (every lane runs this)
            unsigned mine = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const unsigned z = __ballot_sync(kFull, hj == c);
                if (lane == c) mine = (unsigned)__popc(z);
            }
            if (mine) atomicAdd(&s_hist[lane], mine);
            if (hj >= 4) atomicAdd(&s_hist[hj], 1u);
        }
    };

    if constexpr (PERSIST) {
        // Pair indices reach the lanes through two 32-entry register buffers
        // per warp: lane l holds entry l of the current block of 32 pairs and
        // of the next one, which is loaded (coalesced) as soon as the current
        // block is opened, so a pair's indices are on chip when a group needs
        // them.  Blocks come from ranges of `grab` pairs (a multiple of 32)
        // taken from the work counter.
        const unsigned lower = (1u << (grp * G)) - 1u;   // lanes of lower groups
        unsigned long long gcur = 0, gend = 0;
        bool no_more = false;
        // next block of 32 pair indices from the warp's range: base, valid count
        auto next_block = [&](unsigned long long &base, int &valid) {
            valid = 0;
            if (gcur >= gend && !no_more) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(&A.scratch->work, (unsigned long long)A.grab);
                b = __shfl_sync(kFull, b, 0);
                if (b >= (unsigned long long)P) {
                    no_more = true;
                } else {
                    gcur = b;
                    gend = b + A.grab < (unsigned long long)P ? b + A.grab : (unsigned long long)P;
                }
            }
            if (gcur < gend) {
                base = gcur;
                valid = (int)(gend - gcur < 32ull ? gend - gcur : 32ull);
                gcur += valid;
            }
        };
        unsigned long long cbase = 0, nbase = 0;
        int cvalid = 0, nvalid = 0, cpos = 0;
        uint2 cur = make_uint2(0u, 0u), nxt = make_uint2(0u, 0u);
        next_block(cbase, cvalid);
        if (lane < cvalid) cur = __ldg(A.pairs + cbase + lane);
        next_block(nbase, nvalid);
        if (lane < nvalid) nxt = __ldg(A.pairs + nbase + lane);
        for (;;) {
            for (;;) {
                const bool need = !active;
                const unsigned need_mask = __ballot_sync(kFull, need && g == 0);
                if (need_mask == 0) break;
                if (cpos == cvalid) {
                    if (nvalid == 0) break;   // nothing left anywhere
                    cur = nxt;
                    cbase = nbase;
                    cvalid = nvalid;
                    cpos = 0;
                    next_block(nbase, nvalid);
                    if (lane < nvalid) nxt = __ldg(A.pairs + nbase + lane);
                }
                const int avail = cvalid - cpos;
                const int rank = __popc(need_mask & lower);
                const int src = (cpos + rank) & 31;
                const unsigned px = __shfl_sync(kFull, cur.x, src);
                const unsigned py = __shfl_sync(kFull, cur.y, src);
                if (need && rank < avail) start_pair((long long)(cbase + cpos + rank), px, py);
                const int want = __popc(need_mask);
                cpos += want < avail ? want : avail;
            }
            if (!__any_sync(kFull, active)) break;
            step(std::false_type{});
        }
    } else {
        // a fixed share of the pairs per warp: blocks of 32 / G pairs in
        // grid-stride order; a warp moves to its next block when the
        // slowest pair of the current one has stopped
        // (the next block's pair indices are loaded before the current
        // block is worked on)
        const long long per_warp = 32 / G;
        const long long stride = (((long long)gridDim.x * blockDim.x) >> 5) * per_warp;
        long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * per_warp;
        uint2 nxt = make_uint2(0u, 0u);
        if (base + grp < P) nxt = __ldg(A.pairs + base + grp);
        if constexpr (OPEN) {
            // Second pass of the two-pass form: the pairs the first pass left
            // at kOpenStatus.  A warp scans tiles of 512 statuses (16 per
            // lane), lists the open ones in its part of shared memory, and
            // runs them 32 at a time, each from its first step (which repeats
            // the first pass's arithmetic and leaves the pair open) to its stop.
            uint16_t *w_list = reinterpret_cast<uint16_t *>(smem + defer_offset(A.levels)) + (threadIdx.x >> 5) * 512;
            const bool vec = ((uintptr_t)A.status & 15) == 0;
            // tiles from a counter (open pairs cluster where near-duplicate
            // groups put many similar pairs together)
            for (;;) {
                unsigned long long tg = 0;
                if (lane == 0) tg = atomicAdd(&A.scratch->work, 1ull);
                const long long g0 = (long long)__shfl_sync(kFull, tg, 0) * 2048;   // four tiles per grab
                if (g0 >= P) break;
                for (long long t0 = g0; t0 < g0 + 2048 && t0 < P; t0 += 512) {
                    const long long qs = t0 + 16ll * lane;
                    uint32_t open = 0;
                    if (vec && qs + 16 <= P) {
                        open = blsh_eq16(*reinterpret_cast<const uint4 *>(A.status + qs), kOpenStatus);
                    } else {
                        for (int i = 0; i < 16; ++i)
                            if (qs + i < P && A.status[qs + i] == kOpenStatus) open |= 1u << i;
                    }
                    const int c = __popc(open);
                    int incl = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int y = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int total = __shfl_sync(kFull, incl, 31);
                    if (total == 0) continue;
                    __syncwarp();                                  // the previous tile's list has been read
                    int slot = incl - c;
                    for (uint32_t bits = open; bits; bits &= bits - 1) w_list[slot++] = (uint16_t)(16 * lane + __ffs(bits) - 1);
                    __syncwarp();
                    for (int b0 = 0; b0 < total; b0 += 32) {
                        if (b0 + lane < total) {
                            const long long qq = t0 + w_list[b0 + lane];
                            const uint2 pr = __ldg(A.pairs + qq);
                            start_pair(qq, pr.x, pr.y);
                            al = false;                            // Algorithm 2 was decided in the first pass
                        }
                        if (__any_sync(kFull, active)) step(std::true_type{});
                        while (__any_sync(kFull, active)) step(std::false_type{});
                    }
                }
            }
        } else if constexpr (FAST) {
            // Most pairs stop within their first step (the four chunks of the
            // plane), but a warp would otherwise run its later steps for the
            // few that do not, with the other lanes idle.  Pairs Algorithm 1
            // leaves open after the first step (Algorithm 2 decided: h <= 128)
            // are parked in the warp's part of shared memory with their
            // agreements so far, and continued 32 at a time, every lane busy.
            // (Each pair goes through the same chunks and tests, so the outputs
            // are those of the chunk-by-chunk loop.)
            const int wib = threadIdx.x >> 5;
            long long *dq = s_defq + wib * kDefer;
            uint2 *dp = s_defp + wib * kDefer;
            int *dm = s_defm + wib * kDefer;
            int cnt = 0;
            auto drain = [&](int n) {   // the last n (<= 32) parked pairs, one per lane
                __syncwarp();
                if (lane < n) {
                    const int e = cnt - n + lane;
                    q = dq[e];
                    cur_pair = dp[e];
                    m = dm[e];
                    rx = A.sig + (size_t)cur_pair.x * A.W;
                    ry = A.sig + (size_t)cur_pair.y * A.W;
                    j = 4;
                    w = 4;
                    acc = 0;
                    sub = 0;
                    a1 = active = true;
                    al = false;
                } else {
                    a1 = al = active = false;
                }
                __syncwarp();
                cnt -= n;
                while (__any_sync(kFull, active)) step(std::false_type{});
            };
            for (; base < P; base += stride) {
                const uint2 pr = nxt;
                const long long qq = base + grp;
                if (base + stride + grp < P) nxt = __ldg(A.pairs + base + stride + grp);
                if (qq < P) start_pair(qq, pr.x, pr.y);
                if (__any_sync(kFull, active)) step(std::true_type{});   // the first four chunks
                const bool park = active && a1 && !al;
                const unsigned pmask = __ballot_sync(kFull, park);
                if (pmask) {
                    if (park) {
                        const int e = cnt + __popc(pmask & ((1u << lane) - 1u));
                        dq[e] = q;
                        dp[e] = cur_pair;
                        dm[e] = m;
                        a1 = active = false;
                    }
                    cnt += __popc(pmask);
                }
                while (__any_sync(kFull, active)) step(std::false_type{});   // pairs Algorithm 2 still holds open
                if (cnt >= 32) drain(32);
            }
            while (cnt > 0) drain(cnt < 32 ? cnt : 32);
        } else {
            for (; base < P; base += stride) {
                const uint2 pr = nxt;
                const long long qq = base + grp;
                if (base + stride + grp < P) nxt = __ldg(A.pairs + base + stride + grp);
                if (qq < P) start_pair(qq, pr.x, pr.y);
                while (__any_sync(kFull, active)) step(std::false_type{});
            }
        }
    }

    __syncthreads();
    if (A.stop_hist)
        for (int i = threadIdx.x; i < A.levels; i += blockDim.x)
            if (s_hist[i]) atomicAdd(A.stop_hist + i, (unsigned long long)s_hist[i]);
}

// Two-pass form, first pass (cosine, k = 32, upper-range concentration sets,
// Algorithm 2 over at most four chunks): one lane per pair, nothing but the
// pair's first four chunks (the plane's 16 bytes, or the rows' first 16)
// and the tests of levels 0..3 with their thresholds in registers -- the
// decisions of verify_kernel's first step, in the same order.  A pair that
// stops gets its outputs; a pair Algorithm 1 leaves open is marked
// kOpenStatus for the second pass (verify_kernel with OPEN).  A lane takes
// two pairs at a time, so that their loads overlap.  Each lane counts its
// stops per level in registers; the warp adds them once at the end.
template <bool PLANE>
__global__ void __launch_bounds__(256) verify_first_kernel(const VerifyArgs A) {
    __shared__ unsigned s_h[4];
    if (threadIdx.x < 4) s_h[threadIdx.x] = 0;
    int mm[4], clo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        mm[i] = i < A.levels ? __ldg(A.min_matches + i) : 0;
        clo[i] = i < A.levels ? __ldg(A.conc_lo + i) : 0;
    }
    __syncthreads();
    long long P = A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const unsigned valid = A.levels >= 4 ? 0xfu : (1u << A.levels) - 1u;
    // the bit of the chunk after which a level limit is reached
    auto at = [](int lim) { const int d = lim - 1; return d >= 0 && d < 4 ? 1u << d : 0u; };
    const unsigned last = at(A.levels), cap = at(A.cap_levels), lite_last = at(A.lite_levels);
    const int lane = threadIdx.x & 31;
    // a pair's decisions and outputs, given its first four words; returns the
    // level it stops at for the histogram (-1: none counted)
    auto decide = [&](long long q, uint2 pr, uint4 a, uint4 b) -> int {
        const int c0 = 32 - __popc(a.x ^ b.x), c1 = c0 + 32 - __popc(a.y ^ b.y);
        const int c2 = c1 + 32 - __popc(a.z ^ b.z), c3 = c2 + 32 - __popc(a.w ^ b.w);
        auto m_at = [&](int i) { return i == 0 ? c0 : i == 1 ? c1 : i == 2 ? c2 : c3; };
        unsigned prune = 0, conc = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            prune |= (unsigned)(m_at(i) < mm[i]) << i;
            conc |= (unsigned)(m_at(i) >= clo[i]) << i;
        }
        prune &= valid;
        conc &= valid;
        int hj = -1;
        const unsigned s1 = prune | (A.lite ? 0u : conc) | ((last | cap) & valid);
        if (s1) {
            const int i = __ffs(s1) - 1;
            const unsigned bi = 1u << i;
            const int st1 = (prune & bi) ? BLSH_PRUNED
                            : (!A.lite && (conc & bi)) ? BLSH_ACCEPT
                            : (last & bi) ? (A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX)
                                          : BLSH_NEEDS_HASHES;
            const int m1 = m_at(i);
            A.status[q] = (uint8_t)st1;
            if (A.n_used) A.n_used[q] = (uint16_t)((i + 1) * A.k);
            if (A.m_out) A.m_out[q] = (uint16_t)m1;
            if (st1 == BLSH_NEEDS_HASHES) {
                A.need[pr.x] = 1;
                A.need[pr.y] = 1;
            } else {
                if (A.est_out && st1 != BLSH_PRUNED) A.est_out[q] = __ldg(A.est_tab + (size_t)i * A.est_stride + m1);
                hj = i;
            }
        } else {
            A.status[q] = kOpenStatus;
        }
        if (A.lite_levels) {
            const unsigned sl = prune | (lite_last & valid);
            const int i = __ffs(sl) - 1;   // Algorithm 2 stops within these four chunks
            A.lstatus[q] = (prune >> i) & 1u ? BLSH_PRUNED : BLSH_LITE_SURVIVOR;
            if (A.ln_used) A.ln_used[q] = (uint16_t)((i + 1) * A.k);
        }
        return hj;
    };
    auto bad_pair = [&](long long q) {
        A.status[q] = BLSH_BAD_PAIR;
        if (A.n_used) A.n_used[q] = 0;
        if (A.m_out) A.m_out[q] = 0;
        if (A.lite_levels) {
            A.lstatus[q] = BLSH_BAD_PAIR;
            if (A.ln_used) A.ln_used[q] = 0;
        }
        blsh_dev_error(A.scratch, BLSH_ERANGE, 0, 1ull);
    };
    auto row = [&](uint32_t o) { return PLANE ? __ldg(A.plane + o) : ldg4(A.sig + (size_t)o * A.W); };
    unsigned hc0 = 0, hc1 = 0, hc2 = 0, hc3 = 0;   // this lane's stops at levels 0..3
    // two pairs per lane at a time (pairs q and q + stride): both pairs'
    // loads are in flight before either is decided
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < P; base += 2 * stride) {
        const long long qa = base + lane, qb = base + stride + lane;
        uint2 pa = make_uint2(0u, 0u), pb = make_uint2(0u, 0u);
        if (qa < P) pa = __ldg(A.pairs + qa);
        if (qb < P) pb = __ldg(A.pairs + qb);
        const bool oka = qa < P && (long long)pa.x < A.N && (long long)pa.y < A.N;
        const bool okb = qb < P && (long long)pb.x < A.N && (long long)pb.y < A.N;
        uint4 xa = make_uint4(0u, 0u, 0u, 0u), ya = xa, xb = xa, yb = xa;
        if (oka) {
            xa = row(pa.x);
            ya = row(pa.y);
        }
        if (okb) {
            xb = row(pb.x);
            yb = row(pb.y);
        }
        int ha = -1, hb = -1;
        if (oka) ha = decide(qa, pa, xa, ya);
        else if (qa < P) bad_pair(qa);
        if (okb) hb = decide(qb, pb, xb, yb);
        else if (qb < P) bad_pair(qb);
        hc0 += (ha == 0) + (hb == 0);
        hc1 += (ha == 1) + (hb == 1);
        hc2 += (ha == 2) + (hb == 2);
        hc3 += (ha == 3) + (hb == 3);
    }
    {
        const unsigned c0 = __reduce_add_sync(kFull, hc0), c1 = __reduce_add_sync(kFull, hc1);
        const unsigned c2 = __reduce_add_sync(kFull, hc2), c3 = __reduce_add_sync(kFull, hc3);
        const unsigned mine = lane == 0 ? c0 : lane == 1 ? c1 : lane == 2 ? c2 : lane == 3 ? c3 : 0u;
        if (mine) atomicAdd(&s_h[lane], mine);
    }
    __syncthreads();
    if (A.stop_hist && threadIdx.x < 4 && s_h[threadIdx.x])
        atomicAdd(A.stop_hist + threadIdx.x, (unsigned long long)s_h[threadIdx.x]);
}

// The first pass's tests on packed counts.  With k = 32 the cumulative
// disagreements after chunk i are D_i = 32(i+1) - m_i <= 128; the four levels
// sit in two words, level 2w in the low and level 2w+1 in the high half of
// word w, and each of Algorithm 1's tests is an add in every half whose bit 15
// gives the answer (no carry leaves a half: every half stays below 2^16):
//   prune_i  m_i <  mm_i   <=>  D_i >  32(i+1) - mm_i  =: dmax_i   (D_i + 0x7fff - dmax_i >= 0x8000)
//   conc_i   m_i >= clo_i  <=>  D_i <  32(i+1) - clo_i + 1 =: e_i  (0x7fff + e_i - D_i >= 0x8000)
// with dmax_i clamped to [-1, 0x7fff] and e_i to [0, 0x7fff]: a level beyond
// the table's (or, in Algorithm 2, every level's concentration test) gets the
// constant that never fires.
struct FirstConsts {
    unsigned kp[2];      // halves 0x7fff - dmax_i
    unsigned ec[2];      // halves 0x7fff + e_i
    unsigned stop[2];    // bit 15 of a half: the level limit or the hash cap is reached there
    unsigned last[2];    // bit 15: the level limit
    unsigned llast[2];   // bit 15: Algorithm 2's level limit
    int lastcode;        // status of a pair reaching the level limit undecided
};

// One pair's first-pass decisions: st (kOpenStatus when Algorithm 1 goes on
// past the fourth chunk), the level i it stops at and its agreements m
// there; Algorithm 2's status ls and level il.
struct FirstOut {
    int st, i, m, ls, il;
    int m4;   // agreements after chunk 3 (where Algorithm 1 goes on from an open pair)
};

__device__ __forceinline__ FirstConsts first_consts(const VerifyArgs &A) {
    auto at = [](int lim) { const int d = lim - 1; return d >= 0 && d < 4 ? 1u << d : 0u; };
    const unsigned valid = A.levels >= 4 ? 0xfu : (1u << A.levels) - 1u;
    const unsigned last = at(A.levels) & valid, stop = (at(A.levels) | at(A.cap_levels)) & valid;
    const unsigned llast = at(A.lite_levels) & valid;
    FirstConsts c = {};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int w = i >> 1, h = (i & 1) * 16;
        long long dmax = 0x7fff, e = 0;
        if (i < A.levels) {
            dmax = 32ll * (i + 1) - __ldg(A.min_matches + i);
            dmax = dmax < -1 ? -1 : dmax > 0x7fff ? 0x7fff : dmax;
            if (!A.lite) {
                e = 32ll * (i + 1) - __ldg(A.conc_lo + i) + 1;
                e = e < 0 ? 0 : e > 0x7fff ? 0x7fff : e;
            }
        }
        c.kp[w] |= (unsigned)(0x7fff - dmax) << h;
        c.ec[w] |= (unsigned)(0x7fff + e) << h;
        const unsigned bit = 0x8000u << h;
        if ((stop >> i) & 1u) c.stop[w] |= bit;
        if ((last >> i) & 1u) c.last[w] |= bit;
        if ((llast >> i) & 1u) c.llast[w] |= bit;
    }
    c.lastcode = A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX;
    return c;
}

__device__ __forceinline__ FirstOut first_decide(const FirstConsts &c, uint4 a, uint4 b) {
    constexpr unsigned M = 0x80008000u;
    const unsigned d0 = __popc(a.x ^ b.x), d1 = __popc(a.y ^ b.y), d2 = __popc(a.z ^ b.z), d3 = __popc(a.w ^ b.w);
    const unsigned e1 = d0 + d1, e2 = e1 + d2;
    const unsigned w0 = d0 | e1 << 16, w1 = e2 | (e2 + d3) << 16;   // D_0 | D_1, D_2 | D_3
    const unsigned p0 = (w0 + c.kp[0]) & M, p1 = (w1 + c.kp[1]) & M;
    const unsigned q0 = (c.ec[0] - w0) & M, q1 = (c.ec[1] - w1) & M;
    const unsigned s0 = p0 | q0 | c.stop[0], s1 = p1 | q1 | c.stop[1];
    FirstOut o;
    o.st = kOpenStatus;
    o.i = 0;
    o.m = 0;
    o.m4 = 128 - (int)(w1 >> 16);
    if (s0 | s1) {   // the first level with a decision (or the limit)
        const bool lo = s0 != 0;
        const unsigned s = lo ? s0 : s1, w = lo ? w0 : w1, p = lo ? p0 : p1, q = lo ? q0 : q1;
        const unsigned l = lo ? c.last[0] : c.last[1];
        const int h = (s & 0x8000u) ? 0 : 16;
        o.i = (lo ? 0 : 2) + (h >> 4);
        o.m = 32 * (o.i + 1) - (int)((w >> h) & 0xffffu);
        o.st = ((p >> h) & 0x8000u)   ? BLSH_PRUNED
               : ((q >> h) & 0x8000u) ? BLSH_ACCEPT
               : ((l >> h) & 0x8000u) ? c.lastcode
                                      : BLSH_NEEDS_HASHES;
    }
    // Algorithm 2 (fused): its first prune, else its level limit
    const unsigned t0 = p0 | c.llast[0], t1 = p1 | c.llast[1];
    const bool lo2 = t0 != 0;
    const unsigned t = lo2 ? t0 : t1, pp = lo2 ? p0 : p1;
    const int h2 = (t & 0x8000u) ? 0 : 16;
    o.il = (lo2 ? 0 : 2) + (h2 >> 4);
    o.ls = ((pp >> h2) & 0x8000u) ? BLSH_PRUNED : BLSH_LITE_SURVIVOR;
    return o;
}

// The two passes in one kernel, where every output array takes packed
// four-pair stores and P < 2^31.  A warp takes tiles of kTilePairs
// consecutive pairs from a counter.  It runs the first pass over its tile
// four pairs a lane (their indices in two 16-byte loads, their eight rows
// gathered before any is decided, one store per output array for the four:
// 4 statuses in a word, 4 counts in 8 bytes; the decisions of
// verify_first_kernel, taken by first_decide), four quads a lane, and keeps
// the pairs Algorithm 1 leaves open after four chunks in its part of shared
// memory (the pair's offset in the tile and its agreements so far); then it
// continues them 32 at a time, a lane each, from chunk 4 on, with the tests
// of verify_kernel's step (four chunks a step, thresholds in shared memory)
// until each stops.  The open pairs' outputs land in the sectors the first
// pass wrote a moment before, still in L2; a second kernel would scan every
// status again and read each such sector back from DRAM to change a few
// bytes of it.
constexpr int kTilePairs = 512;

template <bool PLANE>
__global__ void __launch_bounds__(256) verify_tile_kernel(const VerifyArgs A) {
    extern __shared__ int32_t s_tab[];
    // minMatches and the concentration bounds of every level, the stop
    // histogram, then each warp's open list: (offset in the tile) | m << 16
    int32_t *s_mm = s_tab, *s_clo = s_tab + A.levels;
    unsigned *s_hist = reinterpret_cast<unsigned *>(s_tab + 2 * A.levels);
    uint32_t *s_open = reinterpret_cast<uint32_t *>(s_tab + 3 * A.levels) + (threadIdx.x >> 5) * kTilePairs;
    for (int i = threadIdx.x; i < A.levels; i += blockDim.x) {
        s_mm[i] = __ldg(A.min_matches + i);
        s_clo[i] = __ldg(A.conc_lo + i);
        s_hist[i] = 0;
    }
    const FirstConsts c = first_consts(A);
    __syncthreads();
    unsigned P = (unsigned)A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0u : (pd < A.P ? (unsigned)pd : P);
    }
    const unsigned long long N = (unsigned long long)A.N;
    const int k = A.k, lane = threadIdx.x & 31;
    auto row = [&](uint32_t o) { return PLANE ? __ldg(A.plane + o) : ldg4(A.sig + (size_t)o * A.W); };
    // stops at levels 0..3 in 16-bit fields, added into hc every 8192 quads
    unsigned h01 = 0, h23 = 0, hc0 = 0, hc1 = 0, hc2 = 0, hc3 = 0, iters = 0;
    auto count = [&](const FirstOut &o) {
        if (o.st != kOpenStatus && o.st != BLSH_NEEDS_HASHES) {
            if (o.i < 2) h01 += 1u << (o.i << 4);
            else h23 += 1u << ((o.i - 2) << 4);
        }
    };
    auto flush = [&]() {
        hc0 += h01 & 0xffffu;
        hc1 += h01 >> 16;
        hc2 += h23 & 0xffffu;
        hc3 += h23 >> 16;
        h01 = h23 = 0;
    };
    auto side = [&](unsigned q, const FirstOut &o, unsigned x, unsigned y) {
        if (o.st == BLSH_NEEDS_HASHES) {
            A.need[x] = 1;
            A.need[y] = 1;
        } else if (A.est_out && o.st != kOpenStatus && o.st != BLSH_PRUNED) {
            A.est_out[q] = __ldg(A.est_tab + o.i * A.est_stride + o.m);
        }
    };
    // one pair by itself (a tail, or a quad naming an object >= N); returns
    // whether it is open
    auto one = [&](unsigned q, uint2 pr, int &m4) -> bool {
        if ((unsigned long long)pr.x < N && (unsigned long long)pr.y < N) {
            const FirstOut o = first_decide(c, row(pr.x), row(pr.y));
            A.status[q] = (uint8_t)o.st;
            if (o.st != kOpenStatus) {
                if (A.n_used) A.n_used[q] = (uint16_t)((o.i + 1) * k);
                if (A.m_out) A.m_out[q] = (uint16_t)o.m;
            }
            if (A.lite_levels) {
                A.lstatus[q] = (uint8_t)o.ls;
                if (A.ln_used) A.ln_used[q] = (uint16_t)((o.il + 1) * k);
            }
            side(q, o, pr.x, pr.y);
            count(o);
            m4 = o.m4;
            return o.st == kOpenStatus;
        }
        A.status[q] = BLSH_BAD_PAIR;
        if (A.n_used) A.n_used[q] = 0;
        if (A.m_out) A.m_out[q] = 0;
        if (A.lite_levels) {
            A.lstatus[q] = BLSH_BAD_PAIR;
            if (A.ln_used) A.ln_used[q] = 0;
        }
        blsh_dev_error(A.scratch, BLSH_ERANGE, 0, 1ull);
        return false;
    };
    auto at = [](int lim, int j) { const int d = lim - 1 - j; return d >= 0 && d < 4 ? 1u << d : 0u; };
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&A.scratch->work, 1ull);
        t = __shfl_sync(kFull, t, 0);
        if (t * kTilePairs >= P) break;
        const unsigned base = (unsigned)t * kTilePairs;
        int n_open = 0;   // the warp's open pairs in this tile so far
        __syncwarp();     // the previous tile's list has been read
#pragma unroll 1
        for (int r = 0; r < kTilePairs / 128; ++r) {
            const unsigned q = base + 128u * r + 4u * lane;
            unsigned om = 0;   // which of the lane's four pairs are open
            int m4[4] = {0, 0, 0, 0};
            if (q + 4 <= P) {
                const uint4 *pp = reinterpret_cast<const uint4 *>(A.pairs) + (q >> 1);
                const uint4 u = __ldcs(pp), v = __ldcs(pp + 1);
                const unsigned mx = max(max(max(u.x, u.y), max(u.z, u.w)), max(max(v.x, v.y), max(v.z, v.w)));
                if ((unsigned long long)mx < N) {
                    const uint4 a0 = row(u.x), b0 = row(u.y), a1 = row(u.z), b1 = row(u.w);
                    const uint4 a2 = row(v.x), b2 = row(v.y), a3 = row(v.z), b3 = row(v.w);
                    const FirstOut o0 = first_decide(c, a0, b0), o1 = first_decide(c, a1, b1);
                    const FirstOut o2 = first_decide(c, a2, b2), o3 = first_decide(c, a3, b3);
                    const unsigned g = q >> 2;
                    reinterpret_cast<unsigned *>(A.status)[g] =
                        (unsigned)o0.st | (unsigned)o1.st << 8 | (unsigned)o2.st << 16 | (unsigned)o3.st << 24;
                    if (A.n_used)
                        reinterpret_cast<uint2 *>(A.n_used)[g] =
                            make_uint2((unsigned)((o0.i + 1) * k) | (unsigned)((o1.i + 1) * k) << 16,
                                       (unsigned)((o2.i + 1) * k) | (unsigned)((o3.i + 1) * k) << 16);
                    if (A.m_out)
                        reinterpret_cast<uint2 *>(A.m_out)[g] =
                            make_uint2((unsigned)o0.m | (unsigned)o1.m << 16, (unsigned)o2.m | (unsigned)o3.m << 16);
                    if (A.lite_levels) {
                        reinterpret_cast<unsigned *>(A.lstatus)[g] =
                            (unsigned)o0.ls | (unsigned)o1.ls << 8 | (unsigned)o2.ls << 16 | (unsigned)o3.ls << 24;
                        if (A.ln_used)
                            reinterpret_cast<uint2 *>(A.ln_used)[g] =
                                make_uint2((unsigned)((o0.il + 1) * k) | (unsigned)((o1.il + 1) * k) << 16,
                                           (unsigned)((o2.il + 1) * k) | (unsigned)((o3.il + 1) * k) << 16);
                    }
                    side(q, o0, u.x, u.y);
                    side(q + 1, o1, u.z, u.w);
                    side(q + 2, o2, v.x, v.y);
                    side(q + 3, o3, v.z, v.w);
                    count(o0);
                    count(o1);
                    count(o2);
                    count(o3);
                    om = (unsigned)(o0.st == kOpenStatus) | (unsigned)(o1.st == kOpenStatus) << 1 |
                         (unsigned)(o2.st == kOpenStatus) << 2 | (unsigned)(o3.st == kOpenStatus) << 3;
                    m4[0] = o0.m4;
                    m4[1] = o1.m4;
                    m4[2] = o2.m4;
                    m4[3] = o3.m4;
                } else {
                    om = (unsigned)one(q, make_uint2(u.x, u.y), m4[0]) | (unsigned)one(q + 1, make_uint2(u.z, u.w), m4[1]) << 1 |
                         (unsigned)one(q + 2, make_uint2(v.x, v.y), m4[2]) << 2 |
                         (unsigned)one(q + 3, make_uint2(v.z, v.w), m4[3]) << 3;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (q + i < P) om |= (unsigned)one(q + i, __ldg(A.pairs + q + i), m4[i]) << i;
            }
            // the open pairs into the warp's list, in lane order
            const int cnt = __popc(om);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            int slot = n_open + incl - cnt;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((om >> i) & 1u) {
                    if (slot < kTilePairs && q + i - base < kTilePairs) s_open[slot] = (q + i - base) | (uint32_t)m4[i] << 16;
                    else blsh_dev_error(A.scratch, BLSH_EDEVICE, -1, 0ull);   // (self-check: no slot)
                    ++slot;
                }
            n_open += __shfl_sync(kFull, incl, 31);
            if (++iters == 8192) {
                flush();
                iters = 0;
            }
        }
        __syncwarp();
        // the tile's open pairs, a lane each, from chunk 4 (the four chunk
        // tests of a step together, the first stop by a bit scan)
        for (int b0 = 0; b0 < n_open; b0 += 32) {
            bool act = b0 + lane < n_open;
            unsigned q = 0;
            int m = 0, j = 4;
            uint2 pr = make_uint2(0u, 0u);
            const uint32_t *rx = A.sig, *ry = A.sig;
            if (act) {
                const uint32_t e = s_open[b0 + lane];
                q = base + (e & 0xffffu);
                m = (int)(e >> 16);
                // self-checks (a failed one reports BLSH_EDEVICE and skips the
                // access): the pair lies below P and names objects below N, a
                // step's words lie inside the row, an estimate inside the table
                if (q >= P) {
                    blsh_dev_error(A.scratch, BLSH_EDEVICE, -1, 0ull);
                    act = false;
                } else {
                    pr = __ldg(A.pairs + q);
                    if ((unsigned long long)pr.x >= N || (unsigned long long)pr.y >= N) {
                        blsh_dev_error(A.scratch, BLSH_EDEVICE, -1, 0ull);
                        act = false;
                    }
                }
                rx = A.sig + (size_t)pr.x * A.W;
                ry = A.sig + (size_t)pr.y * A.W;
            }
            while (__any_sync(kFull, act)) {
                if (act && j + 3 >= A.W) {
                    blsh_dev_error(A.scratch, BLSH_EDEVICE, -1, 0ull);
                    act = false;
                }
                if (act) {
                    const uint4 a = ldg4(rx + j), b = ldg4(ry + j);   // k = 32: chunk j is word j
                    const int c0 = m + 32 - __popc(a.x ^ b.x), c1 = c0 + 32 - __popc(a.y ^ b.y);
                    const int c2 = c1 + 32 - __popc(a.z ^ b.z), c3 = c2 + 32 - __popc(a.w ^ b.w);
                    auto m_at = [&](int i) { return i == 0 ? c0 : i == 1 ? c1 : i == 2 ? c2 : c3; };
                    unsigned valid = 0, prune = 0, conc = 0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int jj = j + i;
                        if (jj < A.levels) {
                            valid |= 1u << i;
                            prune |= (unsigned)(m_at(i) < s_mm[jj]) << i;
                            conc |= (unsigned)(m_at(i) >= s_clo[jj]) << i;
                        }
                    }
                    const unsigned last = at(A.levels, j), cap = at(A.cap_levels, j);
                    const unsigned s1 = (prune | (A.lite ? 0u : conc) | last | cap) & valid;
                    if (s1) {
                        const int i = __ffs(s1) - 1;
                        const unsigned bi = 1u << i;
                        const int st = (prune & bi) ? BLSH_PRUNED
                                       : (!A.lite && (conc & bi)) ? BLSH_ACCEPT
                                       : (last & bi) ? (A.lite ? BLSH_LITE_SURVIVOR : BLSH_ACCEPT_AT_MAX)
                                                     : BLSH_NEEDS_HASHES;
                        const int js = j + i, ms = m_at(i);
                        A.status[q] = (uint8_t)st;
                        if (A.n_used) A.n_used[q] = (uint16_t)((js + 1) * k);
                        if (A.m_out) A.m_out[q] = (uint16_t)ms;
                        if (st == BLSH_NEEDS_HASHES) {
                            A.need[pr.x] = 1;
                            A.need[pr.y] = 1;
                        } else {
                            if (js >= A.levels || ms >= A.est_stride) {
                                blsh_dev_error(A.scratch, BLSH_EDEVICE, -1, 0ull);
                            } else {
                                if (A.est_out && st != BLSH_PRUNED) A.est_out[q] = __ldg(A.est_tab + js * A.est_stride + ms);
                                atomicAdd(&s_hist[js], 1u);
                            }
                        }
                        act = false;
                    } else {
                        m = c3;
                        j += 4;
                    }
                }
            }
        }
    }
    flush();
    {
        const unsigned c0 = __reduce_add_sync(kFull, hc0), c1 = __reduce_add_sync(kFull, hc1);
        const unsigned c2 = __reduce_add_sync(kFull, hc2), c3 = __reduce_add_sync(kFull, hc3);
        const unsigned mine = lane == 0 ? c0 : lane == 1 ? c1 : lane == 2 ? c2 : lane == 3 ? c3 : 0u;
        if (mine && lane < A.levels) atomicAdd(&s_hist[lane], mine);
    }
    __syncthreads();
    if (A.stop_hist)
        for (int i = threadIdx.x; i < A.levels; i += blockDim.x)
            if (s_hist[i]) atomicAdd(A.stop_hist + i, (unsigned long long)s_hist[i]);
}

// plane[i] = words 0..3 of row i
__global__ void __launch_bounds__(256) plane_copy_kernel(const uint32_t *__restrict__ sig, long long N, int W,
                                                         uint4 *__restrict__ plane) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
        plane[i] = ldg4(sig + (size_t)i * W);
}

template <int KIND, int G, int U, bool PERSIST, bool PLANE = false, bool FAST = false, bool OPEN = false>
int launch_kernel(blsh_ctx *ctx, const VerifyArgs &A, const blsh_plan &plan, cudaStream_t s) {
    auto kern = verify_kernel<KIND, G, U, PERSIST, PLANE, FAST, OPEN>;
    // FAST plain form: the parked pairs (kDefer per warp) or, in the second
    // pass of the two-pass form, a tile's open pairs (512 per warp)
    const size_t smem = OPEN ? defer_offset(A.levels) + (size_t)(plan.block / 32) * 512 * sizeof(uint16_t)
                        : FAST && !PERSIST
                            ? defer_offset(A.levels) + (size_t)(plan.block / 32) * kDefer * (8 + 8 + 4)
                            : sizeof(int32_t) * A.levels * (FAST ? 3 : 2);
    if (smem > 48 * 1024) {
        if (smem > ctx->smem_optin) return blsh_fail(ctx, BLSH_EINVAL, "tables too large for shared memory");
        BLSH_CUDA(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    long long grid;
    if (PERSIST) {
        int occ = 0;
        BLSH_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, plan.block, smem));
        if (occ < 1) occ = 1;
        if (plan.ctas_per_sm > 0 && plan.ctas_per_sm < occ) occ = plan.ctas_per_sm;
        grid = (long long)occ * ctx->sm_count;
        BLSH_CUDA(ctx, cudaMemsetAsync(&A.scratch->work, 0, sizeof(unsigned long long), s));
    } else {
        // enough CTAs for two full waves; each warp then loops over its blocks
        const long long per_cta = plan.block / G;
        grid = (A.P + per_cta - 1) / per_cta;
        const long long cap = (long long)ctx->sm_count * (2 * 2048 / plan.block);
        if (grid > cap) grid = cap;
    }
    if (grid == 0) return BLSH_OK;
    if (OPEN) BLSH_CUDA(ctx, cudaMemsetAsync(&A.scratch->work, 0, sizeof(unsigned long long), s));   // tile counter
    blsh_time_start(ctx, s);
    kern<<<(unsigned)grid, plan.block, smem, s>>>(A);
    BLSH_LAUNCHED(ctx, "verify_kernel");
    return BLSH_OK;
}

template <bool PERSIST>
int dispatch(blsh_ctx *ctx, const VerifyArgs &A, const blsh_plan &plan, int kind, cudaStream_t s) {
    if (kind == BLSH_COSINE) {
        // k = 32 (one word per chunk) with upper-range concentration sets: the
        // branch-free four-chunk step
        if (A.chunk_words == 1 && A.conc_upper) {
            // plain form with Algorithm 2 (if any) over at most four chunks:
            // two passes -- every pair's first four chunks in a lean kernel,
            // then the pairs Algorithm 1 leaves open (a few percent)
            if (!PERSIST && A.lite_levels <= 4 && (A.lite_levels == 0 || A.lite_levels <= A.levels)) {
                // four pairs a lane where the outputs take the packed stores
                const bool quad = A.P < (1ll << 31) && blsh_aligned(A.pairs, 16) && blsh_aligned(A.status, 4) &&
                                  blsh_aligned(A.n_used, 8) && blsh_aligned(A.m_out, 8) &&
                                  (!A.lite_levels || (blsh_aligned(A.lstatus, 4) && blsh_aligned(A.ln_used, 8)));
                if (quad) {
                    // both passes in one kernel (verify_tile_kernel): one wave
                    // of resident CTAs, warps taking tiles from a counter
                    if (A.P == 0) return BLSH_OK;
                    const size_t smem = (size_t)A.levels * 3 * sizeof(int32_t) + 8 * kTilePairs * sizeof(uint32_t);
                    int occ = 0;
                    BLSH_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                                       &occ, A.plane ? verify_tile_kernel<true> : verify_tile_kernel<false>, 256, smem));
                    if (occ < 1) occ = 1;
                    const long long tiles = (A.P + kTilePairs - 1) / kTilePairs;
                    const long long blocks = (tiles + 7) / 8, cap = (long long)ctx->sm_count * occ;
                    const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
                    BLSH_CUDA(ctx, cudaMemsetAsync(&A.scratch->work, 0, sizeof(unsigned long long), s));   // tile counter
                    blsh_time_start(ctx, s);
                    if (A.plane) verify_tile_kernel<true><<<grid, 256, smem, s>>>(A);
                    else verify_tile_kernel<false><<<grid, 256, smem, s>>>(A);
                    BLSH_LAUNCHED(ctx, "verify_tile_kernel");
                    return BLSH_OK;
                } else {
                    const long long blocks = (A.P + 255) / 256, cap = (long long)ctx->sm_count * 8;
                    const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
                    if (grid == 0) return BLSH_OK;
                    blsh_time_start(ctx, s);
                    if (A.plane) verify_first_kernel<true><<<grid, 256, 0, s>>>(A);
                    else verify_first_kernel<false><<<grid, 256, 0, s>>>(A);
                }
                BLSH_LAUNCHED(ctx, "verify_first_kernel");
                return A.plane ? launch_kernel<BLSH_COSINE, 1, 1, false, true, true, true>(ctx, A, plan, s)
                               : launch_kernel<BLSH_COSINE, 1, 1, false, false, true, true>(ctx, A, plan, s);
            }
            return A.plane ? launch_kernel<BLSH_COSINE, 1, 1, PERSIST, true, true>(ctx, A, plan, s)
                           : launch_kernel<BLSH_COSINE, 1, 1, PERSIST, false, true>(ctx, A, plan, s);
        }
        return A.plane ? launch_kernel<BLSH_COSINE, 1, 1, PERSIST, true>(ctx, A, plan, s)
                       : launch_kernel<BLSH_COSINE, 1, 1, PERSIST, false>(ctx, A, plan, s);
    }
    switch (plan.group) {
    case 1: return launch_kernel<BLSH_JACCARD, 1, 8, PERSIST>(ctx, A, plan, s);
    case 4: return launch_kernel<BLSH_JACCARD, 4, 2, PERSIST>(ctx, A, plan, s);
    case 8: return launch_kernel<BLSH_JACCARD, 8, 1, PERSIST>(ctx, A, plan, s);
    case 16: return launch_kernel<BLSH_JACCARD, 16, 1, PERSIST>(ctx, A, plan, s);
    case 32: return launch_kernel<BLSH_JACCARD, 32, 1, PERSIST>(ctx, A, plan, s);
    }
    return blsh_fail(ctx, BLSH_EINVAL, "unsupported group size %d", plan.group);
}

}  // namespace

blsh_plan blsh_default_plan(int kind) {
    blsh_plan p;
    p.mode = BLSH_PLAN_PERSISTENT;
    p.group = kind == BLSH_COSINE ? 1 : 8;
    p.block = 256;
    p.grab = kind == BLSH_COSINE ? 128 : 32;
    p.ctas_per_sm = 0;
    return p;
}

// Words moved per group step must not exceed a Jaccard chunk (k words).
int blsh_check_plan(const blsh_plan &plan, int kind, int k) {
    if (plan.mode != BLSH_PLAN_PLAIN && plan.mode != BLSH_PLAN_PERSISTENT) return BLSH_EINVAL;
    if (plan.block != 128 && plan.block != 256 && plan.block != 512) return BLSH_EINVAL;
    if (kind == BLSH_COSINE) {
        if (plan.group != 1) return BLSH_EINVAL;
    } else {
        int wps;
        switch (plan.group) {
        case 1: wps = 32; break;
        case 4: wps = 32; break;
        case 8: wps = 32; break;
        case 16: wps = 64; break;
        case 32: wps = 128; break;
        default: return BLSH_EINVAL;
        }
        if (wps > k) return BLSH_EINVAL;
    }
    if (plan.mode == BLSH_PLAN_PERSISTENT && (plan.grab < 1 || plan.grab > (1 << 20))) return BLSH_EINVAL;
    // (persistent launches round grab up to a multiple of 32)
    if (plan.ctas_per_sm < 0) return BLSH_EINVAL;
    return BLSH_OK;
}

// Cosine signatures larger than this do not stay in L2 between the random
// row reads of the pairs; the first four words of every row (the first 128
// hashes) then go into a dense plane (16 bytes per object) that does, and the
// first step of every pair reads them there.
constexpr long long kPlaneMinBytes = 64ll << 20;

int blsh_launch_verify(blsh_ctx *ctx, const VerifyArgs &A0, const blsh_plan &plan, cudaStream_t s) {
    const int kind = A0.chunk_words == A0.k ? BLSH_JACCARD : BLSH_COSINE;
    VerifyArgs A = A0;
    A.plane = nullptr;
    // the plane lives in the buffer blsh_ctx_reserve allocated; a call with
    // more objects than were reserved reads the rows instead (no allocation
    // here: this is a hot call)
    if (kind == BLSH_COSINE && A.W > 4 && A.N * (long long)A.W * 4 > kPlaneMinBytes && ctx->plane_cap >= A.N) {
        const long long blocks = (A.N + 255) / 256, cap = (long long)ctx->sm_count * 8;
        blsh_time_start(ctx, s);
        plane_copy_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(A.sig, A.N, A.W,
                                                                                  (uint4 *)ctx->plane);
        BLSH_LAUNCHED(ctx, "plane_copy_kernel");
        A.plane = (const uint4 *)ctx->plane;
    }
    if (plan.mode == BLSH_PLAN_PERSISTENT) return dispatch<true>(ctx, A, plan, kind, s);
    return dispatch<false>(ctx, A, plan, kind, s);
}

int blsh_make_verify_args(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                          const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words, uint8_t *status,
                          uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist, VerifyArgs &A) {
    const blsh_params &p = tab->p;
    if (!sig || (P > 0 && (!pairs || !status)))
        return blsh_fail(ctx, BLSH_EINVAL, "pairs, sig and status are required");
    if (P < 0 || N < 0 || N > (1ll << 32)) return blsh_fail(ctx, BLSH_EINVAL, "bad P or N");
    const int need = p.kind == BLSH_JACCARD ? p.n_max : (p.n_max + 31) / 32;
    if (sig_words < need || sig_words % 4)
        return blsh_fail(ctx, BLSH_EINVAL, "sig_words must be a multiple of 4 covering n_max hashes");
    if (!blsh_aligned(sig, 16) || !blsh_aligned(pairs, 8) || !blsh_aligned(n_used, 2) || !blsh_aligned(m, 2) ||
        !blsh_aligned(est, 4) || !blsh_aligned(stop_hist, 8) || !blsh_aligned(P_dev, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    A.pairs = reinterpret_cast<const uint2 *>(pairs);
    A.P = P;
    A.P_dev = reinterpret_cast<const long long *>(P_dev);
    A.sig = sig;
    A.N = N;
    A.W = sig_words;
    A.k = p.k;
    A.chunk_words = p.kind == BLSH_JACCARD ? p.k : p.k / 32;
    A.levels = tab->levels;
    A.lite = 0;
    A.conc_words = tab->conc_words;
    A.est_stride = p.n_max + 1;
    A.min_matches = tab->min_matches;
    A.conc_bits = tab->conc_bits;
    A.conc_lo = tab->conc_lo;
    A.conc_upper = tab->conc_upper ? 1 : 0;
    A.est_tab = tab->est;
    A.status = status;
    A.n_used = n_used;
    A.m_out = m;
    A.est_out = est;
    A.sim_out = nullptr;
    A.stop_hist = reinterpret_cast<unsigned long long *>(stop_hist);
    A.scratch = ctx->scratch;
    A.grab = 0;
    A.lite_levels = 0;
    A.lstatus = nullptr;
    A.ln_used = nullptr;
    A.lsim = nullptr;
    A.cap_levels = A.levels;
    A.need = nullptr;
    A.plane = nullptr;
    return BLSH_OK;
}

// The plan the autotuner chose for these tables, else the default.  (A
// plan stored for destroyed tables whose address was reused may not fit the
// new tables' kind and k; the default is used then.)
blsh_plan blsh_plan_for(blsh_ctx *ctx, const blsh_tables *tab) {
    blsh_plan plan = blsh_default_plan(tab->p.kind);
    std::lock_guard<std::mutex> lk(ctx->mu);
    auto it = ctx->plans.find(tab);
    if (it != ctx->plans.end() && blsh_check_plan(it->second, tab->p.kind, tab->p.k) == BLSH_OK) plan = it->second;
    return plan;
}

extern "C" int blsh_verify_plan(blsh_ctx *ctx, const blsh_tables *tab, const blsh_plan *plan,
                                const uint32_t *pairs, int64_t P, const int64_t *P_dev, const uint32_t *sig,
                                int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used, uint16_t *m,
                                float *est, uint64_t *stop_hist, void *stream) {
    if (!ctx || !tab || !plan) return BLSH_EINVAL;
    if (tab->device != ctx->device) return blsh_fail(ctx, BLSH_EINVAL, "tables built on another device");
    if (blsh_check_plan(*plan, tab->p.kind, tab->p.k) != BLSH_OK)
        return blsh_fail(ctx, BLSH_EINVAL, "invalid plan for this kind and k");
    VerifyArgs A;
    int rc = blsh_make_verify_args(ctx, tab, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est,
                                   stop_hist, A);
    if (rc) return rc;
    A.grab = (plan->grab + 31) / 32 * 32;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    if (stop_hist) BLSH_CUDA(ctx, cudaMemsetAsync(stop_hist, 0, sizeof(uint64_t) * tab->levels, s));
    return blsh_launch_verify(ctx, A, *plan, s);
}

extern "C" int blsh_verify(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                           const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                           uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                           void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    const blsh_plan plan = blsh_plan_for(ctx, tab);
    return blsh_verify_plan(ctx, tab, &plan, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est,
                            stop_hist, stream);
}

extern "C" int blsh_set_plan(blsh_ctx *ctx, const blsh_tables *tab, const blsh_plan *plan) {
    if (!ctx || !tab || !plan) return BLSH_EINVAL;
    if (blsh_check_plan(*plan, tab->p.kind, tab->p.k) != BLSH_OK)
        return blsh_fail(ctx, BLSH_EINVAL, "invalid plan for this kind and k");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->plans[tab] = *plan;
    return BLSH_OK;
}

namespace {

// Times every candidate launch plan for `tab` on the given pairs (one
// untimed call, then three timed ones each) and returns the fastest and its
// time per call.  Outputs are overwritten.
int tune_plans(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P, const uint32_t *sig,
               int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used, uint16_t *m, float *est,
               void *stream, blsh_plan *best, float *best_ms_out) {
    cudaStream_t s = blsh_stream(stream);
    std::vector<blsh_plan> cands;
    const int kind = tab->p.kind;
    const int groups_c[] = {1};
    const int groups_j[] = {1, 4, 8, 16, 32};
    const int *groups = kind == BLSH_COSINE ? groups_c : groups_j;
    const int ng = kind == BLSH_COSINE ? 1 : 5;
    for (int gi = 0; gi < ng; ++gi)
        for (int block : {128, 256, 512}) {
            blsh_plan p;
            p.group = groups[gi];
            p.block = block;
            p.ctas_per_sm = 0;
            p.mode = BLSH_PLAN_PLAIN;
            p.grab = 32;
            if (blsh_check_plan(p, kind, tab->p.k) == BLSH_OK) cands.push_back(p);
            p.mode = BLSH_PLAN_PERSISTENT;
            for (int grab : {32, 128, 512}) {
                p.grab = grab;
                if (blsh_check_plan(p, kind, tab->p.k) == BLSH_OK) cands.push_back(p);
            }
        }
    cudaEvent_t e0, e1;
    BLSH_CUDA(ctx, cudaEventCreate(&e0));
    BLSH_CUDA(ctx, cudaEventCreate(&e1));
    float best_ms = 1e30f;
    blsh_plan best_plan = blsh_default_plan(kind);
    int rc = BLSH_OK;
    for (const blsh_plan &p : cands) {
        rc = blsh_verify_plan(ctx, tab, &p, pairs, P, nullptr, sig, N, sig_words, status, n_used, m, est,
                              nullptr, stream);
        if (rc) break;
        if ((rc = blsh_cuda_check(ctx, cudaEventRecord(e0, s), "event"))) break;
        for (int r = 0; r < 3 && !rc; ++r)
            rc = blsh_verify_plan(ctx, tab, &p, pairs, P, nullptr, sig, N, sig_words, status, n_used, m, est,
                                  nullptr, stream);
        if (rc) break;
        if ((rc = blsh_cuda_check(ctx, cudaEventRecord(e1, s), "event"))) break;
        if ((rc = blsh_cuda_check(ctx, cudaEventSynchronize(e1), "event sync"))) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best_plan = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    *best = best_plan;
    *best_ms_out = best_ms / 3.0f;
    return BLSH_OK;
}

}  // namespace

extern "C" int blsh_autotune(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                             const uint32_t *sig, int64_t N, int32_t sig_words, uint8_t *status,
                             uint16_t *n_used, uint16_t *m, float *est, blsh_plan *best, void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    blsh_device_guard g(ctx->device);
    blsh_plan plan;
    float ms = 0.f;
    const int rc = tune_plans(ctx, tab, pairs, P, sig, N, sig_words, status, n_used, m, est, stream, &plan, &ms);
    if (rc) return rc;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->plans[tab] = plan;
    }
    if (best) *best = plan;
    return BLSH_OK;
}

extern "C" int blsh_autotune_k(blsh_ctx *ctx, const blsh_params *params, const int32_t *ks, int32_t n_ks,
                               const uint32_t *pairs, int64_t P, const uint32_t *sig, int64_t N, int32_t sig_words,
                               uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, blsh_tables **out,
                               blsh_plan *best, float *ms_per_k, void *stream) {
    if (!ctx || !params || !ks || !out) return BLSH_EINVAL;
    *out = nullptr;
    if (n_ks < 1 || n_ks > 8) return blsh_fail(ctx, BLSH_EINVAL, "between 1 and 8 chunk sizes");
    for (int i = 0; i < n_ks; ++i)
        if ((ks[i] != 32 && ks[i] != 64 && ks[i] != 128) || params->n_max % ks[i])
            return blsh_fail(ctx, BLSH_EINVAL, "chunk size %d: not 32, 64 or 128, or not dividing n_max", ks[i]);
    blsh_device_guard g(ctx->device);
    blsh_tables *best_tab = nullptr;
    blsh_plan best_plan = blsh_default_plan(params->kind);
    float best_ms = 1e30f;
    int rc = BLSH_OK;
    for (int i = 0; i < n_ks && rc == BLSH_OK; ++i) {
        blsh_params q = *params;
        q.k = ks[i];
        // Lite's h: the same number of hashes, rounded up to a whole chunk
        q.h = (q.h + q.k - 1) / q.k * q.k;
        if (q.h > q.n_max) q.h = q.n_max;
        blsh_tables *tab = nullptr;
        rc = blsh_tables_build(ctx, &q, &tab, stream);
        if (rc == BLSH_ENUMERIC) rc = BLSH_OK;   // the table is usable; the caller sees near ties in its download
        if (rc) break;
        blsh_plan plan;
        float ms = 0.f;
        rc = tune_plans(ctx, tab, pairs, P, sig, N, sig_words, status, n_used, m, est, stream, &plan, &ms);
        if (ms_per_k) ms_per_k[i] = rc ? -1.f : ms;
        if (rc == BLSH_OK && ms < best_ms) {
            if (best_tab) blsh_tables_destroy(best_tab);
            best_tab = tab;
            best_plan = plan;
            best_ms = ms;
        } else {
            blsh_tables_destroy(tab);
        }
    }
    if (rc) {
        if (best_tab) blsh_tables_destroy(best_tab);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->plans[best_tab] = best_plan;
    }
    *out = best_tab;
    if (best) *best = best_plan;
    return BLSH_OK;
}

namespace {

// Pairs left at BLSH_NEEDS_HASHES, finished over all n_max hashes: one
// thread per pair (they are few), Algorithm 1 from its first chunk, the
// decisions of verify_kernel.  Statuses are read 16 at a time.
__global__ void __launch_bounds__(256) verify_resume_kernel(const VerifyArgs A, int kind, int vec) {
    long long P = A.P;
    if (A.P_dev) {
        const long long pd = *A.P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const int lane = threadIdx.x & 31;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // a warp scans 512 statuses (16 per lane), then works each open pair of
    // them with all its lanes: lane l takes chunk j0 + l of 32 chunks at a
    // time, an inclusive scan gives m after every chunk, and the first chunk
    // whose test stops the pair (the tests of Algorithm 1, in its order) is
    // the one the sequential loop would stop at
    for (long long base = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 512; base < P;
         base += nwarps * 512) {
        const long long q0 = base + 16ll * lane;
        uint32_t hit = 0;
        if (vec && q0 + 16 <= P) {
            hit = blsh_eq16(*reinterpret_cast<const uint4 *>(A.status + q0), BLSH_NEEDS_HASHES);
        } else {
            for (int i = 0; i < 16; ++i)
                if (q0 + i < P && A.status[q0 + i] == BLSH_NEEDS_HASHES) hit |= 1u << i;
        }
        for (unsigned lanes = __ballot_sync(kFull, hit != 0); lanes; lanes &= lanes - 1) {
            const int l = __ffs(lanes) - 1;
            for (uint32_t bits = __shfl_sync(kFull, hit, l); bits; bits &= bits - 1) {
                const long long q = base + 16ll * l + (__ffs(bits) - 1);
                const uint2 pr = __ldg(A.pairs + q);
                const uint32_t *rx = A.sig + (size_t)pr.x * A.W, *ry = A.sig + (size_t)pr.y * A.W;
                int carry = 0, jstop = A.levels - 1, mstop = 0, st = BLSH_ACCEPT_AT_MAX;
                for (int j0 = 0; j0 < A.levels; j0 += 32) {
                    const int j = j0 + lane;
                    int c = 0;
                    if (j < A.levels)
                        for (int w = j * A.chunk_words; w < (j + 1) * A.chunk_words; ++w) {
                            const uint32_t a = __ldg(rx + w), b = __ldg(ry + w);
                            c += kind == BLSH_JACCARD ? (a == b) : 32 - __popc(a ^ b);
                        }
                    int m = c;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int t = __shfl_up_sync(kFull, m, o);
                        if (lane >= o) m += t;
                    }
                    m += carry;
                    int s = -1;
                    if (j < A.levels) {
                        // concentration: m >= conc_lo[j] where every level's set is an upper range
                        const bool conc = A.conc_upper
                                              ? m >= __ldg(A.conc_lo + j)
                                              : (__ldg(A.conc_bits + j * A.conc_words + (m >> 5)) >> (m & 31)) & 1u;
                        if (m < __ldg(A.min_matches + j)) s = BLSH_PRUNED;
                        else if (conc) s = BLSH_ACCEPT;
                        else if (j + 1 == A.levels) s = BLSH_ACCEPT_AT_MAX;
                    }
                    const unsigned stop = __ballot_sync(kFull, s >= 0);
                    if (stop) {
                        const int f = __ffs(stop) - 1;
                        jstop = j0 + f;
                        mstop = __shfl_sync(kFull, m, f);
                        st = __shfl_sync(kFull, s, f);
                        break;
                    }
                    carry = __shfl_sync(kFull, m, 31);
                }
                if (lane == 0) {
                    A.status[q] = (uint8_t)st;
                    if (A.n_used) A.n_used[q] = (uint16_t)((jstop + 1) * A.k);
                    if (A.m_out) A.m_out[q] = (uint16_t)mstop;
                    if (A.est_out && st != BLSH_PRUNED)
                        A.est_out[q] = __ldg(A.est_tab + (size_t)jstop * A.est_stride + mstop);
                    if (A.stop_hist) atomicAdd(A.stop_hist + jstop, 1ull);
                }
            }
        }
    }
}

}  // namespace

extern "C" int blsh_verify_resume(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                                  const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                                  uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                                  void *stream) {
    if (!ctx || !tab) return BLSH_EINVAL;
    if (tab->device != ctx->device) return blsh_fail(ctx, BLSH_EINVAL, "tables built on another device");
    VerifyArgs A;
    int rc = blsh_make_verify_args(ctx, tab, pairs, P, P_dev, sig, N, sig_words, status, n_used, m, est, stop_hist,
                                   A);
    if (rc) return rc;
    if (P == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long warps = (P + 511) / 512;
    const long long cap = (long long)ctx->sm_count * 8;
    const long long blocks = (warps + 7) / 8;
    blsh_time_start(ctx, s);
    verify_resume_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(A, tab->p.kind,
                                                                             blsh_aligned(status, 16) ? 1 : 0);
    BLSH_LAUNCHED(ctx, "verify_resume_kernel");
    return BLSH_OK;
}
