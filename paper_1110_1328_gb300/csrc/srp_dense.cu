// srp_dense.cu -- sign random projections of dense rows (Section 4.2, "LSH
// family"): bit j of row i = [x_i . r_j >= 0].
//
// Tensor-core path (d a multiple of 64, bits a multiple of 256):
//   1. srp_dense_prep: X and R become BF16 pairs hi + lo with
//      hi = bf16(v), lo = bf16(v - hi) (|v - hi - lo| <= 2^-16 |v|), written in
//      the tile layout the tensor cores read (128- and 256-row tiles of 64
//      K-values, 128-byte rows, 16-byte chunks XOR-swizzled by row), plus the
//      L2 norms of the rows of X and the columns of R.
//   2. srp_dense_tc_persistent: one CTA per SM walks tiles of 128 rows x 256
//      bits; the K dimension streams through a two-stage shared-memory ring
//      filled by bulk copies (cp.async.bulk, completion on mbarriers); one
//      thread issues tcgen05.mma (BF16 x BF16 -> FP32 in tensor memory) for
//      hi*hi, hi*lo and lo*hi into one of two accumulators; four epilogue
//      warps read the other accumulator back (tcgen05.ld) and set a bit
//      wherever |p| > margin * |x_i| * |r_j|, queueing every other sign.
//   3. srp_dense_recheck_kernel: each queued sign is recomputed in FP32 with a
//      rigorous error bound, then in FP64 with one, and, if neither can decide
//      it, as the FP64 sum over coordinates 0..d-1 in order -- the oracle's
//      definition -- so every bit is exact whenever the margin bounds the
//      tensor-core error.
// The error of step 2 is at most 3.1 * 2^-16 sum|x_i r_ij| from the split
// plus the FP32 accumulation of 3d products; the rigorous margin used when
// the caller passes margin <= 0 is (2^-14 + 3 d 2^-22) * 1.25, applied to
// |x| |r| >= sum|x_i r_ij|.
//
// Every other shape uses srp_dense_simt_kernel (hashing.cu): FP32 sums with
// the same kind of bound and an FP64 recheck.
#include <cuda_bf16.h>

#include <atomic>

#include "common.cuh"

int blsh_srp_dense_simt(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                        uint32_t *sig, cudaStream_t s);

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int BM = 128;                   // rows of X per CTA
constexpr int BN = 256;                   // bits per CTA
constexpr int BK = 64;                    // K values per stage (128 bytes of BF16 per row)
constexpr int TILE_A = BM * BK * 2;       // 16 KiB
constexpr int TILE_B = BN * BK * 2;       // 32 KiB
constexpr int STAGE_BYTES = 2 * TILE_A + 2 * TILE_B;   // hi and lo of both operands: 96 KiB
constexpr int STAGES = 2;
constexpr long long kWaitPolls = 1ll << 24;

// byte offset of element k (0..63) of row r inside a 128-byte-row tile with
// the 128-byte swizzle: 16-byte chunk c = k/8 is stored at chunk c ^ (r % 8)
__host__ __device__ inline int swz_offset(int r, int k) { return r * 128 + ((((k >> 3) ^ (r & 7))) << 4) + (k & 7) * 2; }

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// ---- preparation --------------------------------------------------------------

// One warp per row of X (rows >= N are zero-filled up to the padded tile);
// lanes take 4 consecutive values at a time.  xnorm: |x| in FP32 rounded up.
__global__ void srp_dense_prep_x(const float *__restrict__ X, long long N, long long Npad, int d,
                                 unsigned char *__restrict__ Xh, unsigned char *__restrict__ Xl,
                                 float *__restrict__ xnorm) {
    const int lane = threadIdx.x & 31;
    const int KT = d / BK;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < Npad; r += warps) {
        const long long mt = r / BM;
        const int rr = (int)(r % BM);
        float ss = 0.0f;
        for (int k0 = 4 * lane; k0 < d; k0 += 128) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < N) v = __ldg(reinterpret_cast<const float4 *>(X + (size_t)r * d + k0));
            const float a[4] = {v.x, v.y, v.z, v.w};
            __nv_bfloat16 hi[4], lo[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                hi[i] = __float2bfloat16_rn(a[i]);
                lo[i] = __float2bfloat16_rn(a[i] - __bfloat162float(hi[i]));
                ss = __fmaf_ru(a[i], a[i], ss);
            }
            const int kt = k0 / BK, kk = k0 % BK;
            const size_t tile = ((size_t)mt * KT + kt) * TILE_A;
            *reinterpret_cast<uint2 *>(Xh + tile + swz_offset(rr, kk)) = *reinterpret_cast<const uint2 *>(hi);
            *reinterpret_cast<uint2 *>(Xl + tile + swz_offset(rr, kk)) = *reinterpret_cast<const uint2 *>(lo);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ss = __fadd_ru(ss, __shfl_xor_sync(kFull, ss, o));
        if (lane == 0) xnorm[r] = __fsqrt_ru(ss) * 1.0001f;
    }
}

// One thread per column j of R (bits): its d values become row j of the B
// operand (B is stored N-major rows of K values) and row j of Rt (FP32 R
// transposed, read by the rechecks).  rnorm: |r_j| rounded up.
__global__ void srp_dense_prep_r(const float *__restrict__ R, int d, int bits, unsigned char *__restrict__ Rh,
                                 unsigned char *__restrict__ Rl, float *__restrict__ rnorm,
                                 float *__restrict__ Rt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= bits) return;
    const int KT = d / BK;
    const int nt = j / BN, jj = j % BN;
    float ss = 0.0f;
    for (int k = 0; k < d; ++k) {
        const float v = __ldg(R + (size_t)k * bits + j);
        const __nv_bfloat16 hi = __float2bfloat16_rn(v);
        const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
        ss = __fmaf_ru(v, v, ss);
        Rt[(size_t)j * d + k] = v;   // column j of R, contiguous, for the rechecks
        const size_t tile = ((size_t)nt * KT + k / BK) * TILE_B;
        *reinterpret_cast<__nv_bfloat16 *>(Rh + tile + swz_offset(jj, k % BK)) = hi;
        *reinterpret_cast<__nv_bfloat16 *>(Rl + tile + swz_offset(jj, k % BK)) = lo;
    }
    rnorm[j] = __fsqrt_ru(ss) * 1.0001f;
}

// ---- tcgen05 / mbarrier / bulk-copy helpers ------------------------------------

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false if the phase did not complete within kWaitPolls polls
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    for (long long i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows
// 128 bytes apart, 8-row groups 1024 bytes apart.
__device__ __forceinline__ unsigned long long smem_desc(const void *p) {
    const unsigned long long addr = smem_u32(p);
    unsigned long long d = 0;
    d |= (addr & 0x3FFFFull) >> 4;          // start address
    d |= 1ull << 16;                         // leading-dimension byte offset (unused for this layout)
    d |= (1024ull >> 4) << 32;               // stride-dimension byte offset
    d |= 1ull << 46;                         // descriptor version
    d |= 2ull << 61;                         // 128-byte swizzle
    return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major, M = 128, N = 256.
constexpr unsigned kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(BN >> 3) << 17) | ((unsigned)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a, unsigned long long b, unsigned acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float (&v)[32]) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// A sign the tensor-core margin cannot decide, when the recheck queue is
// full: FP32 with its bound, else the FP64 sum in coordinate order.
__device__ __noinline__ bool sign_in_line(const float *__restrict__ x, const float *__restrict__ R, int d, int bits,
                                          int col, blsh_dev_scratch *scratch) {
    atomicAdd(&scratch->counters[2], 1ull);
    float acc = 0.0f, mag = 0.0f;
    for (int c = 0; c < d; ++c) {
        const float a = __ldg(x + c), b = __ldg(R + (size_t)c * bits + col);
        acc = __fmaf_rn(a, b, acc);
        mag = __fmaf_rn(fabsf(a), fabsf(b), mag);
    }
    const float bound = 1.25f * (float)d * 5.9604644775390625e-8f * mag + (float)d * 1.4e-45f;
    if (fabsf(acc) > bound) return acc >= 0.0f;
    double s = 0.0;
    for (int c = 0; c < d; ++c) s += (double)__ldg(x + c) * (double)__ldg(R + (size_t)c * bits + col);
    if (s == 0.0) atomicAdd(&scratch->counters[3], 1ull);
    return s >= 0.0;
}

// ---- the persistent, warp-specialised tensor-core kernel -------------------------
//
// One CTA per SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// (tile t: rows 128 (t / tiles_n), bits 256 (t % tiles_n), so consecutive
// tiles of a CTA share their rows of X).  Six warps:
//   warp 0  producer: bulk copies of each K stage into the two-stage ring;
//   warp 1  MMA issuer (one thread): 12 tcgen05.mma per K stage into one of
//           two 256-column accumulators in tensor memory (512 columns), so
//           the epilogue of one tile runs while the next tile accumulates;
//   warps 2-9 epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows of
//           the tile) in columns 128 ((w - 2) / 4) .. +127, tests each value
//           against margin |x_i| |r_j| (margin |r_j| staged in shared memory
//           for all bits), writes the decided bits and queues the others.
// Barriers: full/empty per ring stage (bulk-copy bytes / MMA commit), and
// acc_full/acc_empty per accumulator (MMA commit / 128 epilogue arrivals).
// Every wait is bounded; a role that gives up records the failure and
// stops, and the others give up in turn.
constexpr int kEpiWarps = 8;   // two per TMEM lane quarter, each taking half of a tile's 256 columns
constexpr int kTcThreads = 32 * (2 + kEpiWarps);

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1) srp_dense_tc_persistent(
    const unsigned char *__restrict__ Xh, const unsigned char *__restrict__ Xl, const unsigned char *__restrict__ Rh,
    const unsigned char *__restrict__ Rl, const float *__restrict__ xnorm, const float *__restrict__ rnorm,
    long long N, int d, int bits, float margin, uint32_t *__restrict__ sig, uint2 *__restrict__ queue,
    unsigned long long qcap, unsigned long long *qcount, const float *__restrict__ X, const float *__restrict__ R,
    long long tiles_total, blsh_dev_scratch *scratch) {
    extern __shared__ __align__(1024) unsigned char dyn_smem[];
    unsigned char *ring = reinterpret_cast<unsigned char *>(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    float *s_mr = reinterpret_cast<float *>(ring + (size_t)STAGES * STAGE_BYTES);   // [bits]: margin |r_j|
    for (int j = threadIdx.x; j < bits; j += blockDim.x) s_mr[j] = margin * __ldg(rnorm + j);
    __shared__ __align__(8) unsigned long long full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2];
    __shared__ __align__(8) unsigned long long mma_done;
    __shared__ unsigned tmem_base;
    __shared__ volatile int s_fail;
    const int KT = d / BK;
    const int tiles_n = bits / BN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(&full_bar[st], 1);
            mbar_init(&empty_bar[st], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 32 * kEpiWarps);
        }
        mbar_init(&mma_done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {   // producer
            long long it = 0;
            for (long long t = blockIdx.x; t < tiles_total && !s_fail; t += gridDim.x) {
                const long long mt = t / tiles_n;
                const int nt = (int)(t % tiles_n);
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int st = (int)(it % STAGES);
                    const unsigned use = (unsigned)(it / STAGES);
                    if (!mbar_wait(&empty_bar[st], (use & 1u) ^ 1u)) {   // the MMAs reading stage st are done
                        s_fail = 1;
                        break;
                    }
                    unsigned char *sp = ring + (size_t)st * STAGE_BYTES;
                    const size_t ta = ((size_t)mt * KT + kb) * TILE_A, tb = ((size_t)nt * KT + kb) * TILE_B;
                    mbar_expect_tx(&full_bar[st], STAGE_BYTES);
                    bulk_g2s(sp, Xh + ta, TILE_A, &full_bar[st]);
                    bulk_g2s(sp + TILE_A, Xl + ta, TILE_A, &full_bar[st]);
                    bulk_g2s(sp + 2 * TILE_A, Rh + tb, TILE_B, &full_bar[st]);
                    bulk_g2s(sp + 2 * TILE_A + TILE_B, Rl + tb, TILE_B, &full_bar[st]);
                }
            }
            // the last copy into each stage has landed before the CTA ends
            // (at once when its MMAs consumed it; a bounded wait otherwise)
            for (int st = 0; st < STAGES; ++st)
                if (it > st) mbar_wait(&full_bar[st], (unsigned)(((it - 1 - st) / STAGES) & 1));
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            long long it = 0, tc = 0;
            for (long long t = blockIdx.x; t < tiles_total && !s_fail; t += gridDim.x, ++tc) {
                const int buf = (int)(tc & 1);
                const unsigned use_acc = (unsigned)(tc >> 1);
                if (!mbar_wait(&acc_empty[buf], (use_acc & 1u) ^ 1u)) {   // the epilogue is done with it
                    s_fail = 1;
                    break;
                }
                fence_after();
                const unsigned acc = tmem + (unsigned)(buf * BN);
                bool ok = true;
                for (int kb = 0; kb < KT; ++kb, ++it) {
                    const int st = (int)(it % STAGES);
                    const unsigned use = (unsigned)(it / STAGES);
                    if (!mbar_wait(&full_bar[st], use & 1u)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    unsigned char *sp = ring + (size_t)st * STAGE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {   // K = 16 per MMA: 32 bytes along the 128-byte row
                        const unsigned long long ah = smem_desc(sp + kk * 32), al = smem_desc(sp + TILE_A + kk * 32);
                        const unsigned long long bh = smem_desc(sp + 2 * TILE_A + kk * 32);
                        const unsigned long long bl = smem_desc(sp + 2 * TILE_A + TILE_B + kk * 32);
                        mma_bf16(acc, ah, bh, (kb | kk) != 0);
                        mma_bf16(acc, ah, bl, 1u);
                        mma_bf16(acc, al, bh, 1u);
                    }
                    mma_commit(&empty_bar[st]);   // stage st is free once these MMAs finish
                }
                if (!ok) {
                    s_fail = 1;
                    break;
                }
                mma_commit(&acc_full[buf]);       // the tile's accumulator is final once all its MMAs finish
            }
            // every MMA issued has finished before tensor memory is freed
            mma_commit(&mma_done);
            mbar_wait(&mma_done, 0u);
        }
    } else {   // epilogue warps
        const int ew = warp & 3;                  // TMEM lanes 32 ew .. 32 ew + 31
        const int half = (warp - 2) >> 2;         // columns 128 half .. 128 half + 127
        const int words = bits >> 5;
        long long tc = 0;
        for (long long t = blockIdx.x; t < tiles_total && !s_fail; t += gridDim.x, ++tc) {
            const long long mt = t / tiles_n;
            const int nt = (int)(t % tiles_n);
            const int buf = (int)(tc & 1);
            const unsigned use_acc = (unsigned)(tc >> 1);
            if (!__all_sync(kFull, mbar_wait(&acc_full[buf], use_acc & 1u))) {   // the same verdict for the warp
                s_fail = 1;
                break;
            }
            fence_after();
            const long long row = mt * BM + ew * 32 + lane;
            const float xn = row < N ? __ldg(xnorm + row) : 0.0f;
            constexpr int kBuf = 8;
            unsigned short pend[kBuf];
            int npend = 0;
            for (int c = half * 4; c < half * 4 + 4; ++c) {
                float v[32];
                tmem_ld32(tmem + ((unsigned)(ew * 32) << 16) + (unsigned)(buf * BN + c * 32), v);
                const float *mr = s_mr + nt * BN + c * 32;
                uint32_t word = 0, und = 0;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    word |= (uint32_t)(v[i] >= 0.0f) << i;
                    und |= (uint32_t)!(fabsf(v[i]) > xn * mr[i]) << i;   // inside the margin (or NaN): recheck
                }
                if (row < N) {
                    word &= ~und;
                    for (uint32_t u = und; u; u &= u - 1) {
                        const int i = __ffs(u) - 1;
                        if (npend < kBuf) {
                            pend[npend++] = (unsigned short)(c * 32 + i);
                        } else {
                            word |= (uint32_t)sign_in_line(X + (size_t)row * d, R, d, bits, nt * BN + c * 32 + i,
                                                           scratch) << i;
                        }
                    }
                    sig[(size_t)row * words + nt * (BN / 32) + c] = word;
                }
            }
            // the accumulator may be overwritten now
            fence_before();
            mbar_arrive(&acc_empty[buf]);
            // warp-aggregated append of the undecided signs: one atomic per warp
            int incl = npend;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int wtotal = __shfl_sync(kFull, incl, 31);
            unsigned long long base = 0;
            if (lane == 0 && wtotal) base = atomicAdd(qcount, (unsigned long long)wtotal);
            base = __shfl_sync(kFull, base, 0);
            for (int p = 0; p < npend; ++p) {
                const unsigned long long slot = base + (unsigned long long)(incl - npend + p);
                const int col = nt * BN + pend[p];
                if (slot < qcap) {
                    queue[slot] = make_uint2((uint32_t)row, (uint32_t)col);
                } else if (sign_in_line(X + (size_t)row * d, R, d, bits, col, scratch)) {
                    atomicOr(sig + (size_t)row * words + (col >> 5), 1u << (col & 31));
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && s_fail) blsh_dev_error(scratch, BLSH_EDEVICE, -1, 0ull);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
}

// Queued signs: eight lanes per (row, bit).  Three stages, each with a
// rigorous bound:
//   FP32 partial sums, lane g of the group taking the 16-byte pieces 8i + g
//   of both rows (any summation order errs by at most (d+8) u sum|p|);
//   if undecided, FP64 partial sums of the exact products, lane g owning
//   coordinates [g d/8, (g+1) d/8) (error at most
//   (d+8) 2^-53 sum|p|, so a sign it decides is the sign of the exact sum and
//   of the oracle's sum, which errs by less);
//   if still undecided (exact ties such as zero rows), the FP64 sum over
//   coordinates 0..d-1 in order, lane g continuing lane g-1's running sum --
//   exactly the oracle's sum.
__global__ void __launch_bounds__(256) srp_dense_recheck_kernel(const uint2 *__restrict__ queue,
                                                                unsigned long long qcap,
                                                                const unsigned long long *qcount,
                                                                const float *__restrict__ X,
                                                                const float *__restrict__ Rt, int d, int bits,
                                                                uint32_t *__restrict__ sig,
                                                                blsh_dev_scratch *scratch) {
    const unsigned long long total = *qcount;
    const unsigned long long n = total < qcap ? total : qcap;
    const int lane = threadIdx.x & 31, g = lane & 7;
    const int per = d >> 3;   // coordinates per lane (d is a multiple of 64)
    const unsigned long long groups = (unsigned long long)gridDim.x * (blockDim.x >> 3);
    unsigned long long done = 0, zeros = 0;
    const unsigned long long warp_first = (((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3) & ~3ull;
    for (unsigned long long it0 = warp_first; it0 < n; it0 += groups) {
        const unsigned long long it = it0 + (unsigned long long)(lane >> 3);
        const bool live = it < n;
        uint2 rj = make_uint2(0u, 0u);
        if (live) rj = queue[it];
        const float *xr = X + (size_t)rj.x * d, *rr = Rt + (size_t)rj.y * d;
        const float *x = xr + g * per;
        const float *r = rr + g * per;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
        // FP32 stage: the group's eight lanes read 128 contiguous bytes of each
        // row per step (lane g the 16 bytes at 4 (8 i + g)); the bound holds
        // for any order of the terms
        if (live)
#pragma unroll 4
            for (int i = 0; i < per / 4; ++i) {
                const int c = (8 * i + g) * 4;
                const float4 u = __ldg(reinterpret_cast<const float4 *>(xr + c));
                const float4 v = __ldg(reinterpret_cast<const float4 *>(rr + c));
                a0 = __fmaf_rn(u.x, v.x, a0); a1 = __fmaf_rn(u.y, v.y, a1);
                a2 = __fmaf_rn(u.z, v.z, a2); a3 = __fmaf_rn(u.w, v.w, a3);
                m0 = __fmaf_rn(fabsf(u.x), fabsf(v.x), m0); m1 = __fmaf_rn(fabsf(u.y), fabsf(v.y), m1);
                m2 = __fmaf_rn(fabsf(u.z), fabsf(v.z), m2); m3 = __fmaf_rn(fabsf(u.w), fabsf(v.w), m3);
            }
        float acc = (a0 + a1) + (a2 + a3), mag = (m0 + m1) + (m2 + m3);
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            acc += __shfl_xor_sync(kFull, acc, o);
            mag += __shfl_xor_sync(kFull, mag, o);
        }
        const float bound = 1.25f * (float)(d + 8) * 5.9604644775390625e-8f * mag + (float)(d + 8) * 1.4e-45f;
        bool decided = !live || fabsf(acc) > bound;
        bool bit = acc >= 0.0f;
        if (__any_sync(kFull, !decided)) {
            double p = 0.0, q = 0.0;
            if (!decided)
                for (int c = 0; c < per; ++c) {
                    const double t = (double)__ldg(x + c) * (double)__ldg(r + c);
                    p += t;
                    q += fabs(t);
                }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                p += __shfl_xor_sync(kFull, p, o);
                q += __shfl_xor_sync(kFull, q, o);
            }
            const double bound64 = 1.25 * (double)(d + 8) * 1.1102230246251565e-16 * q + (double)(d + 8) * 5e-324;
            const bool decided64 = decided || fabs(p) > bound64;
            if (!decided && decided64) bit = p >= 0.0;
            if (__any_sync(kFull, !decided64)) {
                double s = 0.0;
                for (int step = 0; step < 8; ++step) {
                    if (g == step && !decided64)
                        for (int c = 0; c < per; ++c) s += (double)__ldg(x + c) * (double)__ldg(r + c);
                    s = __shfl_sync(kFull, s, (lane & 24) | step);
                }
                if (!decided64) {
                    bit = s >= 0.0;
                    zeros += (g == 0 && s == 0.0);
                }
            }
        }
        if (g == 0 && live) {
            if (bit) atomicOr(sig + (size_t)rj.x * (bits >> 5) + (rj.y >> 5), 1u << (rj.y & 31));
            ++done;
        }
    }
    if (done) atomicAdd(&scratch->counters[2], done);
    if (zeros) atomicAdd(&scratch->counters[3], zeros);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct DenseLayout {
    size_t xh, xl, rh, rl, rt, xn, rn, qc, q, total;
    unsigned long long qcap;
};

// Recheck queue capacity: 1/16 of the signs (at least 2^20); signs beyond it
// are decided in line by the tensor-core kernel itself.
unsigned long long queue_cap(long long N, int bits) {
    const unsigned long long all = (unsigned long long)N * bits;
    const unsigned long long c = all / 16;
    return c < (1ull << 20) ? ((1ull << 20) < all ? (1ull << 20) : all) : c;
}

DenseLayout dense_layout(long long N, int d, int bits) {
    const long long Npad = (N + BM - 1) / BM * BM;
    DenseLayout L;
    size_t o = 0;
    L.xh = o; o = up256(o + (size_t)Npad * d * 2);
    L.xl = o; o = up256(o + (size_t)Npad * d * 2);
    L.rh = o; o = up256(o + (size_t)bits * d * 2);
    L.rl = o; o = up256(o + (size_t)bits * d * 2);
    L.rt = o; o = up256(o + (size_t)bits * d * 4);
    L.xn = o; o = up256(o + (size_t)Npad * 4);
    L.rn = o; o = up256(o + (size_t)bits * 4);
    L.qc = o; o = up256(o + 8);
    L.qcap = queue_cap(N, bits);
    L.q = o; o = up256(o + (size_t)L.qcap * 8);
    L.total = o;
    return L;
}

bool tc_shape(long long N, int d, int bits) {
    return N > 0 && d % BK == 0 && bits % BN == 0 && d <= 4096 && (N + BM - 1) / BM <= 65535;
}

}  // namespace

extern "C" int blsh_srp_dense_workspace(int64_t N, int32_t d, int32_t bits, size_t *bytes) {
    if (!bytes || N < 0 || d <= 0 || bits <= 0) return BLSH_EINVAL;
    *bytes = tc_shape(N, d, bits) ? dense_layout(N, d, bits).total : 0;
    return BLSH_OK;
}

extern "C" int blsh_srp_dense(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                              float margin, uint32_t *sig, void *workspace, size_t workspace_bytes, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (!X || !R || !sig) return blsh_fail(ctx, BLSH_EINVAL, "X, R and sig are required");
    if (N < 0 || N >= (1ll << 32) || d <= 0 || bits <= 0 || bits % 32 || bits > 4096 || !(margin == margin))
        return blsh_fail(ctx, BLSH_EINVAL, "bad N, d, bits or margin");
    if (N == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    if (!workspace || !tc_shape(N, d, bits) || !blsh_aligned(X, 16) || !blsh_aligned(R, 16))
        return blsh_srp_dense_simt(ctx, X, N, d, R, bits, sig, s);
    const DenseLayout L = dense_layout(N, d, bits);
    if (workspace_bytes < L.total || !blsh_aligned(workspace, 256))
        return blsh_fail(ctx, BLSH_ETRUNC, "workspace needs %zu bytes, 256-byte aligned", L.total);
    // the margin must cover the tensor-core error: split 3.1 * 2^-16, FP32
    // accumulation of 3d products at 2^-22 each, with a 25% slack
    const float rigorous = 1.25f * (4.0f * 1.52587890625e-5f + 3.0f * (float)d * 2.384185791015625e-7f);
    const float m = margin > rigorous ? margin : rigorous;
    unsigned char *ws = (unsigned char *)workspace;
    const long long Npad = (N + BM - 1) / BM * BM;
    blsh_time_start(ctx, s);
    srp_dense_prep_x<<<(unsigned)((Npad + 7) / 8 < 65535ll * 8 ? (Npad + 7) / 8 : 65535ll * 8), 256, 0, s>>>(
        X, N, Npad, d, ws + L.xh, ws + L.xl, (float *)(ws + L.xn));
    BLSH_LAUNCHED(ctx, "srp_dense_prep_x");
    blsh_time_start(ctx, s);
    srp_dense_prep_r<<<(bits + 127) / 128, 128, 0, s>>>(R, d, bits, ws + L.rh, ws + L.rl, (float *)(ws + L.rn),
                                                        (float *)(ws + L.rt));
    BLSH_LAUNCHED(ctx, "srp_dense_prep_r");
    unsigned long long *qcount = (unsigned long long *)(ws + L.qc);
    uint2 *queue = (uint2 *)(ws + L.q);
    BLSH_CUDA(ctx, cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), s));
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + (size_t)bits * sizeof(float);
    const size_t smem_max = (size_t)STAGES * STAGE_BYTES + 1024 + 4096 * sizeof(float);   // bits <= 4096
    static std::atomic<unsigned long long> opted{0};
    if (ctx->device < 64 && !((opted.load() >> ctx->device) & 1ull)) {
        BLSH_CUDA(ctx, cudaFuncSetAttribute(srp_dense_tc_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_max));
        opted.fetch_or(1ull << ctx->device);
    }
    const long long tiles = (long long)(bits / BN) * (Npad / BM);
    const unsigned grid = (unsigned)(tiles < ctx->sm_count ? tiles : ctx->sm_count);
    blsh_time_start(ctx, s);
    srp_dense_tc_persistent<<<grid, kTcThreads, smem, s>>>(ws + L.xh, ws + L.xl, ws + L.rh, ws + L.rl,
                                                          (float *)(ws + L.xn), (float *)(ws + L.rn), N, d, bits, m,
                                                          sig, queue, L.qcap, qcount, X, R, tiles, ctx->scratch);
    BLSH_LAUNCHED(ctx, "srp_dense_tc_persistent");
    blsh_time_start(ctx, s);
    srp_dense_recheck_kernel<<<ctx->sm_count * 8, 256, 0, s>>>(queue, L.qcap, qcount, X, (float *)(ws + L.rt), d,
                                                                 bits, sig, ctx->scratch);
    BLSH_LAUNCHED(ctx, "srp_dense_recheck_kernel");
    return BLSH_OK;
}
