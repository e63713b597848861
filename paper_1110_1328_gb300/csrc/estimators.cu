// estimators.cu -- the classical estimator of Section 3 (the "LSH Approx"
// comparison mode of Section 5.1) and the learned Beta prior of Section 4.1.
//
//   blsh_estimate_mle: for each pair, m = agreements among hashes 0..n-1 and
//     the maximum-likelihood estimate m/n (Jaccard) or cos(pi (1 - m/n))
//     (cosine: the estimate of the angle is pi (1 - m/n)); a pair is kept
//     iff its estimate exceeds t (Section 2: "pairs ... with estimated
//     similarity greater than the threshold are finally output").  The
//     keep decision is the integer test m > m_star, m_star = the largest m
//     whose estimate is <= t, found on the host in FP64.
//   blsh_fit_beta_prior: exact Jaccard similarities of a sample of candidate
//     pairs, their mean and population variance (divisor r), and the
//     method-of-moments Beta(alpha, beta) (Section 4.1).
#include <math.h>

#include "common.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr double kPi = 3.141592653589793238462643383279502884;

// Eight lanes per pair; lanes stride over the words of the first n hashes.
__global__ void __launch_bounds__(256) mle_kernel(const uint2 *__restrict__ pairs, long long P,
                                                  const long long *P_dev, const uint32_t *__restrict__ sig,
                                                  long long N, int W, int kind, int n, int m_star,
                                                  uint16_t *__restrict__ m_out, float *__restrict__ est_out,
                                                  uint8_t *__restrict__ keep, blsh_dev_scratch *scratch) {
    if (P_dev) {
        const long long pd = *P_dev;
        P = pd < 0 ? 0 : (pd < P ? pd : P);
    }
    const int lane = threadIdx.x & 31, g = lane & 7;
    const long long groups = (long long)gridDim.x * (blockDim.x >> 3);
    const long long first = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
    // all lanes of a warp run the same iterations (the reduction shuffles)
    for (long long q0 = first & ~3ll; q0 < P; q0 += groups) {
        const long long q = q0 + (lane >> 3);
        const bool live = q < P;
        uint2 pr = make_uint2(0u, 0u);
        bool bad = false;
        if (live) {
            pr = __ldg(pairs + q);
            bad = (long long)pr.x >= N || (long long)pr.y >= N;
        }
        int c = 0;
        if (live && !bad) {
            const uint32_t *rx = sig + (size_t)pr.x * W, *ry = sig + (size_t)pr.y * W;
            if (kind == BLSH_JACCARD) {
                for (int i = g; i < n; i += 8) c += __ldg(rx + i) == __ldg(ry + i);
            } else {
                const int words = (n + 31) >> 5;
                for (int i = g; i < words; i += 8) {
                    uint32_t agree = ~(__ldg(rx + i) ^ __ldg(ry + i));
                    const int valid = n - 32 * i;
                    if (valid < 32) agree &= (1u << valid) - 1u;
                    c += __popc(agree);
                }
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
        if (live && g == 0) {
            if (bad) {
                blsh_dev_error(scratch, BLSH_ERANGE, 0, 1ull);
                if (m_out) m_out[q] = 0;
                if (est_out) est_out[q] = __int_as_float(0x7fc00000);
                if (keep) keep[q] = BLSH_BAD_PAIR;
            } else {
                if (m_out) m_out[q] = (uint16_t)c;
                if (est_out) {
                    const double r = (double)c / (double)n;
                    est_out[q] = (float)(kind == BLSH_JACCARD ? r : cos(kPi * (1.0 - r)));
                }
                if (keep) keep[q] = c > m_star ? 1 : 0;
            }
        }
    }
}

// The largest m in [0, n] whose estimate is <= t (-1 if none).
int mle_threshold(int kind, int n, double t) {
    int best = -1;
    for (int m = 0; m <= n; ++m) {
        const double r = (double)m / (double)n;
        const double e = kind == BLSH_JACCARD ? r : cos(kPi * (1.0 - r));
        if (e <= t) best = m;
    }
    return best;
}

// First position in L[0..n) holding a value >= v.
__device__ __forceinline__ long long lower_bound_u32(const uint32_t *L, long long n, uint32_t v) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (__ldg(L + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Warp per sampled pair: |A n B| / |A u B| by searching the shorter row's
// elements in the longer one.
__global__ void __launch_bounds__(256) sample_jaccard_kernel(const uint2 *__restrict__ pairs, long long P,
                                                             const int64_t *__restrict__ indptr,
                                                             const uint32_t *__restrict__ indices, long long N,
                                                             double *__restrict__ sims,
                                                             blsh_dev_scratch *scratch) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long q = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < P; q += warps) {
        const uint2 pr = __ldg(pairs + q);
        if ((long long)pr.x >= N || (long long)pr.y >= N) {
            if (lane == 0) {
                sims[q] = __longlong_as_double(0x7ff8000000000000ll);
                blsh_dev_error(scratch, BLSH_ERANGE, 0, 1ull);
            }
            continue;
        }
        const long long ax = __ldg(indptr + pr.x), ex = __ldg(indptr + pr.x + 1);
        const long long ay = __ldg(indptr + pr.y), ey = __ldg(indptr + pr.y + 1);
        long long s0 = ax, ns = ex - ax, l0 = ay, nl = ey - ay;
        if (nl < ns) { s0 = ay; ns = ey - ay; l0 = ax; nl = ex - ax; }
        long long inter = 0;
        for (long long i = lane; i < ns; i += 32) {
            const uint32_t v = __ldg(indices + s0 + i);
            const long long pos = lower_bound_u32(indices + l0, nl, v);
            inter += pos < nl && __ldg(indices + l0 + pos) == v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) inter += __shfl_xor_sync(kFull, inter, o);
        const long long uni = (ex - ax) + (ey - ay) - inter;
        if (lane == 0) sims[q] = uni == 0 ? 0.0 : __ddiv_rn((double)inter, (double)uni);
    }
}

// One CTA: mean and population variance of the r sims (fixed order: thread
// t sums elements t, t+T, ...; then a fixed tree), and the method-of-moments
// Beta.  out: [mean, var, alpha, beta, fallback flag].
__global__ void __launch_bounds__(256) prior_moments_kernel(const double *__restrict__ sims, long long r,
                                                            double *__restrict__ out) {
    __shared__ double part[256];
    double s = 0.0;
    for (long long i = threadIdx.x; i < r; i += blockDim.x) s += sims[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = part[0] / (double)r;
    __syncthreads();
    double v = 0.0;
    for (long long i = threadIdx.x; i < r; i += blockDim.x) {
        const double d = sims[i] - mean;
        v += d * d;
    }
    part[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double var = part[0] / (double)r;
        double alpha = 1.0, beta = 1.0, fallback = 1.0;
        if (var > 0.0 && var < mean * (1.0 - mean)) {
            const double k = mean * (1.0 - mean) / var - 1.0;
            alpha = mean * k;
            beta = (1.0 - mean) * k;
            fallback = 0.0;
        }
        out[0] = mean;
        out[1] = var;
        out[2] = alpha;
        out[3] = beta;
        out[4] = fallback;
    }
}

}  // namespace

extern "C" int blsh_estimate_mle(blsh_ctx *ctx, int32_t kind, int32_t n_hashes, double t, const uint32_t *pairs,
                                 int64_t P, const int64_t *P_dev, const uint32_t *sig, int64_t N,
                                 int32_t sig_words, uint16_t *m, float *est, uint8_t *keep, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (kind != BLSH_JACCARD && kind != BLSH_COSINE) return blsh_fail(ctx, BLSH_EINVAL, "bad kind");
    if (n_hashes <= 0 || n_hashes > 65535 || P < 0 || N < 0 || N > (1ll << 32) || !sig || (P > 0 && !pairs))
        return blsh_fail(ctx, BLSH_EINVAL, "bad n_hashes, P, N or pointers");
    const long long need = kind == BLSH_JACCARD ? n_hashes : (n_hashes + 31) / 32;
    if (sig_words < need) return blsh_fail(ctx, BLSH_EINVAL, "signature rows shorter than n_hashes");
    if (!blsh_aligned(pairs, 8) || !blsh_aligned(m, 2) || !blsh_aligned(est, 4) || !blsh_aligned(P_dev, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    if (P == 0) return BLSH_OK;
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const int m_star = mle_threshold(kind, n_hashes, t);
    const long long groups = (P + 3) / 4 * 4;
    const long long blocks = (groups * 8 + 255) / 256;
    const long long cap = (long long)ctx->sm_count * 16;
    blsh_time_start(ctx, s);
    mle_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(
        reinterpret_cast<const uint2 *>(pairs), P, reinterpret_cast<const long long *>(P_dev), sig, N, sig_words,
        kind, n_hashes, m_star, m, est, keep, ctx->scratch);
    BLSH_LAUNCHED(ctx, "mle_kernel");
    return BLSH_OK;
}

extern "C" int blsh_fit_beta_prior(blsh_ctx *ctx, const uint32_t *pairs, int64_t r, const int64_t *indptr,
                                   const uint32_t *indices, int64_t N, double *sims, double *out_device,
                                   double *out_host, void *stream) {
    if (!ctx) return BLSH_EINVAL;
    if (r <= 0 || N < 0 || N > (1ll << 32) || !pairs || !indptr || !indices || !sims || !out_device)
        return blsh_fail(ctx, BLSH_EINVAL, "a positive sample and all pointers are required");
    if (!blsh_aligned(pairs, 8) || !blsh_aligned(sims, 8) || !blsh_aligned(out_device, 8) || !blsh_aligned(indptr, 8))
        return blsh_fail(ctx, BLSH_EINVAL, "misaligned pointer");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    const long long cap = (long long)ctx->sm_count * 8;
    const long long blocks = (r + 7) / 8;
    blsh_time_start(ctx, s);
    sample_jaccard_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(
        reinterpret_cast<const uint2 *>(pairs), r, indptr, indices, N, sims, ctx->scratch);
    BLSH_LAUNCHED(ctx, "sample_jaccard_kernel");
    blsh_time_start(ctx, s);
    prior_moments_kernel<<<1, 256, 0, s>>>(sims, r, out_device);
    BLSH_LAUNCHED(ctx, "prior_moments_kernel");
    if (out_host) {
        BLSH_CUDA(ctx, cudaMemcpyAsync(out_host, out_device, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
        BLSH_CUDA(ctx, cudaStreamSynchronize(s));
    }
    return BLSH_OK;
}
