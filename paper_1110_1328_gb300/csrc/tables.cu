// tables.cu -- the Section 4.3 inference tables, built in FP64 on the GPU.
//
// For every level j (n = (j+1) k) one CTA evaluates, for m = 0..n:
//   Pr[S >= t | M(m,n)]                        (Equation pruneProb)
//   S^(m,n), the posterior mode                (Equation map)
//   Pr[|S - S^| < delta | M(m,n)], m >= minMatches   (Equation concentrateProb)
// with the Jaccard posterior Beta(m+alpha, n-m+beta) of Section 4.1 and the
// cosine posterior of r on [0.5, 1] of Section 4.2, and reduces them to
// minMatches(n) and the concentration bitmap.  The incomplete beta is
// evaluated by its continued fraction with the forward (Wallis) recurrence.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTieTol = 1e-9;

// Value of the continued fraction 1 + d1/(1 + d2/(1 + ...)) of
// I_x(a,b) = x^a (1-x)^b / (a B(a,b)) / [1 + d1/(1 + d2/(...))], with
//   d_{2i+1} = -(a+i)(a+b+i) x / ((a+2i)(a+2i+1)),
//   d_{2i}   =  i(b-i) x / ((a+2i-1)(a+2i)),
// by the forward recurrence A_j = A_{j-1} + d_j A_{j-2}, B_j = B_{j-1} + d_j B_{j-2}
// (A_{-1} = 1, B_{-1} = 0, A_0 = B_0 = 1), renormalised so that B_j = 1.
__device__ double cf_forward(double a, double b, double x) {
    double A2 = 1.0, B2 = 0.0;   // A_{j-2}, B_{j-2}
    double A1 = 1.0, B1 = 1.0;   // A_{j-1}, B_{j-1}
    double f = 1.0;
    for (int j = 1; j <= 20000; ++j) {
        double d;
        if (j & 1) {
            const double i = (double)((j - 1) >> 1);
            d = -(a + i) * (a + b + i) * x / ((a + 2.0 * i) * (a + 2.0 * i + 1.0));
        } else {
            const double i = (double)(j >> 1);
            d = i * (b - i) * x / ((a + 2.0 * i - 1.0) * (a + 2.0 * i));
        }
        double A = A1 + d * A2;
        double B = B1 + d * B2;
        if (B == 0.0) B = 1e-300;
        const double inv = 1.0 / B;
        A2 = A1 * inv;
        B2 = B1 * inv;
        A1 = A * inv;
        B1 = 1.0;
        if (fabs(A1 - f) <= 1e-16 * fabs(A1)) {
            f = A1;
            break;
        }
        f = A1;
    }
    return f;
}

__device__ double log_prefactor(double a, double b, double x) {
    // log( x^a (1-x)^b / (a B(a,b)) )
    return a * log(x) + b * log1p(-x) - log(a) - (lgamma(a) + lgamma(b) - lgamma(a + b));
}

// I_x(a,b); small values are always computed directly, never as 1 - (~1).
__device__ double ibeta(double a, double b, double x) {
    if (!(x > 0.0)) return 0.0;
    if (!(x < 1.0)) return 1.0;
    if (x * (a + b + 2.0) < a + 1.0) return exp(log_prefactor(a, b, x)) / cf_forward(a, b, x);
    return 1.0 - exp(log_prefactor(b, a, 1.0 - x)) / cf_forward(b, a, 1.0 - x);
}

// log I_x(a,b), for ratios of tails that may underflow.
__device__ double log_ibeta(double a, double b, double x) {
    if (!(x > 0.0)) return -INFINITY;
    if (!(x < 1.0)) return 0.0;
    if (x * (a + b + 2.0) < a + 1.0) return log_prefactor(a, b, x) - log(cf_forward(a, b, x));
    return log1p(-exp(log_prefactor(b, a, 1.0 - x)) / cf_forward(b, a, 1.0 - x));
}

__device__ double cos_to_r(double c) { return 1.0 - acos(c) / kPi; }
__device__ double r_to_cos(double r) { return cos(kPi * (1.0 - r)); }

struct TabArgs {
    int kind, k, n_max, levels, conc_words;
    double t, eps, delta, gamma, alpha, beta;
    int32_t *min_matches;
    uint32_t *conc_bits;
    int32_t *conc_lo;     // [levels]: the smallest concentrated m (n+1 if none)
    float *est;
    double *prune_prob, *conc_prob;
    int *flags;           // [3]: near ties, non-finite / non-monotone, a level whose concentrated m are no upper range
};

__device__ double mode_estimate(const TabArgs &A, int m, int n) {
    if (A.kind == BLSH_JACCARD) {
        double s = (m + A.alpha - 1.0) / (n + A.alpha + A.beta - 2.0);
        return fmin(1.0, fmax(0.0, s));
    }
    return r_to_cos(fmax((double)m / (double)n, 0.5));
}

// Pr[S >= t | M(m,n)]
__device__ double prune_probability(const TabArgs &A, int m, int n) {
    if (A.kind == BLSH_JACCARD) {
        // 1 - I_t(m+alpha, n-m+beta) as the upper tail I_{1-t}(n-m+beta, m+alpha)
        return ibeta(n - m + A.beta, m + A.alpha, 1.0 - A.t);
    }
    const double tr = cos_to_r(A.t);
    if (tr <= 0.5) return 1.0;
    const double a = m + 1.0, b = n - m + 1.0;
    // (B_1 - B_{t_r}) / (B_1 - B_{0.5}) over the density r^m (1-r)^(n-m)
    return exp(log_ibeta(b, a, 1.0 - tr) - log_ibeta(b, a, 0.5));
}

// Pr[|S - S^| < delta | M(m,n)]
__device__ double concentration(const TabArgs &A, int m, int n) {
    const double s = mode_estimate(A, m, n);
    if (A.kind == BLSH_JACCARD) {
        const double a = m + A.alpha, b = n - m + A.beta;
        const double hi = fmin(1.0, s + A.delta), lo = fmax(0.0, s - A.delta);
        return ibeta(b, a, 1.0 - lo) - ibeta(b, a, 1.0 - hi);
    }
    const double a = m + 1.0, b = n - m + 1.0;
    const double rhi = cos_to_r(fmin(1.0, s + A.delta));
    const double rlo = fmax(0.5, cos_to_r(fmax(-1.0, s - A.delta)));
    const double lden = log_ibeta(b, a, 0.5);
    return exp(log_ibeta(b, a, 1.0 - rlo) - lden) - exp(log_ibeta(b, a, 1.0 - rhi) - lden);
}

__global__ void __launch_bounds__(256) build_tables_kernel(TabArgs A) {
    __shared__ unsigned char bit[BLSH_MAX_NMAX + 1];
    __shared__ unsigned char keep[BLSH_MAX_NMAX + 1];
    __shared__ int s_min;
    const int j = blockIdx.x;
    const int n = (j + 1) * A.k;
    const int W = A.n_max + 1;
    if (threadIdx.x == 0) s_min = n + 1;
    __syncthreads();
    for (int m = threadIdx.x; m <= n; m += blockDim.x) {
        const double pr = prune_probability(A, m, n);
        A.prune_prob[(size_t)j * W + m] = pr;
        const bool ok = pr >= A.eps;
        keep[m] = ok;
        if (ok) atomicMin(&s_min, m);
        if (!isfinite(pr)) atomicOr(&A.flags[1], 1);
        if (fabs(pr - A.eps) < kTieTol) atomicAdd(&A.flags[0], 1);
        A.est[(size_t)j * W + m] = (float)mode_estimate(A, m, n);
    }
    for (int m = n + 1 + threadIdx.x; m < W; m += blockDim.x) {
        A.prune_prob[(size_t)j * W + m] = nan("");
        A.est[(size_t)j * W + m] = 0.0f;
    }
    __syncthreads();
    const int mm = s_min;
    if (threadIdx.x == 0) A.min_matches[j] = mm;
    for (int m = threadIdx.x; m < W; m += blockDim.x) {
        unsigned char c = 0;
        double cp = nan("");
        if (m <= n && m >= mm) {
            if (!keep[m]) atomicOr(&A.flags[1], 2);   // Pr not monotone in m
            cp = concentration(A, m, n);
            if (!isfinite(cp)) atomicOr(&A.flags[1], 1);
            if (fabs(cp - (1.0 - A.gamma)) < kTieTol) atomicAdd(&A.flags[0], 1);
            c = cp >= 1.0 - A.gamma;
        }
        bit[m] = c;
        A.conc_prob[(size_t)j * W + m] = cp;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < A.conc_words; w += blockDim.x) {
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int m = w * 32 + b;
            if (m < W && bit[m]) word |= 1u << b;
        }
        A.conc_bits[(size_t)j * A.conc_words + w] = word;
    }
    // the smallest concentrated m, and whether every m from it up to n is
    // concentrated (an upper range: the verification kernel then tests m >= it
    // instead of reading the bitmap)
    if (threadIdx.x == 0) {
        int lo = n + 1;
        for (int m = mm; m <= n; ++m)
            if (bit[m]) { lo = m; break; }
        for (int m = lo; m <= n; ++m)
            if (!bit[m]) { atomicOr(&A.flags[2], 1); break; }
        A.conc_lo[j] = lo;
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" int blsh_tables_build(blsh_ctx *ctx, const blsh_params *p, blsh_tables **out, void *stream) {
    if (!ctx || !p || !out) return BLSH_EINVAL;
    *out = nullptr;
    if (p->kind != BLSH_JACCARD && p->kind != BLSH_COSINE)
        return blsh_fail(ctx, BLSH_EINVAL, "kind must be BLSH_JACCARD or BLSH_COSINE");
    if (p->k != 32 && p->k != 64 && p->k != 128) return blsh_fail(ctx, BLSH_EINVAL, "k must be 32, 64 or 128");
    if (p->n_max <= 0 || p->n_max > BLSH_MAX_NMAX || p->n_max % p->k)
        return blsh_fail(ctx, BLSH_EINVAL, "n_max must be a positive multiple of k, at most %d", BLSH_MAX_NMAX);
    if (p->h < 0 || p->h > p->n_max || p->h % p->k)
        return blsh_fail(ctx, BLSH_EINVAL, "h must be a multiple of k, at most n_max");
    if (!(p->t > 0 && p->t < 1) || !(p->eps > 0 && p->eps < 1) || !(p->delta > 0 && p->delta < 1) ||
        !(p->gamma > 0 && p->gamma < 1))
        return blsh_fail(ctx, BLSH_EINVAL, "t, eps, delta, gamma must lie in (0, 1)");
    if (p->kind == BLSH_JACCARD && !(p->alpha > 0 && p->beta > 0))
        return blsh_fail(ctx, BLSH_EINVAL, "the Beta prior needs alpha, beta > 0");
    blsh_device_guard g(ctx->device);
    cudaStream_t s = blsh_stream(stream);
    blsh_tables *tab = new blsh_tables();
    tab->p = *p;
    tab->device = ctx->device;
    tab->levels = p->n_max / p->k;
    tab->conc_words = (p->n_max + 1 + 31) / 32;
    const size_t L = tab->levels, W = p->n_max + 1;
    const size_t o_mm = 0;
    const size_t o_lo = align256(o_mm + L * sizeof(int32_t));
    const size_t o_conc = align256(o_lo + L * sizeof(int32_t));
    const size_t o_est = align256(o_conc + L * tab->conc_words * sizeof(uint32_t));
    const size_t o_pr = align256(o_est + L * W * sizeof(float));
    const size_t o_cp = align256(o_pr + L * W * sizeof(double));
    const size_t o_fl = align256(o_cp + L * W * sizeof(double));
    tab->bytes = align256(o_fl + 3 * sizeof(int));
    cudaError_t e = cudaMalloc(&tab->dev, tab->bytes);
    if (e != cudaSuccess) {
        delete tab;
        return blsh_cuda_check(ctx, e, "cudaMalloc(tables)");
    }
    char *base = (char *)tab->dev;
    tab->min_matches = (int32_t *)(base + o_mm);
    tab->conc_lo = (int32_t *)(base + o_lo);
    tab->conc_bits = (uint32_t *)(base + o_conc);
    tab->est = (float *)(base + o_est);
    tab->prune_prob = (double *)(base + o_pr);
    tab->conc_prob = (double *)(base + o_cp);
    tab->flags = (int *)(base + o_fl);
    TabArgs A;
    A.kind = p->kind; A.k = p->k; A.n_max = p->n_max; A.levels = tab->levels; A.conc_words = tab->conc_words;
    A.t = p->t; A.eps = p->eps; A.delta = p->delta; A.gamma = p->gamma; A.alpha = p->alpha; A.beta = p->beta;
    A.min_matches = tab->min_matches; A.conc_bits = tab->conc_bits; A.conc_lo = tab->conc_lo; A.est = tab->est;
    A.prune_prob = tab->prune_prob; A.conc_prob = tab->conc_prob; A.flags = tab->flags;
    int flags[3] = {0, 0, 0};
    e = cudaMemsetAsync(tab->flags, 0, 3 * sizeof(int), s);
    if (e == cudaSuccess) {
        blsh_time_start(ctx, s);
        build_tables_kernel<<<tab->levels, 256, 0, s>>>(A);
        e = cudaGetLastError();
        ctx->launches.fetch_add(1, std::memory_order_relaxed);
        if (e == cudaSuccess) blsh_time_stop(ctx, "build_tables_kernel");
        ctx->timing.open = false;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, tab->flags, sizeof(flags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(tab->dev);
        delete tab;
        return blsh_cuda_check(ctx, e, "building the inference tables");
    }
    tab->near_ties = flags[0];
    tab->numeric_bad = flags[1];
    tab->conc_upper = flags[2] == 0;
    *out = tab;
    if (flags[1])
        return blsh_fail(ctx, BLSH_ENUMERIC, "inference table: %s",
                         (flags[1] & 2) ? "Pr[S>=t|M] not monotone in m" : "non-finite probability");
    return BLSH_OK;
}

extern "C" int blsh_tables_destroy(blsh_tables *tab) {
    if (!tab) return BLSH_OK;
    {
        blsh_device_guard g(tab->device);
        cudaFree(tab->dev);
    }
    delete tab;
    return BLSH_OK;
}

extern "C" int blsh_tables_download(const blsh_tables *tab, blsh_params *params, int32_t *levels,
                                    int32_t *near_ties, int32_t *min_matches, uint8_t *conc, float *est,
                                    double *prune_prob, double *conc_prob) {
    if (!tab) return BLSH_EINVAL;
    blsh_device_guard g(tab->device);
    const size_t L = tab->levels, W = tab->p.n_max + 1;
    if (params) *params = tab->p;
    if (levels) *levels = tab->levels;
    if (near_ties) *near_ties = tab->near_ties;
    if (min_matches && cudaMemcpy(min_matches, tab->min_matches, L * sizeof(int32_t), cudaMemcpyDeviceToHost))
        return BLSH_EDEVICE;
    if (est && cudaMemcpy(est, tab->est, L * W * sizeof(float), cudaMemcpyDeviceToHost)) return BLSH_EDEVICE;
    if (prune_prob && cudaMemcpy(prune_prob, tab->prune_prob, L * W * sizeof(double), cudaMemcpyDeviceToHost))
        return BLSH_EDEVICE;
    if (conc_prob && cudaMemcpy(conc_prob, tab->conc_prob, L * W * sizeof(double), cudaMemcpyDeviceToHost))
        return BLSH_EDEVICE;
    if (conc) {
        std::vector<uint32_t> bits(L * tab->conc_words);
        if (cudaMemcpy(bits.data(), tab->conc_bits, bits.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost))
            return BLSH_EDEVICE;
        for (size_t j = 0; j < L; ++j)
            for (size_t m = 0; m < W; ++m)
                conc[j * W + m] = (bits[j * tab->conc_words + m / 32] >> (m % 32)) & 1u;
    }
    return BLSH_OK;
}
