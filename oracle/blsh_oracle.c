/*
 * blsh_oracle.c -- plain, slow CPU oracle for BayesLSH candidate verification.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this file.  It shares no code, header, table
 * or constant generator with the CUDA library; the two meet only at the seeded
 * inputs drawn by the `synth` module.
 *
 * Everything is computed in FP64 (or exact integers), one pair and one chunk
 * at a time, in the order the paper states it:
 *
 *   - regularised incomplete beta I_x(a,b): Section 4.1 "Inference" (evaluated
 *     by the continued fraction the paper cites, DiDonato & Morris; here with
 *     the modified Lentz method, Lentz 1976 / Thompson & Barnett 1986);
 *   - Jaccard posterior Beta(m+alpha, n-m+beta), Pr[S>=t|M], mode and
 *     concentration: Section 4.1;
 *   - cosine posterior of r on [0.5,1], Pr[S>=t|M], R^ = m/n and
 *     concentration, with r2c / c2r: Section 4.2;
 *   - minMatches(n) and the (m,n) concentration cache: Section 4.3;
 *   - the verification loop: Algorithm 1 (BayesLSH) and Algorithm 2
 *     (BayesLSH-Lite);
 *   - minhash (Section 4.1 "LSH family", with h(x) = (a x + b) mod (2^31-1)),
 *     sign random projections (Section 4.2 "LSH family"), LSH banding
 *     (Section 2, "Candidate generation via LSH");
 *   - the two-byte storage of Gaussian samples (Section 4.3), and codes
 *     generated from a counter (SplitMix64, implemented here and in the
 *     library each from its published definition).
 *
 * Readings of points the paper leaves open or states inconsistently:
 *   - a chunk compares exactly k hashes, n .. n+k-1 (Algorithms 1-2 print a
 *     k+1-term sum);
 *   - Algorithm 1 stops once Pr[|S-S^| < delta | M] >= 1-gamma (the test as
 *     printed in the algorithm is garbled; the Section 4 text states this one);
 *   - Algorithm 1 stops at n = n_max with the current estimate (the paper's
 *     loop has no bound);
 *   - a pair is pruned iff Pr[S>=t|M] < eps (Pr == eps is kept);
 *   - Jaccard mode (m+alpha-1)/(n+alpha+beta-2) (the Beta mode the paper states;
 *     its printed substitution has -1 in the denominator), clamped to [0,1];
 *   - cosine R^ = max(m/n, 0.5) since the posterior lives on [0.5,1]; the
 *     concentration interval is clipped to S^+delta <= 1 and r >= 0.5;
 *   - concentration is tested with >= 1-gamma;
 *   - Lite's exact cosine is an order-independent fixed-point dot product
 *     (every product rounded once to a multiple of 2^-60, summed in int64),
 *     divided by the fixed-point norms.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_JACCARD 0
#define ORC_COSINE 1

#define ORC_PRUNED 0
#define ORC_ACCEPT 1
#define ORC_ACCEPT_AT_MAX 2
#define ORC_LITE_REJECT 3
#define ORC_LITE_ACCEPT 4

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Regularised incomplete beta I_x(a,b) = B_x(a,b) / B(a,b)  (Section 4.1).   */
/* ------------------------------------------------------------------------- */

/* The continued fraction
 *   I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 1 / (1 + d1/(1 + d2/(1 + ...)))
 * with
 *   d_{2i+1} = -(a+i)(a+b+i) x / ((a+2i)(a+2i+1)),   i >= 0
 *   d_{2i}   =  i (b-i) x / ((a+2i-1)(a+2i)),          i >= 1,
 * evaluated by the modified Lentz method.  Returns the value of the tail
 * 1 + d1/(1 + d2/(...)) so the caller divides by it. */
static double orc_cf_tail(double a, double b, double x)
{
    const double tiny = 1e-300;
    double f = 1.0, C = 1.0, D = 0.0;
    for (int j = 1; j <= 20000; j++) {
        double dj;
        if (j & 1) {
            double i = (double)((j - 1) / 2);
            dj = -(a + i) * (a + b + i) * x / ((a + 2.0 * i) * (a + 2.0 * i + 1.0));
        } else {
            double i = (double)(j / 2);
            dj = i * (b - i) * x / ((a + 2.0 * i - 1.0) * (a + 2.0 * i));
        }
        D = 1.0 + dj * D;
        if (fabs(D) < tiny) D = tiny;
        C = 1.0 + dj / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-16) break;
    }
    return f;
}

/* x^a (1-x)^b / (a B(a,b)), in log space. */
static double orc_front(double a, double b, double x)
{
    double lbeta = lgamma(a) + lgamma(b) - lgamma(a + b);
    return exp(a * log(x) + b * log1p(-x) - log(a) - lbeta);
}

/* I_x(a,b) for a, b > 0.  The fraction converges fast for x < (a+1)/(a+b+2);
 * otherwise the symmetry I_x(a,b) = 1 - I_{1-x}(b,a) is used, so a value near
 * 0 is always computed directly (no cancellation in small tails). */
double orc_ibeta(double a, double b, double x)
{
    if (!(x > 0.0)) return 0.0;
    if (!(x < 1.0)) return 1.0;
    if (x < (a + 1.0) / (a + b + 2.0))
        return orc_front(a, b, x) / orc_cf_tail(a, b, x);
    return 1.0 - orc_front(b, a, 1.0 - x) / orc_cf_tail(b, a, 1.0 - x);
}

/* ------------------------------------------------------------------------- */
/* Inference, Jaccard (Section 4.1) and cosine (Section 4.2).                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int kind;
    double t, eps, delta, gamma, alpha, beta;
    int k, n_max;
} orc_params;

static double orc_c2r(double c) { return 1.0 - acos(c) / ORC_PI; }
static double orc_r2c(double r) { return cos(ORC_PI * (1.0 - r)); }

/* log I_x(a,b), so that ratios of two tiny tails do not underflow. */
double orc_log_ibeta(double a, double b, double x)
{
    if (!(x > 0.0)) return -INFINITY;
    if (!(x < 1.0)) return 0.0;
    if (x < (a + 1.0) / (a + b + 2.0)) {
        double lbeta = lgamma(a) + lgamma(b) - lgamma(a + b);
        return a * log(x) + b * log1p(-x) - log(a) - lbeta - log(orc_cf_tail(a, b, x));
    }
    return log1p(-orc_front(b, a, 1.0 - x) / orc_cf_tail(b, a, 1.0 - x));
}

/* Pr[S >= t | M(m,n)]. */
double orc_prune_prob(const orc_params *p, int m, int n)
{
    if (p->kind == ORC_JACCARD) {
        double a = m + p->alpha, b = n - m + p->beta;
        /* 1 - I_t(a,b), written as the upper tail I_{1-t}(b,a). */
        return orc_ibeta(b, a, 1.0 - p->t);
    } else {
        double a = m + 1.0, b = n - m + 1.0;
        double tr = orc_c2r(p->t);
        if (tr <= 0.5) return 1.0;   /* t <= 0: the whole support [0.5,1] lies above t_r */
        /* (B_1 - B_{t_r}) / (B_1 - B_0.5): a ratio of regularised upper tails,
         * I_{1-t_r}(b,a) / I_{0.5}(b,a), taken in log space. */
        return exp(orc_log_ibeta(b, a, 1.0 - tr) - orc_log_ibeta(b, a, 0.5));
    }
}

/* Posterior mode S^ (Equation map). */
double orc_estimate(const orc_params *p, int m, int n)
{
    if (p->kind == ORC_JACCARD) {
        double s = (m + p->alpha - 1.0) / (n + p->alpha + p->beta - 2.0);
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
        return s;
    } else {
        double r = (double)m / (double)n;
        if (r < 0.5) r = 0.5;
        return orc_r2c(r);
    }
}

/* Pr[|S - S^| < delta | M(m,n)] (Equation concentrateProb). */
double orc_conc_prob(const orc_params *p, int m, int n)
{
    double s = orc_estimate(p, m, n);
    if (p->kind == ORC_JACCARD) {
        double a = m + p->alpha, b = n - m + p->beta;
        double hi = s + p->delta, lo = s - p->delta;
        if (hi > 1.0) hi = 1.0;
        if (lo < 0.0) lo = 0.0;
        /* I_hi - I_lo = (1 - I_lo) - (1 - I_hi) as upper tails. */
        return orc_ibeta(b, a, 1.0 - lo) - orc_ibeta(b, a, 1.0 - hi);
    } else {
        double a = m + 1.0, b = n - m + 1.0;
        double shi = s + p->delta, slo = s - p->delta;
        if (shi > 1.0) shi = 1.0;
        if (slo < -1.0) slo = -1.0;
        double rhi = orc_c2r(shi), rlo = orc_c2r(slo);
        if (rlo < 0.5) rlo = 0.5;
        /* (B_{c2r(S^+delta)} - B_{c2r(S^-delta)}) / (B_1 - B_0.5), as upper tails
         * relative to the normaliser I_{0.5}(b,a). */
        double lden = orc_log_ibeta(b, a, 0.5);
        return exp(orc_log_ibeta(b, a, 1.0 - rlo) - lden) - exp(orc_log_ibeta(b, a, 1.0 - rhi) - lden);
    }
}

/* ------------------------------------------------------------------------- */
/* Section 4.3: minMatches(n) and the concentration cache, for n = j k.       */
/* ------------------------------------------------------------------------- */

/* Returns 0, or -1 on bad parameters, or -2 if the linear scan and the binary
 * search for minMatches disagree (a non-monotone Pr[S>=t|M] in m).
 * min_matches [L]; conc [L][n_max+1] (1 = concentrated, only for
 * m >= minMatches); est [L][n_max+1]; prune_out / conc_out optional
 * [L][n_max+1] dumps of the probabilities (NaN where not evaluated). */
int orc_tables(int kind, double t, double eps, double delta, double gamma,
               double alpha, double beta, int k, int n_max,
               int32_t *min_matches, uint8_t *conc, double *est,
               double *prune_out, double *conc_out)
{
    if (k <= 0 || n_max <= 0 || n_max % k != 0) return -1;
    orc_params p = {kind, t, eps, delta, gamma, alpha, beta, k, n_max};
    int L = n_max / k, W = n_max + 1;
    int rc = 0;
    for (int j = 0; j < L; j++) {
        int n = (j + 1) * k;
        /* linear scan: the smallest m with Pr >= eps, n+1 if none */
        int lin = n + 1;
        for (int m = 0; m <= n; m++) {
            double pr = orc_prune_prob(&p, m, n);
            if (prune_out) prune_out[(size_t)j * W + m] = pr;
            if (pr >= eps) { lin = m; break; }
        }
        if (prune_out)
            for (int m = lin + 1; m <= n; m++) prune_out[(size_t)j * W + m] = orc_prune_prob(&p, m, n);
        if (prune_out)
            for (int m = n + 1; m < W; m++) prune_out[(size_t)j * W + m] = NAN;
        /* binary search over m in [0, n+1) on the monotone predicate Pr >= eps */
        int lo = 0, hi = n + 1;
        while (lo < hi) {
            int mid = lo + (hi - lo) / 2;
            if (orc_prune_prob(&p, mid, n) >= eps) hi = mid; else lo = mid + 1;
        }
        if (lo != lin) rc = -2;
        min_matches[j] = lin;
        for (int m = 0; m < W; m++) {
            uint8_t c = 0;
            double cp = NAN;
            if (m <= n && m >= lin) {
                cp = orc_conc_prob(&p, m, n);
                c = (cp >= 1.0 - gamma) ? 1 : 0;
            }
            conc[(size_t)j * W + m] = c;
            if (conc_out) conc_out[(size_t)j * W + m] = cp;
            est[(size_t)j * W + m] = (m <= n) ? orc_estimate(&p, m, n) : NAN;
        }
    }
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 (BayesLSH) and Algorithm 2 (BayesLSH-Lite).                    */
/* ------------------------------------------------------------------------- */

/* Matches among hashes [n, n+k) of rows x and y.  Jaccard rows hold one
 * uint32 minhash per hash; cosine rows hold bit j of hash j in word j/32 at
 * bit position j%32. */
static int orc_chunk_matches(int kind, const uint32_t *sx, const uint32_t *sy, int n, int k)
{
    int m = 0;
    for (int i = n; i < n + k; i++) {
        if (kind == ORC_JACCARD) {
            m += (sx[i] == sy[i]);
        } else {
            uint32_t bx = (sx[i / 32] >> (i % 32)) & 1u;
            uint32_t by = (sy[i / 32] >> (i % 32)) & 1u;
            m += (bx == by);
        }
    }
    return m;
}

/* Returns the number of pairs that named an object >= N (their status is
 * set to 255 and they are otherwise skipped). */
int64_t orc_verify(int kind, int k, int n_max, const int32_t *min_matches, const uint8_t *conc,
                   const double *est_tab, const uint32_t *pairs, int64_t P,
                   const uint32_t *sig, int64_t N, int sig_words,
                   uint8_t *status, uint16_t *n_used, uint16_t *m_out, double *est)
{
    int W = n_max + 1;
    int64_t bad = 0;
    for (int64_t q = 0; q < P; q++) {
        uint32_t x = pairs[2 * q], y = pairs[2 * q + 1];
        if (x >= N || y >= N) { status[q] = 255; n_used[q] = 0; m_out[q] = 0; est[q] = NAN; bad++; continue; }
        const uint32_t *sx = sig + (size_t)x * sig_words, *sy = sig + (size_t)y * sig_words;
        int n = 0, m = 0, st;
        for (;;) {
            m += orc_chunk_matches(kind, sx, sy, n, k);
            n += k;
            int j = n / k - 1;
            if (m < min_matches[j]) { st = ORC_PRUNED; break; }          /* Pr[S>=t|M] < eps */
            if (conc[(size_t)j * W + m]) { st = ORC_ACCEPT; break; }     /* concentrated */
            if (n == n_max) { st = ORC_ACCEPT_AT_MAX; break; }           /* hash budget spent */
        }
        status[q] = (uint8_t)st;
        n_used[q] = (uint16_t)n;
        m_out[q] = (uint16_t)m;
        /* Algorithm 1 outputs S^ only with a kept pair */
        est[q] = st == ORC_PRUNED ? NAN : est_tab[(size_t)(n / k - 1) * W + m];
    }
    return bad;
}

/* Exact Jaccard |A n B| / |A u B| by a merge of two sorted index lists. */
double orc_exact_jaccard(const uint32_t *a, int64_t na, const uint32_t *b, int64_t nb)
{
    int64_t i = 0, j = 0, inter = 0;
    while (i < na && j < nb) {
        if (a[i] == b[j]) { inter++; i++; j++; }
        else if (a[i] < b[j]) i++;
        else j++;
    }
    int64_t uni = na + nb - inter;
    if (uni == 0) return 0.0;
    return (double)inter / (double)uni;
}

/* Fixed-point term: the exact FP64 product of two floats, scaled by 2^60 and
 * rounded to the nearest integer (ties to even). */
static int64_t orc_fx(float u, float v)
{
    return llrint(ldexp((double)u * (double)v, 60));
}

/* Exact cosine of two sparse rows with sorted indices:
 *   D = sum over common indices of fx(x_i, y_i), Nx = sum fx(x_i, x_i), Ny likewise,
 *   s = D / sqrt(Nx * Ny)  (each conversion and operation rounded once in FP64).
 * The int64 sums do not depend on summation order.  Rows must have squared
 * norm below 4; a zero row gives 0. */
double orc_exact_cosine(const uint32_t *ia, const float *va, int64_t na,
                        const uint32_t *ib, const float *vb, int64_t nb)
{
    int64_t D = 0, Nx = 0, Ny = 0;
    for (int64_t i = 0; i < na; i++) Nx += orc_fx(va[i], va[i]);
    for (int64_t j = 0; j < nb; j++) Ny += orc_fx(vb[j], vb[j]);
    int64_t i = 0, j = 0;
    while (i < na && j < nb) {
        if (ia[i] == ib[j]) { D += orc_fx(va[i], vb[j]); i++; j++; }
        else if (ia[i] < ib[j]) i++;
        else j++;
    }
    if (Nx == 0 || Ny == 0) return 0.0;
    return (double)D / sqrt((double)Nx * (double)Ny);
}

/* Algorithm 2.  values == NULL means binary sets (Jaccard); otherwise
 * real-valued rows (cosine).  sim[q] is the exact similarity for pairs that
 * survive pruning and NaN for pruned pairs. */
int64_t orc_verify_lite(int kind, int k, int h, const int32_t *min_matches,
                        const uint32_t *pairs, int64_t P, const uint32_t *sig, int64_t N, int sig_words,
                        const int64_t *indptr, const uint32_t *indices, const float *values, double t,
                        uint8_t *status, uint16_t *n_used, double *sim)
{
    int64_t bad = 0;
    for (int64_t q = 0; q < P; q++) {
        uint32_t x = pairs[2 * q], y = pairs[2 * q + 1];
        if (x >= N || y >= N) { status[q] = 255; n_used[q] = 0; sim[q] = NAN; bad++; continue; }
        const uint32_t *sx = sig + (size_t)x * sig_words, *sy = sig + (size_t)y * sig_words;
        int n = 0, m = 0, pruned = 0;
        while (n < h) {
            m += orc_chunk_matches(kind, sx, sy, n, k);
            n += k;
            if (m < min_matches[n / k - 1]) { pruned = 1; break; }
        }
        n_used[q] = (uint16_t)n;
        if (pruned) { status[q] = ORC_PRUNED; sim[q] = NAN; continue; }
        double s;
        int64_t ax = indptr[x], ex = indptr[x + 1], ay = indptr[y], ey = indptr[y + 1];
        if (values == NULL)
            s = orc_exact_jaccard(indices + ax, ex - ax, indices + ay, ey - ay);
        else
            s = orc_exact_cosine(indices + ax, values + ax, ex - ax, indices + ay, values + ay, ey - ay);
        sim[q] = s;
        status[q] = (s > t) ? ORC_LITE_ACCEPT : ORC_LITE_REJECT;
    }
    return bad;
}

/* ------------------------------------------------------------------------- */
/* Hashes.                                                                    */
/* ------------------------------------------------------------------------- */

/* Minhash (Section 4.1 "LSH family"): sig[i][j] = min over x in S_i of
 * (a_j x + b_j) mod (2^31 - 1), in uint64.  An empty set gives 0xFFFFFFFF. */
void orc_minhash(const int64_t *indptr, const uint32_t *indices, int64_t N, int n_hashes,
                 const uint32_t *a, const uint32_t *b, uint32_t *sig)
{
    const uint64_t p = 2147483647ull;
    for (int64_t i = 0; i < N; i++) {
        for (int j = 0; j < n_hashes; j++) {
            uint64_t best = 0xFFFFFFFFull;
            for (int64_t e = indptr[i]; e < indptr[i + 1]; e++) {
                uint64_t h = ((uint64_t)a[j] * (uint64_t)indices[e] + (uint64_t)b[j]) % p;
                if (h < best) best = h;
            }
            sig[(size_t)i * n_hashes + j] = (uint32_t)best;
        }
    }
}

/* Sign random projection (Section 4.2 "LSH family") of sparse rows:
 * bit j of row i = [ sum_e val_e * R[idx_e][j] >= 0 ], the sum taken in FP64
 * in row order (each product of two floats is exact in FP64).  R is
 * [dim][bits] float32.  Bit j goes to word j/32, position j%32. */
void orc_srp_sparse(const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                    const float *R, int bits, uint32_t *sig)
{
    int W = bits / 32;
    for (int64_t i = 0; i < N; i++) {
        uint32_t *row = sig + (size_t)i * W;
        memset(row, 0, sizeof(uint32_t) * W);
        for (int j = 0; j < bits; j++) {
            double acc = 0.0;
            for (int64_t e = indptr[i]; e < indptr[i + 1]; e++)
                acc += (double)values[e] * (double)R[(size_t)indices[e] * bits + j];
            if (acc >= 0.0) row[j / 32] |= 1u << (j % 32);
        }
    }
}

/* Section 4.3, "Cheaper storage of hash functions": a standard Gaussian
 * sample x, assumed to lie in (-8, 8), is stored in two bytes as
 * q = floor((x + 8) * 2^16 / 16) and read back as q * 16 / 2^16 - 8.
 * floor((x + 8) 2^12) is formed as floor(x 2^12) + 2^15, which is the same
 * integer and involves no rounding (x 2^12 is exact).  Values whose code
 * falls outside [0, 65535] (x < -8, x >= 8) or NaN are clamped (NaN to 0);
 * their number is returned. */
int64_t orc_quantize_gaussian(const float *x, int64_t n, uint16_t *q)
{
    int64_t outside = 0;
    for (int64_t i = 0; i < n; i++) {
        double c = floor((double)x[i] * 4096.0) + 32768.0;
        if (!(c >= 0.0)) { c = 0.0; outside++; }
        else if (c > 65535.0) { c = 65535.0; outside++; }
        q[i] = (uint16_t)c;
    }
    return outside;
}

double orc_dequantize_gaussian(uint16_t q)
{
    return (double)q * 16.0 / 65536.0 - 8.0;
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), as a counter-based generator: output k (k = 0,
 * 1, ...) of the stream started at `seed` is the finaliser applied to
 * seed + (k + 1) * 0x9E3779B97F4A7C15 (mod 2^64). */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Two-byte codes (Section 4.3) of the projection matrix R [dim][bits],
 * generated from a counter instead of stored: entry c = t * bits + j takes
 * SplitMix64 outputs 3c, 3c + 1, 3c + 2 of the stream `seed`, splits them
 * into twelve 16-bit integers u_1..u_12 and sums them (Irwin-Hall: S has
 * mean 12 * 32767.5 = 393210 and standard deviation sqrt(65536^2 - 1), so
 * (S - 393210) / 65536 is a standard normal to within the Irwin-Hall
 * approximation, truncated at +-6).  The code is the Section 4.3 encoding
 * floor((x + 8) 2^16 / 16) of x = (S - 393210) / 65536, i.e.
 * floor((S - 393210) / 16) + 32768, always inside [8192, 57343].  Rows
 * row0 .. row0 + rows - 1 are written to codes [rows][bits]. */
void orc_gaussian_codes(uint64_t seed, int64_t row0, int64_t rows, int bits, uint16_t *codes)
{
    for (int64_t r = 0; r < rows; r++)
        for (int j = 0; j < bits; j++) {
            uint64_t c = (uint64_t)(row0 + r) * (uint64_t)bits + (uint64_t)j;
            int64_t S = 0;
            for (int w = 0; w < 3; w++) {
                uint64_t o = orc_splitmix64_at(seed, 3u * c + (uint64_t)w);
                for (int h = 0; h < 4; h++) S += (int64_t)((o >> (16 * h)) & 0xFFFFu);
            }
            int64_t num = S - 393210;                 /* floor division by 16 */
            int64_t fl = num >= 0 ? num / 16 : -((-num + 15) / 16);
            codes[(size_t)r * bits + j] = (uint16_t)(fl + 32768);
        }
}

/* Sign random projections of sparse rows with R stored in two bytes per
 * entry (Section 4.3): bit j of row i = [ sum_e values[e] * r(indices[e], j)
 * >= 0 ], r the decoded value above, the sum in FP64 in row order. */
void orc_srp_sparse_q16(const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                        const uint16_t *Rq, int bits, uint32_t *sig)
{
    int W = bits / 32;
    for (int64_t i = 0; i < N; i++) {
        uint32_t *row = sig + (size_t)i * W;
        memset(row, 0, sizeof(uint32_t) * W);
        for (int j = 0; j < bits; j++) {
            double acc = 0.0;
            for (int64_t e = indptr[i]; e < indptr[i + 1]; e++)
                acc += (double)values[e] * orc_dequantize_gaussian(Rq[(size_t)indices[e] * bits + j]);
            if (acc >= 0.0) row[j / 32] |= 1u << (j % 32);
        }
    }
}

/* The same for dense rows X [N][d] (sum over coordinates 0..d-1 in order).
 * dots (optional, [N][bits]) receives the FP64 sums. */
void orc_srp_dense(const float *X, int64_t N, int d, const float *R, int bits, uint32_t *sig, double *dots)
{
    int W = bits / 32;
    for (int64_t i = 0; i < N; i++) {
        uint32_t *row = sig + (size_t)i * W;
        memset(row, 0, sizeof(uint32_t) * W);
        for (int j = 0; j < bits; j++) {
            double acc = 0.0;
            for (int c = 0; c < d; c++)
                acc += (double)X[(size_t)i * d + c] * (double)R[(size_t)c * bits + j];
            if (dots) dots[(size_t)i * bits + j] = acc;
            if (acc >= 0.0) row[j / 32] |= 1u << (j % 32);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* LSH banding (Section 2): each band b is the concatenation of `rows` hashes  */
/* b*rows .. b*rows+rows-1; objects that agree on a whole band are candidates. */
/* ------------------------------------------------------------------------- */

static int g_kind, g_rows, g_band, g_words;
static const uint32_t *g_sig;

static uint32_t orc_hash_at(const uint32_t *row, int kind, int i)
{
    if (kind == ORC_JACCARD) return row[i];
    return (row[i / 32] >> (i % 32)) & 1u;
}

static int orc_band_cmp(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    const uint32_t *ra = g_sig + (size_t)a * g_words, *rb = g_sig + (size_t)b * g_words;
    for (int i = g_band * g_rows; i < (g_band + 1) * g_rows; i++) {
        uint32_t ha = orc_hash_at(ra, g_kind, i), hb = orc_hash_at(rb, g_kind, i);
        if (ha != hb) return ha < hb ? -1 : 1;
    }
    return a < b ? -1 : (a > b);
}

static int orc_pair_cmp(const void *pa, const void *pb)
{
    const uint32_t *a = (const uint32_t *)pa, *b = (const uint32_t *)pb;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}

/* Writes the distinct candidate pairs (x < y), sorted by (x, y), into
 * out [cap][2] and returns their number (which may exceed cap, in which case
 * only the count is meaningful).  Returns -1 on allocation failure. */
int64_t orc_lsh_candidates(const uint32_t *sig, int64_t N, int sig_words, int kind, int rows, int bands,
                           uint32_t *out, int64_t cap)
{
    uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
    int64_t n_all = 0, cap_all = 1024;
    uint32_t *all = (uint32_t *)malloc(sizeof(uint32_t) * 2 * cap_all);
    if (!ids || !all) { free(ids); free(all); return -1; }
    g_sig = sig; g_kind = kind; g_rows = rows; g_words = sig_words;
    for (int b = 0; b < bands; b++) {
        for (int64_t i = 0; i < N; i++) ids[i] = (uint32_t)i;
        g_band = b;
        qsort(ids, (size_t)N, sizeof(uint32_t), orc_band_cmp);
        int64_t s = 0;
        while (s < N) {
            int64_t e = s + 1;
            while (e < N) {
                /* same band key? compare hashes, ignoring the id tie-break */
                const uint32_t *ra = sig + (size_t)ids[s] * sig_words, *rb = sig + (size_t)ids[e] * sig_words;
                int same = 1;
                for (int i = b * rows; i < (b + 1) * rows; i++)
                    if (orc_hash_at(ra, kind, i) != orc_hash_at(rb, kind, i)) { same = 0; break; }
                if (!same) break;
                e++;
            }
            for (int64_t u = s; u < e; u++)
                for (int64_t v = u + 1; v < e; v++) {
                    if (n_all == cap_all) {
                        cap_all *= 2;
                        uint32_t *nw = (uint32_t *)realloc(all, sizeof(uint32_t) * 2 * cap_all);
                        if (!nw) { free(ids); free(all); return -1; }
                        all = nw;
                    }
                    uint32_t x = ids[u], y = ids[v];
                    all[2 * n_all] = x < y ? x : y;
                    all[2 * n_all + 1] = x < y ? y : x;
                    n_all++;
                }
            s = e;
        }
    }
    qsort(all, (size_t)n_all, 2 * sizeof(uint32_t), orc_pair_cmp);
    int64_t n_out = 0;
    for (int64_t i = 0; i < n_all; i++) {
        if (i > 0 && all[2 * i] == all[2 * i - 2] && all[2 * i + 1] == all[2 * i - 1]) continue;
        if (n_out < cap) { out[2 * n_out] = all[2 * i]; out[2 * n_out + 1] = all[2 * i + 1]; }
        n_out++;
    }
    free(ids);
    free(all);
    return n_out;
}

/* ------------------------------------------------------------------------- */
/* AllPairs-style candidate generation by prefix filtering (the candidate      */
/* generator Section 5.1 pairs with BayesLSH besides LSH: Bayardo, Ma and      */
/* Srikant, "Scaling up all pairs similarity search", WWW 2007).               */
/*                                                                             */
/* Features are ordered by decreasing document frequency (ties: smaller id).   */
/* Walking a row's features in that order, a running bound b grows by          */
/* |x_f| * maxabs_f (cosine; maxabs_f = the largest |weight| of f over all      */
/* rows), or by 1 per element (Jaccard sets); a feature is indexed once b,     */
/* including it, reaches the row's threshold: t - 1e-9 (cosine), or            */
/* alpha = ceil(t |x| - 1e-9) elements (Jaccard: J(x,y) >= t needs            */
/* |x n y| >= t |x|).  The unindexed prefix U(x) then bounds what it can add    */
/* to any similarity: below t (cosine, sum over U of x_f y_f <= sum |x_f|       */
/* maxabs_f), or fewer than alpha common elements (Jaccard), so a pair         */
/* reaching t shares an indexed feature of x.  The cosine bound is summed in    */
/* fixed point, independently of the order of the terms: each term is the      */
/* exact FP64 product |x_f| maxabs_f scaled by 2^48 and rounded to an integer  */
/* (capped at 2^50, far above any threshold), and the threshold is             */
/* ceil((t - 1e-9) 2^48); the rounding (below 2^-49 per term) is far inside    */
/* the 1e-9 margin.  Rows of more than 4096 elements index every feature.      */
/* Candidates: the distinct pairs (x, y), x < y, with an indexed feature of x  */
/* present in y, sorted by (x, y).                                             */
/* ------------------------------------------------------------------------- */

#define ORC_AP_LONG_ROW 4096

static const int64_t *g_ap_df;

static int orc_ap_cmp(const void *pa, const void *pb)
{
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    if (g_ap_df[a] != g_ap_df[b]) return g_ap_df[a] > g_ap_df[b] ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* indexed[e] = 1 if nonzero e's feature is an indexed feature of its row.
 * values may be NULL for sets (kind == ORC_JACCARD).  Returns 0, or -1 on
 * allocation failure. */
int orc_allpairs_indexed(const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                         int64_t dim, double t, int kind, uint8_t *indexed)
{
    int64_t *df = (int64_t *)calloc((size_t)(dim > 0 ? dim : 1), sizeof(int64_t));
    double *maxabs = (double *)calloc((size_t)(dim > 0 ? dim : 1), sizeof(double));
    uint32_t *feat = (uint32_t *)malloc(sizeof(uint32_t) * ORC_AP_LONG_ROW);
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (dim > 0 ? dim : 1));
    if (!df || !maxabs || !feat || !pos) { free(df); free(maxabs); free(feat); free(pos); return -1; }
    int64_t nnz = indptr[N];
    for (int64_t e = 0; e < nnz; e++) {
        df[indices[e]]++;
        if (kind == ORC_COSINE) {
            double a = fabs((double)values[e]);
            if (a > maxabs[indices[e]]) maxabs[indices[e]] = a;
        }
    }
    g_ap_df = df;
    for (int64_t x = 0; x < N; x++) {
        int64_t s = indptr[x], n = indptr[x + 1] - s;
        if (n > ORC_AP_LONG_ROW) {
            for (int64_t e = s; e < s + n; e++) indexed[e] = 1;
            continue;
        }
        for (int64_t i = 0; i < n; i++) {
            feat[i] = indices[s + i];
            pos[indices[s + i]] = s + i;
        }
        qsort(feat, (size_t)n, sizeof(uint32_t), orc_ap_cmp);
        const double two48 = 281474976710656.0;
        const int64_t thr = (int64_t)ceil((t - 1e-9) * two48);
        const double alpha = ceil(t * (double)n - 1e-9);
        int64_t b = 0;
        for (int64_t i = 0; i < n; i++) {
            int64_t e = pos[feat[i]];
            if (kind == ORC_COSINE) {
                int64_t w = llrint(fabs((double)values[e]) * maxabs[feat[i]] * two48);
                if (w > ((int64_t)1 << 50)) w = (int64_t)1 << 50;
                b += w;
                indexed[e] = b >= thr;
            } else {
                b += 1;
                indexed[e] = (double)b >= alpha;
            }
        }
    }
    free(df); free(maxabs); free(feat); free(pos);
    return 0;
}

/* The candidate pairs (see above) into out [cap][2], sorted by (x, y); returns
 * their number (which may exceed cap: only the count is then meaningful), or
 * -1 on allocation failure. */
int64_t orc_allpairs_candidates(const int64_t *indptr, const uint32_t *indices, const float *values, int64_t N,
                                int64_t dim, double t, int kind, uint32_t *out, int64_t cap)
{
    int64_t nnz = indptr[N];
    uint8_t *ix = (uint8_t *)malloc((size_t)(nnz > 0 ? nnz : 1));
    int64_t *start = (int64_t *)calloc((size_t)dim + 1, sizeof(int64_t));
    if (!ix || !start || orc_allpairs_indexed(indptr, indices, values, N, dim, t, kind, ix) != 0) {
        free(ix); free(start); return -1;
    }
    /* inverted lists of the indexed features: rows in increasing order */
    for (int64_t e = 0; e < nnz; e++)
        if (ix[e]) start[indices[e] + 1]++;
    for (int64_t f = 0; f < dim; f++) start[f + 1] += start[f];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (dim > 0 ? dim : 1));
    uint32_t *rows = (uint32_t *)malloc(sizeof(uint32_t) * (start[dim] > 0 ? start[dim] : 1));
    uint32_t *seen = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
    uint32_t *cand = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
    if (!fill || !rows || !seen || !cand) {
        free(ix); free(start); free(fill); free(rows); free(seen); free(cand); return -1;
    }
    for (int64_t f = 0; f < dim; f++) fill[f] = start[f];
    for (int64_t x = 0; x < N; x++)
        for (int64_t e = indptr[x]; e < indptr[x + 1]; e++)
            if (ix[e]) rows[fill[indices[e]]++] = (uint32_t)x;
    for (int64_t x = 0; x < N; x++) seen[x] = UINT32_MAX;
    int64_t n_all = 0, cap_all = 1024;
    uint32_t *all = (uint32_t *)malloc(sizeof(uint32_t) * 2 * cap_all);
    if (!all) { free(ix); free(start); free(fill); free(rows); free(seen); free(cand); return -1; }
    for (int64_t y = 0; y < N; y++) {
        int64_t nc = 0;
        for (int64_t e = indptr[y]; e < indptr[y + 1]; e++) {
            uint32_t f = indices[e];
            for (int64_t i = start[f]; i < start[f + 1] && rows[i] < (uint32_t)y; i++) {
                uint32_t x = rows[i];
                if (seen[x] != (uint32_t)y) { seen[x] = (uint32_t)y; cand[nc++] = x; }
            }
        }
        for (int64_t i = 0; i < nc; i++) {
            if (n_all == cap_all) {
                cap_all *= 2;
                uint32_t *nw = (uint32_t *)realloc(all, sizeof(uint32_t) * 2 * cap_all);
                if (!nw) { free(ix); free(start); free(fill); free(rows); free(seen); free(cand); free(all); return -1; }
                all = nw;
            }
            all[2 * n_all] = cand[i];
            all[2 * n_all + 1] = (uint32_t)y;
            n_all++;
        }
    }
    qsort(all, (size_t)n_all, 2 * sizeof(uint32_t), orc_pair_cmp);
    for (int64_t i = 0; i < n_all && i < cap; i++) { out[2 * i] = all[2 * i]; out[2 * i + 1] = all[2 * i + 1]; }
    free(ix); free(start); free(fill); free(rows); free(seen); free(cand); free(all);
    return n_all;
}

/* ------------------------------------------------------------------------- */
/* Output: the retained pair indices in input order, and the histogram of the  */
/* chunk at which each pair stopped (the paper's "candidates left vs hashes").  */
/* ------------------------------------------------------------------------- */

int64_t orc_compact(const uint8_t *status, int64_t P, uint32_t keep_mask, int64_t *out_idx)
{
    int64_t n = 0;
    for (int64_t q = 0; q < P; q++)
        if (status[q] < 32 && ((keep_mask >> status[q]) & 1u)) out_idx[n++] = q;
    return n;
}

void orc_stop_hist(const uint16_t *n_used, int64_t P, int k, int L, uint64_t *hist)
{
    memset(hist, 0, sizeof(uint64_t) * L);
    for (int64_t q = 0; q < P; q++) {
        int j = n_used[q] / k - 1;
        if (j >= 0 && j < L) hist[j]++;
    }
}

/* ------------------------------------------------------------------------- */
/* Section 3: the maximum-likelihood estimate over the first n hashes, and the */
/* Section 2 output rule (keep iff the estimate exceeds t).                    */
/* ------------------------------------------------------------------------- */
void orc_estimate_mle(int kind, int n, double t, const uint32_t *pairs, int64_t P, const uint32_t *sig,
                      int sig_words, uint16_t *m_out, double *est, uint8_t *keep)
{
    for (int64_t q = 0; q < P; q++) {
        const uint32_t *sx = sig + (size_t)pairs[2 * q] * sig_words, *sy = sig + (size_t)pairs[2 * q + 1] * sig_words;
        int m = orc_chunk_matches(kind, sx, sy, 0, n);
        double r = (double)m / (double)n;
        double e = kind == ORC_JACCARD ? r : cos(ORC_PI * (1.0 - r));
        m_out[q] = (uint16_t)m;
        est[q] = e;
        keep[q] = e > t;
    }
}

/* Section 4.1 "Choice of prior": method-of-moments Beta from r similarities.
 * out = {mean, variance (divisor r), alpha, beta, fallback}; no Beta fits
 * when the variance is 0 or at least mean (1 - mean): then Beta(1,1). */
void orc_fit_beta_prior(const double *sims, int64_t r, double *out)
{
    double s = 0.0;
    for (int64_t i = 0; i < r; i++) s += sims[i];
    double mean = s / (double)r;
    double v = 0.0;
    for (int64_t i = 0; i < r; i++) v += (sims[i] - mean) * (sims[i] - mean);
    double var = v / (double)r;
    out[0] = mean; out[1] = var; out[2] = 1.0; out[3] = 1.0; out[4] = 1.0;
    if (var > 0.0 && var < mean * (1.0 - mean)) {
        double k = mean * (1.0 - mean) / var - 1.0;
        out[2] = mean * k;
        out[3] = (1.0 - mean) * k;
        out[4] = 0.0;
    }
}
