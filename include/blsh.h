/*
 * blsh.h -- C ABI of libblsh: BayesLSH candidate verification on one GB300
 * (sm_103a).
 *
 * The method is BayesLSH (Satuluri & Parthasarathy, "Bayesian Locality
 * Sensitive Hashing for Fast Similarity Search").  Given candidate pairs, the
 * library compares the pairs' LSH signatures k hashes at a time, prunes a pair
 * as soon as Pr[S >= t | m of n hashes agree] < eps, and stops with the
 * posterior-mode estimate once Pr[|S - S^| < delta | m, n] >= 1 - gamma
 * (Algorithm 1).  BayesLSH-Lite (Algorithm 2) prunes the same way with at most
 * h hashes and computes the exact similarity of the survivors.  Around that
 * sit the producers of the signatures (minhash, Section 4.1; sign random
 * projections, Section 4.2), LSH banding (Section 2) and the inference tables
 * (Section 4.3).
 *
 * Conventions shared by every entry point:
 *   - Every array argument is a DEVICE pointer to memory the caller owns
 *     (allocated with cudaMalloc, PyTorch, ...), unless its comment says
 *     "host".  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Calls are asynchronous on that stream: they enqueue work and
 *     return.  Outputs are valid once the stream has reached that point.
 *   - Every call returns an int status (BLSH_OK = 0 or a BLSH_E* code).
 *     Argument errors are detected on the host and nothing is enqueued.
 *     Errors the GPU detects (a pair naming an object index >= N, an output
 *     larger than its capacity) are recorded in the context and returned by
 *     the next blsh_status() call.  No kernel traps or asserts.
 *   - Hot calls (hashing, banding, verify, compaction) allocate no memory
 *     and never synchronise the stream; blsh_ctx_create, blsh_ctx_reserve
 *     and blsh_tables_build allocate (and synchronise) once, at set-up.
 *   - Calls that share a context must not overlap in time on different
 *     streams: the context owns a small scratch area (work counters, the
 *     device error word) that every call reuses.
 *   - Signature rows are 16-byte aligned: `sig` is 16-byte aligned and
 *     `sig_words` is a multiple of 4.
 */
#ifndef BLSH_H
#define BLSH_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BLSH_API __attribute__((visibility("default")))
#else
#define BLSH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define BLSH_OK 0
#define BLSH_EINVAL 1   /* invalid scalar argument, NULL or misaligned pointer */
#define BLSH_ERANGE 2   /* a pair names an object index >= N (device-detected) */
#define BLSH_ETRUNC 3   /* an output or workspace is smaller than needed */
#define BLSH_ENOMEM 4   /* a context or table allocation failed */
#define BLSH_EDEVICE 5  /* a CUDA runtime call failed (message in blsh_last_error) */
#define BLSH_ENUMERIC 6 /* a table value is non-finite or not monotone in m */
#define BLSH_ESIZE 7    /* the problem is larger than a fixed-size scratch array of the library */

/* ---- similarity kinds (Sections 4.1 and 4.2) ---------------------------- */
#define BLSH_JACCARD 0  /* uint32 minhash values, one per hash */
#define BLSH_COSINE 1   /* sign bits: hash j is bit (j % 32) of word (j / 32) */

/* ---- per-pair outcomes (uint8 status arrays) ---------------------------- */
#define BLSH_PRUNED 0         /* Pr[S >= t | M(m,n)] < eps after the last chunk */
#define BLSH_ACCEPT 1         /* Pr[|S - S^| < delta | M(m,n)] >= 1 - gamma */
#define BLSH_ACCEPT_AT_MAX 2  /* n reached n_max unpruned, not concentrated: kept */
#define BLSH_LITE_REJECT 3    /* Algorithm 2: unpruned, exact similarity <= t */
#define BLSH_LITE_ACCEPT 4    /* Algorithm 2: unpruned, exact similarity > t */
#define BLSH_BAD_PAIR 255     /* the pair names an object >= N; nothing computed */

typedef struct blsh_ctx blsh_ctx;
typedef struct blsh_tables blsh_tables;

/* Parameters of Algorithms 1 and 2 (inputs t, eps, delta, gamma, h; the
 * chunk size k of "compare hashes n to n+k"; Section 5.1 uses k = 32,
 * eps = gamma = 0.03, delta = 0.05, h = 64 Jaccard / 128 cosine) and the
 * Beta(alpha, beta) prior of Section 4.1 (ignored for cosine, whose prior is
 * uniform on r in [0.5, 1], Section 4.2). */
typedef struct blsh_params {
    int32_t kind;   /* BLSH_JACCARD or BLSH_COSINE */
    int32_t k;      /* hashes per chunk: 32, 64 or 128 */
    int32_t n_max;  /* most hashes compared per pair: a multiple of k, <= 4096 */
    int32_t h;      /* Lite: hashes used for pruning, a multiple of k, <= n_max */
    double t;       /* similarity threshold, in (0, 1) */
    double eps;     /* recall parameter, in (0, 1) */
    double delta;   /* accuracy half-width, in (0, 1) */
    double gamma;   /* accuracy failure probability, in (0, 1) */
    double alpha;   /* Jaccard prior Beta(alpha, beta), both > 0 */
    double beta;
} blsh_params;

/* Launch shape of the verification kernel.  Only speed depends on it; the
 * outputs are identical for every valid plan. */
#define BLSH_PLAN_PLAIN 0       /* one launch, one lane group per pair, no refill */
#define BLSH_PLAN_PERSISTENT 1  /* one CTA wave; warps take pairs from an atomic
                                 * work counter and refill lanes as pairs stop */
typedef struct blsh_plan {
    int32_t mode;           /* BLSH_PLAN_PLAIN or BLSH_PLAN_PERSISTENT */
    int32_t group;          /* lanes per pair: 1 (cosine, Jaccard) or 4, 8, 16, 32 (Jaccard) */
    int32_t block;          /* threads per CTA: 128, 256 or 512 */
    int32_t grab;           /* persistent: pairs a warp takes per counter grab (multiple of 32/group) */
    int32_t ctas_per_sm;    /* persistent: CTAs per SM in the single wave (0 = as many as fit) */
} blsh_plan;

/* ---- library and context ------------------------------------------------ */

BLSH_API const char *blsh_version(void);
BLSH_API const char *blsh_strerror(int code);

/* Creates a context bound to CUDA device `device` (made current for the
 * call).  Allocates the context's scratch area (a few KB of device memory).
 * *out receives the handle.  BLSH_EDEVICE if the device does not exist or is
 * not sm_103. */
BLSH_API int blsh_ctx_create(blsh_ctx **out, int device);
BLSH_API int blsh_ctx_destroy(blsh_ctx *ctx);

/* Reserves the context's per-object buffers for signature sets of up to
 * max_objects rows, so that the hot calls need no allocation: the
 * first-words plane of the verification calls (16 bytes per object; words
 * 0..3 of every cosine signature row, Algorithm 1's first step) and Lite's
 * squared-norm buffer (8 bytes per object; Algorithm 2's exact cosine).  A
 * set-up call: it synchronises the device, frees the previous buffers and
 * allocates the new ones (it never shrinks them; 0 releases them).  A
 * verification call over more objects than were reserved takes the slower
 * route with the same outputs (rows read directly, norms formed per pair).
 * BLSH_EINVAL for max_objects outside 0..2^32, BLSH_ENOMEM if the
 * allocation fails.  blsh_ctx_reserved returns the reservation (-1 for a
 * NULL context). */
BLSH_API int blsh_ctx_reserve(blsh_ctx *ctx, int64_t max_objects);
BLSH_API int64_t blsh_ctx_reserved(const blsh_ctx *ctx);

/* Text of the last host-side error on this context (static storage owned by
 * the context, valid until the next call). */
BLSH_API const char *blsh_last_error(const blsh_ctx *ctx);

/* Synchronises `stream`, then returns and clears the first error the GPU
 * recorded since the previous blsh_status (BLSH_ERANGE, BLSH_ETRUNC,
 * BLSH_ENUMERIC) or
 * BLSH_EDEVICE if the stream reported a CUDA error; BLSH_OK otherwise.
 * If `counters` (host, 4 x uint64) is not NULL it receives the running
 * totals since the last call: [0] pairs with an index >= N, [1] outputs
 * truncated, [2] SRP signs rechecked at higher precision, [3] SRP dot
 * products that were exactly zero; they are then reset. */
BLSH_API int blsh_status(blsh_ctx *ctx, void *stream, uint64_t *counters);

/* Number of kernels this context has launched so far (host-side count of
 * every launch the library enqueued through it; replays of a captured CUDA
 * graph are not counted).  -1 for a NULL context. */
BLSH_API int64_t blsh_launch_count(const blsh_ctx *ctx);

/* Per-launch device timing, for profiling a step from the host without a
 * profiler.  blsh_timing_begin allocates 2 * max_launches CUDA events and
 * switches recording on: from then on every kernel the library launches
 * through `ctx` (up to max_launches of them) is bracketed by a start and a
 * stop event recorded on the launch's stream.  Launches enqueued while their
 * stream is being captured into a CUDA graph are not recorded.  Recording
 * costs two event records per launch; it is off by default.  One host thread
 * at a time may launch through a context that is recording.
 * blsh_timing_end waits for the recorded stop events, writes up to `max`
 * records in launch order -- names[i] = the kernel's name (a static string
 * owned by the library; a multi-launch helper such as the exclusive scan
 * is one record), ms[i] = its device time in milliseconds -- sets *n to the
 * number written, releases the events and switches recording off.
 * Errors: BLSH_EINVAL for max_launches outside 1..65536 or missing outputs;
 * BLSH_EDEVICE if an event could not be created or read (recording is then
 * off and the records are dropped). */
BLSH_API int blsh_timing_begin(blsh_ctx *ctx, int32_t max_launches);
BLSH_API int blsh_timing_end(blsh_ctx *ctx, int32_t max, const char **names, float *ms, int32_t *n);

/* ---- Section 4.3 tables -------------------------------------------------- */

/* Builds, in FP64 on the GPU, for n_j = (j+1) k, j = 0 .. n_max/k - 1:
 *   minMatches[j] = the smallest m with Pr[S >= t | M(m, n_j)] >= eps
 *                   (n_j + 1 if none), Section 4.3 "Pre-computation of
 *                   minimum matches";
 *   conc[j][m]    = [Pr[|S - S^| < delta | M(m, n_j)] >= 1 - gamma] for
 *                   m >= minMatches[j] (0 below), Section 4.3 "Cache results
 *                   of inference";
 *   est[j][m]     = S^(m, n_j), the posterior mode (Equation map), as float.
 * Jaccard uses the Beta(m+alpha, n-m+beta) posterior (Section 4.1), cosine
 * the posterior of r on [0.5, 1] mapped by r2c (Section 4.2).
 * Allocates the tables' device memory (freed by blsh_tables_destroy) and
 * synchronises `stream` before returning.  BLSH_EINVAL for parameters out
 * of range; BLSH_ENUMERIC if a probability is non-finite or Pr[S>=t|M] is
 * not monotone in m (the table is still returned). */
BLSH_API int blsh_tables_build(blsh_ctx *ctx, const blsh_params *p, blsh_tables **out, void *stream);
BLSH_API int blsh_tables_destroy(blsh_tables *tab);

/* Host copies of the tables, for checks.  Any pointer may be NULL.
 * levels = n_max / k.  min_matches: int32 [levels]; conc: uint8
 * [levels][n_max+1]; est: float [levels][n_max+1]; prune_prob / conc_prob:
 * double [levels][n_max+1] (conc_prob is NaN where it was not evaluated).
 * near_ties: how many evaluated probabilities lie within 1e-9 of their
 * threshold (eps or 1 - gamma). */
BLSH_API int blsh_tables_download(const blsh_tables *tab, blsh_params *params, int32_t *levels, int32_t *near_ties,
                         int32_t *min_matches, uint8_t *conc, float *est, double *prune_prob,
                         double *conc_prob);

/* ---- signatures ---------------------------------------------------------- */

/* Minhash signatures (Section 4.1, "LSH family"; the family is
 * h_j(x) = (a_j x + b_j) mod (2^31 - 1)):
 *   sig[i][j] = min over x in row i of h_j(x),  j < n_hashes,
 * computed exactly in 64-bit integers.  Rows are CSR: indptr int64 [N+1],
 * indices uint32 [nnz] (elements < 2^31 - 1).  a, b: uint32 [n_hashes] with
 * 1 <= a_j < 2^31 - 1 and b_j < 2^31 - 1.  sig: uint32 [N][n_hashes]; an
 * empty row gives 0xFFFFFFFF.  n_hashes must be a positive multiple of 32. */
BLSH_API int blsh_minhash(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, int64_t N, int32_t n_hashes,
                 const uint32_t *a, const uint32_t *b, uint32_t *sig, void *stream);

/* Sign random projections of sparse rows (Section 4.2, "LSH family"):
 * bit j of row i = [ sum_e values_e * R[indices_e][j] >= 0 ].  R: float
 * [dim][bits], row-major.  sig: uint32 [N][bits/32], bit j at word j/32,
 * position j%32.  The sum is taken in FP32 with a rigorous error bound; a
 * sign the bound cannot decide is recomputed in FP64 in row order, so every
 * bit equals the sign of the FP64 row-order sum.  bits: a positive multiple
 * of 32, at most 4096. */
BLSH_API int blsh_srp_sparse(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices, const float *values,
                    int64_t N, const float *R, int64_t dim, int32_t bits, uint32_t *sig, void *stream);

/* Columns [col_begin, col_begin + col_count) of blsh_srp_sparse's signatures
 * (the same bits), for the rows with row_mask[row] != 0 (uint8 [N], device;
 * NULL: every row); other rows and columns of sig are left as they were.
 * This is how points are hashed only as many times as necessary (Section 3:
 * the hashes beyond those the candidate generation and the first chunks of
 * verification read are computed only for the points whose pairs are still
 * undecided).  bits, col_begin and col_count multiples of 128; R 16-byte
 * aligned.  Errors as blsh_srp_sparse. */
BLSH_API int blsh_srp_sparse_cols(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                  const float *values, int64_t N, const float *R, int64_t dim, int32_t bits,
                                  int32_t col_begin, int32_t col_count, const uint8_t *row_mask, uint32_t *sig,
                                  void *stream);

/* Two-byte storage of the Gaussian projection matrix (Section 4.3, "Cheaper
 * storage of hash functions"): q[i] = floor((x[i] + 8) * 2^16 / 16), the code
 * of a sample assumed to lie in (-8, 8); a code q stands for q * 2^-12 - 8.
 * Codes outside [0, 65535] (x < -8, x >= 8) and NaN inputs are clamped (NaN
 * to 0) and make the next blsh_status return BLSH_ENUMERIC.  x: n floats,
 * q: n uint16 (device, caller-owned).  Asynchronous on `stream`. */
BLSH_API int blsh_quantize_gaussian(blsh_ctx *ctx, const float *x, int64_t n, uint16_t *q, void *stream);

/* The two-byte codes of a Gaussian R [dim][bits] generated from a counter,
 * so that an R too large to store or to copy (a 2^24-term vocabulary at
 * 2,048 bits is 68.7 GB of codes) is made on the device: entry
 * c = t * bits + j sums the twelve 16-bit pieces of SplitMix64 outputs 3c,
 * 3c + 1 and 3c + 2 of the stream `seed` (output k = the SplitMix64
 * finaliser of seed + (k + 1) * 0x9E3779B97F4A7C15; Steele, Lea and Flood,
 * OOPSLA 2014), S, whose (S - 393210) / 65536 is a standard normal to the
 * accuracy of the Irwin-Hall sum of twelve uniforms (truncated at +-6); the
 * code is that value's Section 4.3 encoding, floor((S - 393210) / 16) +
 * 32768, in [8192, 57343].  codes: device uint16 [dim][bits], 16-byte
 * aligned; bits a positive multiple of 8.  The codes feed
 * blsh_srp_sparse_q16. */
BLSH_API int blsh_gaussian_codes(blsh_ctx *ctx, uint64_t seed, int64_t dim, int32_t bits, uint16_t *codes,
                                 void *stream);

/* blsh_srp_sparse with R stored as two-byte codes Rq [dim][bits] (uint16,
 * row-major, from blsh_quantize_gaussian): bit j of row i = [ sum_e
 * values[e] * (Rq[indices[e]][j] * 2^-12 - 8) >= 0 ], each bit equal to the
 * sign of the FP64 sum in row order (the decoded values and the products are
 * exact in FP64).  Half the bytes of the float form are gathered per
 * nonzero.  bits: a positive multiple of 32, at most 4096 (multiples of 256
 * with Rq 16-byte aligned take the 16-byte load path).  Errors as
 * blsh_srp_sparse. */
BLSH_API int blsh_srp_sparse_q16(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                 const float *values, int64_t N, const uint16_t *Rq, int64_t dim, int32_t bits,
                                 uint32_t *sig, void *stream);

/* Columns [col_begin, col_begin + col_count) of blsh_srp_sparse_q16's
 * signatures for the rows with row_mask[row] != 0 (NULL: every row), as
 * blsh_srp_sparse_cols does for a float R.  bits, col_begin and col_count
 * multiples of 128; Rq 8-byte aligned.  Errors as blsh_srp_sparse_q16. */
BLSH_API int blsh_srp_sparse_q16_cols(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                      const float *values, int64_t N, const uint16_t *Rq, int64_t dim, int32_t bits,
                                      int32_t col_begin, int32_t col_count, const uint8_t *row_mask, uint32_t *sig,
                                      void *stream);

/* Sign random projections of dense rows X [N][d] (float, row-major) with
 * R [d][bits] (float, row-major), Section 4.2: bit j of row i =
 * [ sum_c X[i][c] R[c][j] >= 0 ], each bit equal to the sign of the FP64 sum
 * over c = 0..d-1 in order.
 * With a workspace (blsh_srp_dense_workspace bytes, 256-byte aligned; nonzero
 * when d is a multiple of 64 and bits a multiple of 256) the projection runs
 * on the tensor cores: X and R are split into BF16 pairs hi + lo and
 * hi*hi + hi*lo + lo*hi is accumulated in FP32; every product with
 * |p| <= margin * |x_i| * |r_j| is recomputed in FP32 with a rigorous bound
 * and, where that cannot decide it, in FP64.  margin is raised to the
 * tensor-core error bound (about (2^-14 + 3 d 2^-22) * 1.25) when smaller;
 * pass 0 for that bound.  Without a workspace (or for other shapes) the
 * projection runs in FP32 on the CUDA cores with the same rechecks.
 * X and R 16-byte aligned; bits a multiple of 32, at most 4096. */
BLSH_API int blsh_srp_dense_workspace(int64_t N, int32_t d, int32_t bits, size_t *bytes);
BLSH_API int blsh_srp_dense(blsh_ctx *ctx, const float *X, int64_t N, int32_t d, const float *R, int32_t bits,
                            float margin, uint32_t *sig, void *workspace, size_t workspace_bytes, void *stream);

/* ---- candidate generation (Section 2, "Candidate generation via LSH") ---- */

/* Workspace bytes blsh_lsh_candidates takes for these sizes.  The last
 * 64 * N * bands of them are a keep record: the emission's count pass notes
 * there which pairs it keeps, so that its write pass writes them without
 * testing them again.  A workspace smaller by up to that much is accepted;
 * the positions the record then does not cover are tested again (same
 * output, more time), and bytes beyond the size returned extend the record. */
BLSH_API int blsh_lsh_candidates_workspace(int64_t N, int32_t kind, int32_t rows, int32_t bands, size_t *bytes);

/* Band b of object i is its hashes b*rows .. b*rows+rows-1; objects that
 * agree on every hash of at least one band become a candidate pair.  Writes
 * each distinct pair once as (x, y) with x < y, in band order (a pair is
 * written for the first band it collides in), into pairs uint32 [cap][2],
 * and the number of distinct pairs into *n_pairs (device int64).  If that
 * number exceeds cap only the first cap pairs are written and blsh_status
 * reports BLSH_ETRUNC.  Band keys are compared in full (no hash collisions
 * can merge buckets).  Cosine: rows <= 32.  workspace: device, 256-byte
 * aligned, blsh_lsh_candidates_workspace() bytes less at most the keep
 * record's 64 * N * bands (BLSH_ETRUNC below that). */
BLSH_API int blsh_lsh_candidates(blsh_ctx *ctx, const uint32_t *sig, int64_t N, int32_t sig_words, int32_t kind,
                        int32_t rows, int32_t bands, uint32_t *pairs, int64_t cap, int64_t *n_pairs,
                        void *workspace, size_t workspace_bytes, void *stream);

/* Candidate generation by prefix filtering, the AllPairs method (Bayardo, Ma
 * and Srikant, WWW 2007) that Section 5.1 pairs with BayesLSH as the other
 * source of candidates.  Features are ordered by decreasing document
 * frequency (ties: smaller id); walking a row's features in that order, a
 * running bound grows by |x_f| * maxabs_f (cosine: maxabs_f = the largest
 * |weight| of f over all rows; the sum in fixed point, each exact product
 * scaled by 2^48 and rounded to an integer, capped at 2^50) or by 1 (sets),
 * and a feature is indexed once the bound including it reaches the row's
 * threshold (cosine: ceil((t - 1e-9) 2^48); sets: ceil(t |x| - 1e-9)
 * elements, since J >= t needs |x n y| >= t |x|).  Rows of more than 4096
 * elements index every feature.  The candidates are the distinct pairs
 * (x, y), x < y, such that some indexed feature of x occurs in y; every
 * pair whose cosine (non-negative weights) or Jaccard similarity reaches t
 * is among them.  They are written to pairs uint32 [cap][2] in increasing
 * order of (x, y), their number to *n_pairs (device int64).
 * Rows: indptr int64 [N+1] (indptr[N] = nnz, passed from the host too),
 * indices uint32 sorted and distinct within a row, features < dim; values
 * float [nnz] for cosine, NULL for sets.
 * The pairs are formed by sorting the candidate keys of every (row, shared
 * indexed feature), duplicates included: max_dups is the capacity of that
 * key buffer (a part of the workspace).  A call with cap = 0 is a count-only
 * call: it writes the number of such keys to *n_dups (device int64, may be
 * NULL otherwise) and 0 to *n_pairs; size max_dups from it and call again.
 * If the keys exceed max_dups, *n_pairs is 0 and blsh_status reports
 * BLSH_ETRUNC; if the distinct pairs exceed cap, only cap are written and
 * blsh_status reports BLSH_ETRUNC.  workspace: blsh_allpairs_workspace(N,
 * nnz, dim, max_dups) bytes (max_dups = 0 for a count-only call), 256-byte
 * aligned.  Asynchronous on `stream` (no host synchronisation). */
BLSH_API int blsh_allpairs_workspace(int64_t N, int64_t nnz, int64_t dim, int64_t max_dups, size_t *bytes);
BLSH_API int blsh_allpairs_candidates(blsh_ctx *ctx, const int64_t *indptr, const uint32_t *indices,
                                      const float *values, int64_t N, int64_t nnz, int64_t dim, double t,
                                      int32_t kind,
                                      int64_t max_dups, uint32_t *pairs, int64_t cap, int64_t *n_pairs,
                                      int64_t *n_dups, void *workspace, size_t workspace_bytes, void *stream);

/* ---- verification: Algorithms 1 and 2 ------------------------------------ */

/* Algorithm 1 (BayesLSH) for pairs uint32 [P][2] (x, y) over signatures
 * sig uint32 [N][sig_words].  Per pair, chunk j compares hashes j*k ..
 * j*k+k-1 (minhash equality, or XOR + popcount of sign bits) and adds the
 * agreements to m; after it, with n = (j+1) k:
 *   m < minMatches[j]            -> BLSH_PRUNED,
 *   conc[j][m]                   -> BLSH_ACCEPT,
 *   n == n_max                   -> BLSH_ACCEPT_AT_MAX.
 * Outputs per pair: status uint8 [P]; n_used uint16 [P] (hashes compared);
 * m uint16 [P] (agreements); est float [P]: S^(m, n) at the stop for kept
 * pairs (Algorithm 1 outputs an estimate only with a kept pair); the entries
 * of pruned pairs and of BLSH_BAD_PAIR pairs are not written.  n_used, m,
 * est may be NULL.  stop_hist: uint64 [n_max/k] or NULL; entry j counts
 * the pairs that stopped after chunk j (the call overwrites it).
 * P_dev: NULL, or a device int64 holding the pair count; the kernel then
 * reads the count there (clamped to P, which acts as the capacity), so the
 * call can follow a producer on the same stream without a host sync.
 * Uses the plan blsh_autotune stored for these tables, else a default.
 * Cosine signature sets larger than 64 MB (N * sig_words * 4 bytes) with
 * sig_words > 4 and N <= blsh_ctx_reserved(ctx): the call first copies words
 * 0..3 of every row (the first 128 hashes) into the context's plane of N
 * uint4, which stays in L2, and every pair's first step reads them there;
 * with N above the reservation each
 * pair reads its rows (same outputs).  The call allocates nothing and does
 * not synchronise, so it can be captured into a CUDA graph.  This holds for
 * every verification entry point below. */
BLSH_API int blsh_verify(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P, const int64_t *P_dev,
                const uint32_t *sig, int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used,
                uint16_t *m, float *est, uint64_t *stop_hist, void *stream);

/* Lazy hashing (Section 3: each point is hashed only as many times as
 * necessary).  blsh_verify_both_capped is blsh_verify_both reading only the
 * first hash_limit hashes of each signature (a multiple of k, at least h, at
 * most n_max): a pair Algorithm 1 has not decided by then gets status
 * BLSH_NEEDS_HASHES (its n_used and m so far are written, not its estimate,
 * and it is not counted in stop_hist) and sets need[x] = need[y] = 1 (uint8
 * [N], device, cleared by the caller).  Algorithm 2 decides every pair within
 * its h <= hash_limit hashes.  After the remaining hashes of the marked
 * objects are computed (blsh_srp_sparse_cols or blsh_srp_sparse_q16_cols
 * with row_mask = need), blsh_verify_resume finishes
 * the BLSH_NEEDS_HASHES pairs over all n_max hashes and adds their stops to
 * stop_hist (not cleared), leaving every other pair's outputs as they are.
 * Together the two calls give exactly the outputs of blsh_verify_both. */
#define BLSH_NEEDS_HASHES 253
BLSH_API int blsh_verify_both_capped(blsh_ctx *ctx, const blsh_tables *tab, int32_t hash_limit,
                                     const uint32_t *pairs, int64_t P, const int64_t *P_dev, const uint32_t *sig,
                                     int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used, uint16_t *m,
                                     float *est, uint64_t *stop_hist, const int64_t *indptr,
                                     const uint32_t *indices, const float *values, uint8_t *lite_status,
                                     uint16_t *lite_n_used, double *sim, uint8_t *need, void *stream);
BLSH_API int blsh_verify_resume(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                                const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                                uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                                void *stream);

/* Stores `plan` as the launch plan blsh_verify, blsh_verify_lite and
 * blsh_verify_both use for these tables (what blsh_autotune does with the
 * plan it finds).  BLSH_EINVAL for a plan invalid for the tables' kind and k. */
BLSH_API int blsh_set_plan(blsh_ctx *ctx, const blsh_tables *tab, const blsh_plan *plan);

/* The same with an explicit launch plan. */
BLSH_API int blsh_verify_plan(blsh_ctx *ctx, const blsh_tables *tab, const blsh_plan *plan, const uint32_t *pairs,
                     int64_t P, const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                     uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                     void *stream);

/* Algorithm 2 (BayesLSH-Lite): the pruning loop of Algorithm 1 limited to
 * h = tab's params.h hashes, without the concentration test; a pair that is
 * not pruned gets its exact similarity from its rows, by a merge of the
 * sorted index lists: Jaccard |A n B| / |A u B| (values == NULL), or cosine
 * (values != NULL) as D / sqrt(Nx Ny) where D, Nx, Ny are sums of the FP64
 * products x_i y_i, x_i^2, y_i^2 each rounded to a multiple of 2^-60 and
 * added in int64 (independent of summation order; rows need squared norm
 * < 4).  status: BLSH_PRUNED, BLSH_LITE_ACCEPT (s > t) or BLSH_LITE_REJECT;
 * sim: double [P], written for the pairs that survive pruning (the entries
 * of pruned and bad pairs are not written); n_used uint16 [P] or NULL.
 * Rows: indptr int64 [N+1], indices uint32 sorted ascending within a row,
 * values float or NULL.  Cosine: when the survivors outnumber half the rows
 * and N <= blsh_ctx_reserved(ctx), each row's Nx is formed once per call
 * into the context's int64 [N] norm buffer; otherwise each survivor forms
 * its two sums itself (same bits: the sums are order-independent).
 * Survivors are queued (up to 2^23 per call) and spread over the warps; any
 * beyond the queue are finished by a second pass over the statuses. */
BLSH_API int blsh_verify_lite(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                     const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                     const int64_t *indptr, const uint32_t *indices, const float *values, uint8_t *status,
                     uint16_t *n_used, double *sim, void *stream);

/* Algorithms 1 and 2 over the same candidate pairs in one pass: the outputs
 * of blsh_verify (status, n_used, m, est, stop_hist) and of blsh_verify_lite
 * (lite_status, lite_n_used, sim), identical to the two calls made one after
 * the other, with each pair's indices and signature words read once (Algorithm
 * 2's pruning test over the first h hashes is the test Algorithm 1 makes on
 * them).  Arguments and errors as those two calls; lite_n_used may be NULL. */
BLSH_API int blsh_verify_both(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                              const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                              uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist,
                              const int64_t *indptr, const uint32_t *indices, const float *values,
                              uint8_t *lite_status, uint16_t *lite_n_used, double *sim, void *stream);

/* Times candidate plans on the given inputs (outputs are overwritten) and
 * stores the fastest for `tab` in the context; *best (host) receives it.
 * Synchronises `stream`. */
BLSH_API int blsh_autotune(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P, const uint32_t *sig,
                  int64_t N, int32_t sig_words, uint8_t *status, uint16_t *n_used, uint16_t *m, float *est,
                  blsh_plan *best, void *stream);

/* The batching pattern's tuner: the chunk size k ("compare hashes n to
 * n+k" of Algorithm 1) chosen together with the launch plan.  For each
 * k = ks[i] (32, 64 or 128, dividing params->n_max; 1 to 8 of them) it builds
 * the Section 4.3 tables for *params with that k (Lite's h rounded up to a
 * whole chunk, at most n_max), times every launch plan as blsh_autotune does
 * on the given inputs (outputs are overwritten), and keeps the fastest
 * (tables, plan).  *out receives those tables (destroy them with
 * blsh_tables_destroy), *best (host, may be NULL) the plan, which is also
 * stored for them in the context; ms_per_k (host float [n_ks], may be NULL)
 * the best time per call found for each k.  The decisions of Algorithms 1
 * and 2 depend on k (pairs are tested after every k hashes), so the outputs
 * of later calls are those of the chosen k.  Synchronises `stream`.
 * BLSH_EINVAL for a k outside {32, 64, 128} or not dividing n_max. */
BLSH_API int blsh_autotune_k(blsh_ctx *ctx, const blsh_params *params, const int32_t *ks, int32_t n_ks,
                             const uint32_t *pairs, int64_t P, const uint32_t *sig, int64_t N, int32_t sig_words,
                             uint8_t *status, uint16_t *n_used, uint16_t *m, float *est, blsh_tables **out,
                             blsh_plan *best, float *ms_per_k, void *stream);

/* ---- the classical estimator and the learned prior ------------------------- */

/* The maximum-likelihood estimate of Section 3 over a fixed number of hashes
 * (the "LSH Approx" comparison mode of Section 5.1): for each pair,
 * m = agreements among hashes 0 .. n_hashes-1, est = m / n_hashes (Jaccard)
 * or cos(pi (1 - m / n_hashes)) (cosine), keep = [est > t] (Section 2), decided
 * as m > m_star with m_star the largest m whose estimate is <= t (FP64, on
 * the host).  m uint16 [P], est float [P], keep uint8 [P] (BLSH_BAD_PAIR for
 * a pair naming an object >= N); any may be NULL.  P_dev as in blsh_verify. */
BLSH_API int blsh_estimate_mle(blsh_ctx *ctx, int32_t kind, int32_t n_hashes, double t, const uint32_t *pairs,
                               int64_t P, const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words,
                               uint16_t *m, float *est, uint8_t *keep, void *stream);

/* The learned prior of Section 4.1: exact Jaccard similarities of r sampled
 * candidate pairs (sims, device double [r]), their mean s and population
 * variance v (divisor r), and the method-of-moments Beta:
 *   alpha = s (s (1 - s) / v - 1),  beta = (1 - s) (s (1 - s) / v - 1).
 * out_device (device double [5]) = {s, v, alpha, beta, fallback}; when v is 0
 * or v >= s (1 - s) the moments admit no Beta and the uniform Beta(1,1) is
 * returned with fallback = 1.  If out_host (host double [5]) is not NULL the
 * call synchronises `stream` and copies the result there. */
BLSH_API int blsh_fit_beta_prior(blsh_ctx *ctx, const uint32_t *pairs, int64_t r, const int64_t *indptr,
                                 const uint32_t *indices, int64_t N, double *sims, double *out_device,
                                 double *out_host, void *stream);

/* ---- output (the set O of Algorithms 1 and 2) ----------------------------- */

/* Stable compaction: out_idx int64 [cap] receives, in increasing order, the
 * indices q < P (or < *P_dev) with status[q] < 32 and bit status[q] of
 * keep_mask set; *n_out (device int64) their number.  If it exceeds cap only
 * cap indices are written and blsh_status reports BLSH_ETRUNC. */
BLSH_API int blsh_compact(blsh_ctx *ctx, const uint8_t *status, int64_t P, const int64_t *P_dev, uint32_t keep_mask,
                 int64_t *out_idx, int64_t cap, int64_t *n_out, void *stream);

/* The same stable compaction for callers that cannot allocate device memory
 * (no counterpart in the paper; it exists for how the library is embedded).
 * Some callers cannot call cudaMalloc at all -- code running inside a host
 * application that owns every device allocation through its own memory
 * pool, or a plug-in for which any allocation outside that pool is
 * forbidden -- so they cannot create a blsh_ctx, whose scratch area is
 * allocated.  This entry point takes no context and allocates nothing: its
 * scratch is a fixed array of 16384 int64 (128 KiB) in the library's own
 * device memory, which every GPU that loads the library holds until the
 * process exits.  The caller passes the inputs and outputs, as for
 * blsh_compact: status uint8 [P], out_idx int64 [cap], *n_out (device int64)
 * = the number of kept indices (only the first cap are written; there is no
 * context to report truncation, so compare *n_out with cap).
 *   - P (the capacity when P_dev is given) may be at most 67,108,864
 *     (16384 tiles of 4096 statuses); larger P returns BLSH_ESIZE and
 *     enqueues nothing.  BLSH_EINVAL for bad pointers or sizes,
 *     BLSH_EDEVICE for a CUDA error.
 *   - The array's device address belongs to the CUDA context the library's
 *     module is loaded into.  The first call made in each context (the
 *     device's primary context, a context the caller created, or the new
 *     primary context after cudaDeviceReset) looks that address up
 *     (cudaGetSymbolAddress, with the context current) and remembers it for
 *     the context (the last 64 contexts are remembered).  Make that first
 *     call before any stream capture in the context: a first call made while
 *     its stream is being captured returns BLSH_EDEVICE and enqueues
 *     nothing.
 *   - Launch errors are taken from each launch's own return code: an error
 *     left on the calling thread by earlier work is neither returned by this
 *     call nor cleared.
 *   - Every call reuses the same array, which keeps the last call's
 *     contents; each call overwrites every entry it reads, so nothing needs
 *     clearing.  Calls that overlap on the GPU (on different streams, or
 *     from different threads) race on the array and give wrong results:
 *     serialise them. */
BLSH_API int blsh_compact_noalloc(const uint8_t *status, int64_t P, const int64_t *P_dev, uint32_t keep_mask,
                                  int64_t *out_idx, int64_t cap, int64_t *n_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BLSH_H */
