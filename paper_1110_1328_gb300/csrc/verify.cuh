// verify.cuh -- the chunked verification loop of Algorithm 1 (BayesLSH) and
// the pruning loop of Algorithm 2 (BayesLSH-Lite), shared by verify.cu and
// lite.cu.
#pragma once

#include "common.cuh"

// Internal status of a Lite pair that survived pruning and waits for its
// exact similarity.
#define BLSH_LITE_SURVIVOR 254

struct VerifyArgs {
    const uint2 *pairs;
    long long P;                 // pair count, or capacity when P_dev is set
    const long long *P_dev;      // device pair count or NULL
    const uint32_t *sig;
    long long N;
    int W;                       // signature row stride in words
    int k;                       // hashes per chunk
    int chunk_words;             // words per chunk: Jaccard k, cosine k/32
    int levels;                  // chunks at most (n_max/k, or h/k for Lite)
    int lite;                    // Algorithm 2: no concentration test
    int conc_words;              // bitmap words per level
    int est_stride;              // n_max + 1
    const int32_t *min_matches;  // [levels]
    const uint32_t *conc_bits;   // [levels][conc_words]
    const int32_t *conc_lo;      // [levels]: smallest concentrated m, used when conc_upper
    int conc_upper;              // every level's concentrated m are the range [conc_lo, n]
    const float *est_tab;        // [levels][est_stride]
    uint8_t *status;
    uint16_t *n_used;
    uint16_t *m_out;
    float *est_out;
    double *sim_out;             // Lite: unused by the pruning pass (the exact pass writes survivors')
    unsigned long long *stop_hist;
    blsh_dev_scratch *scratch;
    int grab;                    // persistent: pairs per work-counter grab
    // Algorithms 1 and 2 in one pass over the pairs: Algorithm 2's pruning
    // over the first lite_levels chunks (h/k), its outputs below; 0 = one
    // algorithm only
    int lite_levels;
    uint8_t *lstatus;
    uint16_t *ln_used;
    double *lsim;
    // lazily computed hashes: only the first cap_levels chunks are available;
    // a pair still undecided there gets BLSH_NEEDS_HASHES and marks its two
    // objects in need[] (cap_levels == levels: no cap)
    int cap_levels;
    uint8_t *need;
    // cosine: words 0..3 of every row (the first 128 hashes) copied into a
    // dense plane of N entries, or NULL (set by blsh_launch_verify)
    const uint4 *plane;
};

// BLSH_NEEDS_HASHES (blsh.h): an Algorithm 1 pair that needs hashes beyond
// those computed so far (blsh_verify_resume finishes it).

int blsh_launch_verify(blsh_ctx *ctx, const VerifyArgs &A, const blsh_plan &plan, cudaStream_t s);
blsh_plan blsh_default_plan(int kind);
int blsh_check_plan(const blsh_plan &plan, int kind, int k);
int blsh_make_verify_args(blsh_ctx *ctx, const blsh_tables *tab, const uint32_t *pairs, int64_t P,
                          const int64_t *P_dev, const uint32_t *sig, int64_t N, int32_t sig_words, uint8_t *status,
                          uint16_t *n_used, uint16_t *m, float *est, uint64_t *stop_hist, VerifyArgs &A);
blsh_plan blsh_plan_for(blsh_ctx *ctx, const blsh_tables *tab);
