// common.cuh -- internal definitions shared by the libblsh translation units:
// the context and table objects, the device scratch area, error helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <vector>

#include "blsh.h"

#define BLSH_MAX_NMAX 4096
#define BLSH_COMPACT_MAX_CTAS 2048
#define BLSH_RECHECK_CAP (1u << 20)   // queued SRP sign rechecks per call (8 MiB per context)
#define BLSH_LITE_QUEUE_CAP (1u << 23) // queued Lite survivors per call (64 MiB per context)

// Device-side scratch owned by a context.  Every call zeroes what it uses
// before its kernels run (cudaMemsetAsync on the caller's stream).
struct blsh_dev_scratch {
    unsigned int err_code;             // first device-detected error (0 = none)
    unsigned int pad0;
    unsigned long long counters[4];    // bad pairs, truncations, SRP rechecks, SRP zeros
    unsigned long long work;           // verify: next pair handed out
    unsigned long long work2;          // lite: next survivor tile handed out
    unsigned long long work3;          // lite: survivors queued
    unsigned long long recheck_count;  // SRP: signs queued for an FP64 recheck
    unsigned long long band_work[3];   // banding: next chunk of positions (count pass, write pass), record words used
    unsigned long long hash_work;      // sparse projection: next (row, piece) item handed out
    unsigned int norm2_valid;          // Lite: the rows' squared norms were formed for this call
    long long cta_counts[BLSH_COMPACT_MAX_CTAS];  // compaction: kept items per CTA
};

struct blsh_ctx {
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    blsh_dev_scratch *scratch = nullptr;
    uint2 *recheck_queue = nullptr;                   // [BLSH_RECHECK_CAP] (row, bit) of undecided SRP signs
    unsigned long long *lite_queue = nullptr;         // [BLSH_LITE_QUEUE_CAP] Lite survivors (pair indices)
    // per-object buffers, sized by blsh_ctx_reserve (never by a hot call)
    void *plane = nullptr;                            // verification: [plane_cap] first four words of each row
    long long plane_cap = 0;
    void *norm2 = nullptr;                            // Lite (cosine): [norm2_cap] rows' squared norms
    long long norm2_cap = 0;
    char err[512] = {0};
    std::map<const blsh_tables *, blsh_plan> plans;   // autotuned plans
    std::atomic<long long> launches{0};            // kernels launched through this context
    std::mutex mu;
    // per-launch device timing (blsh_timing_begin/_end): while `on`, each
    // launch is bracketed by a pair of events on its stream
    struct {
        bool on = false, open = false;
        int cap = 0, n = 0;
        cudaStream_t s = nullptr;
        std::vector<cudaEvent_t> ev;        // [2 cap]: start, stop of record i
        std::vector<const char *> name;     // [cap]: kernel name of record i
    } timing;
};

struct blsh_tables {
    blsh_params p;
    int device = 0;
    int levels = 0;          // n_max / k
    int conc_words = 0;      // uint32 words per level of the concentration bitmap
    int near_ties = 0;
    int numeric_bad = 0;
    void *dev = nullptr;     // one allocation holding the arrays below
    size_t bytes = 0;
    int32_t *min_matches = nullptr;   // [levels]
    int32_t *conc_lo = nullptr;       // [levels]: smallest concentrated m (n+1 if none)
    bool conc_upper = false;          // every level's concentrated m form the range [conc_lo, n]
    uint32_t *conc_bits = nullptr;    // [levels][conc_words]
    float *est = nullptr;             // [levels][n_max+1]
    double *prune_prob = nullptr;     // [levels][n_max+1]
    double *conc_prob = nullptr;      // [levels][n_max+1]
    int *flags = nullptr;             // [3]: near ties, non-finite / non-monotone, conc not an upper range
};

// Records `fmt` as the context's last error and returns `code`.
int blsh_fail(blsh_ctx *ctx, int code, const char *fmt, ...);

// Maps a CUDA error to BLSH_EDEVICE with a message, or returns BLSH_OK.
int blsh_cuda_check(blsh_ctx *ctx, cudaError_t e, const char *what);

#define BLSH_CUDA(ctx, call)                                      \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return blsh_cuda_check(ctx, e_, #call); \
    } while (0)

// Checks the launch that was just enqueued and counts it.
// Timing of the next launch on stream s: its start event (only while timing
// is on, records remain and s is not being captured into a graph).
static inline void blsh_time_start(blsh_ctx *ctx, cudaStream_t s) {
    auto &T = ctx->timing;
    T.open = false;
    if (!T.on || T.n >= T.cap) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventRecord(T.ev[2 * T.n], s) != cudaSuccess) return;
    T.open = true;
    T.s = s;
}

// The stop event of the launch started by blsh_time_start, named `what`.
static inline void blsh_time_stop(blsh_ctx *ctx, const char *what) {
    auto &T = ctx->timing;
    if (!T.open) return;
    T.open = false;
    if (cudaEventRecord(T.ev[2 * T.n + 1], T.s) == cudaSuccess) T.name[T.n++] = what;
}

// After each kernel launch: the launch error check, the launch count and the
// timing record (`what` is the kernel's name).
#define BLSH_LAUNCHED(ctx, what)                                  \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) {                                  \
            (ctx)->timing.open = false;                           \
            return blsh_cuda_check(ctx, e_, what);                \
        }                                                         \
        (ctx)->launches.fetch_add(1, std::memory_order_relaxed);  \
        blsh_time_stop(ctx, what);                                \
    } while (0)

static inline bool blsh_aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

// Device error reporting: the first error code sticks, counters accumulate.
__device__ __forceinline__ void blsh_dev_error(blsh_dev_scratch *s, unsigned int code, int counter,
                                               unsigned long long n) {
    atomicCAS(&s->err_code, 0u, code);
    if (counter >= 0) atomicAdd(&s->counters[counter], n);
}

// Makes ctx->device current for the duration of a call.
struct blsh_device_guard {
    int prev = -1;
    bool ok = true;
    explicit blsh_device_guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~blsh_device_guard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

static inline cudaStream_t blsh_stream(void *s) { return (cudaStream_t)s; }

// Statuses (one byte each) equal to `val` among the 16 bytes of v: bit i of
// the result for byte i.  Per 32-bit word, x = w ^ (val in every byte); the
// high bit of a byte of ~(((x & 0x7f..) + 0x7f..) | x) is set exactly when
// the byte is zero (no carry crosses a byte), and one multiply gathers the
// four high bits: shifted down by 7 they sit at bits 8k, and the multiplier
// 1 + 2^7 + 2^14 + 2^21 puts byte k's on bit 21 + k with no other term on
// bits 21..24.  About two operations a status instead of seven.
__device__ __forceinline__ uint32_t blsh_eq16(uint4 v, uint32_t val) {
    const uint32_t rep = val * 0x01010101u;
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t x = w[k] ^ rep;
        const uint32_t z = ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
        r |= ((((z >> 7) * 0x00204081u) >> 21) & 0xfu) << (4 * k);
    }
    return r;
}
