// compact_noalloc.cu -- blsh_compact_noalloc: the stable compaction of
// compact.cu for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside a host that owns
// all device memory through its own pool, or a plug-in loaded where any
// allocation outside the pool is forbidden.  They cannot create a blsh_ctx
// (whose scratch area is allocated), so this entry point takes no context and
// keeps its scratch -- one count per tile of 4096 statuses -- in a file-scope
// __device__ array of fixed size.  Every GPU that loads the library holds that
// array until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address.  The device address belongs to the CUDA context the module was
// loaded into, so it is looked up with cudaGetSymbolAddress on the first call
// made in each context (identified by the driver's unique context id, so that
// a context created after cudaDeviceReset, or a second context on the same
// device, gets its own lookup) and cached for later calls.
#include <cuda.h>

#include <mutex>

#include "common.cuh"
#include "scan.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 16;
constexpr long long kTile = kThreads * kPer;            // statuses per tile
constexpr long long kMaxTiles = 16384;                  // scratch: 16384 int64 = 128 KiB
constexpr long long kMaxItems = kTile * kMaxTiles;      // 67,108,864 statuses
constexpr int kCacheSlots = 64;   // contexts remembered (the oldest entry is replaced)

__device__ __align__(256) long long g_tile_scratch[kMaxTiles];

struct ScratchSlot {
    unsigned long long ctx_id = 0;   // 0: empty (the driver's ids start at 1)
    long long *ptr = nullptr;
};
std::mutex g_mu;
ScratchSlot g_slots[kCacheSlots];
int g_next_slot = 0;

__device__ __forceinline__ bool kept(uint8_t st, uint32_t mask) { return st < 32 && ((mask >> st) & 1u); }

__device__ __forceinline__ long long resolve_p(long long P, const long long *P_dev) {
    if (!P_dev) return P;
    const long long pd = *P_dev;
    return pd < 0 ? 0 : (pd < P ? pd : P);
}

// Pass 1: tile t counts its kept statuses into counts[t].  Every tile below
// kMaxTiles that the launch covers is written, kept or not, so nothing has to
// be cleared between calls.
__global__ void __launch_bounds__(kThreads) tile_count(const uint8_t *status, long long P_cap,
                                                       const long long *P_dev, uint32_t mask, long long *counts) {
    const long long P = resolve_p(P_cap, P_dev);
    const long long q0 = (long long)blockIdx.x * kTile;
    long long c = 0;
    for (int i = 0; i < kPer; ++i) {
        const long long q = q0 + (long long)i * kThreads + threadIdx.x;
        if (q < P) c += kept(status[q], mask);
    }
    long long total;
    blsh_scan::block_exclusive<long long>(c, &total);
    if (threadIdx.x == 0) counts[blockIdx.x] = total;
}

// Pass 2: exclusive scan of the tile counts in place, by one CTA; the sum goes
// to *n_out.
__global__ void __launch_bounds__(1024) tile_offsets(long long *counts, long long tiles, long long *n_out) {
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < tiles; c0 += blockDim.x) {
        const long long t = c0 + threadIdx.x;
        const long long v = t < tiles ? counts[t] : 0;
        long long tot;
        const long long ex = blsh_scan::block_exclusive<long long>(v, &tot);
        const long long base = carry;
        if (t < tiles) counts[t] = base + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry = base + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_out = carry;
}

// Pass 3: tile t writes the indices of its kept statuses, in order, from
// offset counts[t]; indices at or beyond cap are dropped.
__global__ void __launch_bounds__(kThreads) tile_write(const uint8_t *status, long long P_cap,
                                                       const long long *P_dev, uint32_t mask,
                                                       const long long *counts, int64_t *out, long long cap) {
    const long long P = resolve_p(P_cap, P_dev);
    const long long q0 = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kPer;
    uint32_t bits = 0;
    int c = 0;
    for (int i = 0; i < kPer; ++i) {
        const long long q = q0 + i;
        if (q < P && kept(status[q], mask)) {
            bits |= 1u << i;
            ++c;
        }
    }
    long long o = counts[blockIdx.x] + blsh_scan::block_exclusive<long long>((long long)c, nullptr);
    for (int i = 0; i < kPer; ++i)
        if ((bits >> i) & 1u) {
            if (o < cap) out[o] = q0 + i;
            ++o;
        }
}

// The driver's id of the calling thread's current context (0 if none),
// through the runtime's driver entry points, so the library needs no link
// against libcuda.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_tile_scratch in the current context: cached per
// context; looked up (cudaGetSymbolAddress) only outside stream capture, since
// the lookup may load the module.  Returns BLSH_OK or BLSH_EDEVICE.
int scratch_for(cudaStream_t s, long long **ptr) {
    // any runtime call binds the device's primary context to a thread that
    // has no current context yet; a capturing stream implies a context
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return BLSH_EDEVICE;
    unsigned long long id = current_context_id();
    if (id == 0 && cs == cudaStreamCaptureStatusNone && cudaFree(nullptr) == cudaSuccess) id = current_context_id();
    if (id == 0) return BLSH_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    for (const ScratchSlot &e : g_slots)
        if (e.ctx_id == id) {
            *ptr = e.ptr;
            return BLSH_OK;
        }
    if (cs != cudaStreamCaptureStatusNone) return BLSH_EDEVICE;   // first call in this context made under capture
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tile_scratch) != cudaSuccess) return BLSH_EDEVICE;
    g_slots[g_next_slot] = ScratchSlot{id, (long long *)p};
    g_next_slot = (g_next_slot + 1) % kCacheSlots;
    *ptr = (long long *)p;
    return BLSH_OK;
}

}  // namespace

extern "C" int blsh_compact_noalloc(const uint8_t *status, int64_t P, const int64_t *P_dev, uint32_t keep_mask,
                                    int64_t *out_idx, int64_t cap, int64_t *n_out, void *stream) {
    if (!n_out || (P > 0 && !status) || (cap > 0 && !out_idx) || P < 0 || cap < 0) return BLSH_EINVAL;
    if (P > kMaxItems) return BLSH_ESIZE;   // more statuses than the fixed scratch covers
    if (!blsh_aligned(out_idx, 8) || !blsh_aligned(n_out, 8) || !blsh_aligned(P_dev, 8)) return BLSH_EINVAL;
    cudaStream_t s = blsh_stream(stream);
    long long *counts = nullptr;
    if (scratch_for(s, &counts) != BLSH_OK) return BLSH_EDEVICE;
    long long tiles = (P + kTile - 1) / kTile;
    if (tiles < 1) tiles = 1;
    // each launch's own error code (cudaLaunchKernel returns it), so an error
    // left on the thread by earlier, unrelated work is neither reported as
    // this call's nor cleared
    const long long *pd = (const long long *)P_dev;
    long long P_cap = P;
    void *count_args[] = {(void *)&status, (void *)&P_cap, (void *)&pd, (void *)&keep_mask, (void *)&counts};
    void *offset_args[] = {(void *)&counts, (void *)&tiles, (void *)&n_out};
    long long cap_ll = cap;
    void *write_args[] = {(void *)&status, (void *)&P_cap, (void *)&pd, (void *)&keep_mask, (void *)&counts,
                          (void *)&out_idx, (void *)&cap_ll};
    cudaError_t e = cudaLaunchKernel((const void *)tile_count, dim3((unsigned)tiles), dim3(kThreads), count_args, 0, s);
    if (e == cudaSuccess)
        e = cudaLaunchKernel((const void *)tile_offsets, dim3(1), dim3(1024), offset_args, 0, s);
    if (e == cudaSuccess)
        e = cudaLaunchKernel((const void *)tile_write, dim3((unsigned)tiles), dim3(kThreads), write_args, 0, s);
    if (e != cudaSuccess) {
        cudaGetLastError();   // the slot now holds this call's launch error
        return BLSH_EDEVICE;
    }
    return BLSH_OK;
}
