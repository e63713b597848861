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
// address; the device address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, with the device
// current) and passed to the kernels.
#include <mutex>

#include "common.cuh"
#include "scan.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 16;
constexpr long long kTile = kThreads * kPer;            // statuses per tile
constexpr long long kMaxTiles = 16384;                  // scratch: 16384 int64 = 128 KiB
constexpr long long kMaxItems = kTile * kMaxTiles;      // 67,108,864 statuses
constexpr int kMaxDevices = 64;

__device__ __align__(256) long long g_tile_scratch[kMaxTiles];

std::mutex g_mu;
long long *g_scratch_ptr[kMaxDevices] = {nullptr};

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

// Device address of g_tile_scratch on the current device, looked up once.
cudaError_t scratch_for(int device, long long **ptr) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_tile_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = (long long *)p;
    }
    *ptr = g_scratch_ptr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" int blsh_compact_noalloc(const uint8_t *status, int64_t P, const int64_t *P_dev, uint32_t keep_mask,
                                    int64_t *out_idx, int64_t cap, int64_t *n_out, void *stream) {
    if (!n_out || (P > 0 && !status) || (cap > 0 && !out_idx) || P < 0 || cap < 0) return BLSH_EINVAL;
    if (P > kMaxItems) return BLSH_ESIZE;   // more statuses than the fixed scratch covers
    if (!blsh_aligned(out_idx, 8) || !blsh_aligned(n_out, 8) || !blsh_aligned(P_dev, 8)) return BLSH_EINVAL;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
        cudaGetLastError();
        return BLSH_EDEVICE;
    }
    long long *counts = nullptr;
    if (scratch_for(device, &counts) != cudaSuccess) {
        cudaGetLastError();
        return BLSH_EDEVICE;
    }
    cudaStream_t s = blsh_stream(stream);
    long long tiles = (P + kTile - 1) / kTile;
    if (tiles < 1) tiles = 1;
    tile_count<<<(unsigned)tiles, kThreads, 0, s>>>(status, P, (const long long *)P_dev, keep_mask, counts);
    tile_offsets<<<1, 1024, 0, s>>>(counts, tiles, (long long *)n_out);
    tile_write<<<(unsigned)tiles, kThreads, 0, s>>>(status, P, (const long long *)P_dev, keep_mask, counts,
                                                    out_idx, cap);
    return cudaGetLastError() == cudaSuccess ? BLSH_OK : BLSH_EDEVICE;
}
