// scan.cuh -- device-wide exclusive prefix sum in three phases (tile sums,
// scan of the tile sums in one CTA, tile scans with their offsets).  Used by
// the banding step for bucket offsets and pair offsets.
#pragma once

#include "common.cuh"

namespace blsh_scan {

constexpr int kThreads = 256;
constexpr int kPerThread = 8;
constexpr int kTile = kThreads * kPerThread;

template <typename T>
__device__ T block_exclusive(T v, T *total) {
    __shared__ T warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        T s = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const T before = wid > 0 ? warp_sums[wid - 1] : T(0);
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    const T r = before + x - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) tile_sums(const T *in, long long n, T *partial) {
    const long long base = (long long)blockIdx.x * kTile;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const long long p = base + (long long)i * kThreads + threadIdx.x;
        if (p < n) s += in[p];
    }
    T total;
    block_exclusive<T>(s, &total);
    if (threadIdx.x == 0) partial[blockIdx.x] = total;
}

// Exclusive scan of partial[0..m) in place by one CTA; *grand = the sum.
template <typename T>
__global__ void __launch_bounds__(1024) scan_partials(T *partial, long long m, T *grand) {
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long c0 = 0; c0 < m; c0 += blockDim.x) {
        const long long p = c0 + threadIdx.x;
        const T v = p < m ? partial[p] : T(0);
        T tot;
        const T ex = block_exclusive<T>(v, &tot);
        const T base = carry;
        if (p < m) partial[p] = base + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry = base + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && grand) *grand = carry;
}

// out[p] = partial[tile] + exclusive scan within the tile (in may equal out).
template <typename T>
__global__ void __launch_bounds__(kThreads) tile_apply(const T *in, T *out, long long n, const T *partial) {
    const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kPerThread;
    T v[kPerThread];
    T s = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const long long p = base + i;
        v[i] = p < n ? in[p] : T(0);
        s += v[i];
    }
    T ex = block_exclusive<T>(s, nullptr) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kPerThread; ++i) {
        const long long p = base + i;
        if (p < n) out[p] = ex;
        ex += v[i];
    }
}

inline long long tiles_for(long long n) { return (n + kTile - 1) / kTile; }

// Exclusive scan of in[0..n) into out (may alias); *grand (device) = total.
// `partial` needs tiles_for(n) elements.
template <typename T>
cudaError_t exclusive_scan(const T *in, T *out, long long n, T *partial, T *grand, cudaStream_t s) {
    const long long tiles = tiles_for(n);
    if (tiles == 0) return cudaMemsetAsync(grand, 0, sizeof(T), s);
    tile_sums<T><<<(unsigned)tiles, kThreads, 0, s>>>(in, n, partial);
    scan_partials<T><<<1, 1024, 0, s>>>(partial, tiles, grand);
    tile_apply<T><<<(unsigned)tiles, kThreads, 0, s>>>(in, out, n, partial);
    return cudaGetLastError();
}

}  // namespace blsh_scan
