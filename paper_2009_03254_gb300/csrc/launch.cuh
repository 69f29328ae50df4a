// Work distribution over one or many volumes.
//
// Every stage kernel receives a Launch: a device table of volumes and a
// few counters.  A single extraction is a table of one entry; a batch is
// a table of many (each volume with its own isovalue, cache and output
// range).  A kernel first turns the per-volume amount of work (tiles,
// chunks or warp tiles: fixed by the volume's size, or read from its
// control block where an earlier kernel of the same extraction set it)
// into a prefix in shared memory, then maps "virtual" work items to
// (volume, local item) by binary search.  Items of one volume keep their
// order, so each volume's look-back chains and outputs are exactly those
// of extracting it alone.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace bcmc {

__device__ __forceinline__ uint32_t ceil_div(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

// pre[v] = sum of count(u) for u < v, for v in [0, n]; returns pre[n].
// Called by all threads of the block (any block size); n <= kMaxBatch.
// Each thread takes a run of consecutive volumes; count() is evaluated
// twice per volume (sum, then placement) instead of being kept.
template <class F>
__device__ __forceinline__ uint32_t block_prefix(uint32_t n, F count, uint32_t *pre) {
    __shared__ uint32_t warp_tot[32];
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint32_t v0 = threadIdx.x * per, v1 = min(n, v0 + per);
    uint32_t sum = 0;
    for (uint32_t v = v0; v < v1; v++) sum += count(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (blockDim.x + 31) >> 5;
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nwarps ? warp_tot[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nwarps) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - sum;
    for (uint32_t v = v0; v < v1; v++) {
        pre[v] = run;
        run += count(v);
    }
    if (v0 < n && v1 == n) pre[n] = run;          // the owner of the last volume writes the total
    if (n == 0 && threadIdx.x == 0) pre[0] = 0;
    __syncthreads();
    return pre[n];
}

// Volume v of a launch: from the parameters (kOne) or the device table.
template <bool kOne>
__device__ __forceinline__ const VolEntry &vol_of(const Launch &L, uint32_t v) {
    if (kOne) return L.one;
    return L.vols[v];
}

// the volume owning virtual item x (x < pre[n]): largest v with pre[v] <= x
__device__ __forceinline__ uint32_t find_vol(const uint32_t *pre, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Work-item bookkeeping of a launch: the per-volume prefix of item counts
// (shared memory, batches only), the volume of item x, its first item and
// its item count.  A single volume needs no table.
template <bool kOne, class F>
__device__ __forceinline__ uint32_t launch_prefix(const Launch &L, F count, uint32_t *pre) {
    if (kOne) return count(0u);
    return block_prefix(L.n, count, pre);
}

template <bool kOne>
__device__ __forceinline__ uint32_t item_vol(const uint32_t *pre, uint32_t n, uint32_t x) {
    return kOne ? 0u : find_vol(pre, n, x);
}

template <bool kOne>
__device__ __forceinline__ uint32_t item_base(const uint32_t *pre, uint32_t v) {
    return kOne ? 0u : pre[v];
}

template <bool kOne>
__device__ __forceinline__ uint32_t vol_items(const uint32_t *pre, uint32_t v, uint32_t total) {
    return kOne ? total : pre[v + 1] - pre[v];
}

}  // namespace bcmc
