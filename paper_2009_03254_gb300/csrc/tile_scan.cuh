// Block-wide helpers of the tile scans (cull, cache update, serving cull):
// per-(round, warp) ballot counts turned into offsets inside a tile, and
// work items taken in order from a launch counter.
#pragma once

#include <cstdint>

#include "kernels.cuh"

namespace bcmc {

// A tile is kR * 256 entries handled by 256 threads in kR rounds; entry
// tile*kR*256 + r*256 + threadIdx.x belongs to round r.  Per (round, warp)
// the warp's ballot gives its 32 flags; a warp scan over the kR*8
// (round, warp) counts gives each group's offset inside the tile.  Large
// tiles keep the tiles of a pass within one wave of resident blocks, so
// the look-back walk stays short.

constexpr int kRounds = kScanTile / kThreads;   // rounds of a cache-update tile

template <int kR>
struct TileScan {
    uint32_t cnt[kR][8];              // per (round, warp): packed counts, then exclusive offsets
    unsigned long long excl;          // tile's exclusive prefix (look-back)
};

// warp 0: turn ts.cnt into exclusive offsets (packed 16-bit fields add
// without carries: a tile holds at most 4096 entries) and return the
// tile's packed total in every lane
template <int kR>
__device__ __forceinline__ uint32_t scan_tile_counts(TileScan<kR> &ts) {
    constexpr int kPer = kR * 8 / 32;
    const int lane = threadIdx.x & 31;
    uint32_t *flat = &ts.cnt[0][0] + kPer * lane;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        v[k] = flat[k];
        sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < kPer; k++) {
        flat[k] = run;
        run += v[k];
    }
    return __shfl_sync(0xffffffffu, incl, 31);
}

// block-wide: take the next work item from a launch counter
__device__ __forceinline__ uint32_t next_item(uint32_t *ctr, uint32_t *slot) {
    if (threadIdx.x == 0) *slot = atomicAdd(ctr, 1u);
    __syncthreads();
    const uint32_t x = *slot;
    __syncthreads();                  // all have read it before thread 0 may overwrite it
    return x;
}

}  // namespace bcmc
