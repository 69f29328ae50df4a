// Active-block selection that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: plug-ins living inside an
// application whose own allocator has already reserved the device memory
// (a second allocator in the same process would fail, or fragment what the
// host application manages), and latency-critical loops where an
// allocation's implicit device synchronisation would stall other work.
// For them this file provides iso_active_blocks_static: the range test and
// ordered compaction of the cull stage, taking the per-block ranges
// straight from the caller, with its only scratch (look-back descriptors, a
// tile counter, a status word and the total) in a fixed file-scope device
// array.
//
// The array is part of the loaded module, so every GPU that loads the
// library holds it (about 256 KiB) until the process exits.  All calls
// share it and it keeps the last call's contents: each call clears the
// part it uses before the selection kernel runs, and two calls whose work
// overlaps on the GPU (for example on two streams) race on it.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "bcmc.h"
#include "common.cuh"

namespace {

constexpr uint32_t kTileBlocks = 2048;                 // 256 threads x 8 rounds, as in the cull kernel
constexpr uint32_t kMaxTiles = 32768;
constexpr uint64_t kMaxBlocks = (uint64_t)kTileBlocks * kMaxTiles;   // 2^26 blocks = 2^32 samples
constexpr uint32_t kCounterSlot = kMaxTiles;           // tile counter
constexpr uint32_t kStatusSlot = kMaxTiles + 1;        // bounded-wait timeout and corrupt-range bits
constexpr uint32_t kTotalSlot = kMaxTiles + 2;         // active blocks, written by the last tile
constexpr uint32_t kCountTimeout = 0xFFFFFFFFu;        // *count after a look-back wait gave up
constexpr uint32_t kCountCorrupt = 0xFFFFFFFEu;        // *count when a range is NaN or has min > max

static __device__ __align__(256) unsigned long long g_scratch[kMaxTiles + 4];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned long long *g_device_ptr[kMaxDevices] = {};

// Host code may not take g_scratch's address itself (in host code the
// name only stands for a host-side shadow); ask the runtime, once per
// device, with that device current.
int scratch_address(unsigned long long **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return ISO_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return ISO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_device_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return ISO_ERR_CUDA;
        }
        g_device_ptr[dev] = static_cast<unsigned long long *>(p);
    }
    *out = g_device_ptr[dev];
    return ISO_OK;
}

__global__ void clear_scratch_kernel(unsigned long long *scratch, uint32_t ntiles) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < ntiles; i += gridDim.x * blockDim.x) scratch[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scratch[kCounterSlot] = 0;
        scratch[kStatusSlot] = 0;
        scratch[kTotalSlot] = 0;
    }
}

// After every tile has finished (stream order): the count, or the code of
// the failure any tile recorded.
__global__ void finish_count_kernel(const unsigned long long *scratch, uint32_t *count) {
    const uint32_t status = (uint32_t)scratch[kStatusSlot];
    *count = (status & bcmc::kStatusTimeout) ? kCountTimeout
             : (status & bcmc::kStatusCorrupt) ? kCountCorrupt
                                                : (uint32_t)scratch[kTotalSlot];
}

// The active test of the cull kernel, with the 3x3x3 min/max taken on the
// fly from the caller's ranges instead of a precomputed hull.
__global__ void __launch_bounds__(256) select_static_kernel(const float *__restrict__ bmin,
                                                            const float *__restrict__ bmax, bcmc::Geom g, float iso,
                                                            uint32_t *ids, uint64_t capacity,
                                                            unsigned long long *scratch, uint32_t ntiles) {
    __shared__ uint32_t cnt[8][8];
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t slab = g.nbx * g.nby;
    uint32_t *status = reinterpret_cast<uint32_t *>(scratch + kStatusSlot);
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + kCounterSlot);
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        uint32_t bits[8];
#pragma unroll
        for (int r = 0; r < 8; r++) {
            const uint32_t b = tile * kTileBlocks + r * 256 + threadIdx.x;
            bool act = false;
            if (b < g.nb) {
                const int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / slab);
                float lo = bmin[b], hi = bmax[b];
                // a range that is not a range (NaN, or min > max) is reported,
                // as iso_load_volume reports it; the neighbours' ranges are
                // each checked by their own thread
                if (!(lo <= hi)) atomicOr(status, bcmc::kStatusCorrupt);
                for (int dz = -1; dz <= 1; dz++)
                    for (int dy = -1; dy <= 1; dy++)
                        for (int dx = -1; dx <= 1; dx++) {
                            const int x = bx + dx, y = by + dy, z = bz + dz;
                            if (x < 0 || y < 0 || z < 0 || x >= (int)g.nbx || y >= (int)g.nby || z >= (int)g.nbz)
                                continue;
                            const uint32_t n = (uint32_t)x + g.nbx * ((uint32_t)y + g.nby * (uint32_t)z);
                            lo = fminf(lo, __ldg(bmin + n));
                            hi = fmaxf(hi, __ldg(bmax + n));
                        }
                act = lo < iso && iso <= hi;
            }
            bits[r] = __ballot_sync(0xffffffffu, act);
            if (lane == 0) cnt[r][warp] = (uint32_t)__popc(bits[r]);
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t *flat = &cnt[0][0];
            const uint32_t a = flat[2 * lane], c = flat[2 * lane + 1];
            uint32_t incl = a + c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            flat[2 * lane] = incl - (a + c);
            flat[2 * lane + 1] = incl - c;
            const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
            const unsigned long long excl = bcmc::lookback_exclusive(scratch, tile, tot, status, bcmc::kStatusTimeout);
            if (lane == 0) {
                s_excl = excl;
                if (tile == ntiles - 1) scratch[kTotalSlot] = excl + tot;
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 8; r++) {
            if (!((bits[r] >> lane) & 1u)) continue;
            const uint64_t at = s_excl + cnt[r][warp] + __popc(bits[r] & lt);
            if (at < capacity) ids[at] = tile * kTileBlocks + r * 256 + threadIdx.x;
        }
        __syncthreads();
    }
}

}  // namespace

extern "C" int iso_active_blocks_static(const float *d_bmin, const float *d_bmax, uint32_t nx, uint32_t ny,
                                        uint32_t nz, float isovalue, uint32_t *d_ids, uint64_t capacity,
                                        uint32_t *d_count, void *stream) {
    if (!d_bmin || !d_bmax || !d_count || (capacity && !d_ids) || !std::isfinite(isovalue) || nx == 0 || ny == 0 ||
        nz == 0)
        return ISO_ERR_INVALID_ARG;
    const auto misaligned = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 3u) != 0; };
    if (misaligned(d_bmin) || misaligned(d_bmax) || misaligned(d_count) || (capacity && misaligned(d_ids)))
        return ISO_ERR_INVALID_ARG;
    const uint64_t nbx = (nx + 3ull) / 4, nby = (ny + 3ull) / 4, nbz = (nz + 3ull) / 4;
    const uint64_t nb = nbx * nby * nbz;
    if (nb > kMaxBlocks) return ISO_ERR_INVALID_ARG;   // more blocks than the fixed scratch covers
    unsigned long long *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != ISO_OK) return rc;
    const bcmc::Geom g{nx, ny, nz, (uint32_t)nbx, (uint32_t)nby, (uint32_t)nbz, (uint32_t)nb, 1u,
                       bcmc::div_magic((uint32_t)nbx), bcmc::div_magic((uint32_t)nby)};
    const uint32_t ntiles = (uint32_t)((nb + kTileBlocks - 1) / kTileBlocks);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    clear_scratch_kernel<<<(ntiles + 255) / 256, 256, 0, st>>>(scratch, ntiles);
    int sms = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return ISO_ERR_CUDA;
    }
    const uint32_t grid = ntiles < (uint32_t)(4 * sms) ? ntiles : (uint32_t)(4 * sms);
    select_static_kernel<<<grid, 256, 0, st>>>(d_bmin, d_bmax, g, isovalue, d_ids, capacity, scratch, ntiles);
    finish_count_kernel<<<1, 1, 0, st>>>(scratch, d_count);
    if (cudaGetLastError() != cudaSuccess) return ISO_ERR_CUDA;
    return ISO_OK;
}
