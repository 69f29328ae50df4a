// Naive data-parallel marching cubes over a dense field: the baseline the
// paper measures before its block method (Section 3.3.3, Table
// "mc_naive_parallel_perf").  Every cell of the volume is classified, the
// cells the surface crosses are compacted, their triangle counts are
// prefix-summed into output offsets, and a second pass over the crossing
// cells writes the triangle soup.  No blocks, ranges or cache take part:
// the input is a decoded float32 field (iso_decode_volume's output, or any
// x-fastest field).
//
//   dense_classify   one pass over all cells (cell c = x + cx*(y + cy*z),
//                    cx = nx-1, cy = ny-1): the 8-bit case of each cell, the
//                    crossing ones (0 < case < 255) compacted in ascending
//                    order with their cases (decoupled look-back)
//   dense_scan       triangles of each crossing cell from the case table,
//                    exclusive prefix sum into 64-bit offsets, the total
//   dense_emit       one thread per crossing cell: its triangles at its
//                    offset, vertices interpolated as in the block path
//
// Triangle order is that of full-volume marching cubes (cells in ascending
// linear order, then table order).  Vertices use the block path's format:
// float4 {x, y, z relative to the origin of the 4x4x4 block holding the
// cell, w = that block's id as uint32 bits}, each coordinate computed by the
// same float32 operations as the block path, so a triangle's bytes equal the
// block path's triangle on the same edges.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "bcmc.h"
#include "common.cuh"
#include "kernels.cuh"
#include "mc_tables.cuh"
#include "tile_scan.cuh"
#include "volume.cuh"

namespace bcmc {

namespace {

constexpr int kDenseRounds = 16;                       // 4096 cells per classify / scan tile
constexpr uint32_t kDenseTile = kDenseRounds * kThreads;

struct DenseTables {
    uint8_t num_tri[256];
    uint8_t tri_edges[256][16];
};

struct DenseArgs {
    const float *f;
    uint32_t nx, ny, nz;
    uint32_t cx, cy;                                   // cells along x and y
    unsigned long long inv_cx, inv_cy;                 // div_magic of cx, cy
    uint64_t ncells;                                   // < 2^32
    uint32_t nbx, nby;                                 // blocks along x and y (vertex block ids)
    float iso;
    uint32_t *active;                                  // crossing cells, ascending
    uint8_t *cases;                                    // their cases
    unsigned long long *desc;                          // look-back descriptors
    uint32_t *ctr;                                     // [0] classify tiles, [1] scan tiles, [2] status
    uint32_t *n_active;                                // written by the last classify tile
    unsigned long long *offsets;                       // first triangle of each crossing cell
    unsigned long long *n_tri;                         // written by the last scan tile
    const DenseTables *tab;
    float4 *out;
    unsigned long long cap;                            // output capacity in triangles
    unsigned long long *edge_ids;                      // optional: 3 global edge ids per triangle
};

__device__ __forceinline__ void cell_xyz(const DenseArgs &a, uint32_t c, uint32_t &x, uint32_t &y, uint32_t &z) {
    const uint32_t q = div_by(c, a.cx, a.inv_cx);
    x = c - q * a.cx;
    z = div_by(q, a.cy, a.inv_cy);
    y = q - z * a.cy;
}

// the 8 corner samples of cell (x, y, z): corner k = (k&1, k>>1&1, k>>2)
__device__ __forceinline__ void corners(const DenseArgs &a, uint32_t x, uint32_t y, uint32_t z, float (&v)[8]) {
    const size_t sy = a.nx, sz = (size_t)a.nx * a.ny;
    const float *p = a.f + (size_t)x + sy * y + sz * z;
    v[0] = __ldg(p);
    v[1] = __ldg(p + 1);
    v[2] = __ldg(p + sy);
    v[3] = __ldg(p + sy + 1);
    v[4] = __ldg(p + sz);
    v[5] = __ldg(p + sz + 1);
    v[6] = __ldg(p + sz + sy);
    v[7] = __ldg(p + sz + sy + 1);
}

__device__ __forceinline__ uint32_t case_of(const float (&v)[8], float iso) {
    uint32_t cs = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) cs |= (v[k] < iso ? 1u : 0u) << k;
    return cs;
}

__global__ void __launch_bounds__(kThreads) dense_classify_kernel(DenseArgs a) {
    __shared__ TileScan<kDenseRounds> ts;
    __shared__ uint32_t bal[kDenseRounds][8];
    __shared__ uint32_t slot_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t ntiles = (uint32_t)((a.ncells + kDenseTile - 1) / kDenseTile);
    while (true) {
        const uint32_t tile = next_item(&a.ctr[0], &slot_x);
        if (tile >= ntiles) break;
        uint8_t cs[kDenseRounds];
#pragma unroll
        for (int r = 0; r < kDenseRounds; r++) {
            const uint64_t c = (uint64_t)tile * kDenseTile + r * kThreads + threadIdx.x;
            uint32_t cv = 0;
            if (c < a.ncells) {
                uint32_t x, y, z;
                cell_xyz(a, (uint32_t)c, x, y, z);
                float v[8];
                corners(a, x, y, z, v);
                cv = case_of(v, a.iso);
            }
            cs[r] = (uint8_t)cv;
            const uint32_t b = __ballot_sync(0xffffffffu, cv != 0u && cv != 255u);
            if (lane == 0) {
                bal[r][warp] = b;
                ts.cnt[r][warp] = (uint32_t)__popc(b);
            }
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t tot = scan_tile_counts(ts);
            const unsigned long long excl = lookback_exclusive(a.desc, tile, tot, &a.ctr[2], kStatusTimeout);
            if (lane == 0) {
                ts.excl = excl;
                if (tile == ntiles - 1) *a.n_active = (uint32_t)(excl + tot);
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kDenseRounds; r++) {
            const uint32_t b = bal[r][warp];
            if (!((b >> lane) & 1u)) continue;
            const uint32_t at = (uint32_t)ts.excl + ts.cnt[r][warp] + __popc(b & lt);
            a.active[at] = tile * kDenseTile + r * kThreads + threadIdx.x;
            a.cases[at] = cs[r];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) dense_scan_kernel(DenseArgs a, uint32_t n_active) {
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t slot_x;
    constexpr int kPT = kDenseRounds;                   // counts per thread, consecutive
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ntiles = (n_active + kDenseTile - 1) / kDenseTile;
    while (true) {
        const uint32_t tile = next_item(&a.ctr[1], &slot_x);
        if (tile >= ntiles) break;
        const uint32_t i0 = tile * kDenseTile + threadIdx.x * kPT;
        uint32_t n[kPT], sum = 0;
#pragma unroll
        for (int k = 0; k < kPT; k++) {
            n[k] = i0 + k < n_active ? a.tab->num_tri[a.cases[i0 + k]] : 0u;
            sum += n[k];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t w = lane < kThreads / 32 ? wsum[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, wi, kThreads / 32 - 1);
            if (lane < kThreads / 32) wsum[lane] = wi - w;
            const unsigned long long excl = lookback_exclusive(a.desc, tile, tot, &a.ctr[2], kStatusTimeoutScan);
            if (lane == 0) {
                s_excl = excl;
                if (tile == ntiles - 1) *a.n_tri = excl + tot;
            }
        }
        __syncthreads();
        unsigned long long run = s_excl + wsum[warp] + (incl - sum);
#pragma unroll
        for (int k = 0; k < kPT; k++) {
            if (i0 + k < n_active) a.offsets[i0 + k] = run;
            run += n[k];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) dense_emit_kernel(DenseArgs a, uint32_t n_active) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_active; i += gridDim.x * blockDim.x) {
        const uint32_t c = a.active[i], cs = a.cases[i];
        uint32_t x, y, z;
        cell_xyz(a, c, x, y, z);
        float v[8];
        corners(a, x, y, z, v);
        const uint32_t bx = x >> 2, by = y >> 2, bz = z >> 2;
        const float wbits = __uint_as_float(bx + a.nbx * (by + a.nby * bz));
        const float fx = (float)(x - 4 * bx), fy = (float)(y - 4 * by), fz = (float)(z - 4 * bz);
        const uint32_t nt = a.tab->num_tri[cs];
        unsigned long long t = a.offsets[i];
        for (uint32_t k = 0; k < nt; k++, t++) {
            if (t >= a.cap) break;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                // edge e = 4*axis + m: its lower corner is (0, m&1, m>>1) on the
                // other two axes in increasing axis order
                const uint32_t e = a.tab->tri_edges[cs][3 * k + j];
                const uint32_t ax = e >> 2, m = e & 3u;
                const uint32_t dx = ax == 0 ? 0u : (m & 1u);
                const uint32_t dy = ax == 0 ? (m & 1u) : (ax == 1 ? 0u : (m >> 1));
                const uint32_t dz = ax == 2 ? 0u : (m >> 1);
                const uint32_t lo = dx + 2 * dy + 4 * dz, hi = lo + (1u << ax);
                const float tt = edge_fraction<false>(a.iso, v[lo], v[hi]);
                float4 p = make_float4(__fadd_rn(fx, (float)dx), __fadd_rn(fy, (float)dy), __fadd_rn(fz, (float)dz),
                                       wbits);
                if (ax == 0) p.x = __fadd_rn(p.x, tt);
                else if (ax == 1) p.y = __fadd_rn(p.y, tt);
                else p.z = __fadd_rn(p.z, tt);
                a.out[3 * t + j] = p;
                if (a.edge_ids) {
                    const unsigned long long gx = x + dx, gy = y + dy, gz = z + dz;
                    a.edge_ids[3 * t + j] = 3ull * (gx + (unsigned long long)a.nx * (gy + (unsigned long long)a.ny * gz)) + ax;
                }
            }
        }
    }
}

}  // namespace

}  // namespace bcmc

using namespace bcmc;
using namespace bcmc_host;

extern "C" int iso_mc_dense(const float *d_field, uint32_t nx, uint32_t ny, uint32_t nz, float isovalue,
                            float *d_vertices, uint64_t capacity_triangles, uint64_t *d_edge_ids,
                            iso_dense_stats *stats, void *stream) {
    if (!d_field || !stats || !std::isfinite(isovalue) || nx == 0 || ny == 0 || nz == 0) return ISO_ERR_INVALID_ARG;
    if (capacity_triangles && !d_vertices) return ISO_ERR_INVALID_ARG;
    const auto misaligned = [](const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (misaligned(d_field, 4) || misaligned(d_vertices, 16) || misaligned(d_edge_ids, 8)) return ISO_ERR_INVALID_ARG;
    *stats = iso_dense_stats{};
    const uint64_t ncells = (uint64_t)(nx - 1) * (ny - 1) * (nz - 1);
    if (ncells >= (1ull << 32)) return ISO_ERR_INVALID_ARG;     // cell ids are 32-bit
    if (ncells == 0) return ISO_OK;                              // a flat volume has no cells
    int dev = 0;
    ISO_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    McTables mt{};
    if (!build_mc_tables(&mt)) return ISO_ERR_CUDA;
    DenseTables ht{};
    std::memcpy(ht.num_tri, mt.num_tri, 256);
    std::memcpy(ht.tri_edges, mt.tri_edges, 256 * 16);
    const uint32_t tiles_c = (uint32_t)((ncells + kDenseTile - 1) / kDenseTile);
    DenseArgs a{};
    a.f = d_field;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.cx = nx - 1;
    a.cy = ny - 1;
    a.inv_cx = div_magic(a.cx);
    a.inv_cy = div_magic(a.cy);
    a.ncells = ncells;
    a.nbx = (nx + 3) / 4;
    a.nby = (ny + 3) / 4;
    a.iso = isovalue;
    a.out = reinterpret_cast<float4 *>(d_vertices);
    a.cap = capacity_triangles;
    a.edge_ids = reinterpret_cast<unsigned long long *>(d_edge_ids);
    // scratch: the crossing cells and their cases (room for every cell), the
    // look-back descriptors, counters, totals and the case table; offsets
    // once the crossing cells are counted
    struct Small {
        uint32_t ctr[4];
        uint32_t n_active;
        uint32_t pad;
        unsigned long long n_tri;
    };
    uint8_t *scratch = nullptr;
    const size_t off_cases = ncells * 4, off_desc = (off_cases + ncells + 255) & ~size_t(255),
                 off_small = off_desc + (size_t)tiles_c * 8, off_tab = (off_small + sizeof(Small) + 255) & ~size_t(255),
                 total = off_tab + sizeof(DenseTables);
    int rc = dalloc_on(&scratch, total, dev, st);
    if (rc) return rc;
    a.active = reinterpret_cast<uint32_t *>(scratch);
    a.cases = scratch + off_cases;
    a.desc = reinterpret_cast<unsigned long long *>(scratch + off_desc);
    Small *small = reinterpret_cast<Small *>(scratch + off_small);
    a.ctr = small->ctr;
    a.n_active = &small->n_active;
    a.n_tri = &small->n_tri;
    a.tab = reinterpret_cast<const DenseTables *>(scratch + off_tab);
    unsigned long long *offsets = nullptr;
    Small h{};
    int occ = 1, sms = 1;
    auto fail = [&](int code) {
        dfree_on(offsets, st);
        dfree_on(scratch, st);
        cudaStreamSynchronize(st);
        (void)cudaGetLastError();
        return code;
    };
    if (cudaMemsetAsync(scratch + off_desc, 0, off_tab - off_desc, st) != cudaSuccess ||
        cudaMemcpyAsync(scratch + off_tab, &ht, sizeof(ht), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dense_classify_kernel, kThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(ISO_ERR_CUDA);
    const uint32_t grid_c = std::max(1u, std::min(tiles_c, (uint32_t)(std::max(1, occ) * sms)));
    dense_classify_kernel<<<grid_c, kThreads, 0, st>>>(a);
    if (cudaMemcpyAsync(&h, small, sizeof(Small), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(ISO_ERR_CUDA);
    if (h.ctr[2] & kStatusAnyTimeout) return fail(ISO_ERR_TIMEOUT);
    stats->n_active_cells = h.n_active;
    if (h.n_active) {
        rc = dalloc_on(&offsets, h.n_active, dev, st);
        if (rc) return fail(rc);
        a.offsets = offsets;
        const uint32_t tiles_s = (h.n_active + kDenseTile - 1) / kDenseTile;
        if (cudaMemsetAsync(a.desc, 0, (size_t)tiles_s * 8, st) != cudaSuccess) return fail(ISO_ERR_CUDA);
        dense_scan_kernel<<<std::max(1u, std::min(tiles_s, (uint32_t)(std::max(1, occ) * sms))), kThreads, 0, st>>>(
            a, h.n_active);
        if (cudaMemcpyAsync(&h, small, sizeof(Small), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(ISO_ERR_CUDA);
        if (h.ctr[2] & kStatusAnyTimeout) return fail(ISO_ERR_TIMEOUT);
        stats->num_triangles = h.n_tri;
        if (h.n_tri <= capacity_triangles && h.n_tri) {
            const uint32_t grid_e = (uint32_t)std::min<uint64_t>((h.n_active + kThreads - 1) / kThreads,
                                                                 (uint64_t)std::max(1, occ) * sms * 4);
            dense_emit_kernel<<<grid_e, kThreads, 0, st>>>(a, h.n_active);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return fail(ISO_ERR_CUDA);
    dfree_on(offsets, st);
    dfree_on(scratch, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(ISO_ERR_CUDA);
    return stats->num_triangles > capacity_triangles ? ISO_ERR_CAPACITY : ISO_OK;
}
