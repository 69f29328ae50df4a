// Triangle stage (paper Sections 4.3-4.5) over the candidate blocks.
//
// Candidates are the active blocks whose 2x2x2 "+group" (the block and its
// +x/+y/+z face, edge and corner neighbours, the only blocks its cells
// read) has a range containing the isovalue; any block with a crossing
// cell is one (its cell's below and above corners lie in the +group), so
// no triangle is lost, and every +neighbour of a candidate is itself
// active and therefore cached.  This is the refinement Section 4.4 notes
// as possible ("checking which side the neighbor was on").
//
// Work split: a CTA takes a tile of 32 consecutive candidates from a
// counter; each of its 8 warps owns 4 consecutive candidates and runs the
// phases on them, meeting the other warps only for the tile's offset:
//   A  slots of each block's 8 blocks of the +group (8 lanes per block)
//   B  stage the 5x5x5 samples in shared memory: 16 float4 rows of the
//      block, its +x face, +y/+z rows, edges and corner (50 loads per
//      block, 2 per lane, issued together)
//   C  classify: four ballots give the 125 below-iso bits; each cell's
//      case is 8 bits picked from them; counts from the case table
//   D  per-block counts -> warp totals -> tile total -> one decoupled
//      look-back per tile: the prefix sum over blocks of Section 4.4 in
//      one pass (per-tile rather than per-warp descriptors keep the walk
//      back short: only the tiles in flight, one per CTA, are pending)
//   E  per-cell offsets (Section 4.5) by two packed warp scans, a
//      triangle -> (block, cell, k) map, then each lane writes whole
//      float4 vertices: a warp's stores cover one contiguous range.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"

namespace bcmc {

namespace {

constexpr int kWarps = kThreads / 32;                 // 8
constexpr int kBlocksPerWarp = 4;
constexpr int kTile = kWarps * kBlocksPerWarp;        // 32 = kMcTileBlocks
static_assert(kTile == kMcTileBlocks, "tile size");
constexpr int kHalo = 200;                            // x + 8y + 40z, x,y,z in [0,5)
constexpr int kTmap = kBlocksPerWarp * 64 * 5;        // triangles a warp can own

struct Smem {
    float halo[kTile][kHalo];
    int32_t nslot[kTile][8];
    uint32_t bid[kTile];
    uint32_t lim[kTile];                              // cells per axis inside the volume, 4 bits each
    uint8_t cases[kTile][64];
    uint16_t tmap[kWarps][kTmap];                     // block-in-warp (2) | cell (6) | k (3)
    uint8_t num_tri[256];
    uint8_t tri_edges[256][16];
    uint32_t edge_info[12];
    uint32_t wtot[kWarps];                            // triangles of each warp's blocks in this tile
    unsigned long long tile_base;                     // triangles before this tile
    uint32_t tile[2];
    uint32_t occ;
    uint32_t status;
};

// Halo load job j of a block (0..63; 50 used): neighbour o, source sample
// index inside that block, destination in the padded halo, float4 or not.
// Packed: valid(1) | vec(1) | o(3) | src(6) | dst(8).
__device__ __forceinline__ uint32_t halo_job(int j) {
    int o = 0, src = 0, dst = 0, vec = 0;
    if (j < 16) {                       // own rows (y, z) = (j & 3, j >> 2)
        o = 0; src = 4 * j; dst = 8 * (j & 3) + 40 * (j >> 2); vec = 1;
    } else if (j < 32) {                // +x face: sample (0, y, z) -> halo (4, y, z)
        const int r = j - 16;
        o = 1; src = 4 * r; dst = 4 + 8 * (r & 3) + 40 * (r >> 2);
    } else if (j < 36) {                // +y rows: (x, 0, z) -> (x, 4, z)
        const int z = j - 32;
        o = 2; src = 16 * z; dst = 32 + 40 * z; vec = 1;
    } else if (j < 40) {                // +z rows: (x, y, 0) -> (x, y, 4)
        const int y = j - 36;
        o = 4; src = 4 * y; dst = 8 * y + 160; vec = 1;
    } else if (j < 44) {                // +xy edge: (0, 0, z) -> (4, 4, z)
        const int z = j - 40;
        o = 3; src = 16 * z; dst = 36 + 40 * z;
    } else if (j < 48) {                // +xz edge: (0, y, 0) -> (4, y, 4)
        const int y = j - 44;
        o = 5; src = 4 * y; dst = 164 + 8 * y;
    } else if (j == 48) {               // +yz row: (x, 0, 0) -> (x, 4, 4)
        o = 6; src = 0; dst = 192; vec = 1;
    } else if (j == 49) {               // corner: (0, 0, 0) -> (4, 4, 4)
        o = 7; src = 0; dst = 196;
    } else {
        return 0;
    }
    return 1u | ((uint32_t)vec << 1) | ((uint32_t)o << 2) | ((uint32_t)src << 5) | ((uint32_t)dst << 11);
}

// padded halo offset of logical sample s = x + 5y + 25z
__device__ __forceinline__ int halo_off(int s) { return (s % 5) + 8 * ((s / 5) % 5) + 40 * (s / 25); }

}  // namespace

__global__ void __launch_bounds__(kThreads, 4) mc_kernel(DevState s, Geom g, int debug) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 256; i += kThreads) sm.num_tri[i] = s.tables[i];
    for (int i = threadIdx.x; i < 256 * 16; i += kThreads) (&sm.tri_edges[0][0])[i] = s.tables[256 + i];
    if (threadIdx.x < 12) {
        const int e = threadIdx.x, a = e >> 2, j0 = e & 1, j1 = (e >> 1) & 1;
        const int dx = a == 0 ? 0 : j0, dy = a == 0 ? j0 : (a == 1 ? 0 : j1), dz = a == 2 ? 0 : j1;
        const int lo = dx + 8 * dy + 40 * dz, hi = lo + (a == 0 ? 1 : (a == 1 ? 8 : 40));
        sm.edge_info[e] = (uint32_t)lo | ((uint32_t)hi << 8) | ((uint32_t)dx << 16) | ((uint32_t)dy << 17) |
                          ((uint32_t)dz << 18) | ((uint32_t)a << 19);
    }
    if (threadIdx.x == 0) {
        sm.status = c->status;
        sm.occ = 0;
    }
    __syncthreads();
    const uint32_t n_cand = c->n_cand;
    const uint32_t ntiles = (n_cand + kTile - 1) / kTile;
    const float iso = c->params.iso;
    const unsigned long long tri_cap = c->params.tri_cap;
    float4 *__restrict__ out = reinterpret_cast<float4 *>(c->params.out);
    const bool failed = (sm.status & (kStatusBudget | kStatusTimeout)) != 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->mc_tiles = failed ? 0u : ntiles;
    if (failed) return;
    const uint32_t slab = g.nbx * g.nby;

    // per-lane constants
    const uint32_t job0 = halo_job(lane), job1 = halo_job(lane + 32);
    int cls[4];
#pragma unroll
    for (int r = 0; r < 4; r++) cls[r] = lane + 32 * r < 125 ? halo_off(lane + 32 * r) : -1;
    int cbase[2], cword[2], cshift[2], chalo[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int cell = lane + 32 * h, cx = cell & 3, cy = (cell >> 2) & 3, cz = cell >> 4;
        cbase[h] = cx + 5 * cy + 25 * cz;
        cword[h] = cbase[h] >> 5;
        cshift[h] = cbase[h] & 31;
        chalo[h] = cx + 8 * cy + 40 * cz;
    }
    (void)chalo;
    const int bq = lane >> 3, bo = lane & 7;
    float *halo_w = &sm.halo[warp * kBlocksPerWarp][0];
    uint32_t occ_local = 0;

    for (uint32_t it = 0;; it++) {
        if (threadIdx.x == 0) sm.tile[it & 1] = atomicAdd(&c->ctr[kCtrMc], 1u);
        __syncthreads();
        const uint32_t tile = sm.tile[it & 1];
        if (tile >= ntiles) break;
        const uint32_t base = tile * kTile;
        const int t0 = warp * kBlocksPerWarp;
        const int nb_w = (int)min((uint32_t)kBlocksPerWarp, n_cand - base > (uint32_t)t0 ? n_cand - base - t0 : 0u);

        // ---- A: +group slots
        if (bq < nb_w) {
            const int t = t0 + bq;
            const uint32_t ai = s.icand[base + t];
            const uint32_t b = s.iactive[ai];
            const uint32_t bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / slab;
            const bool ex = bx + 1 < g.nbx, ey = by + 1 < g.nby, ez = bz + 1 < g.nbz;
            const bool exists = (!(bo & 1) || ex) && (!(bo & 2) || ey) && (!(bo & 4) || ez);
            const uint32_t nbid = b + ((bo & 1) ? 1u : 0u) + ((bo & 2) ? g.nbx : 0u) + ((bo & 4) ? slab : 0u);
            sm.nslot[t][bo] = exists ? s.islot[nbid] : -1;
            if (bo == 0) {
                sm.bid[t] = b;
                const uint32_t lx = min(4u, g.nx - 1 - min(g.nx - 1, 4 * bx));
                const uint32_t ly = min(4u, g.ny - 1 - min(g.ny - 1, 4 * by));
                const uint32_t lz = min(4u, g.nz - 1 - min(g.nz - 1, 4 * bz));
                sm.lim[t] = lx | (ly << 4) | (lz << 8);
            }
        }
        __syncwarp();

        // ---- B: stage samples (all loads first, then all stores)
        float4 v[2 * kBlocksPerWarp];
#pragma unroll
        for (int q = 0; q < kBlocksPerWarp; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t job = h ? job1 : job0;
                v[2 * q + h] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < nb_w && (job & 1u)) {
                    const int32_t sl = sm.nslot[t0 + q][(job >> 2) & 7u];
                    if (sl >= 0) {
                        const float *p = s.slots + (size_t)sl * 64 + ((job >> 5) & 63u);
                        if (job & 2u) v[2 * q + h] = __ldg(reinterpret_cast<const float4 *>(p));
                        else v[2 * q + h].x = __ldg(p);
                    }
                }
            }
#pragma unroll
        for (int q = 0; q < kBlocksPerWarp; q++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t job = h ? job1 : job0;
                if (q < nb_w && (job & 1u)) {
                    float *d = halo_w + q * kHalo + (job >> 11);
                    if (job & 2u) *reinterpret_cast<float4 *>(d) = v[2 * q + h];
                    else *d = v[2 * q + h].x;
                }
            }
        __syncwarp();

        // ---- C: classify and count
        uint32_t n0p = 0, n1p = 0;            // per-cell counts of the 4 blocks, one byte each
#pragma unroll
        for (int q = 0; q < kBlocksPerWarp; q++) {
            if (q >= nb_w) continue;          // warp-uniform
            const float *hb = halo_w + q * kHalo;
            uint32_t m[5];
#pragma unroll
            for (int r = 0; r < 4; r++) m[r] = __ballot_sync(0xffffffffu, cls[r] >= 0 && hb[cls[r]] < iso);
            m[4] = 0;
            const uint32_t lim = sm.lim[t0 + q];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int cell = lane + 32 * h;
                const uint32_t lo = cword[h] == 0 ? m[0] : (cword[h] == 1 ? m[1] : m[2]);
                const uint32_t hi = cword[h] == 0 ? m[1] : (cword[h] == 1 ? m[2] : m[3]);
                const uint32_t W = __funnelshift_r(lo, hi, cshift[h]);
                uint32_t cs = (W & 3u) | ((W >> 3) & 0xCu) | ((W >> 21) & 0x30u) | ((W >> 24) & 0xC0u);
                const bool valid = (uint32_t)(cell & 3) < (lim & 15u) && (uint32_t)((cell >> 2) & 3) < ((lim >> 4) & 15u) &&
                                   (uint32_t)(cell >> 4) < ((lim >> 8) & 15u);
                cs = valid ? cs : 0u;
                sm.cases[t0 + q][cell] = (uint8_t)cs;
                const uint32_t n = sm.num_tri[cs];
                if (h == 0) n0p |= n << (8 * q);
                else n1p |= n << (8 * q);
                if (debug) s.dbg_cases[(size_t)(base + t0 + q) * 64 + cell] = (uint8_t)cs;
            }
        }
        uint32_t i0 = n0p, i1 = n1p;          // inclusive warp scans, 4 byte lanes each (sums <= 160)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a0 = __shfl_up_sync(0xffffffffu, i0, o), a1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) { i0 += a0; i1 += a1; }
        }
        const uint32_t s0 = __shfl_sync(0xffffffffu, i0, 31), s1 = __shfl_sync(0xffffffffu, i1, 31);
        uint32_t btot[kBlocksPerWarp], boff[kBlocksPerWarp], wtot = 0;
#pragma unroll
        for (int q = 0; q < kBlocksPerWarp; q++) {
            btot[q] = ((s0 >> (8 * q)) & 0xFFu) + ((s1 >> (8 * q)) & 0xFFu);
            boff[q] = wtot;
            wtot += btot[q];
        }

        // ---- D: prefix over tiles: warp totals -> tile total -> one
        // decoupled look-back per tile (warp 0), then each warp's base
        if (lane == 0) sm.wtot[warp] = wtot;
        __syncthreads();
        if (warp == 0) {
            const uint32_t mine = lane < kWarps ? sm.wtot[lane] : 0u;
            uint32_t tot = mine;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            const unsigned long long excl = lookback_exclusive(s.desc_mc, tile, tot, &c->status);
            if (lane == 0) {
                sm.tile_base = excl;
                if (tile == ntiles - 1) c->n_tri = excl + tot;
            }
        }
        __syncthreads();
        unsigned long long wbase = sm.tile_base;
        for (int w = 0; w < warp; w++) wbase += sm.wtot[w];
        if (lane == 0) {
            uint32_t occ = 0;
#pragma unroll
            for (int q = 0; q < kBlocksPerWarp; q++) occ += btot[q] > 0;
            occ_local += occ;
        }
        if (debug && lane < nb_w) {
#pragma unroll
            for (int q = 0; q < kBlocksPerWarp; q++)
                if (q == lane) {
                    s.dbg_btri[base + t0 + q] = btot[q];
                    s.dbg_boff[base + t0 + q] = wbase + boff[q];
                }
        }
        if (wtot == 0) continue;

        // ---- E: triangle -> (block, cell, k) map, then vertices
        uint16_t *tm = sm.tmap[warp];
#pragma unroll
        for (int q = 0; q < kBlocksPerWarp; q++) {
            if (q >= nb_w) continue;
            const uint32_t n0 = (n0p >> (8 * q)) & 0xFFu, n1 = (n1p >> (8 * q)) & 0xFFu;
            const uint32_t o0 = boff[q] + ((i0 >> (8 * q)) & 0xFFu) - n0;
            const uint32_t o1 = boff[q] + ((s0 >> (8 * q)) & 0xFFu) + ((i1 >> (8 * q)) & 0xFFu) - n1;
            for (uint32_t k = 0; k < n0; k++) tm[o0 + k] = (uint16_t)((q << 9) | (lane << 3) | k);
            for (uint32_t k = 0; k < n1; k++) tm[o1 + k] = (uint16_t)((q << 9) | ((lane + 32) << 3) | k);
        }
        __syncwarp();
        for (uint32_t vtx = lane; vtx < 3 * wtot; vtx += 32) {
            const uint32_t tri = vtx / 3u, j = vtx - 3u * tri;
            const uint32_t e16 = tm[tri];
            const uint32_t q = e16 >> 9, cell = (e16 >> 3) & 63u, k = e16 & 7u;
            const uint32_t cs = sm.cases[t0 + q][cell];
            const uint32_t info = sm.edge_info[sm.tri_edges[cs][3 * k + j]];
            const int cx = (int)(cell & 3u), cy = (int)((cell >> 2) & 3u), cz = (int)(cell >> 4);
            const float *hb = halo_w + q * kHalo + cx + 8 * cy + 40 * cz;
            const float vlo = hb[info & 0xFFu], vhi = hb[(info >> 8) & 0xFFu];
            const float tt = __fdiv_rn(__fsub_rn(iso, vlo), __fsub_rn(vhi, vlo));
            const int px = cx + (int)((info >> 16) & 1u), py = cy + (int)((info >> 17) & 1u), pz = cz + (int)((info >> 18) & 1u);
            const uint32_t a = (info >> 19) & 3u;
            float4 p = make_float4((float)px, (float)py, (float)pz, __uint_as_float(sm.bid[t0 + q]));
            if (a == 0) p.x = __fadd_rn(p.x, tt);
            else if (a == 1) p.y = __fadd_rn(p.y, tt);
            else p.z = __fadd_rn(p.z, tt);
            const unsigned long long gt = wbase + tri;
            if (gt < tri_cap) {
                out[gt * 3 + j] = p;
                if (debug) {
                    const uint32_t b = sm.bid[t0 + q];
                    const uint32_t bx = b % g.nbx, by = (b / g.nbx) % g.nby, bz = b / slab;
                    const unsigned long long vox = (unsigned long long)(4 * bx + px) +
                        (unsigned long long)g.nx * ((unsigned long long)(4 * by + py) +
                                                    (unsigned long long)g.ny * (unsigned long long)(4 * bz + pz));
                    s.dbg_edges[gt * 3 + j] = 3ull * vox + a;
                }
            }
        }
        __syncwarp();
    }
    if (lane == 0 && occ_local) atomicAdd(&sm.occ, occ_local);
    __syncthreads();
    if (threadIdx.x == 0 && sm.occ) atomicAdd(&c->n_occ, sm.occ);
}

size_t mc_smem_bytes() { return sizeof(Smem); }

void launch_mc(const DevState &s, const Geom &g, bool debug, int grid, cudaStream_t st) {
    mc_kernel<<<grid, kThreads, sizeof(Smem), st>>>(s, g, debug ? 1 : 0);
}

int mc_occupancy() {
    cudaFuncSetAttribute(mc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_kernel, kThreads, sizeof(Smem));
    return occ;
}

}  // namespace bcmc
