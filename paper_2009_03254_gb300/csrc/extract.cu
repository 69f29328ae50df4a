// The per-extraction pipeline (paper Section 4, Fig. "algorithm_sketch"):
//
//   prep    clear counters and look-back descriptors, advance the epoch
//   cull    Section 4.1 + the first step of Algorithm 1: mark active blocks,
//           compact I_active and I_new in one pass, stamp cache hits
//   lru_a   Algorithm 1 (grow, select least recently used free slots,
//           assign, evict) over the used-slot list
//   lru_b   append this epoch's slots to the list (most recent last)
//   decode  Section 4.2.1: decode each new block into its slot
//   mc      Sections 4.3-4.5 (mc.cu): halo staging, classification,
//           per-block counts, single-pass prefix over blocks, vertices
//
// Sizes that only the device knows (n_active, n_new, ...) never come back
// to the host between kernels: the kernels are persistent and take their
// work from counters in the control block.
#include <algorithm>
#include <cstdint>

#include "codec.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace bcmc {

// ================================================================ prep

__global__ void __launch_bounds__(kThreads) prep_kernel(DevState s, uint32_t n_cull_desc, uint32_t n_lru_desc,
                                                         int mc_only) {
    Ctl *c = s.ctl;
    const uint32_t n_mc_desc = c->mc_tiles;   // descriptors the last triangle pass used
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = tid; i < n_mc_desc; i += stride) s.desc_mc[i] = 0;
    if (!mc_only) {
        for (uint32_t i = tid; i < n_cull_desc; i += stride) {
            s.desc_cull[i] = 0;
            s.desc_cand[i] = 0;
        }
        for (uint32_t i = tid; i < n_lru_desc; i += stride) {
            s.desc_lru_a[i] = 0;
            s.desc_lru_b[i] = 0;
        }
    }
    if (tid == 0) {
        if (!mc_only) {
            c->epoch += 1;
            c->n_active = 0;
            c->n_new = 0;
            c->n_cand = 0;
            c->n_assign = 0;
            c->status = 0;
            for (int k = 0; k < kNumCtr; k++) c->ctr[k] = 0;
        }
        c->ctr[kCtrMc] = 0;
        c->n_occ = 0;
        c->n_tri = 0;
    }
}

// ================================================================ tile scan helpers
//
// A tile is kScanTile = kRounds * 256 entries handled by 256 threads in
// kRounds rounds; entry tile*kScanTile + r*256 + threadIdx.x belongs to
// round r.  Per (round, warp) the warp's ballot gives its 32 flags; a
// warp scan over the kRounds*8 (round, warp) counts gives each group's
// offset inside the tile.  Large tiles keep the tiles of a pass within
// one wave of resident blocks, so the look-back walk stays short.

constexpr int kRounds = kScanTile / kThreads;

struct TileScan {
    uint32_t cnt[kRounds][8];         // per (round, warp): packed counts, then exclusive offsets
    unsigned long long excl;          // tile's exclusive prefix (look-back)
    uint32_t tile;
};

// warp 0: turn ts.cnt into exclusive offsets (packed 16-bit fields add
// without carries: a tile holds at most 4096 entries) and return the
// tile's packed total in every lane
__device__ __forceinline__ uint32_t scan_tile_counts(TileScan &ts) {
    constexpr int kPer = kRounds * 8 / 32;
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

// ================================================================ cull (Section 4.1)
//
// Active test: the union of a block's range with each neighbour's range
// contains iso (lo < iso <= hi) for some neighbour or the block itself.
// That holds exactly when lo < iso <= hi for the min/max taken over the
// whole 3x3x3 block neighbourhood, which the loader precomputes (`hull`).
// Active blocks that have a slot are cache hits (slot stamped with the
// epoch: "reset the age"); the others are new.  Active blocks whose
// 2x2x2 +group range (`hull8`) also contains iso are the candidates the
// triangle stage visits; I_cand holds their positions in I_active.

__global__ void __launch_bounds__(kThreads) cull_kernel(DevState s, Geom g, uint32_t ntiles) {
    __shared__ TileScan ts;
    __shared__ TileScan tc;
    __shared__ uint32_t bal[3][kRounds][8];            // active, new, candidate ballots
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t epoch = s.ctl->epoch;
    const float iso = s.ctl->params.iso;
    const uint32_t lt = (1u << lane) - 1u;
    while (true) {
        if (threadIdx.x == 0) ts.tile = atomicAdd(&s.ctl->ctr[kCtrCull], 1u);
        __syncthreads();
        const uint32_t tile = ts.tile;
        if (tile >= ntiles) break;
        float2 h[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; r++) {               // all range loads of the tile first
            const uint32_t b = tile * kScanTile + r * kThreads + threadIdx.x;
            h[r] = b < g.nb ? __ldg(s.hull + b) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            const uint32_t b = tile * kScanTile + r * kThreads + threadIdx.x;
            const bool act = b < g.nb && (h[r].x < iso) && (iso <= h[r].y);
            bool nw = false, cand = false;
            if (act) {
                const float2 h8 = __ldg(s.hull8 + b);
                cand = (h8.x < iso) && (iso <= h8.y);
                const int32_t sl = s.islot[b];
                if (sl >= 0) s.slast[sl] = epoch;
                else nw = true;
            }
            const uint32_t ab = __ballot_sync(0xffffffffu, act);
            const uint32_t nbits = __ballot_sync(0xffffffffu, nw);
            const uint32_t cb = __ballot_sync(0xffffffffu, cand);
            if (lane == 0) {
                bal[0][r][warp] = ab;
                bal[1][r][warp] = nbits;
                bal[2][r][warp] = cb;
                ts.cnt[r][warp] = ((uint32_t)__popc(ab) << 16) | (uint32_t)__popc(nbits);
                tc.cnt[r][warp] = (uint32_t)__popc(cb);
                const uint32_t first = tile * kScanTile + r * kThreads + warp * 32;
                if (first < g.nb) s.mactive[first >> 5] = ab;
            }
        }
        __syncthreads();
        if (warp == 0) {                       // active and new counts
            const uint32_t tot = scan_tile_counts(ts);
            const unsigned long long agg = ((unsigned long long)(tot >> 16) << 31) | (tot & 0xFFFFu);
            const unsigned long long excl = lookback_exclusive(s.desc_cull, tile, agg, &s.ctl->status);
            if (lane == 0) {
                ts.excl = excl;
                if (tile == ntiles - 1) {
                    const unsigned long long incl = excl + agg;
                    s.ctl->n_active = (uint32_t)(incl >> 31);
                    s.ctl->n_new = (uint32_t)(incl & 0x7FFFFFFFu);
                }
            }
        } else if (warp == 1) {                // candidate count, in parallel
            const uint32_t totc = scan_tile_counts(tc);
            const unsigned long long exclc = lookback_exclusive(s.desc_cand, tile, totc, &s.ctl->status);
            if (lane == 0) {
                tc.excl = exclc;
                if (tile == ntiles - 1) s.ctl->n_cand = (uint32_t)(exclc + totc);
            }
        }
        __syncthreads();
        const uint32_t act_base = (uint32_t)(ts.excl >> 31), new_base = (uint32_t)(ts.excl & 0x7FFFFFFFu);
        const uint32_t cand_base = (uint32_t)tc.excl;
#pragma unroll 4
        for (int r = 0; r < kRounds; r++) {
            const uint32_t b = tile * kScanTile + r * kThreads + threadIdx.x;
            const uint32_t ab = bal[0][r][warp], nbits = bal[1][r][warp], cb = bal[2][r][warp];
            const uint32_t off = ts.cnt[r][warp];
            if ((ab >> lane) & 1u) s.iactive[act_base + (off >> 16) + __popc(ab & lt)] = b;
            if ((cb >> lane) & 1u) s.icand[cand_base + tc.cnt[r][warp] + __popc(cb & lt)] = b;
            if ((nbits >> lane) & 1u) s.inew[new_base + (off & 0xFFFFu) + __popc(nbits & lt)] = b;
        }
        __syncthreads();
    }
}

// ================================================================ cache update (Algorithm 1)
//
// The paper keeps an age per slot, sorts the free slots by age and hands
// the oldest to the new blocks.  Here a slot stores the epoch of its last
// use (S_last; age = epoch - S_last), and the sort is replaced by a list
// kept in least-recently-used order: slots [u, S) have never been used
// (S_last = 0, the oldest, in index order) and lbuf[lpar][0..u) lists the
// used slots by (S_last, index).  Each update:
//   lru_a  keeps the list's entries that were not hit this epoch, in
//          order; the first `from_used` of them (after the never-used
//          slots) go to the new blocks, the rest move to the new list;
//   lru_b  appends every slot stamped this epoch, by index.
// The new list is again ordered by (S_last, index), so the slots handed
// out are exactly those a stable sort by descending age would put first.
// Growth (more new blocks than free slots) extends [u, S) to
// max(2S, S + n_new - n_avail) slots, capped; new slots count as never
// used, i.e. they have the highest age.

__device__ __forceinline__ void assign_slot(const DevState &s, uint32_t slot, uint32_t r, uint32_t epoch) {
    const uint32_t b = s.inew[r];
    const int32_t old = s.sblock[slot];
    if (old >= 0) s.islot[old] = -1;           // evict
    s.sblock[slot] = (int32_t)b;
    s.islot[b] = (int32_t)slot;
    s.slast[slot] = epoch;
    s.newslot[r] = slot;
}

__global__ void __launch_bounds__(kThreads) lru_a_kernel(DevState s) {
    __shared__ TileScan ts;
    __shared__ uint32_t s_status;
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_status = c->status;
    __syncthreads();
    if (s_status & kStatusTimeout) {           // counts from the cull may be short: change nothing
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            c->S_next = c->S;
            c->u_next = c->u;
            c->n_assign = 0;
        }
        return;
    }
    const uint32_t epoch = c->epoch, n_active = c->n_active, n_new = c->n_new;
    const uint32_t S = c->S, u = c->u, cap = c->cap, lpar = c->lpar;
    const uint32_t n_hit = n_active - n_new;
    const uint32_t n_avail = S - n_hit;
    uint32_t S2 = S;
    if (n_new > n_avail) S2 = min(cap, max(2u * S, S + (n_new - n_avail)));
    const bool fits = n_new <= S2 - n_hit;
    const uint32_t n_assign = fits ? n_new : 0u;
    const uint32_t from_unused = min(n_assign, S2 - u);
    const uint32_t from_used = n_assign - from_unused;
    const uint32_t avail_used = u - n_hit;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->S_next = S2;
        c->u_next = u + from_unused;
        c->from_unused = from_unused;
        c->from_used = from_used;
        c->keep_base = avail_used - from_used;
        c->n_assign = n_assign;
        if (!fits) atomicOr(&c->status, (uint32_t)kStatusBudget);
    }
    const uint32_t *L = s.lbuf[lpar];
    uint32_t *Ln = s.lbuf[lpar ^ 1u];
    const uint32_t ntiles = (u + kScanTile - 1) / kScanTile;
    while (true) {
        if (threadIdx.x == 0) ts.tile = atomicAdd(&c->ctr[kCtrLruA], 1u);
        __syncthreads();
        const uint32_t tile = ts.tile;
        if (tile >= ntiles) break;
        uint32_t bits[kRounds], slot[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            slot[r] = i < u ? L[i] : 0u;
        }
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            const bool av = i < u && s.slast[slot[r]] != epoch;
            bits[r] = __ballot_sync(0xffffffffu, av);
            if (lane == 0) ts.cnt[r][warp] = (uint32_t)__popc(bits[r]);
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t tot = scan_tile_counts(ts);
            const unsigned long long excl = lookback_exclusive(s.desc_lru_a, tile, tot, &c->status);
            if (lane == 0) ts.excl = excl;
        }
        __syncthreads();
        const uint32_t base = (uint32_t)ts.excl;
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            if (!((bits[r] >> lane) & 1u)) continue;
            const uint32_t rank = base + ts.cnt[r][warp] + __popc(bits[r] & lt);
            if (rank < from_used) assign_slot(s, slot[r], from_unused + rank, epoch);
            else Ln[rank - from_used] = slot[r];
        }
        __syncthreads();
    }
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < from_unused; r += gridDim.x * blockDim.x)
        assign_slot(s, u + r, r, epoch);
}

__global__ void __launch_bounds__(kThreads) lru_b_kernel(DevState s) {
    __shared__ TileScan ts;
    __shared__ uint32_t s_status;
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    if (threadIdx.x == 0) s_status = c->status;
    __syncthreads();
    if (s_status & kStatusTimeout) return;
    const uint32_t epoch = c->epoch, S2 = c->S_next, keep = c->keep_base;
    uint32_t *Ln = s.lbuf[c->lpar ^ 1u];
    const uint32_t ntiles = (S2 + kScanTile - 1) / kScanTile;
    while (true) {
        if (threadIdx.x == 0) ts.tile = atomicAdd(&c->ctr[kCtrLruB], 1u);
        __syncthreads();
        const uint32_t tile = ts.tile;
        if (tile >= ntiles) break;
        uint32_t bits[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            const bool used_now = i < S2 && s.slast[i] == epoch;
            bits[r] = __ballot_sync(0xffffffffu, used_now);
            if (lane == 0) ts.cnt[r][warp] = (uint32_t)__popc(bits[r]);
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t tot = scan_tile_counts(ts);
            const unsigned long long excl = lookback_exclusive(s.desc_lru_b, tile, tot, &c->status);
            if (lane == 0) ts.excl = excl;
        }
        __syncthreads();
        const uint32_t base = keep + (uint32_t)ts.excl;
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            if (!((bits[r] >> lane) & 1u)) continue;
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            Ln[base + ts.cnt[r][warp] + __popc(bits[r] & lt)] = i;
        }
        __syncthreads();
    }
}

// ================================================================ decode (Section 4.2.1)

constexpr int kDecodeThreads = 128;

__global__ void __launch_bounds__(kDecodeThreads) decode_new_kernel(DevState s, Geom g) {
    __shared__ uint64_t planes[32 * kDecodeThreads];
    Ctl *c = s.ctl;
    if (c->status & kStatusTimeout) return;      // no barrier in this kernel: per-thread exit is safe
    const uint32_t n = c->n_assign;
    if (blockIdx.x == 0 && threadIdx.x == 0) {   // commit the cache update
        c->S = c->S_next;
        c->u = c->u_next;
        c->lpar ^= 1u;
    }
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint32_t b = s.inew[r];
        const uint32_t slot = s.newslot[r];
        float v[64];
        decode_block(s.bits + (size_t)b * g.rate, g.rate, v, planes + threadIdx.x, kDecodeThreads);
        float4 *dst = reinterpret_cast<float4 *>(s.slots + (size_t)slot * 64);
#pragma unroll
        for (int i = 0; i < 16; i++) dst[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
}

// ================================================================ load-time and utility kernels

// per block: min/max of the block ranges over its 3x3x3 block neighbourhood
// (hull) and over its 2x2x2 +group (hull8)
__global__ void hull_kernel(const float *__restrict__ bmin, const float *__restrict__ bmax, float2 *hull,
                            float2 *hull8, Geom g) {
    const uint32_t slab = g.nbx * g.nby;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < g.nb; b += gridDim.x * blockDim.x) {
        const int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / slab);
        float lo = bmin[b], hi = bmax[b], lo8 = lo, hi8 = hi;
        for (int dz = -1; dz <= 1; dz++) {
            const int z = bz + dz;
            if (z < 0 || z >= (int)g.nbz) continue;
            for (int dy = -1; dy <= 1; dy++) {
                const int y = by + dy;
                if (y < 0 || y >= (int)g.nby) continue;
                for (int dx = -1; dx <= 1; dx++) {
                    const int x = bx + dx;
                    if (x < 0 || x >= (int)g.nbx) continue;
                    const uint32_t n = (uint32_t)x + g.nbx * ((uint32_t)y + g.nby * (uint32_t)z);
                    lo = fminf(lo, bmin[n]);
                    hi = fmaxf(hi, bmax[n]);
                    if (dx >= 0 && dy >= 0 && dz >= 0) {
                        lo8 = fminf(lo8, bmin[n]);
                        hi8 = fmaxf(hi8, bmax[n]);
                    }
                }
            }
        }
        hull[b] = make_float2(lo, hi);
        hull8[b] = make_float2(lo8, hi8);
    }
}

__global__ void reset_cache_kernel(DevState s) {
    Ctl *c = s.ctl;
    const uint32_t cap = c->cap;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        const int32_t b = s.sblock[i];
        if (b >= 0) s.islot[b] = -1;
        s.sblock[i] = -1;
        s.slast[i] = 0;
    }
}

__global__ void reset_ctl_kernel(DevState s) {
    s.ctl->u = 0;
    s.ctl->lpar = 0;
}

__global__ void gather_slots_kernel(const float *__restrict__ slots, const int32_t *__restrict__ islot,
                                    const uint32_t *__restrict__ ids, uint64_t n, float *out, int32_t *missing) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n * 64; i += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t sl = islot[ids[i / 64]];
        if (sl < 0) {
            *missing = 1;
            out[i] = 0.0f;
        } else {
            out[i] = slots[(size_t)sl * 64 + (i % 64)];
        }
    }
}

// ================================================================ launchers

void launch_prep(const DevState &s, uint32_t n_cull_desc, uint32_t n_lru_desc, bool mc_only, int grid,
                 cudaStream_t st) {
    prep_kernel<<<grid, kThreads, 0, st>>>(s, n_cull_desc, n_lru_desc, mc_only ? 1 : 0);
}

void launch_cull(const DevState &s, const Geom &g, int grid, cudaStream_t st) {
    const uint32_t ntiles = (g.nb + kScanTile - 1) / kScanTile;
    cull_kernel<<<(int)std::min<uint32_t>(ntiles, (uint32_t)grid), kThreads, 0, st>>>(s, g, ntiles);
}

void launch_lru(const DevState &s, int grid_a, int grid_b, cudaStream_t st) {
    lru_a_kernel<<<grid_a, kThreads, 0, st>>>(s);
    lru_b_kernel<<<grid_b, kThreads, 0, st>>>(s);
}

void launch_decode_new(const DevState &s, const Geom &g, int grid, cudaStream_t st) {
    decode_new_kernel<<<grid, kDecodeThreads, 0, st>>>(s, g);
}

void launch_hull(const float *bmin, const float *bmax, float2 *hull, float2 *hull8, const Geom &g,
                 cudaStream_t st) {
    const uint32_t blocks = std::min<uint32_t>((g.nb + 255) / 256, 65535u * 4);
    hull_kernel<<<blocks, 256, 0, st>>>(bmin, bmax, hull, hull8, g);
}

void launch_reset_cache(const DevState &s, cudaStream_t st) {
    reset_cache_kernel<<<1024, 256, 0, st>>>(s);
    reset_ctl_kernel<<<1, 1, 0, st>>>(s);
}

void launch_gather_slots(const float *slots, const int32_t *islot, const uint32_t *ids, uint64_t n, float *out,
                         int32_t *missing, cudaStream_t st) {
    if (n == 0) return;
    const uint64_t blocks = std::min<uint64_t>((n * 64 + 255) / 256, 65535u);
    gather_slots_kernel<<<(unsigned)blocks, 256, 0, st>>>(slots, islot, ids, n, out, missing);
}

Grids compute_grids(int sm_count) {
    Grids gr{};
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cull_kernel, kThreads, 0);
    gr.cull = std::max(1, occ) * sm_count;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lru_a_kernel, kThreads, 0);
    gr.lru_a = std::max(1, occ) * sm_count;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lru_b_kernel, kThreads, 0);
    gr.lru_b = std::max(1, occ) * sm_count;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_new_kernel, kDecodeThreads, 0);
    gr.decode = std::max(1, occ) * sm_count;
    mc_grids(sm_count, &gr);
    gr.prep = 2 * sm_count;
    return gr;
}

}  // namespace bcmc
