// The per-extraction pipeline (paper Section 4, Fig. "algorithm_sketch"):
//
//   prep    clear counters and look-back descriptors, advance the epoch
//   cull    Section 4.1 + the first step of Algorithm 1: mark active blocks,
//           compact I_active, I_new and the candidates in one pass, stamp
//           cache hits
//   lru_a   Algorithm 1 (grow, select least recently used free slots,
//           assign, evict) over the used-slot list
//   lru_b   append this epoch's slots to the list (most recent last)
//   decode  Section 4.2.1: decode each new block into its slot
//   mc      Sections 4.3-4.5 (mc.cu): count, scan, emit
//
// Sizes that only the device knows (n_active, n_new, ...) never come back
// to the host between kernels: the kernels are persistent and take their
// work from the volumes' control blocks.  Every kernel runs over a Launch
// (launch.cuh): one volume, or a batch of volumes in the same launches.
// The work a kernel assigns to each volume is computed only from values
// no kernel of the same launch changes, so all blocks agree on it.
#include <algorithm>
#include <cstdint>

#include "codec.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "launch.cuh"
#include "tile_scan.cuh"

namespace bcmc {

// ================================================================ prep

template <bool kOne>
__global__ void __launch_bounds__(kThreads) prep_kernel(Launch L) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t v = 0; v < L.n; v++) {
        const VolEntry &e = vol_of<kOne>(L, v);
        const DevState &s = e.s;
        const uint32_t n_mc_desc = s.ctl->mc_tiles;   // descriptors the last triangle pass used
        for (uint32_t i = tid; i < n_mc_desc; i += stride) {
            s.desc_mc[i] = 0;
            s.desc_occ[i] = 0;
            if (s.desc_vtx) s.desc_vtx[i] = 0;
        }
        for (uint32_t i = tid; i < e.n_cull_desc; i += stride) {
            s.desc_cull[i] = 0;
            s.desc_cand[i] = 0;
        }
        for (uint32_t i = tid; i < e.n_lru_desc; i += stride) {
            s.desc_lru_a[i] = 0;
            s.desc_lru_b[i] = 0;
        }
    }
    for (uint32_t v = tid; v < L.n; v += stride) {
        Ctl *c = vol_of<kOne>(L, v).s.ctl;
        c->epoch += 1;
        c->n_active = 0;
        c->n_new = 0;
        c->n_cand = 0;
        c->n_assign = 0;
        c->status = 0;
        c->n_occ = 0;
        c->n_tri = 0;
        c->n_vtx = 0;
    }
    if (tid < kNumLaunchCounters) L.ctr[tid] = 0;
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
// triangle stage visits (ascending block ids).

template <int kR>
struct CullSmem {
    TileScan<kR> ts, tc;
    uint32_t bal[3][kR][8];           // active, new, candidate ballots
};

// kSeg: the variant that reads segment ranges first (where a volume has them)
template <int kR, bool kSeg>
__device__ __forceinline__ void cull_tile(const DevState &s, const Geom &g, uint32_t tile, uint32_t ntiles,
                                          CullSmem<kR> &sm) {
    constexpr uint32_t kTile = kR * kThreads;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t epoch = s.ctl->epoch;
    const float iso = s.ctl->params.iso;
    const Params &prm = s.ctl->params;
    const bool all = (prm.flags & kParamAllBlocks) != 0;             // the full-volume baseline
    // a wave's block-id window (everything outside it is treated as inactive)
    const bool win = (prm.flags & kParamWindow) != 0;
    const uint32_t w_lo = win ? prm.win_lo : 0u, w_act = win ? prm.win_act_hi : g.nb,
                   w_cand = win ? prm.win_cand_hi : g.nb;
    // groups of kHalf rounds (two groups for tiles of 2048 and 4096 blocks,
    // four for 8192); in each, every load (3x3x3 hull, +group hull, slot)
    // is issued before any of it is used, so a tile waits for one memory
    // round trip per group rather than one per round
    constexpr int kHalf = kR >= 16 ? 8 : kR / 2;
#pragma unroll
    for (int half = 0; half < kR / kHalf; half++) {
        // with segment ranges, a block's reads are skipped when its segment's
        // range cannot hold the isovalue (a whole round of 256 blocks spans 4
        // segments: the warp's 32 lanes read one, a broadcast)
        uint32_t live = ~0u;
        if (kSeg && s.seg != nullptr && !all) {   // uniform
            float2 sh[kHalf];
#pragma unroll
            for (int i = 0; i < kHalf; i++) {
                const uint32_t b = tile * kTile + (half * kHalf + i) * kThreads + threadIdx.x;
                sh[i] = b < g.nb ? __ldg(s.seg + b / kSegBlocks) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int i = 0; i < kHalf; i++)
                if (!((sh[i].x < iso) && (iso <= sh[i].y))) live &= ~(1u << i);
        }
        float2 h[kHalf], h8[kHalf];
        int32_t sl[kHalf];
#pragma unroll
        for (int i = 0; i < kHalf; i++) {
            const uint32_t b = tile * kTile + (half * kHalf + i) * kThreads + threadIdx.x;
            const bool in = b < g.nb && (!kSeg || ((live >> i) & 1u));
            h[i] = in ? __ldg(s.hull + b) : make_float2(0.f, 0.f);
            h8[i] = in ? __ldg(s.hull8 + b) : make_float2(0.f, 0.f);
            sl[i] = in ? s.islot[b] : -1;
        }
#pragma unroll
        for (int i = 0; i < kHalf; i++) {
            const int r = half * kHalf + i;
            const uint32_t b = tile * kTile + r * kThreads + threadIdx.x;
            const bool act = b < g.nb && b >= w_lo && b < w_act && (all || ((h[i].x < iso) && (iso <= h[i].y)));
            const bool cand = act && b < w_cand && (all || ((h8[i].x < iso) && (iso <= h8[i].y)));
            const bool nw = act && sl[i] < 0;
            if (act && sl[i] >= 0) s.slast[sl[i]] = epoch;       // a hit: the slot's age resets
            const uint32_t ab = __ballot_sync(0xffffffffu, act);
            const uint32_t nbits = __ballot_sync(0xffffffffu, nw);
            const uint32_t cb = __ballot_sync(0xffffffffu, cand);
            if (lane == 0) {
                sm.bal[0][r][warp] = ab;
                sm.bal[1][r][warp] = nbits;
                sm.bal[2][r][warp] = cb;
                sm.ts.cnt[r][warp] = ((uint32_t)__popc(ab) << 16) | (uint32_t)__popc(nbits);
                sm.tc.cnt[r][warp] = (uint32_t)__popc(cb);
                const uint32_t first = tile * kTile + r * kThreads + warp * 32;
                if (first < g.nb) s.mactive[first >> 5] = ab;
            }
        }
    }
    __syncthreads();
    // test hook: tile 0 keeps its prefixes to itself, so the other tiles'
    // waits run out (after a short limit) and the extraction reports a timeout
    const bool withhold = (prm.flags & kParamTestWithhold) != 0;
    const bool publish = !(withhold && tile == 0);
    const int spin_limit = withhold ? kTestSpinLimit : kSpinLimit;
    if (warp == 0) {                       // active and new counts
        const uint32_t tot = scan_tile_counts(sm.ts);
        const unsigned long long agg = ((unsigned long long)(tot >> 16) << 31) | (tot & 0xFFFFu);
        const unsigned long long excl =
            publish ? lookback_exclusive(s.desc_cull, tile, agg, &s.ctl->status, kStatusTimeout, spin_limit) : 0ull;
        if (lane == 0) {
            sm.ts.excl = excl;
            if (tile == ntiles - 1) {
                const unsigned long long incl = excl + agg;
                s.ctl->n_active = (uint32_t)(incl >> 31);
                s.ctl->n_new = (uint32_t)(incl & 0x7FFFFFFFu);
            }
        }
    } else if (warp == 1) {                // candidate count, in parallel
        const uint32_t totc = scan_tile_counts(sm.tc);
        const unsigned long long exclc =
            publish ? lookback_exclusive(s.desc_cand, tile, totc, &s.ctl->status, kStatusTimeout, spin_limit) : 0ull;
        if (lane == 0) {
            sm.tc.excl = exclc;
            if (tile == ntiles - 1) s.ctl->n_cand = (uint32_t)(exclc + totc);
        }
    }
    __syncthreads();
    const uint32_t act_base = (uint32_t)(sm.ts.excl >> 31), new_base = (uint32_t)(sm.ts.excl & 0x7FFFFFFFu);
    const uint32_t cand_base = (uint32_t)sm.tc.excl;
#pragma unroll 4
    for (int r = 0; r < kR; r++) {
        const uint32_t b = tile * kTile + r * kThreads + threadIdx.x;
        const uint32_t ab = sm.bal[0][r][warp], nbits = sm.bal[1][r][warp], cb = sm.bal[2][r][warp];
        const uint32_t off = sm.ts.cnt[r][warp];
        const uint32_t ai = act_base + (off >> 16) + __popc(ab & lt);
        const uint32_t ci = cand_base + sm.tc.cnt[r][warp] + __popc(cb & lt);
        const uint32_t ni = new_base + (off & 0xFFFFu) + __popc(nbits & lt);
        if (s.iactive && ((ab >> lane) & 1u) && ai < s.list_cap) s.iactive[ai] = b;
        if (((cb >> lane) & 1u) && ci < s.list_cap) s.icand[ci] = b;
        if (((nbits >> lane) & 1u) && ni < s.list_cap) s.inew[ni] = b;
    }
    __syncthreads();
}

template <int kR, bool kOne, bool kSeg>
__global__ void __launch_bounds__(kThreads) cull_kernel(Launch L) {
    __shared__ CullSmem<kR> sm;
    __shared__ uint32_t pre[kMaxBatch + 1];
    __shared__ uint32_t slot_x;
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) { return ceil_div(vol_of<kOne>(L, v).g.nb, kR * kThreads); }, pre);
    while (true) {
        const uint32_t x = next_item(&L.ctr[kLcCull], &slot_x);
        if (x >= total) break;
        const uint32_t v = item_vol<kOne>(pre, L.n, x);
        const VolEntry &e = vol_of<kOne>(L, v);
        cull_tile<kR, kSeg>(e.s, e.g, x - item_base<kOne>(pre, v), vol_items<kOne>(pre, v, total), sm);
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

__device__ __forceinline__ void assign_slot(const DevState &s, uint32_t slot, uint32_t r, uint32_t epoch,
                                            uint32_t nb) {
    const uint32_t b = s.inew[r];
    if (!in_bounds(slot < s.ctl->cap && b < nb && r < s.list_cap, &s.ctl->status)) return;
    const int32_t old = s.sblock[slot];
    if (old >= 0 && in_bounds((uint32_t)old < nb, &s.ctl->status)) s.islot[old] = -1;   // evict
    s.sblock[slot] = (int32_t)b;
    s.islot[b] = (int32_t)slot;
    s.slast[slot] = epoch;
    s.newslot[r] = slot;
}

struct LruPlan {
    uint32_t S2, n_assign, from_unused, from_used, avail_used;
    bool fits;
};

// the update's sizes, from values the cull fixed
__device__ __forceinline__ LruPlan lru_plan(const Ctl *c) {
    LruPlan p;
    const uint32_t n_active = c->n_active, n_new = c->n_new, S = c->S, u = c->u, cap = c->cap;
    const uint32_t n_hit = n_active - n_new;
    const uint32_t n_avail = S - n_hit;
    p.S2 = S;
    if (n_new > n_avail) p.S2 = min(cap, max(2u * S, S + (n_new - n_avail)));
    p.fits = n_new <= p.S2 - n_hit;
    p.n_assign = p.fits ? n_new : 0u;
    p.from_unused = min(p.n_assign, p.S2 - u);
    p.from_used = p.n_assign - p.from_unused;
    p.avail_used = u - n_hit;
    return p;
}

// Work items of a volume in lru_a: [plan] [tiles of the used-slot list]
// [chunks of direct assignments from never-used slots].  After a cull
// timeout the counts may be short: only the plan item runs (no change).
constexpr uint32_t kAssignChunk = 1024;

__device__ __forceinline__ uint32_t lru_a_items(const Ctl *c) {
    if (c->status & kStatusTimeout) return 1u;
    const LruPlan p = lru_plan(c);
    return 1u + ceil_div(c->u, kScanTile) + ceil_div(p.from_unused, kAssignChunk);
}

template <bool kOne>
__global__ void __launch_bounds__(kThreads) lru_a_kernel(Launch L) {
    __shared__ TileScan<kRounds> ts;
    __shared__ uint32_t pre[kMaxBatch + 1];
    __shared__ uint32_t slot_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t total =
        launch_prefix<kOne>(L, [&](uint32_t v) { return lru_a_items(vol_of<kOne>(L, v).s.ctl); }, pre);
    while (true) {
        const uint32_t x = next_item(&L.ctr[kLcLruA], &slot_x);
        if (x >= total) break;
        const uint32_t v = item_vol<kOne>(pre, L.n, x);
        const DevState &s = vol_of<kOne>(L, v).s;
        Ctl *c = s.ctl;
        const uint32_t item = x - item_base<kOne>(pre, v);
        const uint32_t epoch = c->epoch, u = c->u, nb = vol_of<kOne>(L, v).g.nb;
        if (item == 0) {                                // the plan
            if (threadIdx.x == 0) {
                c->lpar_next = c->lpar ^ 1u;
                if (c->status & kStatusTimeout) {
                    c->S_next = c->S;
                    c->u_next = u;
                    c->n_assign = 0;
                    c->keep_base = 0;
                } else {
                    const LruPlan p = lru_plan(c);
                    c->S_next = p.S2;
                    c->u_next = u + p.from_unused;
                    c->from_unused = p.from_unused;
                    c->from_used = p.from_used;
                    c->keep_base = p.avail_used - p.from_used;
                    c->n_assign = p.n_assign;
                    if (!p.fits) atomicOr(&c->status, (uint32_t)kStatusBudget);
                }
            }
            continue;                                   // block-uniform
        }
        const LruPlan p = lru_plan(c);
        const uint32_t ntiles = ceil_div(u, kScanTile);
        if (item <= ntiles) {                           // a tile of the used-slot list
            const uint32_t tile = item - 1;
            const uint32_t *Lst = s.lbuf[c->lpar];
            uint32_t *Ln = s.lbuf[c->lpar ^ 1u];
            uint32_t bits[kRounds], slot[kRounds];
#pragma unroll
            for (int r = 0; r < kRounds; r++) {
                const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
                slot[r] = i < u ? Lst[i] : 0u;
            }
            uint32_t last[kRounds];           // all gathers issued before any is used
#pragma unroll
            for (int r = 0; r < kRounds; r++) {
                const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
                last[r] = i < u ? s.slast[slot[r]] : epoch;
            }
#pragma unroll
            for (int r = 0; r < kRounds; r++) {
                bits[r] = __ballot_sync(0xffffffffu, last[r] != epoch);
                if (lane == 0) ts.cnt[r][warp] = (uint32_t)__popc(bits[r]);
            }
            __syncthreads();
            if (warp == 0) {
                const uint32_t tot = scan_tile_counts(ts);
                const unsigned long long excl = lookback_exclusive(s.desc_lru_a, tile, tot, &c->status, kStatusTimeoutLru);
                if (lane == 0) ts.excl = excl;
            }
            __syncthreads();
            const uint32_t base = (uint32_t)ts.excl;
#pragma unroll
            for (int r = 0; r < kRounds; r++) {
                if (!((bits[r] >> lane) & 1u)) continue;
                const uint32_t rank = base + ts.cnt[r][warp] + __popc(bits[r] & lt);
                if (rank < p.from_used) assign_slot(s, slot[r], p.from_unused + rank, epoch, nb);
                else if (in_bounds(rank - p.from_used < c->cap, &c->status)) Ln[rank - p.from_used] = slot[r];
            }
            __syncthreads();
        } else {                                        // never-used slots go straight to new blocks
            const uint32_t r0 = (item - 1 - ntiles) * kAssignChunk, r1 = min(p.from_unused, r0 + kAssignChunk);
            for (uint32_t r = r0 + threadIdx.x; r < r1; r += kThreads) assign_slot(s, u + r, r, epoch, nb);
        }
    }
}

// lru_b's work: every slot stamped this epoch (hits and new assignments),
// by index, appended after the list's surviving part.  Run by its own
// kernel, or by the 256-thread decode kernel once its blocks are decoded
// (the decode commits the update meanwhile: nothing here reads what the
// commit changes).  Called by all threads of the block.
template <bool kOne>
__device__ __forceinline__ void lru_b_work(const Launch &L, TileScan<kRounds> &ts, uint32_t *pre, uint32_t *slot_x) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    // after a cull timeout the volume's cache is emptied by the host: no tiles
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) {
            const Ctl *c = vol_of<kOne>(L, v).s.ctl;
            return (c->status & kStatusTimeout) ? 0u : ceil_div(c->S_next, kScanTile);
        },
        pre);
    while (true) {
        const uint32_t x = next_item(&L.ctr[kLcLruB], slot_x);
        if (x >= total) break;
        const uint32_t v = item_vol<kOne>(pre, L.n, x);
        const DevState &s = vol_of<kOne>(L, v).s;
        Ctl *c = s.ctl;
        const uint32_t tile = x - item_base<kOne>(pre, v);
        const uint32_t epoch = c->epoch, S2 = c->S_next, keep = c->keep_base;
        uint32_t *Ln = s.lbuf[c->lpar_next];
        uint32_t bits[kRounds], last[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; r++) {   // all loads first
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            last[r] = i < S2 ? s.slast[i] : ~epoch;
        }
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            bits[r] = __ballot_sync(0xffffffffu, last[r] == epoch);
            if (lane == 0) ts.cnt[r][warp] = (uint32_t)__popc(bits[r]);
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t tot = scan_tile_counts(ts);
            const unsigned long long excl = lookback_exclusive(s.desc_lru_b, tile, tot, &c->status, kStatusTimeoutLru);
            if (lane == 0) ts.excl = excl;
        }
        __syncthreads();
        const uint32_t base = keep + (uint32_t)ts.excl;
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            if (!((bits[r] >> lane) & 1u)) continue;
            const uint32_t i = tile * kScanTile + r * kThreads + threadIdx.x;
            const uint32_t at = base + ts.cnt[r][warp] + __popc(bits[r] & lt);
            if (in_bounds(at < c->cap, &c->status)) Ln[at] = i;
        }
        __syncthreads();
    }
}

template <bool kOne>
__global__ void __launch_bounds__(kThreads) lru_b_kernel(Launch L) {
    __shared__ TileScan<kRounds> ts;
    __shared__ uint32_t pre[kMaxBatch + 1];
    __shared__ uint32_t slot_x;
    lru_b_work<kOne>(L, ts, pre, &slot_x);
}

// ================================================================ decode (Section 4.2.1)
//
// Chunks of kDecodeThreads new blocks; each warp of a chunk stages its 32
// blocks' words in shared memory with coalesced loads and decodes them one
// per lane (codec.cuh).  Chunk 0 of every volume (each volume has at least
// one) also commits the volume's cache update.  With 256-thread blocks the
// kernel then does lru_b's work (the list for the next update, which
// nothing before then reads): its memory latency hides behind the decoding
// and one launch and grid-wide wait fewer run per extraction.

template <int kDecodeThreads>
constexpr bool decode_runs_lru_b() { return kDecodeThreads == kThreads; }

template <int kDecodeThreads, bool kOne>
__global__ void __launch_bounds__(kDecodeThreads, 768 / kDecodeThreads) decode_new_kernel(Launch L) {   // 24 warps/SM
    // dynamic: the plane columns (32 words per thread), then one staging
    // area per warp for the launch's largest rate
    extern __shared__ uint64_t dsm[];
    __shared__ uint32_t pre[kMaxBatch + 1];
    __shared__ TileScan<kRounds> ts;                  // lru_b's work
    __shared__ uint32_t slot_x;
    const uint32_t warp = threadIdx.x >> 5;
    const DecodeSmem sm = decode_smem_layout(dsm, kDecodeThreads, kOne ? L.one.g.rate : L.max_rate);
    load_group_table(sm.tab);
    __syncthreads();
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) { return max(1u, ceil_div(vol_of<kOne>(L, v).s.ctl->n_assign, kDecodeThreads)); },
        pre);
    for (uint32_t x = blockIdx.x; x < total; x += gridDim.x) {
        const uint32_t v = item_vol<kOne>(pre, L.n, x);
        const DevState &s = vol_of<kOne>(L, v).s;
        Ctl *c = s.ctl;
        const uint32_t chunk = x - item_base<kOne>(pre, v);
        if (c->status & kStatusAnyTimeout) continue;  // block-uniform: no barrier in this loop
        if (chunk == 0 && threadIdx.x == 0) {         // commit the cache update
            c->S = c->S_next;
            c->u = c->u_next;
            c->lpar = c->lpar_next;
        }
        const uint32_t n_assign = c->n_assign;
        const uint32_t r0 = chunk * kDecodeThreads + warp * 32u;
        if (r0 >= n_assign) continue;                 // warp-uniform
        const uint32_t r = r0 + (threadIdx.x & 31u);
        const uint32_t rate = vol_of<kOne>(L, v).g.rate;
        bool have = r < n_assign;
        const uint32_t b = have ? s.inew[r] : 0u;
        const uint32_t slot = have ? s.newslot[r] : 0u;
        have = have && in_bounds(b < vol_of<kOne>(L, v).g.nb && slot < c->cap, &c->status);
        stage_blocks<true>(s.bits, rate, b, have, sm.stage);
        if (!have) continue;
        float val[64];
        decode_staged(sm.stage + (threadIdx.x & 31u) * (2u * rate + 1u), rate, sm.tab, val, sm.planes + threadIdx.x,
                      kDecodeThreads);
        float4 *dst = reinterpret_cast<float4 *>(s.slots + (size_t)slot * 64);
#pragma unroll
        for (int i = 0; i < 16; i++) dst[i] = make_float4(val[4 * i], val[4 * i + 1], val[4 * i + 2], val[4 * i + 3]);
    }
    if constexpr (decode_runs_lru_b<kDecodeThreads>()) {
        __syncthreads();                              // `pre` is lru_b's from here
        lru_b_work<kOne>(L, ts, pre, &slot_x);
    }
}

// ================================================================ batch bookkeeping

__global__ void batch_params_kernel(Launch L, const float *__restrict__ iso) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < L.n; v += gridDim.x * blockDim.x) {
        Params &p = L.vols[v].s.ctl->params;
        p.iso = iso[v];
        p.format = kVertexFloat4;
        p.flags = 0;
    }
}

// One block: place the volumes' surfaces one after another in the batch's
// output (volume v starts after the triangles of volumes 0..v-1 and may
// use the rest of the buffer).
__global__ void __launch_bounds__(kThreads) batch_offsets_kernel(Launch L, const BatchOut *__restrict__ bo,
                                                                 unsigned long long *tri_base) {
    __shared__ unsigned long long warp_tot[kThreads / 32];
    const uint32_t per = (L.n + kThreads - 1) / kThreads;
    const uint32_t v0 = threadIdx.x * per;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long sum = 0;
    for (uint32_t k = 0; k < per; k++)
        if (v0 + k < L.n) sum += L.vols[v0 + k].s.ctl->n_tri;
    unsigned long long incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long run = incl - sum;
    for (int w = 0; w < warp; w++) run += warp_tot[w];
    const unsigned long long out = bo->out, cap = bo->tri_cap;
    for (uint32_t k = 0; k < per; k++) {
        const uint32_t v = v0 + k;
        if (v >= L.n) break;
        Ctl *c = L.vols[v].s.ctl;
        tri_base[v] = run;
        c->params.out = out + run * 3 * sizeof(float4);
        c->params.tri_cap = run < cap ? cap - run : 0ull;
        run += c->n_tri;
        if (v == L.n - 1) tri_base[L.n] = run;
    }
}

// copy every volume's control block into one array (one readback)
__global__ void batch_gather_kernel(Launch L, Ctl *dst) {
    constexpr uint32_t kWords = sizeof(Ctl) / 4;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n * kWords; i += gridDim.x * blockDim.x)
        reinterpret_cast<uint32_t *>(dst)[i] =
            reinterpret_cast<const uint32_t *>(L.vols[i / kWords].s.ctl)[i % kWords];
}

// ================================================================ waves (over-budget extraction)

// Active blocks of each z-layer of blocks (a layer is nbx*nby consecutive
// ids): the host packs layers into waves whose active blocks fit the cache.
__global__ void __launch_bounds__(kThreads) count_layers_kernel(const float2 *__restrict__ hull, Geom g, float iso,
                                                                uint32_t *layer_active) {
    const uint32_t slab = g.nbx * g.nby;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < g.nb; b += gridDim.x * blockDim.x) {
        const float2 h = __ldg(hull + b);
        const bool act = (h.x < iso) && (iso <= h.y);
        // lanes of a warp usually share a layer: one atomic per (warp, layer)
        const uint32_t z = b / slab;
        const uint32_t peers = __match_any_sync(__activemask(), z);
        const uint32_t n = __popc(__ballot_sync(__activemask(), act) & peers);
        if (n && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&layer_active[z], n);
    }
}

void launch_count_layers(const float2 *hull, const Geom &g, float iso, uint32_t *layer_active, cudaStream_t st) {
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((g.nb + kThreads - 1) / kThreads, 65535u));
    count_layers_kernel<<<blocks, kThreads, 0, st>>>(hull, g, iso, layer_active);
}

// ================================================================ load-time and utility kernels

// per block: min/max of the block ranges over its 3x3x3 block neighbourhood
// (hull) and over its 2x2x2 +group (hull8)
__global__ void hull_kernel(const float *__restrict__ bmin, const float *__restrict__ bmax, float2 *hull,
                            float2 *hull8, Geom g, uint32_t *status) {
    const uint32_t slab = g.nbx * g.nby;
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < g.nb; b += gridDim.x * blockDim.x) {
        const int bx = (int)(b % g.nbx), by = (int)((b / g.nbx) % g.nby), bz = (int)(b / slab);
        float lo = bmin[b], hi = bmax[b], lo8 = lo, hi8 = hi;
        if (!(lo <= hi)) atomicOr(status, (uint32_t)kStatusCorrupt);   // NaN, or min > max
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

// One warp per segment of kSegBlocks consecutive blocks: the min of their
// hulls' lows and the max of their highs.  A block is active only if
// lo < iso <= hi for its own hull, which lies within its segment's.
__global__ void seg_hull_kernel(const float2 *__restrict__ hull, float2 *seg, uint32_t nb) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nseg = (nb + kSegBlocks - 1) / kSegBlocks;
    for (uint32_t q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nseg; q += (gridDim.x * blockDim.x) >> 5) {
        float lo = INFINITY, hi = -INFINITY;
        for (uint32_t k = lane; k < kSegBlocks; k += 32) {
            const uint64_t b = (uint64_t)q * kSegBlocks + k;
            if (b < nb) {
                const float2 h = hull[b];
                lo = fminf(lo, h.x);
                hi = fmaxf(hi, h.y);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) seg[q] = make_float2(lo, hi);
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

// the decode kernel's dynamic shared memory for a launch
size_t decode_smem(const Launch &L, int threads) {
    return decode_smem_bytes((uint32_t)threads, L.vols ? L.max_rate : L.one.g.rate);
}

// Algorithm 1 after the cull (both list kernels), then the decode
template <bool kOne>
void cache_update(const Launch &L, const Plan &pl, cudaStream_t st, cudaEvent_t *ev, cudaEvent_t bits_ready) {
    lru_a_kernel<kOne><<<pl.lru_a, kThreads, 0, st>>>(L);
    if (pl.decode_tile != kThreads) lru_b_kernel<kOne><<<pl.lru_b, kThreads, 0, st>>>(L);   // else the decode's
    if (ev) cudaEventRecord(ev[3], st);
    if (bits_ready) cudaStreamWaitEvent(st, bits_ready, 0);   // the bitstream may still be on its way
    if (pl.decode_tile == 64) decode_new_kernel<64, kOne><<<pl.decode, 64, decode_smem(L, 64), st>>>(L);
    else if (pl.decode_tile == 256) decode_new_kernel<256, kOne><<<pl.decode, 256, decode_smem(L, 256), st>>>(L);
    else decode_new_kernel<128, kOne><<<pl.decode, 128, decode_smem(L, 128), st>>>(L);
    if (ev) cudaEventRecord(ev[4], st);
}

template <bool kOne>
void cull_only(const Launch &L, const Plan &pl, cudaStream_t st) {
    // volumes with segment ranges (the largest) take 8192-block tiles: half
    // the look-back walks of 4096-block tiles, whose depth grows with the
    // tiles in flight
    if (kOne ? L.one.s.seg != nullptr : L.seg_any != 0) cull_kernel<32, kOne, true><<<pl.cull, kThreads, 0, st>>>(L);
    else if (pl.cull_tile == 2048) cull_kernel<8, kOne, false><<<pl.cull, kThreads, 0, st>>>(L);
    else cull_kernel<16, kOne, false><<<pl.cull, kThreads, 0, st>>>(L);
}

template <bool kOne>
void front(const Launch &L, const Plan &pl, cudaStream_t st, cudaEvent_t *ev, cudaEvent_t bits_ready) {
    prep_kernel<kOne><<<pl.prep, kThreads, 0, st>>>(L);
    if (ev) cudaEventRecord(ev[1], st);
    cull_only<kOne>(L, pl, st);
    if (ev) cudaEventRecord(ev[2], st);
    cache_update<kOne>(L, pl, st, ev, bits_ready);
}

void launch_cull(const Launch &L, const Plan &pl, cudaStream_t st) {
    if (L.vols) cull_only<false>(L, pl, st);
    else cull_only<true>(L, pl, st);
}

void launch_front(const Launch &L, const Plan &pl, cudaStream_t st, cudaEvent_t *ev, cudaEvent_t bits_ready) {
    if (L.vols) front<false>(L, pl, st, ev, bits_ready);
    else front<true>(L, pl, st, ev, bits_ready);
}

void launch_cache_update(const Launch &L, const Plan &pl, cudaStream_t st) {
    if (L.vols) cache_update<false>(L, pl, st, nullptr, nullptr);
    else cache_update<true>(L, pl, st, nullptr, nullptr);
}

void launch_batch_params(const Launch &L, const float *d_iso, cudaStream_t st) {
    batch_params_kernel<<<(L.n + 255) / 256, 256, 0, st>>>(L, d_iso);
}

void launch_batch_offsets(const Launch &L, const BatchOut *bo, unsigned long long *tri_base, cudaStream_t st) {
    batch_offsets_kernel<<<1, kThreads, 0, st>>>(L, bo, tri_base);
}

void launch_batch_gather(const Launch &L, Ctl *dst, cudaStream_t st) {
    const uint32_t words = L.n * (uint32_t)(sizeof(Ctl) / 4);
    batch_gather_kernel<<<(words + 255) / 256, 256, 0, st>>>(L, dst);
}

void launch_hull(const float *bmin, const float *bmax, float2 *hull, float2 *hull8, float2 *seg, const Geom &g,
                 uint32_t *status, cudaStream_t st) {
    const uint32_t blocks = std::min<uint32_t>((g.nb + 255) / 256, 65535u * 4);
    hull_kernel<<<blocks, 256, 0, st>>>(bmin, bmax, hull, hull8, g, status);
    if (seg) {
        const uint32_t nseg = (g.nb + kSegBlocks - 1) / kSegBlocks;
        seg_hull_kernel<<<std::min<uint32_t>((nseg + 7) / 8, 65535u * 4), 256, 0, st>>>(hull, seg, g.nb);
    }
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

// the limit is set for the largest rate, so any launch fits
template <bool kOne>
void set_decode_attributes() {
    cudaFuncSetAttribute(decode_new_kernel<64, kOne>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)decode_smem_bytes(64, 32));
    cudaFuncSetAttribute(decode_new_kernel<128, kOne>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)decode_smem_bytes(128, 32));
    cudaFuncSetAttribute(decode_new_kernel<256, kOne>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)decode_smem_bytes(256, 32));
}

template <bool kOne>
Plan limits_of(const Plan &tiles, uint32_t rate, bool seg) {
    Plan pl = tiles;
    int occ = 0;
    if (seg) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cull_kernel<32, kOne, true>, kThreads, 0);
    else if (tiles.cull_tile == 2048) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cull_kernel<8, kOne, false>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cull_kernel<16, kOne, false>, kThreads, 0);
    pl.cull = std::max(1, occ);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lru_a_kernel<kOne>, kThreads, 0);
    pl.lru_a = std::max(1, occ);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lru_b_kernel<kOne>, kThreads, 0);
    pl.lru_b = std::max(1, occ);
    set_decode_attributes<false>();
    set_decode_attributes<true>();
    if (tiles.decode_tile == 64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_new_kernel<64, kOne>, 64, decode_smem_bytes(64, rate));
    else if (tiles.decode_tile == 256)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_new_kernel<256, kOne>, 256,
                                                      decode_smem_bytes(256, rate));
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, decode_new_kernel<128, kOne>, 128,
                                                       decode_smem_bytes(128, rate));
    pl.decode = std::max(1, occ);
    mc_occupancy(&pl, kOne);
    pl.prep = 2;
    return pl;
}

Plan occupancy_limits(const Plan &tiles, bool single, uint32_t rate, bool seg) {
    return single ? limits_of<true>(tiles, rate, seg) : limits_of<false>(tiles, rate, seg);
}

bool valid_tiles(const Plan &pl) {
    return (pl.cull_tile == 2048 || pl.cull_tile == 4096) &&
           (pl.decode_tile == 64 || pl.decode_tile == 128 || pl.decode_tile == 256) &&
           (pl.count_tile == 16 || pl.count_tile == 32 || pl.count_tile == 64) &&
           (pl.scan_tile == 1024 || pl.scan_tile == 2048 || pl.scan_tile == 4096) &&
           (pl.emit_tile == 16 || pl.emit_tile == 32 || pl.emit_tile == 64);
}

}  // namespace bcmc
