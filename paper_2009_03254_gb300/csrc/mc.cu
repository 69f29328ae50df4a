// Triangle stage (paper Sections 4.3-4.5) over the candidate blocks, in
// the paper's two passes.
//
// Candidates are the active blocks whose 2x2x2 "+group" (the block and its
// +x/+y/+z face, edge and corner neighbours, the only blocks its cells
// read) has a range containing the isovalue; any block with a crossing
// cell is one (its cell's below and above corners lie in the +group), so
// no triangle is lost, and every +neighbour of a candidate is itself
// active and therefore cached.  This is the refinement Section 4.4 notes
// as possible ("checking which side the neighbor was on").
//
//   count   Section 4.4: stage each candidate's 5x5x5 samples, classify its
//           64 cells, write its triangle count
//   scan    prefix sum of the counts over the candidates (block offsets
//           and the total), single pass with decoupled look-back
//   emit    Section 4.5: stage and classify again, per-cell offsets by
//           warp scans, then one triangle (three float4 vertices) per lane
//
// Both passes give each warp 4 consecutive candidates at a time (a "warp
// tile") and no warp ever waits for another one:
//   A  slots of each block's 8 blocks of the +group (8 lanes per block)
//   B  stage the samples in shared memory: 16 float4 rows of the block,
//      its +x face, +y/+z rows, edges and corner (50 loads per block, 2
//      per lane, issued together)
//   C  classify: four ballots give the 125 below-iso bits; each cell's
//      case is 8 bits picked from them; counts from the case table
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"
#include "mc_tables.cuh"

namespace bcmc {

namespace {

constexpr int kWarps = kThreads / 32;                 // 8
constexpr int kBPW = 4;                               // candidates per warp tile
constexpr int kHalo = 200;                            // x + 8y + 40z, x,y,z in [0,5)
constexpr int kTmap = kBPW * 64 * 5;                  // triangles a warp tile can hold
constexpr int kScanItems = 2048;                      // counts per scan tile

struct WarpTile {                                     // one warp's shared-memory area
    float halo[kBPW][kHalo];
    int32_t nslot[kBPW][8];
    uint32_t bid[kBPW];
    uint32_t lim[kBPW];                               // cells per axis inside the volume, 4 bits each
    uint8_t cases[kBPW][64];
};

struct CountSmem {
    WarpTile w[kWarps];
    uint8_t num_tri[256];
    uint32_t occ;
};

struct EmitSmem {
    WarpTile w[kWarps];
    float4 stage[kWarps][96];                         // 32 triangles' vertices per warp
    uint16_t tmap[kWarps][kTmap];                     // block-in-tile (2) | cell (6) | k (3)
    uint32_t tri_row[256 * kMaxTriPerCell];           // 3 edge numbers of each table triangle, packed
    uint8_t num_tri[256];
    uint32_t edge_info[12];
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

// Per-lane constants of phases B and C.
struct LaneConst {
    uint32_t job0, job1;                // halo jobs lane and lane + 32
    int cls[4];                         // halo offsets of samples lane + 32r (or -1)
    int cword[2], cshift[2];            // where each of the lane's two cells starts in the 128-bit mask
    __device__ __forceinline__ void init(int lane) {
        job0 = halo_job(lane);
        job1 = halo_job(lane + 32);
#pragma unroll
        for (int r = 0; r < 4; r++) cls[r] = lane + 32 * r < 125 ? halo_off(lane + 32 * r) : -1;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int cell = lane + 32 * h, base = (cell & 3) + 5 * ((cell >> 2) & 3) + 25 * (cell >> 4);
            cword[h] = base >> 5;
            cshift[h] = base & 31;
        }
    }
};

// Phases A-C for the warp tile starting at candidate `base` (nb_w of
// kBPW slots used).  Leaves cases in wt.cases when kKeepCases and returns
// the per-cell triangle counts of the lane's two cells, packed one byte
// per block: n0p for cell lane, n1p for cell lane + 32.
// `b` is this lane's block (candidate base + lane/8), loaded by the caller
// one warp tile ahead.
template <bool kKeepCases, bool kDebug>
__device__ __forceinline__ void stage_and_classify(const DevState &s, const Geom &g, float iso, uint32_t base,
                                                   int nb_w, uint32_t b, WarpTile &wt, const LaneConst &lc,
                                                   const uint8_t *num_tri, uint32_t &n0p, uint32_t &n1p) {
    const int lane = threadIdx.x & 31, bq = lane >> 3, bo = lane & 7;
    const uint32_t slab = g.nbx * g.nby;
    // ---- A: +group slots
    if (bq < nb_w) {
        uint32_t bx, by, bz;
        block_coords(g, b, bx, by, bz);
        const bool ex = bx + 1 < g.nbx, ey = by + 1 < g.nby, ez = bz + 1 < g.nbz;
        const bool exists = (!(bo & 1) || ex) && (!(bo & 2) || ey) && (!(bo & 4) || ez);
        const uint32_t nbid = b + ((bo & 1) ? 1u : 0u) + ((bo & 2) ? g.nbx : 0u) + ((bo & 4) ? slab : 0u);
        wt.nslot[bq][bo] = exists ? s.islot[nbid] : -1;
        if (bo == 0) {
            wt.bid[bq] = b;
            const uint32_t lx = min(4u, g.nx - 1 - min(g.nx - 1, 4 * bx));
            const uint32_t ly = min(4u, g.ny - 1 - min(g.ny - 1, 4 * by));
            const uint32_t lz = min(4u, g.nz - 1 - min(g.nz - 1, 4 * bz));
            wt.lim[bq] = lx | (ly << 4) | (lz << 8);
        }
    }
    __syncwarp();
    // ---- B: stage samples (all loads first, then all stores)
    float4 v[2 * kBPW];
#pragma unroll
    for (int q = 0; q < kBPW; q++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t job = h ? lc.job1 : lc.job0;
            v[2 * q + h] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q < nb_w && (job & 1u)) {
                const int32_t sl = wt.nslot[q][(job >> 2) & 7u];
                if (sl >= 0) {
                    const float *p = s.slots + (size_t)sl * 64 + ((job >> 5) & 63u);
                    if (job & 2u) v[2 * q + h] = __ldg(reinterpret_cast<const float4 *>(p));
                    else v[2 * q + h].x = __ldg(p);
                }
            }
        }
#pragma unroll
    for (int q = 0; q < kBPW; q++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t job = h ? lc.job1 : lc.job0;
            if (q < nb_w && (job & 1u)) {
                float *d = &wt.halo[q][0] + (job >> 11);
                if (job & 2u) *reinterpret_cast<float4 *>(d) = v[2 * q + h];
                else *d = v[2 * q + h].x;
            }
        }
    __syncwarp();
    // ---- C: classify and count
    n0p = 0;
    n1p = 0;
#pragma unroll
    for (int q = 0; q < kBPW; q++) {
        if (q >= nb_w) continue;          // warp-uniform
        const float *hb = &wt.halo[q][0];
        uint32_t m[4];
#pragma unroll
        for (int r = 0; r < 4; r++) m[r] = __ballot_sync(0xffffffffu, lc.cls[r] >= 0 && hb[lc.cls[r]] < iso);
        const uint32_t lim = wt.lim[q];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int cell = lane + 32 * h;
            const uint32_t lo = lc.cword[h] == 0 ? m[0] : (lc.cword[h] == 1 ? m[1] : m[2]);
            const uint32_t hi = lc.cword[h] == 0 ? m[1] : (lc.cword[h] == 1 ? m[2] : m[3]);
            const uint32_t W = __funnelshift_r(lo, hi, lc.cshift[h]);
            uint32_t cs = (W & 3u) | ((W >> 3) & 0xCu) | ((W >> 21) & 0x30u) | ((W >> 24) & 0xC0u);
            const bool valid = (uint32_t)(cell & 3) < (lim & 15u) &&
                               (uint32_t)((cell >> 2) & 3) < ((lim >> 4) & 15u) &&
                               (uint32_t)(cell >> 4) < ((lim >> 8) & 15u);
            cs = valid ? cs : 0u;
            if (kKeepCases) wt.cases[q][cell] = (uint8_t)cs;
            if (kDebug) s.dbg_cases[(size_t)(base + q) * 64 + cell] = (uint8_t)cs;
            const uint32_t n = num_tri[cs];
            if (h == 0) n0p |= n << (8 * q);
            else n1p |= n << (8 * q);
        }
    }
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

}  // namespace

// ================================================================ count (Section 4.4)

template <bool kDebug>
__global__ void __launch_bounds__(kThreads) mc_count_kernel(DevState s, Geom g) {
    __shared__ CountSmem sm;
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 256; i += kThreads) sm.num_tri[i] = s.tables[i];
    if (threadIdx.x == 0) sm.occ = 0;
    __syncthreads();
    const bool failed = (c->status & (kStatusBudget | kStatusTimeout)) != 0;   // nothing below changes it
    const uint32_t n_cand = failed ? 0u : c->n_cand;
    const float iso = c->params.iso;
    const uint32_t nwt = (n_cand + kBPW - 1) / kBPW;
    LaneConst lc;
    lc.init(lane);
    WarpTile &wt = sm.w[warp];
    uint32_t occ = 0;
    const uint32_t stride = gridDim.x * kWarps;
    uint32_t t = blockIdx.x * kWarps + warp;
    const uint32_t bq = (uint32_t)lane >> 3;
    uint32_t b_next = t < nwt && t * kBPW + bq < n_cand ? s.icand[t * kBPW + bq] : 0u;
    for (; t < nwt; t += stride) {
        const uint32_t base = t * kBPW;
        const int nb_w = (int)min((uint32_t)kBPW, n_cand - base);
        const uint32_t b = b_next;
        const uint32_t tn = t + stride;                   // next warp tile's block, loaded early
        b_next = tn < nwt && tn * kBPW + bq < n_cand ? s.icand[tn * kBPW + bq] : 0u;
        uint32_t n0p, n1p;
        stage_and_classify<false, kDebug>(s, g, iso, base, nb_w, b, wt, lc, sm.num_tri, n0p, n1p);
        const uint32_t r0 = warp_sum(n0p), r1 = warp_sum(n1p);   // per-byte sums <= 160: no carries
        if (lane < nb_w) {
            const uint32_t cnt = ((r0 >> (8 * lane)) & 0xFFu) + ((r1 >> (8 * lane)) & 0xFFu);
            s.counts[base + lane] = cnt;
            occ += cnt > 0;
        }
    }
    occ = warp_sum(occ);
    if (lane == 0 && occ) atomicAdd(&sm.occ, occ);
    __syncthreads();
    if (threadIdx.x == 0 && sm.occ) atomicAdd(&c->n_occ, sm.occ);
}

// ================================================================ scan (Section 4.4)
//
// Exclusive prefix of the candidates' counts -> 64-bit offsets; the last
// tile writes the total.  kScanItems counts per tile, 8 per thread.

__global__ void __launch_bounds__(kThreads) mc_scan_kernel(DevState s) {
    __shared__ uint32_t wsum[kWarps];
    __shared__ unsigned long long s_excl;
    __shared__ uint32_t s_tile, s_status;
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) s_status = c->status;      // one read per block: the loop below has barriers
    __syncthreads();
    const bool failed = (s_status & (kStatusBudget | kStatusTimeout)) != 0;
    const uint32_t n = failed ? 0u : c->n_cand;
    const uint32_t ntiles = (n + kScanItems - 1) / kScanItems;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->mc_tiles = ntiles;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&c->ctr[kCtrMc], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t i0 = tile * kScanItems + threadIdx.x * 8;
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            v[k] = i0 + k < n ? s.counts[i0 + k] : 0u;
            sum += v[k];
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
            const uint32_t w = lane < kWarps ? wsum[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, wi, kWarps - 1);
            if (lane < kWarps) wsum[lane] = wi - w;                      // exclusive warp offsets
            const unsigned long long excl = lookback_exclusive(s.desc_mc, tile, tot, &c->status);
            if (lane == 0) {
                s_excl = excl;
                if (tile == ntiles - 1) c->n_tri = excl + tot;
            }
        }
        __syncthreads();
        unsigned long long run = s_excl + wsum[warp] + (incl - sum);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (i0 + k < n) s.offsets[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
    }
}

// ================================================================ emit (Section 4.5)

template <bool kDebug>
__global__ void __launch_bounds__(kThreads) mc_emit_kernel(DevState s, Geom g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EmitSmem &sm = *reinterpret_cast<EmitSmem *>(smem_raw);
    Ctl *c = s.ctl;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < 256; i += kThreads) sm.num_tri[i] = s.tables[i];
    for (int i = threadIdx.x; i < 256 * kMaxTriPerCell; i += kThreads) {
        const uint8_t *e = s.tables + 256 + (i / kMaxTriPerCell) * 16 + 3 * (i % kMaxTriPerCell);
        sm.tri_row[i] = (uint32_t)e[0] | ((uint32_t)e[1] << 8) | ((uint32_t)e[2] << 16);
    }
    if (threadIdx.x < 12) {
        // edge e: lower corner (dx,dy,dz), axis a; halo offsets of its two samples
        const int e = threadIdx.x, a = e >> 2, j0 = e & 1, j1 = (e >> 1) & 1;
        const int dx = a == 0 ? 0 : j0, dy = a == 0 ? j0 : (a == 1 ? 0 : j1), dz = a == 2 ? 0 : j1;
        const int lo = dx + 8 * dy + 40 * dz, hi = lo + (a == 0 ? 1 : (a == 1 ? 8 : 40));
        sm.edge_info[e] = (uint32_t)lo | ((uint32_t)hi << 8) | ((uint32_t)dx << 16) | ((uint32_t)dy << 17) |
                          ((uint32_t)dz << 18) | ((uint32_t)a << 19);
    }
    __syncthreads();
    const bool failed = (c->status & (kStatusBudget | kStatusTimeout)) != 0;
    const uint32_t n_cand = failed ? 0u : c->n_cand;
    const float iso = c->params.iso;
    const unsigned long long tri_cap = c->params.tri_cap;
    float4 *__restrict__ out = reinterpret_cast<float4 *>(c->params.out);
    const uint32_t nwt = (n_cand + kBPW - 1) / kBPW;
    const uint32_t slab = g.nbx * g.nby;
    (void)slab;
    LaneConst lc;
    lc.init(lane);
    WarpTile &wt = sm.w[warp];
    uint16_t *tm = sm.tmap[warp];
    float4 *stage = sm.stage[warp];
    const uint32_t stride = gridDim.x * kWarps;
    uint32_t t = blockIdx.x * kWarps + warp;
    const uint32_t bq = (uint32_t)lane >> 3;
    uint32_t b_next = t < nwt && t * kBPW + bq < n_cand ? s.icand[t * kBPW + bq] : 0u;
    for (; t < nwt; t += stride) {
        const uint32_t base = t * kBPW;
        const int nb_w = (int)min((uint32_t)kBPW, n_cand - base);
        const uint32_t b = b_next;
        const uint32_t tn = t + stride;                   // next warp tile's block, loaded early
        b_next = tn < nwt && tn * kBPW + bq < n_cand ? s.icand[tn * kBPW + bq] : 0u;
        uint32_t n0p, n1p;
        stage_and_classify<true, false>(s, g, iso, base, nb_w, b, wt, lc, sm.num_tri, n0p, n1p);
        // per-cell offsets inside the warp tile: two packed scans (byte q = block q)
        uint32_t i0 = n0p, i1 = n1p;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a0 = __shfl_up_sync(0xffffffffu, i0, o), a1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) { i0 += a0; i1 += a1; }
        }
        const uint32_t s0 = __shfl_sync(0xffffffffu, i0, 31), s1 = __shfl_sync(0xffffffffu, i1, 31);
        uint32_t wtot = 0;
#pragma unroll
        for (int q = 0; q < kBPW; q++) {
            if (q >= nb_w) continue;
            const uint32_t n0 = (n0p >> (8 * q)) & 0xFFu, n1 = (n1p >> (8 * q)) & 0xFFu;
            const uint32_t b0 = (s0 >> (8 * q)) & 0xFFu;
            const uint32_t o0 = wtot + ((i0 >> (8 * q)) & 0xFFu) - n0;
            const uint32_t o1 = wtot + b0 + ((i1 >> (8 * q)) & 0xFFu) - n1;
            for (uint32_t k = 0; k < n0; k++) tm[o0 + k] = (uint16_t)((q << 9) | (lane << 3) | k);
            for (uint32_t k = 0; k < n1; k++) tm[o1 + k] = (uint16_t)((q << 9) | ((lane + 32) << 3) | k);
            wtot += b0 + ((s1 >> (8 * q)) & 0xFFu);
        }
        if (wtot == 0) continue;                       // warp-uniform
        const unsigned long long gbase = s.offsets[base];
        __syncwarp();
        // one triangle per lane; its three vertices go through the warp's
        // staging area so that each store instruction writes 512
        // contiguous bytes
        for (uint32_t t0 = 0; t0 < wtot; t0 += 32) {
            const uint32_t tri = t0 + lane;
            if (tri < wtot) {
                const uint32_t e16 = tm[tri];
                const uint32_t q = e16 >> 9, cell = (e16 >> 3) & 63u, k = e16 & 7u;
                const uint32_t row = sm.tri_row[wt.cases[q][cell] * kMaxTriPerCell + k];
                const int cx = (int)(cell & 3u), cy = (int)((cell >> 2) & 3u), cz = (int)(cell >> 4);
                const float *hb = &wt.halo[q][0] + cx + 8 * cy + 40 * cz;
                const float wbits = __uint_as_float(wt.bid[q]);
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const uint32_t info = sm.edge_info[(row >> (8 * j)) & 0xFFu];
                    const float vlo = hb[info & 0xFFu], vhi = hb[(info >> 8) & 0xFFu];
                    // t = (iso - v_lo) / (v_hi - v_lo) through the reciprocal: within
                    // 2 ulp of the correctly rounded quotient (positions within 1e-6)
                    const float tt = __fdividef(__fsub_rn(iso, vlo), __fsub_rn(vhi, vlo));
                    const uint32_t a = (info >> 19) & 3u;
                    float4 p = make_float4((float)(cx + (int)((info >> 16) & 1u)),
                                           (float)(cy + (int)((info >> 17) & 1u)),
                                           (float)(cz + (int)((info >> 18) & 1u)), wbits);
                    if (a == 0) p.x = __fadd_rn(p.x, tt);
                    else if (a == 1) p.y = __fadd_rn(p.y, tt);
                    else p.z = __fadd_rn(p.z, tt);
                    stage[3 * lane + j] = p;
                    if (kDebug) {
                        const unsigned long long gt = gbase + tri;
                        uint32_t bx, by, bz;
                        block_coords(g, wt.bid[q], bx, by, bz);
                        const unsigned long long px = 4ull * bx + cx + ((info >> 16) & 1u);
                        const unsigned long long py = 4ull * by + cy + ((info >> 17) & 1u);
                        const unsigned long long pz = 4ull * bz + cz + ((info >> 18) & 1u);
                        if (gt < tri_cap)
                            s.dbg_edges[gt * 3 + j] =
                                3ull * (px + (unsigned long long)g.nx * (py + (unsigned long long)g.ny * pz)) + a;
                    }
                }
            }
            __syncwarp();
            const uint32_t nv = 3 * min(32u, wtot - t0);             // vertices in this chunk
            const unsigned long long v0 = (gbase + t0) * 3;          // first vertex of the chunk
            const unsigned long long vcap = tri_cap * 3;
#pragma unroll
            for (int r = 0; r < 3; r++) {
                const uint32_t f = lane + 32 * r;
                if (f < nv && v0 + f < vcap) out[v0 + f] = stage[f];
            }
            __syncwarp();
        }
    }
}

// ================================================================ launchers

void launch_mc(const DevState &s, const Geom &g, bool debug, bool emit_only, const Grids &gr, cudaStream_t st) {
    if (!emit_only) {
        if (debug) mc_count_kernel<true><<<gr.mc_count, kThreads, 0, st>>>(s, g);
        else mc_count_kernel<false><<<gr.mc_count, kThreads, 0, st>>>(s, g);
        mc_scan_kernel<<<gr.mc_scan, kThreads, 0, st>>>(s);
    }
    if (debug) mc_emit_kernel<true><<<gr.mc_emit, kThreads, sizeof(EmitSmem), st>>>(s, g);
    else mc_emit_kernel<false><<<gr.mc_emit, kThreads, sizeof(EmitSmem), st>>>(s, g);
}

void mc_grids(int sm_count, Grids *gr) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_count_kernel<false>, kThreads, 0);
    gr->mc_count = std::max(1, occ) * sm_count;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_scan_kernel, kThreads, 0);
    gr->mc_scan = std::max(1, occ) * sm_count;
    cudaFuncSetAttribute(mc_emit_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EmitSmem));
    cudaFuncSetAttribute(mc_emit_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(EmitSmem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_emit_kernel<false>, kThreads, sizeof(EmitSmem));
    gr->mc_emit = std::max(1, occ) * sm_count;
}

}  // namespace bcmc
