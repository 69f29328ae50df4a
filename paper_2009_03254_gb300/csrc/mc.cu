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
//           and the total) and compaction of the occupied candidates, one
//           pass with two decoupled look-backs
//   emit    Section 4.5, over the occupied candidates only: stage the
//           samples (the cases kept by count arrive by asynchronous copies),
//           per-cell offsets by warp scans, then one triangle (three
//           vertices) per lane
//
// Both passes give each warp 4 consecutive candidates at a time (a "warp
// tile") and no warp ever waits for another one:
//   A  slots of each block's 8 blocks of the +group (8 lanes per block)
//   B  stage the samples in shared memory: 16 float4 rows of the block,
//      its +x face, +y/+z rows, edges and corner (50 loads per block, 2
//      per lane, issued two blocks at a time), unpadded: sample
//      x + 5y + 25z
//   C  classify: four ballots give the 125 below-iso bits; each cell's
//      case is 8 bits picked from them; counts from the case table
//
// Over a batch, warp tiles are numbered volume after volume; a warp tile
// never spans two volumes.
//
// Indexed mesh (the alternative output Section 4.5 mentions: vertices
// shared within a block).  A block's vertices are the cut edges of its
// 5x5x5 window: edges between two window samples, exactly one of them
// below the isovalue, that belong to at least one of the block's cells
// inside the volume.  The case table uses every cut edge of a cell, so
// these are exactly the edges the block's triangles use.  An edge is named
// by its axis a and lower sample s = x + 5y + 25z; a block's vertices are
// ordered by a, then s.  The cut edges of one axis form a 125-bit mask:
// the below mask XOR itself shifted by the axis step (1, 5, 25), limited
// to the window; lane 4a + r of a warp holds word r of axis a.  Count adds
// the number of cut edges, scan a third prefix sum, and emit lists the
// tile's vertices in shared memory, computes one vertex per lane (the
// triangle soup's arithmetic) and writes each triangle corner as its
// edge's rank: the vertices before its word plus a popcount.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "kernels.cuh"
#include "launch.cuh"
#include "mc_tables.cuh"

namespace bcmc {

namespace {

constexpr int kBPW = 4;                               // candidates per warp tile
constexpr int kHalo = 128;                            // x + 5y + 25z, x,y,z in [0,5)
constexpr int kTmap = kBPW * 64 * 5;                  // triangles a warp tile can hold
constexpr int kWinWords = 3 * 6 * 4;                  // window rows (indexed meshes), then
constexpr int kWinTable = kWinWords + 32;             // a per-lane word for blocks inside the volume

struct WarpTile {                                     // one warp's shared-memory area
    float halo[kBPW][kHalo];
    int32_t nslot[kBPW][8];
    uint32_t bid[kBPW];
    uint32_t lim[kBPW];                               // cells per axis inside the volume, 4 bits each
    uint8_t cases[kBPW][64];
};

template <int kW>                                     // warps per CTA
struct CountSmem {
    WarpTile w[kW];
    uint32_t win[kWinTable];                          // window rows (indexed meshes)
    uint8_t num_tri[256];
};

template <int kW, bool kIdx>
struct EmitSmem {
    WarpTile w[kW];
    float4 stage[kW][kIdx ? 24 : 96];                 // 32 triangles' vertices (indexed: indices) per warp
    uint16_t tmap[kW][kTmap];                         // block-in-tile (2) | cell (6) | k (3)
    uint16_t tri_row[256 * kMaxTriPerCell];           // 3 edge numbers of each table triangle, 4 bits each
    uint8_t num_tri[256];
    float4 edge_f[12];                                // (dx, dy, dz) and, as bits, the packed edge info
    // indexed: per block, the 12 cut-edge words, then (from word 12) the
    // vertices of the tile before each word
    alignas(16) uint32_t cut[kIdx ? kW : 1][kBPW][24];
    uint32_t win[kIdx ? kWinTable : 1];               // window rows
};

// Halo load job j of a block (0..63; 50 used): neighbour o, source sample
// index inside that block, destination sample x + 5y + 25z of the window,
// a row of 4 samples (one float4 load, four stores) or one sample.
// Packed: valid(1) | vec(1) | o(3) | src(6) | dst(8).
__device__ __forceinline__ uint32_t halo_job(int j) {
    int o = 0, src = 0, dst = 0, vec = 0;
    if (j < 16) {                       // own rows (y, z) = (j & 3, j >> 2)
        o = 0; src = 4 * j; dst = 5 * (j & 3) + 25 * (j >> 2); vec = 1;
    } else if (j < 32) {                // +x face: sample (0, y, z) -> halo (4, y, z)
        const int r = j - 16;
        o = 1; src = 4 * r; dst = 4 + 5 * (r & 3) + 25 * (r >> 2);
    } else if (j < 36) {                // +y rows: (x, 0, z) -> (x, 4, z)
        const int z = j - 32;
        o = 2; src = 16 * z; dst = 20 + 25 * z; vec = 1;
    } else if (j < 40) {                // +z rows: (x, y, 0) -> (x, y, 4)
        const int y = j - 36;
        o = 4; src = 4 * y; dst = 5 * y + 100; vec = 1;
    } else if (j < 44) {                // +xy edge: (0, 0, z) -> (4, 4, z)
        const int z = j - 40;
        o = 3; src = 16 * z; dst = 24 + 25 * z;
    } else if (j < 48) {                // +xz edge: (0, y, 0) -> (4, y, 4)
        const int y = j - 44;
        o = 5; src = 4 * y; dst = 104 + 5 * y;
    } else if (j == 48) {               // +yz row: (x, 0, 0) -> (x, 4, 4)
        o = 6; src = 0; dst = 120; vec = 1;
    } else if (j == 49) {               // corner: (0, 0, 0) -> (4, 4, 4)
        o = 7; src = 0; dst = 124;
    } else {
        return 0;
    }
    return 1u | ((uint32_t)vec << 1) | ((uint32_t)o << 2) | ((uint32_t)src << 5) | ((uint32_t)dst << 11);
}

// Per-lane constants of phases B and C.
struct LaneConst {
    uint32_t job0, job1;                // halo jobs lane and lane + 32
    int cls[4];                         // samples lane + 32r (or -1 past the window)
    // where each of the lane's two cells starts in the 128-bit mask: cell
    // lane (z 0..1) starts in word 0 or 1, cell lane + 32 (z 2..3) in word
    // 1 or 2; `up` says the later of the two, `cshift` the bit in it
    bool up[2];
    int cshift[2];
    __device__ __forceinline__ void init(int lane) {
        job0 = halo_job(lane);
        job1 = halo_job(lane + 32);
#pragma unroll
        for (int r = 0; r < 4; r++) cls[r] = lane + 32 * r < 125 ? lane + 32 * r : -1;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int cell = lane + 32 * h, base = (cell & 3) + 5 * ((cell >> 2) & 3) + 25 * (cell >> 4);
            up[h] = (base >> 5) != h;
            cshift[h] = base & 31;
        }
    }
};

// 16-byte global -> shared copy that completes asynchronously (L2 only)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// the 8-bit case of a cell from the 32 mask bits starting at its lower corner
// (corner c at bit (c&1) + 5((c>>1)&1) + 25(c>>2))
__device__ __forceinline__ uint32_t case_bits(uint32_t W) {
    return (W & 3u) | ((W >> 3) & 0xCu) | ((W >> 21) & 0x30u) | ((W >> 24) & 0xC0u);
}

// the 128-bit below-iso mask of a staged block: bit i of word r says
// sample s = 32r + i (s = x + 5y + 25z, s < 125) is below the isovalue
__device__ __forceinline__ void below_mask(const float *hb, const LaneConst &lc, float iso, uint32_t m[4]) {
#pragma unroll
    for (int r = 0; r < 4; r++) m[r] = __ballot_sync(0xffffffffu, lc.cls[r] >= 0 && hb[lc.cls[r]] < iso);
}

// Window rows: word r of row k of axis a has bit i set when sample
// s = 32r + i (s < 125) has coordinate <= k - 1 along a (row 0: none).
__host__ __device__ constexpr uint32_t window_row_word(int a, int k, int r) {
    uint32_t w = 0;
    for (int i = 0; i < 32; i++) {
        const int s = 32 * r + i, c = a == 0 ? s % 5 : (a == 1 ? (s / 5) % 5 : s / 25);
        if (s < 125 && c <= k - 1) w |= 1u << i;
    }
    return w;
}

// copy of the window rows into shared memory (word a*24 + k*4 + r), then
// at word 72 + lane the window word lane_cut_word takes for a block with
// all its cells inside the volume (0 for lanes 12-31)
__device__ __forceinline__ void load_window_rows(uint32_t *win) {
    for (int i = threadIdx.x; i < kWinTable; i += blockDim.x) {
        if (i < kWinWords) {
            win[i] = window_row_word(i / 24, (i / 4) % 6, i % 4);
        } else {
            const int k = i - kWinWords, a = k >> 2, r = k & 3;
            win[i] = k < 12 ? window_row_word(0, a == 0 ? 4 : 5, r) & window_row_word(1, a == 1 ? 4 : 5, r) &
                                  window_row_word(2, a == 2 ? 4 : 5, r)
                            : 0u;
        }
    }
}

// This lane's word of a block's cut edges (lanes 0-11: axis lane / 4,
// word lane % 4; 0 in the other lanes), from the block's below mask m: bit
// i is set when the edge from sample 32r + i along axis a (steps 1, 5, 25)
// crosses the isovalue and belongs to one of the block's cells inside the
// volume (lim: cells per axis inside, 4 bits each).  Such an edge exists
// when every axis has a cell; its samples lie in [0, l] on the other axes
// and it starts below l along its own.
__device__ __forceinline__ uint32_t lane_cut_word(const uint32_t m[4], uint32_t lim, const uint32_t *win) {
    const int lane = threadIdx.x & 31, a = min(lane >> 2, 2), r = lane & 3;
    const uint32_t lo = (r & 2) ? ((r & 1) ? m[3] : m[2]) : ((r & 1) ? m[1] : m[0]);
    const uint32_t hi = (r & 2) ? ((r & 1) ? 0u : m[3]) : ((r & 1) ? m[2] : m[1]);
    const uint32_t far = __funnelshift_r(lo, hi, a == 0 ? 1 : (a == 1 ? 5 : 25));   // bit i: sample s + step
    uint32_t w;
    if (lim == 0x444u) {                                // warp-uniform: the common case
        w = win[kWinWords + lane];
    } else {
        const uint32_t lx = lim & 15u, ly = (lim >> 4) & 15u, lz = lim >> 8;
        w = win[(a == 0 ? lx : lx + 1) * 4 + r] & win[24 + (a == 1 ? ly : ly + 1) * 4 + r] &
            win[48 + (a == 2 ? lz : lz + 1) * 4 + r];
        w = (lane < 12 && lx && ly && lz) ? w : 0u;
    }
    return (lo ^ far) & w;
}

// Phases A-C for the warp tile starting at candidate `base` (count pass)
// or at occupied candidate `base` (emit pass), nb_w of kBPW slots used.
// Returns the per-cell triangle counts of the lane's two cells, packed one
// byte per block: n0p for cell lane, n1p for cell lane + 32.  The count
// pass (kEmit false) classifies and, when there is room for them
// (keeps_cases), stores the cases; the emit pass leaves the cases in
// wt.cases, reading the stored ones instead of classifying again under the
// same test.  `b` is
// this lane's block (block lane/8 of the tile) and `ci` its position in
// the candidate list, loaded by the caller one warp tile ahead.
//
// With `indexed` (count pass only), nv_lane receives, in lane q, the number
// of cut edges (vertices of the indexed mesh) of block q; `win` is the
// window-row table in shared memory.
//
// With `cut_dst` (emit pass of an indexed extraction), the 12 cut-edge
// words count kept for each of the tile's blocks are copied to
// cut_dst + 24q (asynchronously, like the cases; the caller waits).
// whether the count pass keeps the cases (and the emit pass reads them):
// there is room for all of them (n_cand is final before the count starts)
__device__ __forceinline__ bool keeps_cases(const DevState &s) {
    return s.cases != nullptr && s.ctl->n_cand <= s.case_cap;
}

template <bool kEmit>
__device__ __forceinline__ void stage_and_classify(const DevState &s, const Geom &g, float iso, uint32_t base,
                                                   int nb_w, uint32_t b, uint32_t ci, WarpTile &wt,
                                                   const LaneConst &lc, const uint8_t *num_tri, uint32_t &n0p,
                                                   uint32_t &n1p, bool indexed, const uint32_t *win,
                                                   uint32_t &nv_lane, uint32_t *cut_dst = nullptr) {
    const int lane = threadIdx.x & 31, bq = lane >> 3, bo = lane & 7;
    const uint32_t slab = g.nbx * g.nby;
    const bool keep = keeps_cases(s);                     // uniform
    const bool stored = kEmit && keep;
    // The stored cases of the tile's blocks, copied to shared memory while
    // the samples are staged (16 lanes x 16 bytes; both ends 16-byte
    // aligned).  The emit pass's blocks are occupied candidates, not
    // consecutive ones: block q's position in the candidate list is `ci` of
    // lane 8q.
    if (stored || (kEmit && cut_dst)) {   // uniform
        // lanes 0-15: the cases of block lane / 4; lanes 16-27: the cut-edge
        // words of block (lane - 16) / 3, 16 bytes each
        const int qk = (cut_dst && lane >= 16) ? min((lane - 16) / 3, 3) : (lane >> 2);
        const uint32_t cq = __shfl_sync(0xffffffffu, ci, qk * 8);
        if (stored && lane < 4 * nb_w)
            cp_async16(&wt.cases[lane >> 2][16 * (lane & 3)], s.cases + (size_t)cq * 64 + 16 * (lane & 3));
        if (cut_dst && lane >= 16 && lane < 16 + 3 * nb_w) {
            const int k = (lane - 16) % 3;
            cp_async16(cut_dst + 24 * qk + 4 * k, s.cutw + (size_t)cq * 12 + 4 * k);
        }
    }
    // ---- A: +group slots
    if (bq < nb_w) {
        uint32_t bx, by, bz;
        block_coords(g, b, bx, by, bz);
        const bool ex = bx + 1 < g.nbx, ey = by + 1 < g.nby, ez = bz + 1 < g.nbz;
        const bool exists = (!(bo & 1) || ex) && (!(bo & 2) || ey) && (!(bo & 4) || ez);
        const uint32_t nbid = b + ((bo & 1) ? 1u : 0u) + ((bo & 2) ? g.nbx : 0u) + ((bo & 4) ? slab : 0u);
        wt.nslot[bq][bo] = exists && in_bounds(nbid < g.nb, &s.ctl->status) ? s.islot[nbid] : -1;
        if (bo == 0) {
            wt.bid[bq] = b;
            const uint32_t lx = min(4u, g.nx - 1 - min(g.nx - 1, 4 * bx));
            const uint32_t ly = min(4u, g.ny - 1 - min(g.ny - 1, 4 * by));
            const uint32_t lz = min(4u, g.nz - 1 - min(g.nz - 1, 4 * bz));
            wt.lim[bq] = lx | (ly << 4) | (lz << 8);
        }
    }
    __syncwarp();
    // ---- B: stage samples, two blocks at a time (all their loads first,
    // then all their stores)
#pragma unroll
    for (int half = 0; half < 2; half++) {
        float4 v[kBPW];
#pragma unroll
        for (int qq = 0; qq < kBPW / 2; qq++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int q = 2 * half + qq;
                const uint32_t job = h ? lc.job1 : lc.job0;
                v[2 * qq + h] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q < nb_w && (job & 1u)) {
                    const int32_t sl = wt.nslot[q][(job >> 2) & 7u];
                    if (sl >= 0 && in_bounds((uint32_t)sl < s.ctl->cap, &s.ctl->status)) {
                        const float *p = s.slots + (size_t)sl * 64 + ((job >> 5) & 63u);
                        if (job & 2u) v[2 * qq + h] = __ldg(reinterpret_cast<const float4 *>(p));
                        else v[2 * qq + h].x = __ldg(p);
                    }
                }
            }
#pragma unroll
        for (int qq = 0; qq < kBPW / 2; qq++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int q = 2 * half + qq;
                const uint32_t job = h ? lc.job1 : lc.job0;
                if (q < nb_w && (job & 1u)) {
                    float *d = &wt.halo[q][0] + (job >> 11);
                    d[0] = v[2 * qq + h].x;
                    if (job & 2u) {
                        d[1] = v[2 * qq + h].y;
                        d[2] = v[2 * qq + h].z;
                        d[3] = v[2 * qq + h].w;
                    }
                }
            }
    }
    __syncwarp();
    // ---- C: classify (or take the stored cases) and count
    n0p = 0;
    n1p = 0;
#pragma unroll
    for (int q = 0; q < kBPW; q++) {
        if (q >= nb_w) continue;          // warp-uniform
        uint32_t cs[2];
        if (stored) {
            if (q == 0) {                 // the copies issued before staging
                cp_async_wait_all();
                __syncwarp();
            }
            cs[0] = wt.cases[q][lane];
            cs[1] = wt.cases[q][lane + 32];
        } else {
            uint32_t m[4];
            below_mask(&wt.halo[q][0], lc, iso, m);
            const uint32_t lim = wt.lim[q];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t lo = lc.up[h] ? m[h + 1] : m[h];
                const uint32_t hi = lc.up[h] ? m[h + 2] : m[h + 1];
                cs[h] = case_bits(__funnelshift_r(lo, hi, lc.cshift[h]));
            }
            if (lim != 0x444u) {          // warp-uniform: cells past the volume's last sample are empty
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t cell = (uint32_t)lane + 32u * h;
                    const bool valid = (cell & 3u) < (lim & 15u) && ((cell >> 2) & 3u) < ((lim >> 4) & 15u) &&
                                       (cell >> 4) < (lim >> 8);
                    cs[h] = valid ? cs[h] : 0u;
                }
            }
            if (!kEmit && keep) {         // uniform: keep them for the emit pass
#pragma unroll
                for (int h = 0; h < 2; h++)
                    if (in_bounds(base + q < s.list_cap, &s.ctl->status))
                        s.cases[(size_t)(base + q) * 64 + lane + 32 * h] = (uint8_t)cs[h];
            }
            // uniform: count the cut edges, keep the words for emit; a block
            // without triangles has none (a cut edge makes its cell cross),
            // and nothing reads its words
            if (!kEmit && indexed && __any_sync(0xffffffffu, (num_tri[cs[0]] | num_tri[cs[1]]) != 0u)) {
                const uint32_t w = lane_cut_word(m, lim, win);
                const uint32_t nv = __reduce_add_sync(0xffffffffu, __popc(w));
                if (lane == q) nv_lane = nv;
                if (lane < 12 && in_bounds(base + q < s.list_cap, &s.ctl->status))
                    s.cutw[(size_t)(base + q) * 12 + lane] = w;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (kEmit && !stored) wt.cases[q][lane + 32 * h] = (uint8_t)cs[h];
            const uint32_t n = num_tri[cs[h]];
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

// candidates the triangle stage visits: none once the cache update failed
// (both bits are final before the count kernel starts)
__device__ __forceinline__ uint32_t mc_candidates(const Ctl *c) {
    return (c->status & (kStatusBudget | kStatusTimeout | kStatusTimeoutLru)) ? 0u : c->n_cand;
}

// A warp tile located in the launch: volume, first entry, entries used,
// and for this lane's block (entry first + lane/8) its position in the
// candidate list and its block id, read ahead.  The count pass walks the
// candidates; the emit pass walks the occupied ones (kOcc).
struct TileRef {
    uint32_t v, base, nb_w, b, ci;
};

template <bool kOne, bool kOcc = false>
__device__ __forceinline__ TileRef locate_tile(const Launch &L, const uint32_t *pre, uint32_t t, uint32_t total) {
    TileRef r{0u, 0u, 0u, 0u, 0u};
    if (t >= total) return r;
    r.v = item_vol<kOne>(pre, L.n, t);
    const DevState &s = vol_of<kOne>(L, r.v).s;
    const uint32_t n = kOcc ? s.ctl->n_occ : s.ctl->n_cand;
    r.base = (t - item_base<kOne>(pre, r.v)) * kBPW;
    r.nb_w = min((uint32_t)kBPW, n - r.base);
    const uint32_t i = r.base + ((uint32_t)(threadIdx.x & 31) >> 3);
    if (i < n) {
        r.ci = kOcc ? s.iocc[i] : i;
        r.b = s.icand[r.ci];
    }
    return r;
}

}  // namespace

// ================================================================ count (Section 4.4)

template <int kW, bool kOne, bool kIdx>
__global__ void __launch_bounds__(32 * kW, 40 / kW) mc_count_kernel(Launch L) {   // 1280 threads per SM
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CountSmem<kW> &sm = *reinterpret_cast<CountSmem<kW> *>(smem_raw);
    __shared__ uint32_t pre[kMaxBatch + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint8_t *tables = vol_of<kOne>(L, 0).s.tables;
    for (int i = threadIdx.x; i < 256; i += 32 * kW) sm.num_tri[i] = tables[i];
    if (kIdx) load_window_rows(sm.win);
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) { return ceil_div(mc_candidates(vol_of<kOne>(L, v).s.ctl), kBPW); }, pre);
    __syncthreads();                                      // the table
    LaneConst lc;
    lc.init(lane);
    WarpTile &wt = sm.w[warp];
    const uint32_t stride = gridDim.x * kW;
    uint32_t t = blockIdx.x * kW + warp;
    TileRef nxt = locate_tile<kOne>(L, pre, t, total);
    for (; t < total; t += stride) {
        const TileRef cur = nxt;
        nxt = locate_tile<kOne>(L, pre, t + stride, total);   // next warp tile's block, loaded early
        const DevState &s = vol_of<kOne>(L, cur.v).s;
        const float iso = s.ctl->params.iso;
        uint32_t n0p, n1p, nv = 0;
        stage_and_classify<false>(s, vol_of<kOne>(L, cur.v).g, iso, cur.base, (int)cur.nb_w, cur.b, 0u, wt, lc,
                                  sm.num_tri, n0p, n1p, kIdx, sm.win, nv);
        const uint32_t r0 = warp_sum(n0p), r1 = warp_sum(n1p);   // per-byte sums <= 160: no carries
        if (lane < (int)cur.nb_w)       // triangles (<= 320) in the low 16 bits, vertices (<= 300) above
            s.counts[cur.base + lane] = ((r0 >> (8 * lane)) & 0xFFu) + ((r1 >> (8 * lane)) & 0xFFu) + (nv << 16);
    }
}

// ================================================================ scan (Section 4.4)
//
// Exclusive prefix of the candidates' counts -> 64-bit offsets, and the
// compacted positions of the occupied candidates (I_occ: the blocks the
// emit pass visits, Section 4.4); the last tile of a volume writes both
// totals.  kScanItems = 256 * kPT counts per tile, kPT per thread.  Every volume has at least one item; its item 0
// records how many look-back descriptors the volume used (the next prep
// clears them).

template <int kPT, bool kOne>
__global__ void __launch_bounds__(kThreads) mc_scan_kernel(Launch L) {
    constexpr int kWarps = kThreads / 32;
    constexpr uint32_t kScanItems = kThreads * kPT;
    __shared__ uint32_t wsum[kWarps], wocc[kWarps], wvtx[kWarps];
    __shared__ unsigned long long s_excl[3];
    __shared__ uint32_t pre[kMaxBatch + 1];
    __shared__ uint32_t s_item;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) { return max(1u, ceil_div(mc_candidates(vol_of<kOne>(L, v).s.ctl), kScanItems)); },
        pre);
    while (true) {
        if (threadIdx.x == 0) s_item = atomicAdd(&L.ctr[kLcScan], 1u);
        __syncthreads();
        const uint32_t x = s_item;
        __syncthreads();
        if (x >= total) break;
        const uint32_t v = item_vol<kOne>(pre, L.n, x);
        const DevState &s = vol_of<kOne>(L, v).s;
        Ctl *c = s.ctl;
        const uint32_t tile = x - item_base<kOne>(pre, v);
        const uint32_t n = mc_candidates(c);
        const uint32_t ntiles = ceil_div(n, kScanItems);
        if (tile == 0 && threadIdx.x == 0) c->mc_tiles = ntiles;
        if (ntiles == 0) continue;                        // block-uniform
        const bool indexed = (c->params.flags & kParamIndexed) != 0;   // block-uniform
        const uint32_t i0 = tile * kScanItems + threadIdx.x * kPT;
        uint32_t v8[kPT], sum = 0, occ = 0, vsum = 0;
        const bool full = i0 + kPT <= n;                  // the thread's counts in 16-byte loads
        if (full) {
#pragma unroll
            for (int k = 0; k < kPT / 4; k++) {
                const uint4 q = __ldg(reinterpret_cast<const uint4 *>(s.counts + i0) + k);
                v8[4 * k] = q.x;
                v8[4 * k + 1] = q.y;
                v8[4 * k + 2] = q.z;
                v8[4 * k + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kPT; k++) v8[k] = i0 + k < n ? s.counts[i0 + k] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kPT; k++) {
            sum += v8[k] & 0xFFFFu;                       // triangles | vertices << 16
            vsum += v8[k] >> 16;
            occ += (v8[k] & 0xFFFFu) != 0u;
        }
        // triangles in the low 20 bits, occupied candidates above (a warp
        // holds at most 32 * 16 * 320 triangles and 512 candidates: no carry)
        const uint32_t own = sum | (occ << 20);
        uint32_t incl = own, vincl = vsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (indexed) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, vincl, o);
                if (lane >= o) vincl += t;
            }
        }
        if (lane == 31) {
            wsum[warp] = incl & 0xFFFFFu;
            wocc[warp] = incl >> 20;
            wvtx[warp] = vincl;
        }
        __syncthreads();
        // warp 0: triangle offsets; warp 1: occupied positions; warp 2: vertex offsets
        if (warp < 2 || (warp == 2 && indexed)) {
            uint32_t *ws = warp == 0 ? wsum : (warp == 1 ? wocc : wvtx);
            const uint32_t w = lane < kWarps ? ws[lane] : 0u;
            uint32_t wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            const uint32_t tot = __shfl_sync(0xffffffffu, wi, kWarps - 1);
            if (lane < kWarps) ws[lane] = wi - w;                        // exclusive warp offsets
            unsigned long long *desc = warp == 0 ? s.desc_mc : (warp == 1 ? s.desc_occ : s.desc_vtx);
            const unsigned long long excl = lookback_exclusive(desc, tile, tot, &c->status, kStatusTimeoutScan);
            if (lane == 0) {
                s_excl[warp] = excl;
                if (tile == ntiles - 1) {
                    if (warp == 0) c->n_tri = excl + tot;
                    else if (warp == 1) c->n_occ = (uint32_t)(excl + tot);
                    else c->n_vtx = excl + tot;
                }
            }
        }
        __syncthreads();
        const uint32_t before = incl - own;                              // this thread's exclusive prefix in the warp
        unsigned long long run = s_excl[0] + wsum[warp] + (before & 0xFFFFFu);
        uint32_t orun = (uint32_t)s_excl[1] + wocc[warp] + (before >> 20);
        if (indexed) {
            unsigned long long vrun = s_excl[2] + wvtx[warp] + (vincl - vsum);
#pragma unroll
            for (int k = 0; k < kPT; k++) {
                if (i0 + k < n) s.offsets[i0 + k] = run;
                if ((v8[k] & 0xFFFFu) && in_bounds(orun < s.list_cap, &c->status)) {
                    s.voff[orun] = vrun;
                    s.iocc[orun++] = i0 + k;
                }
                run += v8[k] & 0xFFFFu;
                vrun += v8[k] >> 16;
            }
        } else {
            unsigned long long ofs[kPT];
#pragma unroll
            for (int k = 0; k < kPT; k++) {
                ofs[k] = run;
                if (v8[k] && in_bounds(orun < s.list_cap, &c->status)) s.iocc[orun++] = i0 + k;
                run += v8[k];
            }
            if (full) {
#pragma unroll
                for (int k = 0; k < kPT / 2; k++)
                    reinterpret_cast<ulonglong2 *>(s.offsets + i0)[k] = make_ulonglong2(ofs[2 * k], ofs[2 * k + 1]);
            } else {
#pragma unroll
                for (int k = 0; k < kPT; k++)
                    if (i0 + k < n) s.offsets[i0 + k] = ofs[k];
            }
        }
    }
}

// ================================================================ emit (Section 4.5)

template <int kW, bool kDebug, bool kOne, bool kIdx>
__device__ __forceinline__ void emit_body(const Launch &L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EmitSmem<kW, kIdx> &sm = *reinterpret_cast<EmitSmem<kW, kIdx> *>(smem_raw);
    __shared__ uint32_t pre[kMaxBatch + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint8_t *tables = vol_of<kOne>(L, 0).s.tables;
    for (int i = threadIdx.x; i < 256; i += 32 * kW) sm.num_tri[i] = tables[i];
    for (int i = threadIdx.x; i < 256 * kMaxTriPerCell; i += 32 * kW) {
        const uint8_t *e = tables + 256 + (i / kMaxTriPerCell) * 16 + 3 * (i % kMaxTriPerCell);
        sm.tri_row[i] = (uint16_t)(e[0] | (e[1] << 4) | (e[2] << 8));
    }
    if (kIdx) load_window_rows(sm.win);
    if (threadIdx.x < 12) {
        // edge e: lower corner (dx,dy,dz), axis a; halo offsets of its two samples
        const int e = threadIdx.x, a = e >> 2, j0 = e & 1, j1 = (e >> 1) & 1;
        const int dx = a == 0 ? 0 : j0, dy = a == 0 ? j0 : (a == 1 ? 0 : j1), dz = a == 2 ? 0 : j1;
        const int lo = dx + 5 * dy + 25 * dz, hi = lo + (a == 0 ? 1 : (a == 1 ? 5 : 25));
        sm.edge_f[e] = make_float4((float)dx, (float)dy, (float)dz,
                                   __uint_as_float((uint32_t)lo | ((uint32_t)hi << 8) | ((uint32_t)dx << 16) |
                                                   ((uint32_t)dy << 17) | ((uint32_t)dz << 18) | ((uint32_t)a << 19)));
    }
    // all failure bits are final before this kernel starts
    const uint32_t total = launch_prefix<kOne>(
        L, [&](uint32_t v) {
            const Ctl *c = vol_of<kOne>(L, v).s.ctl;
            return (c->status & (kStatusBudget | kStatusAnyTimeout | kStatusSkip)) ? 0u : ceil_div(c->n_occ, kBPW);
        },
        pre);
    __syncthreads();                                      // the tables
    LaneConst lc;
    lc.init(lane);
    WarpTile &wt = sm.w[warp];
    uint16_t *tm = sm.tmap[warp];
    float4 *stage = sm.stage[warp];
    const uint32_t stride = gridDim.x * kW;
    uint32_t t = blockIdx.x * kW + warp;
    TileRef nxt = locate_tile<kOne, true>(L, pre, t, total);
    for (; t < total; t += stride) {
        const TileRef cur = nxt;
        nxt = locate_tile<kOne, true>(L, pre, t + stride, total);   // next warp tile's blocks, loaded early
        const DevState &s = vol_of<kOne>(L, cur.v).s;
        const Geom &g = vol_of<kOne>(L, cur.v).g;
        const Ctl *c = s.ctl;
        const float iso = c->params.iso;
        const unsigned long long tri_cap = c->params.tri_cap;
        const bool packed = c->params.format == kVertexPacked;     // warp-uniform
        float4 *__restrict__ out = reinterpret_cast<float4 *>(c->params.out);
        const uint32_t base = cur.base;
        const int nb_w = (int)cur.nb_w;
        uint32_t n0p, n1p, unused = 0;
        stage_and_classify<true>(s, g, iso, base, nb_w, cur.b, cur.ci, wt, lc, sm.num_tri, n0p, n1p, false, nullptr,
                                 unused, kIdx ? &sm.cut[warp][0][0] : nullptr);
        // consecutive occupied candidates have adjacent outputs (the empty
        // ones between them add nothing): the tile starts at its first block's
        const uint32_t first_ci = __shfl_sync(0xffffffffu, cur.ci, 0);
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
        for (int q = 0; q < kBPW; q++)
            if (q < nb_w) wtot += ((s0 >> (8 * q)) & 0xFFu) + ((s1 >> (8 * q)) & 0xFFu);
        if (wtot == 0) continue;                       // warp-uniform
        const unsigned long long gbase = s.offsets[first_ci];
        unsigned long long vt = 0;                     // indexed: the tile's first vertex
        if constexpr (kIdx) {
            // Per block, lanes 0-11 take one word each of its cut edges and the
            // vertices of the tile before it (an exclusive scan over the lanes,
            // in vertex order: axis, then sample), and list the word's edges
            // in the vertex map `tm` at their ranks.
            vt = s.voff[base];
            cp_async_wait_all();                       // the words (and cases) copied during staging
            __syncwarp();
            uint32_t nvt = 0;
            const int lk = lane % 12, la = lk >> 2, lr = lk & 3;
            for (int qq = 0; qq < nb_w; qq += 2) {     // lanes 0-11: block qq, lanes 12-23: block qq + 1
                const int q = qq + (lane >= 12 ? 1 : 0);
                uint32_t w = (lane < 24 && q < nb_w) ? sm.cut[warp][q][lk] : 0u;
                const uint32_t n = __popc(w);
                uint32_t incl = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += x;
                }
                uint32_t rank = nvt + incl - n;        // the tile's vertices before this word
                if (lane < 24 && q < nb_w) sm.cut[warp][q][12 + lk] = rank;
                while (w) {                            // this word's edges: (block, sample, axis)
                    const uint32_t i = __ffs(w) - 1;
                    w &= w - 1;
                    tm[rank++] = (uint16_t)((q << 9) | ((32 * lr + i) << 2) | la);
                }
                nvt += __shfl_sync(0xffffffffu, incl, 23);
            }
            __syncwarp();
            // one vertex per lane, the triangle soup's arithmetic; consecutive
            // lanes write consecutive vertices
            const unsigned long long vcap = c->params.vert_cap;
            for (uint32_t k = lane; k < nvt; k += 32) {
                const uint32_t e = tm[k];
                const uint32_t q = e >> 9, smp = (e >> 2) & 127u, ax = e & 3u;
                const uint32_t sx = smp % 5u, sy = (smp / 5u) % 5u, sz = smp / 25u;
                const float *hp = &wt.halo[q][0] + smp;
                const float vlo = hp[0], vhi = hp[ax == 0 ? 1 : (ax == 1 ? 5 : 25)];
                float px = (float)sx, py = (float)sy, pz = (float)sz;
                float tt;
                if (!packed) tt = edge_fraction<false>(iso, vlo, vhi);
                else tt = edge_fraction<true>(iso, vlo, vhi);
                if (ax == 0) px = __fadd_rn(px, tt);
                else if (ax == 1) py = __fadd_rn(py, tt);
                else pz = __fadd_rn(pz, tt);
                if (vt + k < vcap) {
                    if (!packed) {
                        out[vt + k] = make_float4(px, py, pz, __uint_as_float(wt.bid[q]));
                    } else {
                        const uint32_t qx = (uint32_t)__float2int_rn(__fmul_rn(px, 255.75f));
                        const uint32_t qy = (uint32_t)__float2int_rn(__fmul_rn(py, 255.75f));
                        const uint32_t qz = (uint32_t)__float2int_rn(__fmul_rn(pz, 255.75f));
                        reinterpret_cast<uint2 *>(out)[vt + k] = make_uint2(qx | (qy << 10) | (qz << 20), wt.bid[q]);
                    }
                }
            }
            vt += c->params.vtx_base;                  // indices count the vertices of earlier waves
            __syncwarp();                              // the vertex map is read: tm takes the triangles
        }
        // each lane lists its two cells' triangles at their offsets (unrolled,
        // predicated stores: the counts differ from lane to lane)
        uint32_t tacc = 0;
#pragma unroll 1
        for (int q = 0; q < nb_w; q++) {
            const uint32_t n0 = (n0p >> (8 * q)) & 0xFFu, n1 = (n1p >> (8 * q)) & 0xFFu;
            const uint32_t b0 = (s0 >> (8 * q)) & 0xFFu;
            const uint32_t o0 = tacc + ((i0 >> (8 * q)) & 0xFFu) - n0;
            const uint32_t o1 = tacc + b0 + ((i1 >> (8 * q)) & 0xFFu) - n1;
#pragma unroll
            for (uint32_t k = 0; k < kMaxTriPerCell; k++) {
                if (k < n0) tm[o0 + k] = (uint16_t)((q << 9) | (lane << 3) | k);
                if (k < n1) tm[o1 + k] = (uint16_t)((q << 9) | ((lane + 32) << 3) | k);
            }
            tacc += b0 + ((s1 >> (8 * q)) & 0xFFu);
        }
        __syncwarp();
        // one triangle per lane; its three vertices (or, indexed, its three
        // vertex indices) go through the warp's staging area so that each
        // store instruction writes contiguous bytes; vertices are stored evict-first
        // (a surface is several times the L2, and the hulls, slot map and
        // cached blocks the next extraction reads should stay there)
        for (uint32_t t0 = 0; t0 < wtot; t0 += 32) {
            const uint32_t tri = t0 + lane;
            if (tri < wtot) {
                const uint32_t e16 = tm[tri];
                const uint32_t q = e16 >> 9, cell = (e16 >> 3) & 63u, k = e16 & 7u;
                const uint32_t row = sm.tri_row[wt.cases[q][cell] * kMaxTriPerCell + k];
                const int cx = (int)(cell & 3u), cy = (int)((cell >> 2) & 3u), cz = (int)(cell >> 4);
                const float *hb = &wt.halo[q][0] + cx + 5 * cy + 25 * cz;
                const float wbits = __uint_as_float(wt.bid[q]);
                const float fx = (float)cx, fy = (float)cy, fz = (float)cz;
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const float4 ef = sm.edge_f[(row >> (4 * j)) & 0xFu];
                    const uint32_t info = __float_as_uint(ef.w);
                    const uint32_t a = (info >> 19) & 3u;
                    if constexpr (kIdx) {
                        // the rank of the edge among the tile's vertices: those
                        // before its word, then its word's bits below it
                        const int smp = cx + (int)((info >> 16) & 1u) + 5 * (cy + (int)((info >> 17) & 1u)) +
                                        25 * (cz + (int)((info >> 18) & 1u));
                        const uint32_t *cw = sm.cut[warp][q] + 4 * a + (smp >> 5);
                        const uint32_t rank = cw[12] + __popc(cw[0] & ((1u << (smp & 31)) - 1u));
                        reinterpret_cast<uint32_t *>(stage)[3 * lane + j] = (uint32_t)(vt + rank);
                    } else {
                        const float vlo = hb[info & 0xFFu], vhi = hb[(info >> 8) & 0xFFu];
                        float4 p = make_float4(__fadd_rn(fx, ef.x), __fadd_rn(fy, ef.y), __fadd_rn(fz, ef.z), wbits);
                        if (!packed) {
                            // t through the reciprocal: within 2 ulp of the correctly
                            // rounded quotient (positions within 1e-6)
                            const float tt = edge_fraction<false>(iso, vlo, vhi);
                            if (a == 0) p.x = __fadd_rn(p.x, tt);
                            else if (a == 1) p.y = __fadd_rn(p.y, tt);
                            else p.z = __fadd_rn(p.z, tt);
                            stage[3 * lane + j] = p;
                        } else {
                            // the 10-bit code round(p / 4 * 1023) decides an integer, so every
                            // step is one IEEE float32 operation (the division correctly
                            // rounded), as the oracle computes it
                            const float tt = edge_fraction<true>(iso, vlo, vhi);
                            if (a == 0) p.x = __fadd_rn(p.x, tt);
                            else if (a == 1) p.y = __fadd_rn(p.y, tt);
                            else p.z = __fadd_rn(p.z, tt);
                            const uint32_t qx = (uint32_t)__float2int_rn(__fmul_rn(p.x, 255.75f));
                            const uint32_t qy = (uint32_t)__float2int_rn(__fmul_rn(p.y, 255.75f));
                            const uint32_t qz = (uint32_t)__float2int_rn(__fmul_rn(p.z, 255.75f));
                            reinterpret_cast<uint2 *>(stage)[3 * lane + j] = make_uint2(qx | (qy << 10) | (qz << 20),
                                                                                         wt.bid[q]);
                        }
                    }
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
            const uint32_t nv = 3 * min(32u, wtot - t0);             // vertices (or indices) in this chunk
            const unsigned long long v0 = (gbase + t0) * 3;          // first of the chunk
            const unsigned long long vcap = tri_cap * 3;
            if constexpr (kIdx) {
                uint32_t *oi = reinterpret_cast<uint32_t *>(c->params.idx_out);
                const uint32_t *st = reinterpret_cast<const uint32_t *>(stage);
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    const uint32_t f = lane + 32 * r;
                    if (f < nv && v0 + f < vcap) oi[v0 + f] = st[f];
                }
            } else if (!packed) {
                if (v0 + 96 <= vcap) {                 // warp-uniform: the whole chunk fits
#pragma unroll
                    for (int r = 0; r < 3; r++) {
                        const uint32_t f = lane + 32 * r;
                        if (f < nv) __stcs(&out[v0 + f], stage[f]);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 3; r++) {
                        const uint32_t f = lane + 32 * r;
                        if (f < nv && v0 + f < vcap) __stcs(&out[v0 + f], stage[f]);
                    }
                }
            } else {
                uint2 *out2 = reinterpret_cast<uint2 *>(out);
                const uint2 *st2 = reinterpret_cast<const uint2 *>(stage);
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    const uint32_t f = lane + 32 * r;
                    if (f < nv && v0 + f < vcap) __stcs(&out2[v0 + f], st2[f]);
                }
            }
            __syncwarp();
        }
    }
}

// the triangle soup; registers bounded for 32 warps per SM (the staging
// holds two blocks' loads at a time, so 64 registers suffice)
template <int kW, bool kDebug, bool kOne>
__global__ void __launch_bounds__(32 * kW, 32 / kW) mc_emit_kernel(Launch L) {
    emit_body<kW, kDebug, kOne, false>(L);
}

// the indexed mesh (single volumes); registers bounded for 32 warps per SM
// (at 24 warps it measured 219 against 158 us per surface on noise512)
template <int kW, bool kDebug>
__global__ void __launch_bounds__(32 * kW, 32 / kW) mc_emit_indexed_kernel(Launch L) {
    emit_body<kW, kDebug, true, true>(L);
}

// ================================================================ launchers

namespace {

template <int kW, bool kOne, bool kIdx>
void count_w(const Launch &L, int grid, cudaStream_t st) {
    mc_count_kernel<kW, kOne, kIdx><<<grid, 32 * kW, sizeof(CountSmem<kW>), st>>>(L);
}

template <int kW, bool kOne, bool kIdx>
void emit_w(const Launch &L, bool debug, int grid, cudaStream_t st) {
    constexpr size_t bytes = sizeof(EmitSmem<kW, kIdx>);
    if constexpr (kIdx) {
        if (debug) mc_emit_indexed_kernel<kW, true><<<grid, 32 * kW, bytes, st>>>(L);
        else mc_emit_indexed_kernel<kW, false><<<grid, 32 * kW, bytes, st>>>(L);
    } else {
        if (debug) mc_emit_kernel<kW, true, kOne><<<grid, 32 * kW, bytes, st>>>(L);
        else mc_emit_kernel<kW, false, kOne><<<grid, 32 * kW, bytes, st>>>(L);
    }
}

// resident CTAs per SM of `kernel` (at least 1)
template <class K>
int occupancy(K kernel, int threads, size_t smem) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();
        occ = 1;
    }
    return std::max(1, occ);
}

template <class K>
void raise_smem(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int kW>
int emit_occupancy(bool single) {
    raise_smem(mc_emit_kernel<kW, false, false>, sizeof(EmitSmem<kW, false>));
    raise_smem(mc_emit_kernel<kW, true, false>, sizeof(EmitSmem<kW, false>));
    raise_smem(mc_emit_kernel<kW, false, true>, sizeof(EmitSmem<kW, false>));
    raise_smem(mc_emit_kernel<kW, true, true>, sizeof(EmitSmem<kW, false>));
    raise_smem(mc_emit_indexed_kernel<kW, false>, sizeof(EmitSmem<kW, true>));
    raise_smem(mc_emit_indexed_kernel<kW, true>, sizeof(EmitSmem<kW, true>));
    // every kernel launched with this CTA count must fit it: a CTA beyond
    // the resident ones would start only when a whole CTA has finished, and
    // its statically assigned tiles would trail the rest
    if (single)
        return std::min({occupancy(mc_emit_kernel<kW, false, true>, 32 * kW, sizeof(EmitSmem<kW, false>)),
                         occupancy(mc_emit_kernel<kW, true, true>, 32 * kW, sizeof(EmitSmem<kW, false>)),
                         occupancy(mc_emit_indexed_kernel<kW, false>, 32 * kW, sizeof(EmitSmem<kW, true>)),
                         occupancy(mc_emit_indexed_kernel<kW, true>, 32 * kW, sizeof(EmitSmem<kW, true>))});
    return std::min(occupancy(mc_emit_kernel<kW, false, false>, 32 * kW, sizeof(EmitSmem<kW, false>)),
                    occupancy(mc_emit_kernel<kW, true, false>, 32 * kW, sizeof(EmitSmem<kW, false>)));
}

template <int kW>
int count_occupancy(bool single) {
    raise_smem(mc_count_kernel<kW, false, false>, sizeof(CountSmem<kW>));
    raise_smem(mc_count_kernel<kW, true, false>, sizeof(CountSmem<kW>));
    raise_smem(mc_count_kernel<kW, true, true>, sizeof(CountSmem<kW>));
    if (single)   // the soup's and the indexed mesh's counts share the CTA count
        return std::min(occupancy(mc_count_kernel<kW, true, false>, 32 * kW, sizeof(CountSmem<kW>)),
                        occupancy(mc_count_kernel<kW, true, true>, 32 * kW, sizeof(CountSmem<kW>)));
    return occupancy(mc_count_kernel<kW, false, false>, 32 * kW, sizeof(CountSmem<kW>));
}

template <bool kOne, bool kIdx>
void count_any(const Launch &L, const Plan &pl, cudaStream_t st) {
    if (pl.count_tile == 16) count_w<4, kOne, kIdx>(L, pl.mc_count, st);
    else if (pl.count_tile == 64) count_w<16, kOne, kIdx>(L, pl.mc_count, st);
    else count_w<8, kOne, kIdx>(L, pl.mc_count, st);
}

template <bool kOne>
void scan_any(const Launch &L, const Plan &pl, cudaStream_t st) {
    if (pl.scan_tile == 1024) mc_scan_kernel<4, kOne><<<pl.mc_scan, kThreads, 0, st>>>(L);
    else if (pl.scan_tile == 4096) mc_scan_kernel<16, kOne><<<pl.mc_scan, kThreads, 0, st>>>(L);
    else mc_scan_kernel<8, kOne><<<pl.mc_scan, kThreads, 0, st>>>(L);
}

template <bool kOne, bool kIdx>
void emit_any(const Launch &L, bool debug, const Plan &pl, cudaStream_t st) {
    if (pl.emit_tile == 16) emit_w<4, kOne, kIdx>(L, debug, pl.mc_emit, st);
    else if (pl.emit_tile == 64) emit_w<16, kOne, kIdx>(L, debug, pl.mc_emit, st);
    else emit_w<8, kOne, kIdx>(L, debug, pl.mc_emit, st);
}

}  // namespace

// tile = candidates per CTA round = 4 per warp
void launch_mc_count(const Launch &L, bool /*debug*/, const Plan &pl, cudaStream_t st, bool indexed) {
    if (L.vols) count_any<false, false>(L, pl, st);
    else if (indexed) count_any<true, true>(L, pl, st);
    else count_any<true, false>(L, pl, st);
}

void launch_mc_scan(const Launch &L, const Plan &pl, cudaStream_t st) {
    if (L.vols) scan_any<false>(L, pl, st);
    else scan_any<true>(L, pl, st);
}

// the indexed mesh is made for single volumes only
void launch_mc_emit(const Launch &L, bool debug, const Plan &pl, cudaStream_t st, bool indexed) {
    if (L.vols) emit_any<false, false>(L, debug, pl, st);
    else if (indexed) emit_any<true, true>(L, debug, pl, st);
    else emit_any<true, false>(L, debug, pl, st);
}

template <int kPT>
int scan_occupancy(bool single) {
    int occ = 0;
    if (single) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_scan_kernel<kPT, true>, kThreads, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mc_scan_kernel<kPT, false>, kThreads, 0);
    return occ;
}

void mc_occupancy(Plan *pl, bool single) {
    // every variant's shared-memory limit is raised, whichever is asked for
    const int e4 = emit_occupancy<4>(single), e8 = emit_occupancy<8>(single), e16 = emit_occupancy<16>(single);
    pl->mc_emit = std::max(1, pl->emit_tile == 16 ? e4 : (pl->emit_tile == 64 ? e16 : e8));
    const int c4 = count_occupancy<4>(single), c8 = count_occupancy<8>(single),
              c16 = count_occupancy<16>(single);
    pl->mc_count = std::max(1, pl->count_tile == 16 ? c4 : (pl->count_tile == 64 ? c16 : c8));
    const int occ = pl->scan_tile == 1024 ? scan_occupancy<4>(single)
                                          : (pl->scan_tile == 4096 ? scan_occupancy<16>(single)
                                                                   : scan_occupancy<8>(single));
    pl->mc_scan = std::max(1, occ);
}

}  // namespace bcmc
