// Kernel launchers of the extraction pipeline (implemented in extract.cu
// and codec.cu).  Every launcher only queues work on `st`.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace bcmc {

// Device pointers of one volume, passed to kernels by value.
struct DevState {
    const uint64_t *bits;      // nb * rate words
    const float2 *hull;        // per block: min/max over its 3x3x3 block neighbourhood
    const float2 *hull8;       // per block: min/max over its 2x2x2 +group
    const float2 *seg;         // per segment of 64 consecutive blocks: the hull of their hulls (null:
                               // the range test reads every block's hull)
    uint32_t *mactive;         // M_active bitmask, ceil(nb/32) words
    uint32_t *iactive;         // I_active (kept only for debugging: nothing downstream reads it; else null)
    uint32_t *inew;            // I_new
    uint32_t *icand;           // candidates: ids of the blocks the triangle stage visits (ascending)
    uint32_t list_cap;         // room of I_active, I_new and the candidates: min(nb, slot cap); longer
                               // lists mean more active blocks than slots, which the cache update refuses
    int32_t *islot;            // I_slot: block -> slot or -1
    uint32_t *slast;           // S_last: slot -> epoch of last use (0 = never)
    int32_t *sblock;           // S_block: slot -> block or -1
    uint32_t *lbuf[2];         // used-slot list, least recently used first (double buffered)
    uint32_t *newslot;         // slot given to I_new[r]
    float *slots;              // decoded blocks, 64 floats per slot
    unsigned long long *desc_cull, *desc_cand, *desc_lru_a, *desc_lru_b, *desc_mc;
    Ctl *ctl;
    const uint8_t *tables;     // num_tri[256] then tri_edges[256][16]
    uint32_t *counts;          // triangles of each candidate
    unsigned long long *offsets; // exclusive prefix of counts: first triangle of each candidate
    uint32_t *iocc;            // I_occ: positions in the candidate list of the occupied candidates (ascending)
    unsigned long long *desc_occ;  // look-back descriptors of the occupied count (next to desc_mc)
    unsigned long long *desc_vtx;  // look-back descriptors of the vertex count (next to desc_occ; null
                                   // where indexed meshes are never made)
    unsigned long long *voff;      // indexed mesh: first vertex of each occupied candidate (null until
                                   // the first indexed extraction)
    uint32_t *cutw;                // indexed mesh: 12 cut-edge words per candidate, written by count and
                                   // read by emit (null until the first indexed extraction)
    uint8_t *cases;            // 64 cell cases per candidate, written by the count pass and read by
                               // emit instead of classifying again (null: emit classifies)
    unsigned long long case_cap;   // candidates `cases` holds: with more, both passes act as if it were null
    // debug copy (null unless the volume was loaded with ISO_DEBUG)
    unsigned long long *dbg_edges;
};

// One volume of a launch: its device state, geometry and the sizes of
// its look-back descriptor arrays.  Kept in device memory (a table of one
// entry for a single extraction, of many for a batch).
struct VolEntry {
    DevState s;
    Geom g;
    uint32_t n_cull_desc, n_lru_desc;
};

constexpr uint32_t kMaxBatch = 1024;     // volumes per launch

// What every stage kernel receives: the volumes and the launch's work
// counters (kNumLaunchCounters words, cleared by the prep kernel).  A
// single volume travels by value in the launch parameters (`one`, with
// vols == nullptr and n == 1), so its kernels read its pointers from the
// constant bank; a batch passes a device table.
struct Launch {
    const VolEntry *vols;
    uint32_t n;
    uint32_t *ctr;
    VolEntry one;
    uint32_t max_rate = 0;   // batches: the largest rate among the volumes (sizes the decoder's staging)
    uint32_t seg_any = 0;    // batches: some volume has segment ranges (the range test's segment variant)
};

// How a launch sequence runs: the CTAs of each persistent kernel and the
// tile size of each kernel that has a choice.  Any choice computes the
// same results; the batch autotuner picks the fastest.
struct Plan {
    int prep, cull, lru_a, lru_b, decode, mc_count, mc_scan, mc_emit;   // CTAs per launch
    int cull_tile;       // block ranges per cull tile: 2048 or 4096
    int decode_tile;     // new blocks per decode CTA (one per thread): 64, 128 or 256
    int count_tile;      // candidates per count CTA round (4 per warp): 16, 32 or 64
    int scan_tile;       // counts per offset-scan tile: 1024, 2048 or 4096
    int emit_tile;       // candidates per emit CTA round (4 per warp): 16, 32 or 64
};

constexpr int kThreads = 256;
constexpr int kScanTile = 4096;          // entries per tile of the cache-update scans
constexpr int kMinCullTile = 2048;       // smallest cull tile (sizes the cull descriptors)
constexpr int kMinMcScanTile = 1024;     // smallest offset-scan tile (sizes its descriptors)
constexpr int kDefaultCullTile = 4096, kDefaultDecodeTile = 128, kDefaultCountTile = 32,
              kDefaultScanTile = 2048, kDefaultEmitTile = 32;

// The isovalue, output buffer and its capacity are read from Ctl::params.
// Front of the pipeline: prep, cull, cache update (two kernels), decode.
// With `ev`, events ev[1..4] are recorded after prep, cull, cache update
// and decode.
// (with bits_ready, the decode waits for that event: an upload still in flight)
void launch_front(const Launch &L, const Plan &pl, cudaStream_t st, cudaEvent_t *ev,
                  cudaEvent_t bits_ready = nullptr);
// the cache update and decode alone (after a cull that set n_active/n_new)
void launch_cache_update(const Launch &L, const Plan &pl, cudaStream_t st);
// the range test alone (Ctl counters and look-back descriptors cleared by the caller)
void launch_cull(const Launch &L, const Plan &pl, cudaStream_t st);
// triangle stage: count, scan, emit.  A batch places the volumes' outputs
// between scan and emit; a rerun into a larger output runs emit alone.
void launch_mc_count(const Launch &L, bool debug, const Plan &pl, cudaStream_t st, bool indexed = false);
void launch_mc_scan(const Launch &L, const Plan &pl, cudaStream_t st);
void launch_mc_emit(const Launch &L, bool debug, const Plan &pl, cudaStream_t st, bool indexed = false);
// batches: per-volume isovalues from a packed array; the volumes' outputs
// placed one after another in `bo->out` (tri_base[v] = first triangle of
// volume v, tri_base[n] = total); control blocks gathered for one readback
struct BatchOut {
    unsigned long long out;        // float4 * vertex buffer
    unsigned long long tri_cap;    // its capacity in triangles
};
void launch_batch_params(const Launch &L, const float *d_iso, cudaStream_t st);
void launch_batch_offsets(const Launch &L, const BatchOut *bo, unsigned long long *tri_base, cudaStream_t st);
void launch_batch_gather(const Launch &L, Ctl *dst, cudaStream_t st);

// the blocks' hulls and, with `seg`, the segments' (64 consecutive blocks each)
void launch_hull(const float *bmin, const float *bmax, float2 *hull, float2 *hull8, float2 *seg, const Geom &g,
                 uint32_t *status, cudaStream_t st);
constexpr uint32_t kSegBlocks = 64;                  // blocks per segment of the segment ranges
constexpr uint64_t kSegmentCullMinBlocks = 1ull << 28;   // default: segment ranges from this many blocks
void launch_reset_cache(const DevState &s, cudaStream_t st);
void launch_encode(const float *field, const Geom &g, uint64_t *bits, float *bmin, float *bmax, cudaStream_t st);
void launch_decode_list(const uint64_t *bits, uint32_t rate, const uint32_t *ids, uint64_t n, float *out,
                        cudaStream_t st);
void launch_decode_volume(const uint64_t *bits, const Geom &g, float *field, cudaStream_t st);
// waves: active blocks of each z-layer of blocks (layer_active zeroed by the caller)
void launch_count_layers(const float2 *hull, const Geom &g, float iso, uint32_t *layer_active, cudaStream_t st);
void launch_gather_slots(const float *slots, const int32_t *islot, const uint32_t *ids, uint64_t n, float *out,
                         int32_t *missing, cudaStream_t st);

// The most CTAs of each kernel one SM holds, for the tile variants in
// `tiles`, in single-volume or batch launches (CTA fields of the result;
// tile fields copied).  Also raises the shared-memory limits of every
// kernel that needs more than the default.
Plan occupancy_limits(const Plan &tiles, bool single, uint32_t rate, bool seg = false);
void mc_occupancy(Plan *pl, bool single);
// tile sizes that the kernels are compiled for
bool valid_tiles(const Plan &pl);

}  // namespace bcmc
