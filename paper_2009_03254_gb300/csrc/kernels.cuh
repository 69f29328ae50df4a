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
    uint32_t *mactive;         // M_active bitmask, ceil(nb/32) words
    uint32_t *iactive;         // I_active
    uint32_t *inew;            // I_new
    uint32_t *icand;           // candidates: ids of the blocks the triangle stage visits (ascending)
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
    // debug copies (null unless the volume was loaded with ISO_DEBUG)
    uint8_t *dbg_cases;        // 64 per candidate block
    unsigned long long *dbg_edges;
};

struct Grids {                 // CTAs per launch, from occupancy at load time
    int prep, cull, lru_a, lru_b, decode, mc_count, mc_scan, mc_emit;
};

constexpr int kThreads = 256;
constexpr int kScanTile = 4096;          // entries per tile of the cull / cache scans

// The isovalue, output buffer and its capacity are read from Ctl::params.
void launch_prep(const DevState &s, uint32_t n_cull_desc, uint32_t n_lru_desc, bool mc_only, int grid,
                 cudaStream_t st);
void launch_cull(const DevState &s, const Geom &g, int grid, cudaStream_t st);
void launch_lru(const DevState &s, int grid_a, int grid_b, cudaStream_t st);
void launch_decode_new(const DevState &s, const Geom &g, int grid, cudaStream_t st);
// triangle stage: count, scan, emit (emit_only: just the last, into a new output)
void launch_mc(const DevState &s, const Geom &g, bool debug, bool emit_only, const Grids &gr, cudaStream_t st);
void launch_hull(const float *bmin, const float *bmax, float2 *hull, float2 *hull8, const Geom &g,
                 cudaStream_t st);
void launch_reset_cache(const DevState &s, cudaStream_t st);
void launch_encode(const float *field, const Geom &g, uint64_t *bits, float *bmin, float *bmax, cudaStream_t st);
void launch_decode_list(const uint64_t *bits, uint32_t rate, const uint32_t *ids, uint64_t n, float *out,
                        cudaStream_t st);
void launch_gather_slots(const float *slots, const int32_t *islot, const uint32_t *ids, uint64_t n, float *out,
                         int32_t *missing, cudaStream_t st);

// occupancy-derived persistent grid sizes
Grids compute_grids(int sm_count);
void mc_grids(int sm_count, Grids *gr);   // also raises the emit kernel's shared-memory limit

}  // namespace bcmc
