// Host-side state of a loaded volume and the helpers the C ABI's entry
// points share (api.cu: single volumes; batch.cu: batches).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "bcmc.h"
#include "common.cuh"
#include "kernels.cuh"

struct iso_volume {
    int device = 0;
    cudaStream_t stream = nullptr;
    bcmc::Geom g{};
    uint32_t flags = 0;
    bcmc::DevState s{};
    bcmc::Plan plan{};                // CTAs and tile sizes of the launches
    bcmc::Plan want{};                // the launch shape asked for (iso_set_shape; zeros: defaults)
    uint32_t cap = 0;                 // physical slots
    uint32_t n_cull_desc = 0, n_lru_desc = 0;
    bcmc::Ctl *host_ctl = nullptr;    // pinned mirror for the one readback
    bcmc::Params *host_params = nullptr;   // pinned: this extraction's isovalue, output and capacity
    cudaStream_t capture_stream = nullptr;
    // ISO_ASYNC_UPLOAD: the bitstream's copy runs on its own stream; the
    // first extraction's decode waits for `uploaded`, every other call waits
    // on the host (upload_pending until then)
    cudaStream_t upload_stream = nullptr;
    cudaEvent_t uploaded = nullptr;
    bool upload_pending = false;
    // ISO_ASYNC_UPLOAD: the load's range check is read by the first call on
    // the volume (check_pending until then); `corrupt` makes every call fail
    bool check_pending = false;
    bool corrupt = false;
    // one extraction: params copy, the stage kernels, count readback; one
    // graph per kind (0: triangle soup, 1: indexed mesh, 2: the soup up to
    // the scan, 3: the emission alone)
    cudaGraph_t graph[4] = {};
    cudaGraphExec_t gexec[4] = {};
    bool use_graph = true;
    uint32_t test_flags = 0;          // ParamFlags of the test hook (iso_set_test_fault)
    uint64_t extractions = 0;         // full extractions run so far (graphs are captured after kGraphAfter)
    // owned device allocations
    uint64_t *bits = nullptr;
    float *bmin = nullptr, *bmax = nullptr;   // staging of host block ranges during the load only
    float2 *hull = nullptr, *hull8 = nullptr;
    float2 *seg = nullptr;            // segment ranges (ISO_SEGMENT_CULL, or large volumes by default)
    uint8_t *tables = nullptr;
    unsigned long long dbg_edges_cap = 0;   // in vertices
    unsigned long long last_vtx = 0;        // vertices of the last indexed extraction
    bool profiling = false;
    cudaEvent_t ev[ISO_NUM_STAGES + 2] = {};   // stage boundaries, then the start of a separate emission
    bool split_emit = false;                   // the last emission ran apart from the count and scan
    float stage_ms[ISO_NUM_STAGES] = {};
    unsigned long long last_tris = 0;
    uint32_t last_n_active = 0, last_n_new = 0, last_n_cand = 0, last_slots = 0;
};

namespace bcmc_host {

// An NVTX range over a library call or one of its phases, so that a
// profiler can group and filter the kernels each one launches (e.g. ncu
// --nvtx --nvtx-include "iso_extract emit/"); without a tool attached the
// push and pop return at once.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define ISO_CK(call)                                                          \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) {                                              \
            (void)cudaGetLastError();                                         \
            return e_ == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA; \
        }                                                                     \
    } while (0)

// A caller's device pointer that its element type (or the vector stores
// and bulk copies that write it) cannot use: not a multiple of `align` bytes.
inline bool misaligned(const void *p, uintptr_t align) { return ((uintptr_t)p & (align - 1)) != 0; }

// Stream-ordered allocation from the library's pool of `dev`, ordered on `st`.
int dalloc_bytes(void **p, size_t bytes, int dev, cudaStream_t st);
void dfree_on(void *p, cudaStream_t st);

template <typename T>
int dalloc_on(T **p, size_t count, int dev, cudaStream_t st) {
    return dalloc_bytes(reinterpret_cast<void **>(p), count * sizeof(T), dev, st);
}

#define ISO_CK_RC(call)          \
    do {                         \
        const int rc_ = (call);  \
        if (rc_) return rc_;     \
    } while (0)

struct DeviceGuard {              // make a device current for the call
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Error of an extraction from its status bits.  After a timeout the
// volume's cache bookkeeping may be inconsistent: it is emptied on the
// volume's stream (and that stream synchronised).
int status_to_error(iso_volume *v, uint32_t st);

void fill_stats(const bcmc::Ctl &c, iso_stats *st, uint32_t reruns);

// The plan of launches over volumes with `total_blocks` blocks and
// `total_slots` cache slots together.  `want` (may be NULL) gives CTAs per
// SM per kernel (0 = the kernel's occupancy limit; larger values are
// clamped to it) and tile sizes (0 = default); the result holds CTAs per
// launch (times the SM count, but no more than the launch can have work
// items) and the tile sizes.
bcmc::Plan launch_plan(const bcmc::Plan *want, int device, uint64_t total_blocks, uint64_t total_slots,
                       uint32_t n_vols, bool single, uint32_t max_rate, bool seg = false);

// the tile fields of `want`, defaults where 0
bcmc::Plan default_tiles(const bcmc::Plan *want);

// a launch shape as a requested plan (ISO_ERR_INVALID_ARG for tiles no kernel has)
int shape_to_want(const iso_launch_shape *shape, bcmc::Plan *out);

// the launch shape that runs for a requested plan (CTAs clamped to the occupancy limits)
iso_launch_shape shape_of(const bcmc::Plan &want, int device, bool single, uint32_t max_rate, bool seg = false);

// largest CTAs per SM of each kernel for these tile sizes, in single-volume
// or batch launches whose largest rate is max_rate (cached per device)
bcmc::Plan occupancy_limits_of(int device, const bcmc::Plan &tiles, bool single, uint32_t max_rate,
                               bool seg = false);

// the verdict of an asynchronous load's range check (waits for the load's
// own work, not for the bitstream): ISO_ERR_CORRUPT for ranges that are not
// ranges, from then on for every call
int check_load(iso_volume *v);

// check_load, then wait on the host for an asynchronous upload still in flight
int finish_upload(iso_volume *v);

// device address of the single-volume work counters (inside the control block)
inline uint32_t *single_counters(const iso_volume *v) {
    return reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(v->s.ctl) + offsetof(bcmc::Ctl, ctr));
}

}  // namespace bcmc_host
