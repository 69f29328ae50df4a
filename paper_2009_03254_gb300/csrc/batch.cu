// Batched extraction (C ABI in include/bcmc.h): many loaded volumes, each
// at its own isovalue, through the same persistent launches.  Every stage
// kernel takes a table of the volumes and numbers its work items volume
// after volume (launch.cuh), so one launch per stage serves the whole
// batch; the sequence (isovalues in, stages, output placement, one
// readback) is captured once as a CUDA graph.  Each volume keeps its own
// cache and control block, so its results equal those of extracting it
// alone.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "bcmc.h"
#include "common.cuh"
#include "kernels.cuh"
#include "volume.cuh"

using namespace bcmc;
using namespace bcmc_host;

namespace {
constexpr int kBatchEvents = 8;   // before, after prep, cull, cache update, decode, count, scan, emit
constexpr int kKernels = 6;       // tuned kernels: cull, cache update, decode, count, scan, emit
constexpr int kVariants = 3;      // tile-size variants per kernel (at most)
}  // namespace

struct iso_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t n = 0;
    std::vector<iso_volume *> vols;
    VolEntry *d_entries = nullptr;
    uint32_t *d_ctr = nullptr;            // the launch's work counters
    float *d_iso = nullptr;
    BatchOut *d_bo = nullptr;
    unsigned long long *d_tri_base = nullptr;
    Ctl *d_ctls = nullptr;                // control blocks gathered for the readback
    float *h_iso = nullptr;               // pinned mirrors
    BatchOut *h_bo = nullptr;
    Ctl *h_ctls = nullptr;
    unsigned long long *h_tri_base = nullptr;
    Plan want{};                          // launch shape: CTAs per SM and tiles, 0 = default
    Plan plan{};                          // what runs
    uint64_t total_blocks = 0, total_slots = 0;
    uint32_t max_rate = 1;                // the largest rate among the volumes
    uint32_t seg_any = 0;                 // some volume has segment ranges
    cudaStream_t capture_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool use_graph = true;
    cudaEvent_t ev[kBatchEvents] = {};
};

namespace {

Launch launch_of(const iso_batch *b) {
    return Launch{b->d_entries, b->n, b->d_ctr, VolEntry{}, b->max_rate, b->seg_any};
}

// per tuned kernel: its CTA field and tile field in a Plan (tile: null
// for the cache update, which has one tile size), and the tile variants
int *ctas_field(Plan &p, int k) {
    int *f[kKernels] = {&p.cull, &p.lru_a, &p.decode, &p.mc_count, &p.mc_scan, &p.mc_emit};
    return f[k];
}

int *tile_field(Plan &p, int k) {
    int *f[kKernels] = {&p.cull_tile, nullptr, &p.decode_tile, &p.count_tile, &p.scan_tile, &p.emit_tile};
    return f[k];
}

constexpr int kTileVariants[kKernels][kVariants] = {
    {2048, 4096, 4096}, {0, 0, 0}, {64, 128, 256}, {16, 32, 64}, {1024, 2048, 4096}, {16, 32, 64}};
constexpr int kNumVariants[kKernels] = {2, 1, 3, 3, 3, 3};

void set_ctas(Plan &p, int k, int ctas) {
    *ctas_field(p, k) = ctas;
    if (k == 1) p.lru_b = ctas;            // both cache-update kernels share one setting
}

void drop_graph(iso_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

void apply_shape(iso_batch *b, const Plan &want) {
    b->want = want;
    b->plan = launch_plan(&b->want, b->device, b->total_blocks, b->total_slots, b->n, false, b->max_rate,
                          b->seg_any != 0);
    drop_graph(b);
}

// Queue one batch extraction on `st`; with `prof`, events between the kernels.
int enqueue_batch(iso_batch *b, cudaStream_t st, bool prof) {
    const Launch L = launch_of(b);
    ISO_CK(cudaMemcpyAsync(b->d_iso, b->h_iso, b->n * sizeof(float), cudaMemcpyHostToDevice, st));
    ISO_CK(cudaMemcpyAsync(b->d_bo, b->h_bo, sizeof(BatchOut), cudaMemcpyHostToDevice, st));
    if (prof) cudaEventRecord(b->ev[0], st);
    launch_batch_params(L, b->d_iso, st);
    launch_front(L, b->plan, st, prof ? b->ev : nullptr);
    launch_mc_count(L, false, b->plan, st);
    if (prof) cudaEventRecord(b->ev[5], st);
    launch_mc_scan(L, b->plan, st);
    if (prof) cudaEventRecord(b->ev[6], st);
    launch_batch_offsets(L, b->d_bo, b->d_tri_base, st);
    launch_mc_emit(L, false, b->plan, st);
    if (prof) cudaEventRecord(b->ev[7], st);
    launch_batch_gather(L, b->d_ctls, st);
    ISO_CK(cudaMemcpyAsync(b->h_ctls, b->d_ctls, b->n * sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    ISO_CK(cudaMemcpyAsync(b->h_tri_base, b->d_tri_base, (b->n + 1) * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st));
    ISO_CK(cudaGetLastError());
    return ISO_OK;
}

int ensure_graph(iso_batch *b) {
    if (b->gexec) return ISO_OK;
    if (!b->capture_stream) ISO_CK(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    ISO_CK(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_batch(b, b->capture_stream, false);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
    if (rc != ISO_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return rc != ISO_OK ? rc : ISO_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        b->gexec = nullptr;
        (void)cudaGetLastError();
        return ISO_ERR_CUDA;
    }
    b->graph = g;
    return ISO_OK;
}

// run the batch (isovalues and output already in the pinned mirrors)
int run_batch(iso_batch *b, bool prof) {
    if (!prof && b->use_graph && ensure_graph(b) != ISO_OK) b->use_graph = false;
    if (!prof && b->use_graph && b->gexec) {
        ISO_CK(cudaGraphLaunch(b->gexec, b->stream));
    } else {
        const int rc = enqueue_batch(b, b->stream, prof);
        if (rc) return rc;
    }
    ISO_CK(cudaStreamSynchronize(b->stream));
    return ISO_OK;
}

// Mirror each control block into its volume; per-volume errors (a timeout
// empties that volume's cache).  Returns the first error.
int finish_batch(iso_batch *b, iso_stats *stats, int *status) {
    int first = ISO_OK;
    for (uint32_t i = 0; i < b->n; i++) {
        iso_volume *v = b->vols[i];
        *v->host_ctl = b->h_ctls[i];
        v->last_n_active = v->host_ctl->n_active;
        v->last_n_new = v->host_ctl->n_new;
        v->last_n_cand = v->host_ctl->n_cand;
        v->last_slots = v->host_ctl->S;
        v->last_tris = v->host_ctl->n_tri;
        const int rc = status_to_error(v, v->host_ctl->status);
        if (stats) fill_stats(*v->host_ctl, &stats[i], 0);
        if (status) status[i] = rc;
        if (rc && !first) first = rc;
    }
    return first;
}

int reset_caches(iso_batch *b) {
    for (iso_volume *v : b->vols) launch_reset_cache(v->s, b->stream);
    ISO_CK(cudaGetLastError());
    ISO_CK(cudaStreamSynchronize(b->stream));
    return ISO_OK;
}

void free_batch(iso_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->device);
    void *ptrs[] = {b->d_entries, b->d_ctr, b->d_iso, b->d_bo, b->d_tri_base, b->d_ctls};
    for (void *p : ptrs) dfree_on(p, b->stream);
    cudaStreamSynchronize(b->stream);
    (void)cudaGetLastError();
    void *host[] = {b->h_iso, b->h_bo, b->h_ctls, b->h_tri_base};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    drop_graph(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (cudaEvent_t &e : b->ev)
        if (e) cudaEventDestroy(e);
    delete b;
}

int set_inputs(iso_batch *b, const float *isovalues, float *d_vertices, uint64_t capacity_triangles) {
    if (!isovalues || (!d_vertices && capacity_triangles) || misaligned(d_vertices, 16)) return ISO_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < b->n; i++)
        if (!std::isfinite(isovalues[i])) return ISO_ERR_INVALID_ARG;
    std::memcpy(b->h_iso, isovalues, b->n * sizeof(float));
    *b->h_bo = BatchOut{(unsigned long long)(uintptr_t)d_vertices, capacity_triangles};
    return ISO_OK;
}

}  // namespace

extern "C" {

int iso_batch_create(iso_batch **out, iso_volume *const *volumes, uint32_t n, void *stream) {
    if (!out || !volumes || n == 0 || n > kMaxBatch) return ISO_ERR_INVALID_ARG;
    *out = nullptr;
    int dev = 0;
    ISO_CK(cudaGetDevice(&dev));
    std::vector<iso_volume *> vols(volumes, volumes + n);
    for (iso_volume *v : vols)
        if (!v || v->device != dev || (v->flags & ISO_DEBUG)) return ISO_ERR_INVALID_ARG;
    {
        std::vector<iso_volume *> sorted = vols;
        std::sort(sorted.begin(), sorted.end());
        if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) return ISO_ERR_INVALID_ARG;
    }
    for (iso_volume *v : vols) ISO_CK_RC(finish_upload(v));   // batches read the bitstreams on their own stream
    iso_batch *b = new (std::nothrow) iso_batch();
    if (!b) return ISO_ERR_OOM;
    b->device = dev;
    b->stream = (cudaStream_t)stream;
    b->n = n;
    b->vols = vols;
    int rc = ISO_OK;
#define TRY(x)                              \
    do {                                    \
        rc = (x);                           \
        if (rc) { free_batch(b); return rc; } \
    } while (0)
    TRY(dalloc_on(&b->d_entries, n, dev, b->stream));
    TRY(dalloc_on(&b->d_ctr, kNumLaunchCounters, dev, b->stream));
    TRY(dalloc_on(&b->d_iso, n, dev, b->stream));
    TRY(dalloc_on(&b->d_bo, 1, dev, b->stream));
    TRY(dalloc_on(&b->d_tri_base, n + 1, dev, b->stream));
    TRY(dalloc_on(&b->d_ctls, n, dev, b->stream));
    if (cudaMallocHost((void **)&b->h_iso, n * sizeof(float)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_bo, sizeof(BatchOut)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_ctls, n * sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_tri_base, (n + 1) * sizeof(unsigned long long)) != cudaSuccess) {
        (void)cudaGetLastError();
        free_batch(b);
        return ISO_ERR_OOM;
    }
    for (cudaEvent_t &e : b->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            (void)cudaGetLastError();
            free_batch(b);
            return ISO_ERR_CUDA;
        }
    std::vector<VolEntry> entries(n);
    for (uint32_t i = 0; i < n; i++) {
        const iso_volume *v = vols[i];
        entries[i] = VolEntry{v->s, v->g, v->n_cull_desc, v->n_lru_desc};
        b->total_blocks += v->g.nb;
        b->total_slots += v->cap;
        b->max_rate = std::max(b->max_rate, v->g.rate);
        if (v->seg) b->seg_any = 1;
    }
    // the volumes' own streams may still hold work (a cache reset, a free)
    for (iso_volume *v : vols)
        if (cudaStreamSynchronize(v->stream) != cudaSuccess) {
            (void)cudaGetLastError();
            free_batch(b);
            return ISO_ERR_CUDA;
        }
    if (cudaMemcpyAsync(b->d_entries, entries.data(), n * sizeof(VolEntry), cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(b->d_ctr, 0, kNumLaunchCounters * sizeof(uint32_t), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        (void)cudaGetLastError();
        free_batch(b);
        return ISO_ERR_CUDA;
    }
#undef TRY
    apply_shape(b, Plan{});
    *out = b;
    return ISO_OK;
}

int iso_batch_extract(iso_batch *b, const float *isovalues, float *d_vertices, uint64_t capacity_triangles,
                      uint64_t *tri_offsets, iso_stats *stats, int *status) {
    NvtxRange nvtx("iso_batch_extract");
    if (!b || !tri_offsets) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    int rc = set_inputs(b, isovalues, d_vertices, capacity_triangles);
    if (rc) return rc;
    rc = run_batch(b, false);
    if (rc) return rc;
    for (uint32_t i = 0; i <= b->n; i++) tri_offsets[i] = b->h_tri_base[i];
    rc = finish_batch(b, stats, status);
    if (rc) return rc;
    return b->h_tri_base[b->n] > capacity_triangles ? ISO_ERR_CAPACITY : ISO_OK;
}

int iso_batch_set_shape(iso_batch *b, const iso_launch_shape *shape) {
    if (!b || !shape) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    Plan w{};
    const int rc = shape_to_want(shape, &w);
    if (rc) return rc;
    apply_shape(b, w);
    return ISO_OK;
}

int iso_batch_get_shape(const iso_batch *b, iso_launch_shape *shape) {
    if (!b || !shape) return ISO_ERR_INVALID_ARG;
    *shape = shape_of(b->want, b->device, false, b->max_rate, b->seg_any != 0);
    return ISO_OK;
}

int iso_batch_tune(iso_batch *b, const float *isovalues, float *d_vertices, uint64_t capacity_triangles,
                   int trials, iso_launch_shape *best, float *best_ms) {
    if (!b || trials < 1) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    int rc = set_inputs(b, isovalues, d_vertices, capacity_triangles);
    if (rc) return rc;
    const Plan keep = b->want;
    // one cold run with `want`: per-kernel times (ms) and the total
    auto timed = [&](const Plan &want, float *kernel_ms, float *total_ms) -> int {
        b->plan = launch_plan(&want, b->device, b->total_blocks, b->total_slots, b->n, false, b->max_rate,
                              b->seg_any != 0);
        int r = reset_caches(b);
        if (r) return r;
        r = run_batch(b, true);
        if (r) return r;
        r = finish_batch(b, nullptr, nullptr);
        if (r) return r;
        for (int k = 0; k < kKernels; k++) {   // events k+1 .. k+2 bracket kernel k
            float ms = 0.f;
            ISO_CK(cudaEventElapsedTime(&ms, b->ev[k + 1], b->ev[k + 2]));
            kernel_ms[k] = ms;
        }
        ISO_CK(cudaEventElapsedTime(total_ms, b->ev[0], b->ev[7]));
        return ISO_OK;
    };
    float best_t[kKernels];
    int best_tile[kKernels], best_ctas[kKernels];
    for (int k = 0; k < kKernels; k++) {
        best_t[k] = std::numeric_limits<float>::infinity();
        best_tile[k] = 0;
        best_ctas[k] = 0;
    }
    for (int i = 0; i < kVariants; i++) {
        Plan tiles{};
        for (int k = 0; k < kKernels; k++)
            if (tile_field(tiles, k)) *tile_field(tiles, k) = kTileVariants[k][std::min(i, kNumVariants[k] - 1)];
        Plan lim = occupancy_limits_of(b->device, default_tiles(&tiles), false, b->max_rate, b->seg_any != 0);
        int cmax = 1;
        for (int k = 0; k < kKernels; k++) cmax = std::max(cmax, *ctas_field(lim, k));
        for (int c = 1; c <= cmax; c++) {
            Plan want = tiles;
            for (int k = 0; k < kKernels; k++) set_ctas(want, k, std::min(c, *ctas_field(lim, k)));
            float kt[kKernels], tot = 0.f, mins[kKernels];
            for (int k = 0; k < kKernels; k++) mins[k] = std::numeric_limits<float>::infinity();
            for (int t = 0; t < trials; t++) {
                rc = timed(want, kt, &tot);
                if (rc) { apply_shape(b, keep); return rc; }
                for (int k = 0; k < kKernels; k++) mins[k] = std::min(mins[k], kt[k]);
            }
            for (int k = 0; k < kKernels; k++) {
                // only settings not timed before: a new tile variant, CTAs within the limit
                if (i >= kNumVariants[k] || c > *ctas_field(lim, k)) continue;
                if (mins[k] < best_t[k]) {
                    best_t[k] = mins[k];
                    best_tile[k] = tile_field(tiles, k) ? *tile_field(tiles, k) : 0;
                    best_ctas[k] = c;
                }
            }
        }
    }
    Plan chosen{};
    for (int k = 0; k < kKernels; k++) {
        set_ctas(chosen, k, best_ctas[k]);
        if (tile_field(chosen, k)) *tile_field(chosen, k) = best_tile[k];
    }
    float default_ms = std::numeric_limits<float>::infinity(), chosen_ms = default_ms;
    for (int t = 0; t < trials; t++) {
        float kt[kKernels], tot = 0.f;
        rc = timed(Plan{}, kt, &tot);
        if (rc) { apply_shape(b, keep); return rc; }
        default_ms = std::min(default_ms, tot);
        rc = timed(chosen, kt, &tot);
        if (rc) { apply_shape(b, keep); return rc; }
        chosen_ms = std::min(chosen_ms, tot);
    }
    apply_shape(b, chosen_ms <= default_ms ? chosen : Plan{});
    rc = reset_caches(b);
    if (rc) return rc;
    if (best) rc = iso_batch_get_shape(b, best);
    if (best_ms) {
        best_ms[0] = default_ms;
        best_ms[1] = std::min(chosen_ms, default_ms);
    }
    return rc;
}

void iso_batch_release(iso_batch *b) { free_batch(b); }

}  // extern "C"
