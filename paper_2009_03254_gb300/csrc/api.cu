// Host side of the C ABI declared in include/bcmc.h.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <utility>
#include <vector>

#include "bcmc.h"
#include "common.cuh"
#include "kernels.cuh"
#include "mc_tables.cuh"

using namespace bcmc;

#include "volume.cuh"

using namespace bcmc_host;

namespace bcmc_host {

// Device memory comes from one library-owned, stream-ordered pool per
// device that keeps freed memory for reuse (release threshold raised), so
// loading and releasing volumes repeatedly does not pay for cudaMalloc and
// cudaFree (which synchronises the device) each time.
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
struct OccEntry {
    int device;
    int key[8];                   // tile sizes, single/batch, largest rate, segment ranges
    Plan limits;
};
std::vector<OccEntry> g_occ;      // occupancy limits per (device, tile variants)

cudaMemPool_t device_pool(int dev) {
    if (dev < 0 || dev >= kMaxPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

// A caller's allocator (iso_set_allocator); every allocation it makes is
// remembered with its free function and device, so it goes back to it.
struct HookAllocator {
    iso_alloc_fn alloc = nullptr;
    iso_free_fn free = nullptr;
    void *ctx = nullptr;
    int device = 0;
};
std::mutex g_alloc_mutex;
HookAllocator g_hook;
std::unordered_map<void *, HookAllocator> g_hooked;

// A volume's pinned host mirrors (control block and parameters, one block)
// and its upload stream are kept for the next volume when it is released:
// pinning and unpinning host memory and creating a stream each cost tens of
// microseconds, which a loop that loads and releases volumes one after
// another would otherwise pay with the GPU idle.
constexpr size_t kParamsOffset = (sizeof(Ctl) + 255) / 256 * 256;
constexpr size_t kPinnedBlockBytes = kParamsOffset + (sizeof(Params) + 255) / 256 * 256;
constexpr size_t kPinnedKeep = 64;                 // blocks kept (a few KB each)
constexpr size_t kStreamsKeep = 8;                 // upload streams kept per device
std::mutex g_reuse_mutex;
std::vector<void *> g_pinned_free;
std::vector<std::pair<int, cudaStream_t>> g_streams_free;   // (device, stream)

void *pinned_take() {
    {
        std::lock_guard<std::mutex> lock(g_reuse_mutex);
        if (!g_pinned_free.empty()) {
            void *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, kPinnedBlockBytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_give(void *p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lock(g_reuse_mutex);
        if (g_pinned_free.size() < kPinnedKeep) {
            g_pinned_free.push_back(p);
            return;
        }
    }
    cudaFreeHost(p);
}

// a non-blocking stream of the current device (`dev`)
cudaError_t stream_take(int dev, cudaStream_t *st) {
    {
        std::lock_guard<std::mutex> lock(g_reuse_mutex);
        for (size_t i = g_streams_free.size(); i-- > 0;)
            if (g_streams_free[i].first == dev) {
                *st = g_streams_free[i].second;
                g_streams_free.erase(g_streams_free.begin() + (long)i);
                return cudaSuccess;
            }
    }
    return cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
}

// an idle stream (the caller synchronised it) of device `dev`
void stream_give(int dev, cudaStream_t st) {
    if (!st) return;
    {
        std::lock_guard<std::mutex> lock(g_reuse_mutex);
        size_t n = 0;
        for (const auto &e : g_streams_free) n += e.first == dev;
        if (n < kStreamsKeep) {
            g_streams_free.emplace_back(dev, st);
            return;
        }
    }
    cudaStreamDestroy(st);
}

int dalloc_bytes(void **p, size_t bytes, int dev, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    HookAllocator h;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        h = g_hook;
    }
    if (h.alloc) {
        void *q = h.alloc(bytes, dev, st, h.ctx);
        if (!q) return ISO_ERR_OOM;
        h.device = dev;
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        g_hooked[q] = h;
        *p = q;
        return ISO_OK;
    }
    cudaMemPool_t pool = device_pool(dev);
    if (pool) {
        cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
        if (e == cudaErrorMemoryAllocation) {   // what the pool keeps may be what is missing: trim, retry once
            (void)cudaGetLastError();
            int cur = 0;
            cudaGetDevice(&cur);
            cudaSetDevice(dev);
            const bool ok = cudaDeviceSynchronize() == cudaSuccess && cudaMemPoolTrimTo(pool, 0) == cudaSuccess;
            cudaSetDevice(cur);
            (void)cudaGetLastError();
            if (ok) e = cudaMallocFromPoolAsync(p, bytes, pool, st);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            *p = nullptr;
            return e == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA;
        }
    } else {
        ISO_CK(cudaMalloc(p, bytes));
    }
    return ISO_OK;
}

void dfree_on(void *p, cudaStream_t st) {
    if (!p) return;
    HookAllocator h;
    bool hooked = false;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mutex);
        auto it = g_hooked.find(p);
        if (it != g_hooked.end()) {
            h = it->second;
            g_hooked.erase(it);
            hooked = true;
        }
    }
    if (hooked) h.free(p, h.device, st, h.ctx);
    else cudaFreeAsync(p, st);
}

int shape_to_want(const iso_launch_shape *shape, Plan *out) {
    Plan w{};
    // CTAs per SM beyond any occupancy limit mean "the limit"; tile sizes
    // are checked exactly (values that do not fit an int are invalid)
    auto c = [](uint32_t x) { return (int)std::min<uint32_t>(x, 1024u); };
    auto t = [](uint32_t x) { return x > 65536u ? -1 : (int)x; };
    w.cull = c(shape->cull_ctas);
    w.cull_tile = t(shape->cull_tile);
    w.lru_a = w.lru_b = c(shape->cache_update_ctas);
    w.decode = c(shape->decode_ctas);
    w.decode_tile = t(shape->decode_tile);
    w.mc_count = c(shape->count_ctas);
    w.count_tile = t(shape->count_tile);
    w.mc_scan = c(shape->scan_ctas);
    w.scan_tile = t(shape->scan_tile);
    w.mc_emit = c(shape->emit_ctas);
    w.emit_tile = t(shape->emit_tile);
    if (!valid_tiles(default_tiles(&w))) return ISO_ERR_INVALID_ARG;
    *out = w;
    return ISO_OK;
}

iso_launch_shape shape_of(const Plan &want, int device, bool single, uint32_t max_rate, bool seg) {
    // CTAs per SM that run: the requested number clamped to the occupancy limit
    const Plan tiles = default_tiles(&want);
    const Plan lim = occupancy_limits_of(device, tiles, single, max_rate, seg);
    auto run = [](int w, int mx) { return (uint32_t)(w > 0 ? std::min(w, mx) : mx); };
    return iso_launch_shape{run(want.cull, lim.cull), (uint32_t)tiles.cull_tile, run(want.lru_a, lim.lru_a),
                            run(want.decode, lim.decode), (uint32_t)tiles.decode_tile,
                            run(want.mc_count, lim.mc_count), (uint32_t)tiles.count_tile,
                            run(want.mc_scan, lim.mc_scan), (uint32_t)tiles.scan_tile,
                            run(want.mc_emit, lim.mc_emit), (uint32_t)tiles.emit_tile};
}

int check_load(iso_volume *v) {
    if (v->check_pending) {
        v->check_pending = false;
        ISO_CK(cudaStreamSynchronize(v->stream));        // the hulls and the readback of their verdict
        if (v->host_ctl->status & kStatusCorrupt) v->corrupt = true;
    }
    return v->corrupt ? ISO_ERR_CORRUPT : ISO_OK;
}

int finish_upload(iso_volume *v) {
    if (!v) return ISO_OK;
    const int rc = check_load(v);
    if (rc || !v->upload_pending) return rc;
    v->upload_pending = false;
    ISO_CK(cudaEventSynchronize(v->uploaded));
    return ISO_OK;
}

Plan default_tiles(const Plan *want) {
    Plan t{};
    t.cull_tile = want && want->cull_tile ? want->cull_tile : kDefaultCullTile;
    t.decode_tile = want && want->decode_tile ? want->decode_tile : kDefaultDecodeTile;
    t.count_tile = want && want->count_tile ? want->count_tile : kDefaultCountTile;
    t.scan_tile = want && want->scan_tile ? want->scan_tile : kDefaultScanTile;
    t.emit_tile = want && want->emit_tile ? want->emit_tile : kDefaultEmitTile;
    return t;
}

Plan occupancy_limits_of(int device, const Plan &tiles, bool single, uint32_t max_rate, bool seg) {
    const int key[8] = {tiles.cull_tile, tiles.decode_tile, tiles.count_tile, tiles.scan_tile, tiles.emit_tile,
                        single ? 1 : 0, (int)max_rate, seg ? 1 : 0};
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    for (const OccEntry &e : g_occ)
        if (e.device == device && std::equal(key, key + 8, e.key)) return e.limits;
    OccEntry e{device, {key[0], key[1], key[2], key[3], key[4], key[5], key[6], key[7]},
               occupancy_limits(tiles, single, max_rate, seg)};
    g_occ.push_back(e);
    return e.limits;
}

Plan launch_plan(const Plan *want, int device, uint64_t total_blocks, uint64_t total_slots, uint32_t n_vols,
                 bool single, uint32_t max_rate, bool seg) {
    const Plan tiles = default_tiles(want);
    const Plan lim = occupancy_limits_of(device, tiles, single, max_rate, seg);
    Plan use = lim;
    if (want) {
        int *dst = &use.prep;
        const int *src = &want->prep, *mx = &lim.prep;
        for (int k = 0; k < 8; k++) dst[k] = src[k] > 0 ? std::min(src[k], mx[k]) : mx[k];
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0) {
        (void)cudaGetLastError();
        sms = 1;
    }
    int *ctas = &use.prep;
    for (int k = 0; k < 8; k++) ctas[k] = std::max(1, ctas[k]) * sms;
    // no more CTAs than work items (each bound holds for any isovalue)
    auto clamp = [](int &grid, uint64_t items) {
        grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)grid, items));
    };
    auto tiles_of = [&](uint64_t n, int tile) { return (n + tile - 1) / tile + n_vols; };
    clamp(use.cull, tiles_of(total_blocks, use.cull_tile));
    clamp(use.lru_a, 2 * tiles_of(total_slots, kScanTile) + n_vols);
    clamp(use.lru_b, tiles_of(total_slots, kScanTile));
    clamp(use.decode, tiles_of(total_slots, use.decode_tile));
    clamp(use.mc_count, tiles_of(total_slots, use.count_tile));
    clamp(use.mc_emit, tiles_of(total_slots, use.emit_tile));
    clamp(use.mc_scan, tiles_of(total_slots, use.scan_tile));
    return use;
}

// After a timeout the cache bookkeeping may be inconsistent: empty it so
// the next extraction starts from a clean state.
int status_to_error(iso_volume *v, uint32_t st) {
    if (st & kStatusBounds) return ISO_ERR_BOUNDS;
    if (st & kStatusAnyTimeout) {
        launch_reset_cache(v->s, v->stream);
        cudaStreamSynchronize(v->stream);
        (void)cudaGetLastError();
        return ISO_ERR_TIMEOUT;
    }
    if (st & kStatusBudget) return ISO_ERR_BUDGET;
    return ISO_OK;
}

void fill_stats(const Ctl &c, iso_stats *st, uint32_t reruns) {
    st->num_triangles = c.n_tri;
    st->n_active = c.n_active;
    st->n_new = c.n_new;
    st->n_occupied = c.n_occ;
    st->n_slots = c.S;
    st->cache_bytes = (uint64_t)c.S * 256ull;
    st->epoch = c.epoch;
    st->reruns = reruns;
    st->n_candidates = c.n_cand;
    st->waves = 1;
    st->num_vertices = 0;
}

}  // namespace bcmc_host

namespace {

#define CK(call) ISO_CK(call)

// allocations of a volume are ordered on its stream
template <typename T>
int dalloc(iso_volume *v, T **p, size_t count) {
    return dalloc_on(p, count, v->device, v->stream);
}

int geometry(uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate, Geom *g) {
    if (nx == 0 || ny == 0 || nz == 0 || rate < 1 || rate > 32) return ISO_ERR_INVALID_ARG;
    const uint64_t nbx = (nx + 3ull) / 4, nby = (ny + 3ull) / 4, nbz = (nz + 3ull) / 4;
    const uint64_t nb = nbx * nby * nbz;
    if (nb >= (1ull << 31)) return ISO_ERR_INVALID_ARG;   // ids and packed counters are 31-bit
    *g = Geom{nx, ny, nz, (uint32_t)nbx, (uint32_t)nby, (uint32_t)nbz, (uint32_t)nb, rate,
              div_magic((uint32_t)nbx), div_magic((uint32_t)nby)};
    return ISO_OK;
}

int free_volume(iso_volume *v) {
    if (!v) return ISO_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(v->device);
    if (v->upload_stream) cudaStreamSynchronize(v->upload_stream);   // nothing is freed under a copy in flight
    DevState &s = v->s;
    void *ptrs[] = {v->bits, v->bmin, v->bmax, v->hull, v->hull8, v->seg, v->tables, s.mactive, s.iactive, s.inew, s.icand,
                    s.islot, s.slast, s.sblock, s.lbuf[0], s.lbuf[1], s.newslot, s.slots, s.desc_cull, s.desc_cand,
                    s.desc_lru_a, s.desc_lru_b, s.desc_mc, s.ctl, s.counts, s.offsets, s.iocc, s.cases, s.dbg_edges,
                    s.voff, s.cutw};
    for (void *p : ptrs) dfree_on(p, v->stream);
    cudaStreamSynchronize(v->stream);
    (void)cudaGetLastError();
    pinned_give(v->host_ctl);            // the block that also holds host_params
    for (int k = 0; k < 4; k++) {
        if (v->gexec[k]) cudaGraphExecDestroy(v->gexec[k]);
        if (v->graph[k]) cudaGraphDestroy(v->graph[k]);
    }
    if (v->capture_stream) cudaStreamDestroy(v->capture_stream);
    stream_give(v->device, v->upload_stream);   // synchronised above
    if (v->uploaded) cudaEventDestroy(v->uploaded);
    for (cudaEvent_t &e : v->ev)
        if (e) cudaEventDestroy(e);
    cudaSetDevice(dev);
    delete v;
    return ISO_OK;
}

constexpr uint64_t kGraphAfter = 8;   // extractions of a volume before its passes are captured as graphs

// What one queued pass runs: the whole extraction, the stages up to the
// scan (the size becomes known), or the emission alone (after the count and
// scan of the same isovalue).
enum class Phase { kAll, kCount, kEmit };

// Queue one extraction pass on `st`: copy the parameters in, run the
// stages, copy the control block out.  Events between the stages are
// recorded when profiling (never inside a captured graph).
int enqueue_pipeline(iso_volume *v, cudaStream_t st, Phase phase, bool prof, bool indexed) {
    const bool debug = (v->flags & ISO_DEBUG) != 0;
    const Launch L{nullptr, 1u, single_counters(v), VolEntry{v->s, v->g, v->n_cull_desc, v->n_lru_desc}};
    CK(cudaMemcpyAsync(&v->s.ctl->params, v->host_params, sizeof(Params), cudaMemcpyHostToDevice, st));
    if (prof) cudaEventRecord(phase == Phase::kEmit ? v->ev[ISO_NUM_STAGES + 1] : v->ev[0], st);
    if (phase != Phase::kEmit) {
        launch_front(L, v->plan, st, prof ? v->ev : nullptr, v->upload_pending ? v->uploaded : nullptr);
        launch_mc_count(L, debug, v->plan, st, indexed);
        if (prof) cudaEventRecord(v->ev[5], st);
        launch_mc_scan(L, v->plan, st);
        if (prof) cudaEventRecord(v->ev[6], st);
    }
    if (phase != Phase::kCount) {
        launch_mc_emit(L, debug, v->plan, st, indexed);
        if (prof) cudaEventRecord(v->ev[7], st);
    }
    CK(cudaMemcpyAsync(v->host_ctl, v->s.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaGetLastError());
    return ISO_OK;
}

int graph_kind(Phase phase, bool indexed) {
    return phase == Phase::kAll ? (indexed ? 1 : 0) : (phase == Phase::kCount ? 2 : 3);
}

// Capture an extraction pass once per volume and kind (on a private stream:
// the legacy default stream cannot be captured); launches then go to the
// volume's stream.  Every per-extraction input comes through Params, so a
// graph never needs updating.
int ensure_graph(iso_volume *v, Phase phase, bool indexed) {
    const int k = graph_kind(phase, indexed);
    if (v->gexec[k]) return ISO_OK;
    if (!v->capture_stream) CK(cudaStreamCreateWithFlags(&v->capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(v->capture_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_pipeline(v, v->capture_stream, phase, false, indexed);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(v->capture_stream, &g);
    if (rc != ISO_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();
        return rc != ISO_OK ? rc : ISO_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&v->gexec[k], g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        v->gexec[k] = nullptr;
        (void)cudaGetLastError();
        return ISO_ERR_CUDA;
    }
    v->graph[k] = g;
    return ISO_OK;
}

void collect_stage_times(iso_volume *v) {
    if (!v->profiling) return;
    for (int k = 0; k < ISO_NUM_STAGES; k++) {
        float ms = 0.0f;
        // a separate emission is timed from its own start event
        cudaEvent_t from = (k == ISO_NUM_STAGES - 1 && v->split_emit) ? v->ev[ISO_NUM_STAGES + 1] : v->ev[k];
        if (cudaEventElapsedTime(&ms, from, v->ev[k + 1]) != cudaSuccess) {
            (void)cudaGetLastError();
            ms = -1.0f;
        }
        v->stage_ms[k] = ms;
    }
}

// debug mode: make sure the per-vertex edge-id buffer can hold T triangles
int ensure_debug_edges(iso_volume *v, unsigned long long tris) {
    if (!(v->flags & ISO_DEBUG) || 3ull * tris <= v->dbg_edges_cap) return ISO_OK;
    CK(cudaStreamSynchronize(v->stream));
    dfree_on(v->s.dbg_edges, v->stream);
    v->s.dbg_edges = nullptr;
    const unsigned long long want = std::max(3ull * tris, 3ull * 1024);
    int rc = dalloc(v, &v->s.dbg_edges, want);
    if (rc) { v->dbg_edges_cap = 0; return rc; }
    v->dbg_edges_cap = want;
    return ISO_OK;
}

// run the pipeline into `out` (capacity cap_tris); returns the error of
// the run, with the control block mirrored on the host
struct Window {                    // a wave: block ids [lo, act_hi) may be active, [lo, cand_hi) candidates
    uint32_t lo, cand_hi, act_hi;
};

struct Indexed {                   // indexed-mesh outputs of one pass
    uint32_t *idx;                 // 3 * cap_tris indices
    unsigned long long vert_cap;   // vertices the vertex buffer holds
    unsigned long long vtx_base;   // added to every index
};

// the first-vertex array of the occupied candidates and the candidates'
// cut-edge words, made at the first indexed extraction
int ensure_voff(iso_volume *v) {
    if (!v->s.voff) {
        const int rc = dalloc(v, &v->s.voff, v->s.list_cap);
        if (rc) return rc;
    }
    if (!v->s.cutw) return dalloc(v, &v->s.cutw, (size_t)v->s.list_cap * 12);
    return ISO_OK;
}

int run(iso_volume *v, float iso, void *out, unsigned long long cap_tris, Phase phase = Phase::kAll,
        uint32_t format = kVertexFloat4, uint32_t flags = 0, const Window *w = nullptr,
        const Indexed *ix = nullptr) {
    NvtxRange nvtx(phase == Phase::kCount ? "iso_extract count" : (phase == Phase::kEmit ? "iso_extract emit"
                                                                                        : "iso_extract"));
    int rc = check_load(v);
    if (rc) return rc;
    rc = ensure_debug_edges(v, cap_tris);
    if (rc) return rc;
    if (ix && (rc = ensure_voff(v)) != ISO_OK) return rc;
    *v->host_params = Params{iso,
                             format,
                             flags | v->test_flags | (w ? (uint32_t)kParamWindow : 0u) |
                                 (ix ? (uint32_t)kParamIndexed : 0u),
                             w ? w->lo : 0u,
                             w ? w->cand_hi : 0u,
                             w ? w->act_hi : 0u,
                             cap_tris,
                             (unsigned long long)(uintptr_t)out,
                             ix ? (unsigned long long)(uintptr_t)ix->idx : 0ull,
                             ix ? ix->vert_cap : 0ull,
                             ix ? ix->vtx_base : 0ull};
    // a pass is captured once the volume has been extracted kGraphAfter
    // times: capturing and instantiating costs about as much as four graph
    // launches save, so a volume extracted only a few times runs plain
    const bool indexed = ix != nullptr;
    const uint64_t before = v->extractions - (phase == Phase::kEmit ? 1 : 0);   // extractions before this one
    const bool graph = v->use_graph && !(v->flags & ISO_DEBUG) && !v->profiling && before >= kGraphAfter;
    if (phase != Phase::kEmit) v->extractions++;
    if (graph && ensure_graph(v, phase, indexed) != ISO_OK) v->use_graph = false;   // plain launches
    const int gk = graph_kind(phase, indexed);
    if (graph && v->gexec[gk]) {
        CK(cudaGraphLaunch(v->gexec[gk], v->stream));
    } else {
        rc = enqueue_pipeline(v, v->stream, phase, v->profiling, indexed);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(v->stream));
    v->upload_pending = false;                   // the decode waited for it
    if (phase != Phase::kCount) {
        v->split_emit = phase == Phase::kEmit;
        collect_stage_times(v);
    }
    if (phase != Phase::kEmit) {
        v->last_n_active = v->host_ctl->n_active;
        v->last_n_new = v->host_ctl->n_new;
        v->last_n_cand = v->host_ctl->n_cand;
        v->last_slots = v->host_ctl->S;
    }
    v->last_tris = v->host_ctl->n_tri;
    v->last_vtx = indexed ? v->host_ctl->n_vtx : 0ull;
    return status_to_error(v, v->host_ctl->status);
}

// A surface whose active blocks do not fit in the cache, extracted in
// waves: consecutive ranges of z-layers of blocks whose active blocks,
// together with those of the next layer (the +z neighbours of the last
// layer's candidates), fit in the cache.  Each wave is one extraction
// restricted to its block-id window; the waves' triangles are appended in
// order, which is the single-pass order (ascending block id).
int run_waves(iso_volume *v, float iso, void *out, unsigned long long cap_tris, uint32_t format,
              unsigned long long *total, iso_stats *st, const Indexed *ix) {
    const Geom &g = v->g;
    const uint32_t slab = g.nbx * g.nby;
    std::vector<uint32_t> layer(g.nbz);
    {
        uint32_t *d_layers = nullptr;
        int rc = dalloc(v, &d_layers, g.nbz);
        if (rc) return rc;
        bool ok = cudaMemsetAsync(d_layers, 0, (size_t)g.nbz * 4, v->stream) == cudaSuccess;
        if (ok) {
            launch_count_layers(v->hull, g, iso, d_layers, v->stream);
            ok = cudaMemcpyAsync(layer.data(), d_layers, (size_t)g.nbz * 4, cudaMemcpyDeviceToHost, v->stream) ==
                     cudaSuccess &&
                 cudaStreamSynchronize(v->stream) == cudaSuccess;
        }
        dfree_on(d_layers, v->stream);
        if (!ok) {
            (void)cudaGetLastError();
            return ISO_ERR_CUDA;
        }
    }
    auto at = [&](uint32_t z) -> uint64_t { return z < g.nbz ? layer[z] : 0; };
    std::vector<std::pair<uint32_t, uint32_t>> waves;   // candidate layers [z0, z1)
    for (uint32_t z = 0; z < g.nbz;) {
        if (at(z) + at(z + 1) > v->cap) return ISO_ERR_BUDGET;   // not even one layer fits
        uint64_t acc = at(z);
        uint32_t z1 = z + 1;
        while (z1 < g.nbz && acc + at(z1) + at(z1 + 1) <= v->cap) acc += at(z1++);
        waves.emplace_back(z, z1);
        z = z1;
    }
    // bytes a triangle (soup) or a vertex (indexed) takes in `out`
    const size_t vbytes = ix ? (format == kVertexPacked ? 8 : 16) : (format == kVertexPacked ? 24 : 48);
    unsigned long long tot = 0, vtot = 0;
    uint64_t n_active = 0, n_new = 0, n_cand = 0, n_occ = 0;
    for (uint32_t z = 0; z < g.nbz; z++) n_active += layer[z];
    for (const auto &wz : waves) {
        const Window w{wz.first * slab, std::min(g.nb, wz.second * slab), std::min(g.nb, (wz.second + 1) * slab)};
        const unsigned long long room = cap_tris > tot ? cap_tris - tot : 0ull;
        int rc;
        if (ix) {
            // this wave's vertices follow the earlier waves' and its indices count them
            const unsigned long long vroom = ix->vert_cap > vtot ? ix->vert_cap - vtot : 0ull;
            const Indexed wx{(ix->idx && room) ? ix->idx + 3 * tot : nullptr, vroom, ix->vtx_base + vtot};
            void *wout = (out && vroom) ? static_cast<char *>(out) + vtot * vbytes : nullptr;
            rc = run(v, iso, wout, wx.idx ? room : 0ull, Phase::kAll, format, 0u, &w, &wx);
        } else {
            void *wout = (out && room) ? static_cast<char *>(out) + tot * vbytes : nullptr;
            rc = run(v, iso, wout, room, Phase::kAll, format, 0u, &w);
        }
        if (rc) return rc;
        const Ctl &c = *v->host_ctl;
        tot += c.n_tri;
        vtot += ix ? c.n_vtx : 0ull;
        n_new += c.n_new;
        n_cand += c.n_cand;
        n_occ += c.n_occ;
    }
    *total = tot;
    v->last_tris = tot;
    v->last_vtx = vtot;
    if (st) {
        fill_stats(*v->host_ctl, st, 0);
        st->num_triangles = tot;
        st->n_active = (uint32_t)std::min<uint64_t>(n_active, 0xFFFFFFFFu);
        st->n_new = (uint32_t)std::min<uint64_t>(n_new, 0xFFFFFFFFu);
        st->n_candidates = (uint32_t)std::min<uint64_t>(n_cand, 0xFFFFFFFFu);
        st->n_occupied = (uint32_t)std::min<uint64_t>(n_occ, 0xFFFFFFFFu);
        st->waves = (uint32_t)waves.size();
        st->num_vertices = vtot;
    }
    return ISO_OK;
}

// One extraction into a caller buffer: a single pass, or waves when the
// surface's active blocks exceed the cache.  *total receives T.
int extract_to(iso_volume *v, float iso, void *out, unsigned long long cap_tris, uint32_t format, uint32_t flags,
               iso_stats *stats, unsigned long long *total, const Indexed *ix = nullptr) {
    int rc = run(v, iso, out, cap_tris, Phase::kAll, format, flags, nullptr, ix);
    if (rc == ISO_ERR_BUDGET && !(flags & kParamAllBlocks))
        return run_waves(v, iso, out, cap_tris, format, total, stats, ix);
    *total = v->host_ctl->n_tri;
    if (stats) {
        fill_stats(*v->host_ctl, stats, 0);
        stats->num_vertices = ix ? v->host_ctl->n_vtx : 0ull;
    }
    return rc;
}

// built once per process (a function-local static: thread-safe initialisation,
// so volumes may be loaded from several threads)
bool build_tables_once(McTables *t) {
    struct Built {
        bool ok;
        McTables tables;
    };
    static const Built built = [] {
        Built b{};
        b.ok = build_mc_tables(&b.tables) && b.tables.max_tri <= kMaxTriPerCell;
        return b;
    }();
    if (!built.ok) return false;
    *t = built.tables;
    return true;
}

}  // namespace

extern "C" {

int iso_set_shape(iso_volume *v, const iso_launch_shape *shape) {
    if (!v || !shape) return ISO_ERR_INVALID_ARG;
    Plan w{};
    const int rc = shape_to_want(shape, &w);
    if (rc) return rc;
    DeviceGuard dg(v->device);
    CK(cudaStreamSynchronize(v->stream));
    v->want = w;
    v->plan = launch_plan(&v->want, v->device, v->g.nb, v->cap, 1, true, v->g.rate, v->seg != nullptr);
    for (int k = 0; k < 4; k++) {            // the captured passes hold the old launch shape
        if (v->gexec[k]) cudaGraphExecDestroy(v->gexec[k]);
        if (v->graph[k]) cudaGraphDestroy(v->graph[k]);
        v->gexec[k] = nullptr;
        v->graph[k] = nullptr;
    }
    CK(cudaGetLastError());
    return ISO_OK;
}

int iso_get_shape(const iso_volume *v, iso_launch_shape *shape) {
    if (!v || !shape) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    *shape = shape_of(v->want, v->device, true, v->g.rate, v->seg != nullptr);
    return ISO_OK;
}

int iso_set_allocator(iso_alloc_fn alloc, iso_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return ISO_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    g_hook.alloc = alloc;
    g_hook.free = free_fn;
    g_hook.ctx = alloc ? ctx : nullptr;
    return ISO_OK;
}

int iso_release_cached_memory(int device) {
    if (device < 0 || device >= kMaxPoolDevices) return ISO_ERR_INVALID_ARG;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_pool_mutex);
        pool = g_pool[device];
    }
    if (!pool) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(device);
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
        (void)cudaGetLastError();
        return ISO_ERR_CUDA;
    }
    // and the pinned host mirrors and upload streams kept for later loads
    std::vector<void *> pinned;
    std::vector<cudaStream_t> streams;
    {
        std::lock_guard<std::mutex> lock(g_reuse_mutex);
        pinned.swap(g_pinned_free);
        for (size_t i = g_streams_free.size(); i-- > 0;)
            if (g_streams_free[i].first == device) {
                streams.push_back(g_streams_free[i].second);
                g_streams_free.erase(g_streams_free.begin() + (long)i);
            }
    }
    for (void *p : pinned) cudaFreeHost(p);
    for (cudaStream_t st : streams) cudaStreamDestroy(st);
    (void)cudaGetLastError();
    return ISO_OK;
}

const char *iso_error_string(int status) {
    switch (status) {
        case ISO_ERR_CORRUPT: return "block ranges are not ranges (NaN, or min > max)";
        case ISO_ERR_BOUNDS: return "a device index failed its bounds check (checked build)";
        case ISO_OK: return "ok";
        case ISO_ERR_INVALID_ARG: return "invalid argument";
        case ISO_ERR_OOM: return "out of memory";
        case ISO_ERR_BUDGET: return "active blocks exceed the cache budget";
        case ISO_ERR_CUDA: return "CUDA runtime error";
        case ISO_ERR_TIMEOUT: return "device-side wait timed out";
        case ISO_ERR_CAPACITY: return "output buffer too small";
        case ISO_PENDING: return "request not finished yet";
        default: return "unknown status";
    }
}

int iso_mc_case_table(uint8_t *num_tri, uint8_t *tri_edges) {
    if (!num_tri || !tri_edges) return ISO_ERR_INVALID_ARG;
    McTables t;
    if (!build_tables_once(&t)) return ISO_ERR_INVALID_ARG;
    std::memcpy(num_tri, t.num_tri, 256);
    std::memcpy(tri_edges, t.tri_edges, 256 * 16);
    return ISO_OK;
}

int iso_load_volume(iso_volume **out, const void *compressed, size_t compressed_bytes, uint32_t nx, uint32_t ny,
                    uint32_t nz, uint32_t rate_bits, const float *block_min, const float *block_max,
                    const iso_options *opt) {
    NvtxRange nvtx("iso_load_volume");
    if (!out || !compressed || !block_min || !block_max) return ISO_ERR_INVALID_ARG;
    *out = nullptr;
    Geom g;
    int rc = geometry(nx, ny, nz, rate_bits, &g);
    if (rc) return rc;
    if (compressed_bytes != (size_t)g.nb * g.rate * 8) return ISO_ERR_INVALID_ARG;
    iso_options o{};
    if (opt) o = *opt;
    double frac = o.initial_cache_fraction > 0 ? o.initial_cache_fraction : 0.1;

    iso_volume *v = new (std::nothrow) iso_volume();
    if (!v) return ISO_ERR_OOM;
    if (cudaGetDevice(&v->device) != cudaSuccess) { (void)cudaGetLastError(); delete v; return ISO_ERR_CUDA; }
    v->stream = (cudaStream_t)o.stream;
    v->g = g;
    v->flags = o.flags;
    uint64_t cap = g.nb;
    if (o.cache_budget_bytes) cap = std::min<uint64_t>(cap, o.cache_budget_bytes / 256);
    if (cap == 0) { delete v; return ISO_ERR_BUDGET; }
    v->cap = (uint32_t)cap;
    uint32_t s0 = (uint32_t)std::min<double>((double)cap, std::ceil(frac * g.nb));
    s0 = std::max<uint32_t>(s0, 1);

#define TRY(x)                              \
    do {                                    \
        rc = (x);                           \
        if (rc) { free_volume(v); return rc; } \
    } while (0)

    DevState &s = v->s;
    const size_t words = (size_t)g.nb * g.rate;
    const uint32_t nwords = (g.nb + 31) / 32;
    // descriptors for the smallest tile of each scan (any plan may run)
    v->n_cull_desc = (g.nb + kMinCullTile - 1) / kMinCullTile;
    v->n_lru_desc = (v->cap + kScanTile - 1) / kScanTile;
    const uint32_t n_mc_desc = (v->cap + kMinMcScanTile - 1) / kMinMcScanTile;   // candidates <= cap
    const bool on_device = (o.flags & ISO_INPUT_ON_DEVICE) != 0;
    TRY(dalloc(v, &v->bits, words));
    if (!on_device) {                 // staging for host ranges (freed once the hulls exist)
        TRY(dalloc(v, &v->bmin, g.nb));
        TRY(dalloc(v, &v->bmax, g.nb));
    }
    TRY(dalloc(v, &v->hull, g.nb));
    TRY(dalloc(v, &v->hull8, g.nb));
    const bool segments = (o.flags & ISO_SEGMENT_CULL) ||
                          (!(o.flags & ISO_NO_SEGMENT_CULL) && (uint64_t)g.nb >= kSegmentCullMinBlocks);
    if (segments) TRY(dalloc(v, &v->seg, (g.nb + kSegBlocks - 1) / kSegBlocks));
    TRY(dalloc(v, &v->tables, 256 + 256 * 16));
    TRY(dalloc(v, &s.mactive, nwords));
    s.list_cap = std::min<uint32_t>(g.nb, v->cap);
    if (v->flags & ISO_DEBUG) TRY(dalloc(v, &s.iactive, s.list_cap));
    TRY(dalloc(v, &s.inew, s.list_cap));
    TRY(dalloc(v, &s.icand, s.list_cap));
    TRY(dalloc(v, &s.islot, g.nb));
    TRY(dalloc(v, &s.slast, v->cap));
    TRY(dalloc(v, &s.sblock, v->cap));
    TRY(dalloc(v, &s.lbuf[0], v->cap));
    TRY(dalloc(v, &s.lbuf[1], v->cap));
    TRY(dalloc(v, &s.newslot, v->cap));
    TRY(dalloc(v, &s.slots, (size_t)v->cap * 64));
    TRY(dalloc(v, &s.desc_cull, v->n_cull_desc));
    TRY(dalloc(v, &s.desc_cand, v->n_cull_desc));
    TRY(dalloc(v, &s.desc_lru_a, v->n_lru_desc));
    TRY(dalloc(v, &s.desc_lru_b, v->n_lru_desc));
    // triangle offsets, then occupied counts, then vertex offsets (indexed meshes)
    TRY(dalloc(v, &s.desc_mc, 3 * (size_t)n_mc_desc));
    s.desc_occ = s.desc_mc + n_mc_desc;
    s.desc_vtx = s.desc_occ + n_mc_desc;
    TRY(dalloc(v, &s.ctl, 1));
    TRY(dalloc(v, &s.counts, v->cap));
    TRY(dalloc(v, &s.offsets, v->cap));
    TRY(dalloc(v, &s.iocc, s.list_cap));
    // the count pass keeps each candidate's cases for the emit pass when they
    // take at most 8 GB (else emit classifies again); debug volumes always
    if ((v->flags & ISO_DEBUG) || (uint64_t)s.list_cap * 64 <= (8ull << 30)) {
        TRY(dalloc(v, &s.cases, (size_t)s.list_cap * 64));
        s.case_cap = s.list_cap;
    }
    {
        char *block = static_cast<char *>(pinned_take());
        if (!block) {
            free_volume(v);
            return ISO_ERR_OOM;
        }
        v->host_ctl = reinterpret_cast<Ctl *>(block);
        v->host_params = reinterpret_cast<Params *>(block + kParamsOffset);
    }
    v->use_graph = !(o.flags & ISO_NO_GRAPH);
    s.bits = v->bits;
    s.hull = v->hull;
    s.hull8 = v->hull8;
    s.seg = v->seg;
    s.tables = v->tables;

    McTables t;
    if (!build_tables_once(&t)) { free_volume(v); return ISO_ERR_CUDA; }
    uint8_t table_bytes[256 + 256 * 16];
    std::memcpy(table_bytes, t.num_tri, 256);
    std::memcpy(table_bytes + 256, t.tri_edges, 256 * 16);

    const cudaMemcpyKind kind = (o.flags & ISO_INPUT_ON_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaStream_t st = v->stream;
#define TRYC(x)                                                            \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) { (void)cudaGetLastError(); free_volume(v); \
            return e_ == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA; } \
    } while (0)
    if (!on_device) {
        TRYC(cudaMemcpyAsync(v->bmin, block_min, (size_t)g.nb * 4, kind, st));
        TRYC(cudaMemcpyAsync(v->bmax, block_max, (size_t)g.nb * 4, kind, st));
    }
    // the bitstream after the ranges (which the hulls need first); an
    // asynchronous upload is queued last, once the load's own work is done,
    // so that no copy of the load waits behind it on the copy engine
    const bool async_bits = (o.flags & ISO_ASYNC_UPLOAD) && !on_device;
    if (!async_bits) TRYC(cudaMemcpyAsync(v->bits, compressed, words * 8, kind, st));

    TRYC(cudaMemcpyAsync(v->tables, table_bytes, sizeof(table_bytes), cudaMemcpyHostToDevice, st));
    TRYC(cudaMemsetAsync(s.islot, 0xFF, (size_t)g.nb * 4, st));
    TRYC(cudaMemsetAsync(s.sblock, 0xFF, (size_t)v->cap * 4, st));
    TRYC(cudaMemsetAsync(s.slast, 0, (size_t)v->cap * 4, st));
    TRYC(cudaMemsetAsync(s.mactive, 0, (size_t)nwords * 4, st));
    TRYC(cudaMemsetAsync(s.desc_mc, 0, (size_t)n_mc_desc * 24, st));
    // index lists start as valid ids, so that even a pass cut short by a
    // device-side timeout only ever indexes inside the volume and the cache
    if (s.iactive) TRYC(cudaMemsetAsync(s.iactive, 0, (size_t)s.list_cap * 4, st));
    TRYC(cudaMemsetAsync(s.inew, 0, (size_t)s.list_cap * 4, st));
    TRYC(cudaMemsetAsync(s.icand, 0, (size_t)s.list_cap * 4, st));
    TRYC(cudaMemsetAsync(s.newslot, 0, (size_t)v->cap * 4, st));
    TRYC(cudaMemsetAsync(s.lbuf[0], 0, (size_t)v->cap * 4, st));
    TRYC(cudaMemsetAsync(s.lbuf[1], 0, (size_t)v->cap * 4, st));
    Ctl c0{};
    c0.S = s0;
    c0.cap = v->cap;
    *v->host_ctl = c0;
    TRYC(cudaMemcpyAsync(s.ctl, v->host_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    // the ranges are needed only for the hulls (device inputs are read in place)
    launch_hull(on_device ? block_min : v->bmin, on_device ? block_max : v->bmax, v->hull, v->hull8, v->seg, g,
                &s.ctl->status, st);
    TRYC(cudaGetLastError());
    dfree_on(v->bmin, st);
    dfree_on(v->bmax, st);
    v->bmin = v->bmax = nullptr;
    TRYC(cudaMemcpyAsync(v->host_ctl, s.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    if (async_bits) {
        // Nothing waits here: the range check's verdict is read by the first
        // call on the volume (check_load), and the bitstream goes on a stream
        // of its own after the load's work on `st` (so no copy of the load
        // queues behind it); the first extraction's decode waits for it.
        cudaEvent_t queued = nullptr;
        TRYC(stream_take(v->device, &v->upload_stream));
        TRYC(cudaEventCreateWithFlags(&v->uploaded, cudaEventDisableTiming));
        TRYC(cudaEventCreateWithFlags(&queued, cudaEventDisableTiming));
        const cudaError_t e1 = cudaEventRecord(queued, st);
        const cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(v->upload_stream, queued, 0) : e1;
        cudaEventDestroy(queued);
        TRYC(e2);
        TRYC(cudaMemcpyAsync(v->bits, compressed, words * 8, kind, v->upload_stream));
        TRYC(cudaEventRecord(v->uploaded, v->upload_stream));
        v->upload_pending = true;
        v->check_pending = true;
    } else {
        TRYC(cudaStreamSynchronize(st));
        if (v->host_ctl->status & kStatusCorrupt) {   // ranges that are not ranges: nothing to cull with
            free_volume(v);
            return ISO_ERR_CORRUPT;
        }
    }
    // single-volume defaults from a sweep of every tile variant and CTA count
    // on the 512^3 benchmark: 4096-count scan tiles at one CTA per SM (the
    // other kernels' defaults were already best; 128-block decode CTAs, with
    // the list append in its own kernel, beat 256-block CTAs that append
    // after decoding: 91.0 + 8.5 against 103.8 us per surface)
    v->want = Plan{};
    v->want.scan_tile = 4096;
    v->want.mc_scan = 1;
    v->plan = launch_plan(&v->want, v->device, g.nb, v->cap, 1, true, g.rate, v->seg != nullptr);
    TRYC(cudaGetLastError());
    *out = v;
    return ISO_OK;
#undef TRY
#undef TRYC
}

int iso_extract_into(iso_volume *v, float isovalue, float *d_vertices, uint64_t capacity_triangles,
                     iso_stats *stats) {
    if (!v || !std::isfinite(isovalue) || (!d_vertices && capacity_triangles) || misaligned(d_vertices, 16))
        return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    unsigned long long total = 0;
    const int rc = extract_to(v, isovalue, d_vertices, capacity_triangles, kVertexFloat4, 0u, stats, &total);
    if (rc) return rc;
    return total > capacity_triangles ? ISO_ERR_CAPACITY : ISO_OK;
}

int iso_extract_all_blocks_into(iso_volume *v, float isovalue, float *d_vertices, uint64_t capacity_triangles,
                     iso_stats *stats) {
    if (!v || !std::isfinite(isovalue) || (!d_vertices && capacity_triangles) || misaligned(d_vertices, 16))
        return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    unsigned long long total = 0;
    const int rc = extract_to(v, isovalue, d_vertices, capacity_triangles, kVertexFloat4, kParamAllBlocks, stats, &total);
    if (rc) return rc;
    return total > capacity_triangles ? ISO_ERR_CAPACITY : ISO_OK;
}

int iso_extract_indexed_into(iso_volume *v, float isovalue, int vertex_format, void *d_vertices,
                             uint64_t capacity_vertices, uint32_t *d_indices, uint64_t capacity_triangles,
                             iso_stats *stats) {
    if (!v || !std::isfinite(isovalue) || (!d_vertices && capacity_vertices) || (!d_indices && capacity_triangles) ||
        (vertex_format != ISO_VERTEX_FLOAT4 && vertex_format != ISO_VERTEX_PACKED) ||
        misaligned(d_vertices, vertex_format == ISO_VERTEX_FLOAT4 ? 16 : 8) || misaligned(d_indices, 4))
        return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    unsigned long long total = 0;
    const Indexed ix{d_indices, capacity_vertices, 0ull};
    const uint32_t format = vertex_format == ISO_VERTEX_PACKED ? kVertexPacked : kVertexFloat4;
    iso_stats local{};
    iso_stats *st = stats ? stats : &local;
    const int rc = extract_to(v, isovalue, d_vertices, capacity_triangles, format, 0u, st, &total, &ix);
    if (rc) return rc;
    // indices are uint32
    if (st->num_vertices > 0xFFFFFFFFull) return ISO_ERR_CAPACITY;
    return (total > capacity_triangles || st->num_vertices > capacity_vertices) ? ISO_ERR_CAPACITY : ISO_OK;
}

int iso_decode_volume(const uint64_t *d_bits, uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate_bits,
                      float *d_field, void *stream) {
    if (!d_bits || !d_field) return ISO_ERR_INVALID_ARG;
    Geom g;
    int rc = geometry(nx, ny, nz, rate_bits, &g);
    if (rc) return rc;
    launch_decode_volume(d_bits, g, d_field, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return ISO_OK;
}

int iso_extract_packed_into(iso_volume *v, float isovalue, uint32_t *d_vertices, uint64_t capacity_triangles,
                     iso_stats *stats) {
    if (!v || !std::isfinite(isovalue) || (!d_vertices && capacity_triangles) || misaligned(d_vertices, 8))
        return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    unsigned long long total = 0;
    const int rc = extract_to(v, isovalue, d_vertices, capacity_triangles, kVertexPacked, 0u, stats, &total);
    if (rc) return rc;
    return total > capacity_triangles ? ISO_ERR_CAPACITY : ISO_OK;
}

int iso_extract(iso_volume *v, float isovalue, iso_mesh *out) {
    if (!v || !out || !std::isfinite(isovalue)) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    std::memset(out, 0, sizeof(*out));
    // the stages up to the scan; the mesh is then allocated at its exact size
    // and the emission runs alone
    int rc = run(v, isovalue, nullptr, 0, Phase::kCount);
    float4 *buf = nullptr;
    uint32_t reruns = 0;
    unsigned long long guess = 0;
    if (rc == ISO_ERR_BUDGET) {           // too many active blocks for the cache: waves
        // first guess: the last surface's size plus a margin; with no history,
        // 2 per block up to 2^24 (a larger surface runs the waves again)
        guess = v->last_tris ? v->last_tris + v->last_tris / 4 + 4096
                             : std::min<unsigned long long>(2ull * v->g.nb + 4096, 1ull << 24);
        {
            const int arc = dalloc(v, &buf, guess * 3);
            if (arc) return arc;
        }
        unsigned long long total = 0;
        rc = run_waves(v, isovalue, buf, guess, kVertexFloat4, &total, &out->stats, nullptr);
        if (rc == ISO_OK && total > guess) {   // the waves again into a buffer of the right size
            dfree_on(buf, v->stream);
            buf = nullptr;
            const int arc = dalloc(v, &buf, std::max(total, 1ull) * 3);
            if (arc) return arc;
            guess = std::max(total, 1ull);
            rc = run_waves(v, isovalue, buf, guess, kVertexFloat4, &total, &out->stats, nullptr);
            out->stats.reruns = 1;
        }
        if (rc) {
            dfree_on(buf, v->stream);
            cudaStreamSynchronize(v->stream);
            return rc;
        }
        out->d_vertices = reinterpret_cast<float *>(buf);
        out->num_triangles = total;
        out->capacity_triangles = guess;
        return ISO_OK;
    }
    if (rc == ISO_OK) {
        guess = std::max(v->host_ctl->n_tri, 1ull);
        const int arc = dalloc(v, &buf, guess * 3);
        if (arc) return arc;
        rc = run(v, isovalue, buf, guess, Phase::kEmit);
    }
    if (rc) {
        dfree_on(buf, v->stream);
        cudaStreamSynchronize(v->stream);
        fill_stats(*v->host_ctl, &out->stats, reruns);
        return rc;
    }
    out->d_vertices = reinterpret_cast<float *>(buf);
    out->num_triangles = v->host_ctl->n_tri;
    out->capacity_triangles = guess;
    fill_stats(*v->host_ctl, &out->stats, reruns);
    return ISO_OK;
}

int iso_mesh_release(iso_volume *v, iso_mesh *m) {
    if (!m) return ISO_ERR_INVALID_ARG;
    if (!m->d_vertices) return ISO_OK;
    if (!v) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    dfree_on(m->d_vertices, v->stream);
    CK(cudaGetLastError());
    m->d_vertices = nullptr;
    m->num_triangles = 0;
    m->capacity_triangles = 0;
    return ISO_OK;
}

void iso_release(iso_volume *v) { free_volume(v); }

int iso_set_stream(iso_volume *v, void *stream) {
    if (!v) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    CK(cudaStreamSynchronize(v->stream));
    v->stream = (cudaStream_t)stream;
    return ISO_OK;
}

int iso_set_profiling(iso_volume *v, int on) {
    if (!v) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    if (on && !v->ev[0]) {
        for (cudaEvent_t &e : v->ev) CK(cudaEventCreate(&e));
    }
    v->profiling = on != 0;
    return ISO_OK;
}

int iso_stage_times(iso_volume *v, float *ms, int n) {
    if (!v || !ms || n < ISO_NUM_STAGES) return ISO_ERR_INVALID_ARG;
    for (int k = 0; k < ISO_NUM_STAGES; k++) ms[k] = v->profiling ? v->stage_ms[k] : 0.0f;
    return ISO_OK;
}

int iso_set_test_fault(iso_volume *v, uint32_t what) {
    if (!v || (what & ~ISO_TEST_WITHHOLD_PREFIX)) return ISO_ERR_INVALID_ARG;
    v->test_flags = (what & ISO_TEST_WITHHOLD_PREFIX) ? (uint32_t)kParamTestWithhold : 0u;
    return ISO_OK;
}

int iso_cache_reset(iso_volume *v) {
    if (!v) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    launch_reset_cache(v->s, v->stream);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(v->stream));
    return ISO_OK;
}

int iso_encode_field(const float *d_field, uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate_bits,
                     uint64_t *d_bits, float *d_bmin, float *d_bmax, void *stream) {
    if (!d_field || !d_bits || !d_bmin || !d_bmax) return ISO_ERR_INVALID_ARG;
    Geom g;
    int rc = geometry(nx, ny, nz, rate_bits, &g);
    if (rc) return rc;
    launch_encode(d_field, g, d_bits, d_bmin, d_bmax, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return ISO_OK;
}

int iso_decode_blocks(const uint64_t *d_bits, uint32_t rate_bits, const uint32_t *d_ids, uint64_t n, float *d_out,
                      void *stream) {
    if (rate_bits < 1 || rate_bits > 32) return ISO_ERR_INVALID_ARG;
    if (n == 0) return ISO_OK;
    if (!d_bits || !d_ids || !d_out) return ISO_ERR_INVALID_ARG;
    launch_decode_list(d_bits, rate_bits, d_ids, n, d_out, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return ISO_OK;
}

int iso_debug_get(iso_volume *v, int which, void *host_dst, size_t bytes, uint64_t *count) {
    if (!v || !count) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    const bool dbg = (v->flags & ISO_DEBUG) != 0;
    const void *src = nullptr;
    uint64_t n = 0;
    size_t elem = 0;
    switch (which) {
        case ISO_DBG_ACTIVE_IDS:
            if (!dbg) return ISO_ERR_INVALID_ARG;
            src = v->s.iactive; n = std::min<uint64_t>(v->last_n_active, v->s.list_cap); elem = 4; break;
        case ISO_DBG_NEW_IDS: src = v->s.inew; n = std::min<uint64_t>(v->last_n_new, v->s.list_cap); elem = 4; break;
        case ISO_DBG_SLOT_OF_BLOCK: src = v->s.islot; n = v->g.nb; elem = 4; break;
        case ISO_DBG_BLOCK_OF_SLOT: src = v->s.sblock; n = v->last_slots; elem = 4; break;
        case ISO_DBG_SLOT_LAST_USE: src = v->s.slast; n = v->last_slots; elem = 4; break;
        case ISO_DBG_ACTIVE_MASK: src = v->s.mactive; n = (v->g.nb + 31) / 32; elem = 4; break;
        case ISO_DBG_CELL_CASES:
            if (!dbg || !v->s.cases) return ISO_ERR_INVALID_ARG;
            src = v->s.cases; n = 64ull * std::min<uint64_t>(v->last_n_cand, v->s.list_cap); elem = 1; break;
        case ISO_DBG_BLOCK_TRIS: src = v->s.counts; n = v->last_n_cand; elem = 4; break;
        case ISO_DBG_BLOCK_OFFSETS: src = v->s.offsets; n = v->last_n_cand; elem = 8; break;
        case ISO_DBG_CANDIDATES: src = v->s.icand; n = std::min<uint64_t>(v->last_n_cand, v->s.list_cap); elem = 4; break;
        case ISO_DBG_EDGE_IDS:
            if (!dbg) return ISO_ERR_INVALID_ARG;
            src = v->s.dbg_edges;
            n = std::min<unsigned long long>(3ull * v->last_tris, v->dbg_edges_cap);
            elem = 8;
            break;
        default: return ISO_ERR_INVALID_ARG;
    }
    *count = n;
    if (n == 0) return ISO_OK;
    if (!host_dst || bytes < n * elem) return ISO_ERR_CAPACITY;
    CK(cudaStreamSynchronize(v->stream));
    CK(cudaMemcpy(host_dst, src, n * elem, cudaMemcpyDeviceToHost));
    return ISO_OK;
}

int iso_debug_read_blocks(iso_volume *v, const uint32_t *ids, uint64_t n, float *host_out) {
    if (!v || (n && (!ids || !host_out))) return ISO_ERR_INVALID_ARG;
    if (n == 0) return ISO_OK;
    DeviceGuard dg(v->device);
    for (uint64_t i = 0; i < n; i++)
        if (ids[i] >= v->g.nb) return ISO_ERR_INVALID_ARG;
    uint32_t *d_ids = nullptr;
    float *d_out = nullptr;
    int32_t *d_missing = nullptr;
    int rc = dalloc(v, &d_ids, n);
    if (!rc) rc = dalloc(v, &d_out, n * 64);
    if (!rc) rc = dalloc(v, &d_missing, 1);
    if (!rc && cudaStreamSynchronize(v->stream) != cudaSuccess) rc = ISO_ERR_CUDA;
    int32_t missing = 0;
    if (!rc && (cudaMemcpy(d_ids, ids, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(d_missing, 0, 4) != cudaSuccess))
        rc = ISO_ERR_CUDA;
    if (!rc) {
        launch_gather_slots(v->s.slots, v->s.islot, d_ids, n, d_out, d_missing, v->stream);
        if (cudaStreamSynchronize(v->stream) != cudaSuccess ||
            cudaMemcpy(host_out, d_out, n * 64 * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&missing, d_missing, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = ISO_ERR_CUDA;
    }
    (void)cudaGetLastError();
    dfree_on(d_ids, v->stream);
    dfree_on(d_out, v->stream);
    dfree_on(d_missing, v->stream);
    cudaStreamSynchronize(v->stream);
    if (rc) return rc;
    return missing ? ISO_ERR_INVALID_ARG : ISO_OK;
}

}  // extern "C"
