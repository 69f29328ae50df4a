// Serving (C ABI in include/bcmc.h): isovalue requests on one resident
// volume, answered in ticks.  A tick takes up to kMaxServe queued requests:
//   front (once per tick)
//     serve_prep     clear the tick's counters and descriptors
//     serve_cull     one pass over the block ranges for all the tick's
//                    isovalues (Section 4.1): the union of their active sets
//                    and each request's own candidate list
//     cache update   Algorithm 1 and the decode (Section 4.2) on the union
//   then, one request per step, in arrival order
//     count, scan    Sections 4.3-4.4 over the request's candidates (the
//                    request is a "view" of the volume: own control block,
//                    candidates, counts and offsets; shared cache)
//     readback       its triangle count; the host allocates its mesh
//     emit           Section 4.5
// A request finishes as soon as its own emission is done: later requests
// of the tick never delay it, while the cull, cache update and decode are
// paid once for the whole tick.  Decoded blocks and all metadata stay
// resident between ticks.  The union is what the tick's cache update
// protects, so every slot a request of the running tick reads stays pinned
// until the tick ends.  If the union does not fit in the cache budget, the
// tick's requests go back to the queue and the next ticks take half as
// many (down to one).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "bcmc.h"
#include "common.cuh"
#include "kernels.cuh"
#include "launch.cuh"
#include "tile_scan.cuh"
#include "volume.cuh"

namespace bcmc {

constexpr int kMaxServe = 8;          // requests per tick

struct ServeArgs {
    VolEntry base;                    // the volume; base.s.ctl carries the tick's union
    uint32_t k;                       // requests in this tick
    float iso[kMaxServe];
    Ctl *ctl[kMaxServe];              // per-request control blocks
    uint32_t *icand[kMaxServe];       // per-request candidate lists
    unsigned long long *desc_cand[kMaxServe];
    unsigned long long *desc_mc[kMaxServe];
    unsigned long long *desc_occ[kMaxServe];
    uint32_t cand_cap;                // room of each candidate list
};

__global__ void __launch_bounds__(kThreads) serve_prep_kernel(ServeArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const DevState &s = a.base.s;
    for (uint32_t i = tid; i < a.base.n_cull_desc; i += stride) s.desc_cull[i] = 0;
    for (uint32_t i = tid; i < a.base.n_lru_desc; i += stride) {
        s.desc_lru_a[i] = 0;
        s.desc_lru_b[i] = 0;
    }
    for (uint32_t j = 0; j < a.k; j++) {
        for (uint32_t i = tid; i < a.base.n_cull_desc; i += stride) a.desc_cand[j][i] = 0;
        const uint32_t n_mc = a.ctl[j]->mc_tiles;      // descriptors the request slot's last scan used
        for (uint32_t i = tid; i < n_mc; i += stride) {
            a.desc_mc[j][i] = 0;
            a.desc_occ[j][i] = 0;
        }
    }
    if (tid == 0) {
        Ctl *c = s.ctl;
        c->epoch += 1;
        c->n_active = 0;
        c->n_new = 0;
        c->n_cand = 0;
        c->n_assign = 0;
        c->status = 0;
        c->n_occ = 0;
        c->n_tri = 0;
        for (int i = 0; i < kNumLaunchCounters; i++) c->ctr[i] = 0;
    }
    if (tid < a.k) {
        Ctl *c = a.ctl[tid];
        c->cap = s.ctl->cap;                            // the shared cache's slot capacity
        c->n_cand = 0;
        c->n_tri = 0;
        c->n_occ = 0;
        c->status = 0;
        c->params.iso = a.iso[tid];
        for (int i = 0; i < kNumLaunchCounters; i++) c->ctr[i] = 0;   // the request's own launches
    }
}

// The cull of Section 4.1 for all the tick's isovalues in one pass over
// the block ranges: a block is in the union when it is active for any of
// them; it is a candidate of request j when it is active for iso_j and
// its +group range contains iso_j (as in the single-volume cull).  Hits
// of the union are stamped with the epoch; the union's active and new
// lists feed the cache update.
struct ServeCullSmem {
    TileScan<kRounds> ts;                     // union: active << 16 | new
    TileScan<kRounds> tc[kMaxServe];          // candidates of each request
    uint32_t bal[2 + kMaxServe][kRounds][8];  // union active, new, candidates
};

__global__ void __launch_bounds__(kThreads) serve_cull_kernel(ServeArgs a) {
    __shared__ ServeCullSmem sm;
    __shared__ uint32_t slot_x;
    constexpr uint32_t kTile = kRounds * kThreads;
    const DevState &s = a.base.s;
    const Geom &g = a.base.g;
    Ctl *c = s.ctl;
    const uint32_t k = a.k;
    const uint32_t ntiles = ceil_div(g.nb, kTile);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t epoch = c->epoch;
    while (true) {
        const uint32_t tile = next_item(&c->ctr[kLcCull], &slot_x);
        if (tile >= ntiles) break;
        float2 h[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; r++) {
            const uint32_t b = tile * kTile + r * kThreads + threadIdx.x;
            h[r] = b < g.nb ? __ldg(s.hull + b) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < kRounds; r++) {               // unrolled: h[] stays in registers
            const uint32_t b = tile * kTile + r * kThreads + threadIdx.x;
            uint32_t am = 0, cm = 0;
            if (b < g.nb) {
#pragma unroll
                for (int j = 0; j < kMaxServe; j++)
                    if (j < (int)k && h[r].x < a.iso[j] && a.iso[j] <= h[r].y) am |= 1u << j;
            }
            bool nw = false;
            if (am) {
                const float2 h8 = __ldg(s.hull8 + b);
#pragma unroll
                for (int j = 0; j < kMaxServe; j++)
                    if (((am >> j) & 1u) && h8.x < a.iso[j] && a.iso[j] <= h8.y) cm |= 1u << j;
                const int32_t sl = s.islot[b];
                if (sl >= 0) s.slast[sl] = epoch;
                else nw = true;
            }
            const uint32_t ab = __ballot_sync(0xffffffffu, am != 0);
            const uint32_t nbits = __ballot_sync(0xffffffffu, nw);
            if (lane == 0) {
                sm.bal[0][r][warp] = ab;
                sm.bal[1][r][warp] = nbits;
                sm.ts.cnt[r][warp] = ((uint32_t)__popc(ab) << 16) | (uint32_t)__popc(nbits);
                const uint32_t first = tile * kTile + r * kThreads + warp * 32;
                if (first < g.nb) s.mactive[first >> 5] = ab;
            }
            for (uint32_t j = 0; j < k; j++) {                 // k is uniform
                const uint32_t cb = __ballot_sync(0xffffffffu, (cm >> j) & 1u);
                if (lane == 0) {
                    sm.bal[2 + j][r][warp] = cb;
                    sm.tc[j].cnt[r][warp] = (uint32_t)__popc(cb);
                }
            }
        }
        __syncthreads();
        // scan q = 0 is the union, q = j + 1 request j; warp w takes q = w, w + 8
        for (uint32_t q = warp; q <= k; q += kThreads / 32) {
            if (q == 0) {
                const uint32_t tot = scan_tile_counts(sm.ts);
                const unsigned long long agg = ((unsigned long long)(tot >> 16) << 31) | (tot & 0xFFFFu);
                const unsigned long long excl = lookback_exclusive(s.desc_cull, tile, agg, &c->status, kStatusTimeout);
                if (lane == 0) {
                    sm.ts.excl = excl;
                    if (tile == ntiles - 1) {
                        const unsigned long long incl = excl + agg;
                        c->n_active = (uint32_t)(incl >> 31);
                        c->n_new = (uint32_t)(incl & 0x7FFFFFFFu);
                    }
                }
            } else {
                const uint32_t j = q - 1;
                const uint32_t tot = scan_tile_counts(sm.tc[j]);
                const unsigned long long excl = lookback_exclusive(a.desc_cand[j], tile, tot, &a.ctl[j]->status,
                                                                   kStatusTimeout);
                if (lane == 0) {
                    sm.tc[j].excl = excl;
                    if (tile == ntiles - 1) a.ctl[j]->n_cand = (uint32_t)(excl + tot);
                }
            }
        }
        __syncthreads();
        const uint32_t act_base = (uint32_t)(sm.ts.excl >> 31), new_base = (uint32_t)(sm.ts.excl & 0x7FFFFFFFu);
#pragma unroll 2
        for (int r = 0; r < kRounds; r++) {
            const uint32_t b = tile * kTile + r * kThreads + threadIdx.x;
            const uint32_t ab = sm.bal[0][r][warp], nbits = sm.bal[1][r][warp];
            const uint32_t off = sm.ts.cnt[r][warp];
            const uint32_t ai = act_base + (off >> 16) + __popc(ab & lt);
            const uint32_t ni = new_base + (off & 0xFFFFu) + __popc(nbits & lt);
            if (s.iactive && ((ab >> lane) & 1u) && ai < s.list_cap) s.iactive[ai] = b;
            if (((nbits >> lane) & 1u) && ni < s.list_cap) s.inew[ni] = b;
            for (uint32_t j = 0; j < k; j++) {
                // a list longer than its room means more active blocks than
                // cache slots: the cache update fails the tick, nothing reads it
                const uint32_t cb = sm.bal[2 + j][r][warp];
                const uint32_t at = (uint32_t)sm.tc[j].excl + sm.tc[j].cnt[r][warp] + __popc(cb & lt);
                if (((cb >> lane) & 1u) && at < a.cand_cap) a.icand[j][at] = b;
            }
        }
        __syncthreads();
    }
}

// the union's failures (budget, a timeout) are every request's
__global__ void serve_status_kernel(ServeArgs a) {
    const uint32_t j = threadIdx.x;
    if (j < a.k) a.ctl[j]->status |= a.base.s.ctl->status & (kStatusBudget | kStatusAnyTimeout);
}

}  // namespace bcmc

using namespace bcmc;
using namespace bcmc_host;

namespace {

struct Request {
    uint64_t ticket;
    float iso;
};

struct Done {
    int status;
    iso_mesh mesh;
};

struct Slot {                           // device state of one request position in a tick
    Ctl *ctl = nullptr;
    uint32_t *icand = nullptr, *counts = nullptr;
    unsigned long long *offsets = nullptr, *desc_cand = nullptr, *desc_mc = nullptr, *desc_occ = nullptr;
    uint32_t *iocc = nullptr;
};

}  // namespace

struct iso_server {
    iso_volume *v = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t max_batch = 4, limit = 4;  // requests per tick; current limit after budget failures
    uint64_t vertex_budget = 0;         // 0 = none
    uint32_t format = kVertexFloat4;    // vertex format of the meshes
    uint64_t tri_bytes = 48;            // their bytes per triangle
    uint32_t cand_cap = 0;              // room of each request's candidate list
    uint64_t held_bytes = 0;            // finished meshes not yet taken
    Slot slots[kMaxServe];
    VolEntry views[kMaxServe];          // per-request views of the volume (by value into each launch)
    Ctl *h_ctl = nullptr;               // pinned: one request's control block, read back
    Params *h_params = nullptr;         // pinned: one request's output
    Plan view_plan{};                   // launches over one view
    uint64_t next_ticket = 1;
    std::deque<Request> queue;
    std::vector<Request> tick;          // the running tick's requests
    uint32_t tick_next = 0;             // next of them to emit
    Ctl tick_union{};                   // the tick's union figures (for the stats)
    std::map<uint64_t, Done> done;
};

namespace {

ServeArgs serve_args(const iso_server *sv, const std::vector<Request> &reqs) {
    ServeArgs a{};
    const iso_volume *v = sv->v;
    a.base = VolEntry{v->s, v->g, v->n_cull_desc, v->n_lru_desc};
    a.k = (uint32_t)reqs.size();
    for (uint32_t j = 0; j < a.k; j++) {
        a.iso[j] = reqs[j].iso;
        a.ctl[j] = sv->slots[j].ctl;
        a.icand[j] = sv->slots[j].icand;
        a.desc_cand[j] = sv->slots[j].desc_cand;
        a.desc_mc[j] = sv->slots[j].desc_mc;
        a.desc_occ[j] = sv->slots[j].desc_occ;
    }
    a.cand_cap = sv->cand_cap;
    return a;
}

void free_server(iso_server *sv) {
    if (!sv) return;
    DeviceGuard dg(sv->device);
    for (auto &kv : sv->done)
        if (kv.second.mesh.d_vertices) dfree_on(kv.second.mesh.d_vertices, sv->stream);
    for (Slot &s : sv->slots) {
        void *p[] = {s.ctl, s.icand, s.counts, s.offsets, s.desc_cand, s.desc_mc, s.iocc};
        for (void *x : p) dfree_on(x, sv->stream);
    }
    cudaStreamSynchronize(sv->stream);
    (void)cudaGetLastError();
    if (sv->h_ctl) cudaFreeHost(sv->h_ctl);
    if (sv->h_params) cudaFreeHost(sv->h_params);
    delete sv;
}

void finish(iso_server *sv, const Request &r, int status, const Ctl *c, float *buf) {
    Done d{};
    d.status = status;
    d.mesh.d_vertices = buf;
    if (c) {
        d.mesh.num_triangles = buf ? c->n_tri : 0;
        d.mesh.capacity_triangles = buf ? c->n_tri : 0;
        Ctl s = sv->tick_union;         // the tick's cache figures, the request's own surface figures
        s.n_tri = c->n_tri;
        s.n_occ = c->n_occ;
        s.n_cand = c->n_cand;
        fill_stats(s, &d.mesh.stats, 0);
    }
    if (buf) sv->held_bytes += sv->tri_bytes * c->n_tri;
    sv->done[r.ticket] = d;
}

void requeue_rest(iso_server *sv) {     // the tick's unfinished requests, in order, to the queue's front
    for (uint32_t j = (uint32_t)sv->tick.size(); j-- > sv->tick_next;) sv->queue.push_front(sv->tick[j]);
    sv->tick.clear();
    sv->tick_next = 0;
}

// The front of a tick over the queue's first requests.  Returns ISO_OK
// (with sv->tick set, or the requests re-queued or finished), or a CUDA
// error.
int start_tick(iso_server *sv, uint32_t *completed) {
    iso_volume *v = sv->v;
    cudaStream_t st = sv->stream;
    const uint32_t k = std::min<uint32_t>(sv->limit, (uint32_t)sv->queue.size());
    sv->tick.clear();
    for (uint32_t j = 0; j < k; j++) {
        sv->tick.push_back(sv->queue.front());
        sv->queue.pop_front();
    }
    sv->tick_next = 0;
    const ServeArgs a = serve_args(sv, sv->tick);
    const Launch single{nullptr, 1u, single_counters(v), a.base};
    serve_prep_kernel<<<v->plan.prep, kThreads, 0, st>>>(a);
    serve_cull_kernel<<<v->plan.cull, kThreads, 0, st>>>(a);
    launch_cache_update(single, v->plan, st);
    serve_status_kernel<<<1, kMaxServe, 0, st>>>(a);
    ISO_CK(cudaMemcpyAsync(v->host_ctl, v->s.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    ISO_CK(cudaGetLastError());
    ISO_CK(cudaStreamSynchronize(st));
    const Ctl uni = *v->host_ctl;
    sv->tick_union = uni;
    v->last_n_active = uni.n_active;
    v->last_n_new = uni.n_new;
    v->last_n_cand = 0;
    v->last_slots = uni.S;
    if (uni.status & kStatusAnyTimeout) {
        status_to_error(v, uni.status);   // empties the cache
        for (const Request &r : sv->tick) finish(sv, r, ISO_ERR_TIMEOUT, nullptr, nullptr);
        *completed += k;
        sv->tick.clear();
        return ISO_OK;
    }
    if (uni.status & kStatusBudget) {
        if (k > 1) {                      // too many decodes at once: fewer requests per tick
            requeue_rest(sv);
            sv->limit = std::max(1u, k / 2);
            return ISO_OK;
        }
        finish(sv, sv->tick[0], ISO_ERR_BUDGET, nullptr, nullptr);
        *completed += 1;
        sv->tick.clear();
        return ISO_OK;
    }
    sv->limit = std::min(sv->max_batch, sv->limit * 2);
    return ISO_OK;
}

// Count, scan and emit the tick's next request.  A mesh that does not fit
// the vertex budget sends it and the rest of the tick back to the queue.
int emit_next(iso_server *sv, uint32_t *completed) {
    cudaStream_t st = sv->stream;
    const uint32_t j = sv->tick_next;
    const Request r = sv->tick[j];
    const VolEntry &view = sv->views[j];
    Ctl *dctl = sv->slots[j].ctl;
    uint32_t *ctr = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(dctl) + offsetof(Ctl, ctr));
    const Launch L{nullptr, 1u, ctr, view};
    launch_mc_count(L, false, sv->view_plan, st);
    launch_mc_scan(L, sv->view_plan, st);
    ISO_CK(cudaMemcpyAsync(sv->h_ctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    ISO_CK(cudaGetLastError());
    ISO_CK(cudaStreamSynchronize(st));
    const Ctl c = *sv->h_ctl;
    if (c.status & (kStatusAnyTimeout | kStatusBounds)) {
        finish(sv, r, (c.status & kStatusBounds) ? ISO_ERR_BOUNDS : ISO_ERR_TIMEOUT, &c, nullptr);
        sv->tick_next++;
        *completed += 1;
        return ISO_OK;
    }
    const uint64_t bytes = sv->tri_bytes * c.n_tri;
    if (sv->vertex_budget && sv->held_bytes > 0 && sv->held_bytes + bytes > sv->vertex_budget) {
        requeue_rest(sv);                 // wait until the held meshes are taken
        return ISO_OK;
    }
    float *buf = nullptr;
    if (c.n_tri) {
        const int rc = dalloc_on(&buf, (size_t)c.n_tri * (sv->tri_bytes / 4), sv->device, st);
        if (rc) {
            finish(sv, r, rc, &c, nullptr);
            sv->tick_next++;
            *completed += 1;
            return ISO_OK;
        }
    }
    *sv->h_params = Params{r.iso, sv->format, 0u, 0u, 0u, 0u, c.n_tri, (unsigned long long)(uintptr_t)buf};
    ISO_CK(cudaMemcpyAsync(&dctl->params, sv->h_params, sizeof(Params), cudaMemcpyHostToDevice, st));
    launch_mc_emit(L, false, sv->view_plan, st);
    ISO_CK(cudaGetLastError());
    ISO_CK(cudaStreamSynchronize(st));
    finish(sv, r, ISO_OK, &c, buf);
    sv->tick_next++;
    *completed += 1;
    return ISO_OK;
}

}  // namespace

extern "C" {

int iso_server_create(iso_server **out, iso_volume *v, const iso_server_options *opt) {
    if (!out || !v || (v->flags & ISO_DEBUG)) return ISO_ERR_INVALID_ARG;
    *out = nullptr;
    iso_server_options o{};
    if (opt) o = *opt;
    if (o.max_batch > (uint32_t)kMaxServe) return ISO_ERR_INVALID_ARG;
    if (o.vertex_format != ISO_VERTEX_FLOAT4 && o.vertex_format != ISO_VERTEX_PACKED) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    ISO_CK_RC(finish_upload(v));             // the server reads the bitstream on its own stream
    iso_server *sv = new (std::nothrow) iso_server();
    if (!sv) return ISO_ERR_OOM;
    sv->v = v;
    sv->device = v->device;
    sv->stream = (cudaStream_t)o.stream;
    sv->max_batch = o.max_batch ? o.max_batch : 4;
    sv->limit = sv->max_batch;
    sv->vertex_budget = o.vertex_budget_bytes;
    sv->format = o.vertex_format == ISO_VERTEX_PACKED ? kVertexPacked : kVertexFloat4;
    sv->tri_bytes = o.vertex_format == ISO_VERTEX_PACKED ? 24 : 48;
    const size_t cand = std::min<size_t>(v->cap, v->g.nb);       // candidates of an admitted tick <= cap
    sv->cand_cap = (uint32_t)cand;
    const size_t n_mc_desc = (cand + kMinMcScanTile - 1) / kMinMcScanTile;
    int rc = ISO_OK;
#define TRY(x)                                   \
    do {                                         \
        rc = (x);                                \
        if (rc) { free_server(sv); return rc; }  \
    } while (0)
    for (uint32_t j = 0; j < sv->max_batch; j++) {
        Slot &s = sv->slots[j];
        TRY(dalloc_on(&s.ctl, 1, sv->device, sv->stream));
        TRY(cudaMemsetAsync(s.ctl, 0, sizeof(Ctl), sv->stream) == cudaSuccess ? ISO_OK   // no field undefined
                                                                              : ((void)cudaGetLastError(), ISO_ERR_CUDA));
        TRY(dalloc_on(&s.icand, cand, sv->device, sv->stream));
        TRY(dalloc_on(&s.counts, cand, sv->device, sv->stream));
        TRY(dalloc_on(&s.offsets, cand, sv->device, sv->stream));
        TRY(dalloc_on(&s.desc_cand, v->n_cull_desc, sv->device, sv->stream));
        TRY(dalloc_on(&s.desc_mc, 2 * n_mc_desc, sv->device, sv->stream));
        s.desc_occ = s.desc_mc + n_mc_desc;
        TRY(dalloc_on(&s.iocc, cand, sv->device, sv->stream));
        DevState d = v->s;                // the volume's cache and geometry, the request's own lists
        d.ctl = s.ctl;
        d.icand = s.icand;
        d.counts = s.counts;
        d.offsets = s.offsets;
        d.desc_cand = s.desc_cand;
        d.desc_mc = s.desc_mc;
        d.desc_occ = s.desc_occ;
        d.iocc = s.iocc;
        d.cases = nullptr;                // a request's emit classifies (no per-request case store)
        sv->views[j] = VolEntry{d, v->g, v->n_cull_desc, v->n_lru_desc};
    }
    if (cudaMallocHost((void **)&sv->h_ctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&sv->h_params, sizeof(Params)) != cudaSuccess) {
        (void)cudaGetLastError();
        free_server(sv);
        return ISO_ERR_OOM;
    }
    cudaStream_t st = sv->stream;
    bool ok = cudaStreamSynchronize(v->stream) == cudaSuccess;
    for (uint32_t j = 0; ok && j < sv->max_batch; j++) {
        ok = cudaMemsetAsync(sv->slots[j].ctl, 0, sizeof(Ctl), st) == cudaSuccess &&
             cudaMemsetAsync(sv->slots[j].icand, 0, cand * 4, st) == cudaSuccess &&
             cudaMemsetAsync(sv->slots[j].desc_mc, 0, n_mc_desc * 16, st) == cudaSuccess;
    }
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_server(sv);
        return ISO_ERR_CUDA;
    }
#undef TRY
    sv->view_plan = launch_plan(nullptr, sv->device, v->g.nb, cand, 1, true, v->g.rate);
    *out = sv;
    return ISO_OK;
}

int iso_server_submit(iso_server *sv, float isovalue, uint64_t *ticket) {
    if (!sv || !ticket || !std::isfinite(isovalue)) return ISO_ERR_INVALID_ARG;
    *ticket = sv->next_ticket++;
    sv->queue.push_back(Request{*ticket, isovalue});
    return ISO_OK;
}

int iso_server_step(iso_server *sv, uint32_t *completed) {
    NvtxRange nvtx("iso_server_step");
    if (!sv) return ISO_ERR_INVALID_ARG;
    uint32_t n = 0;
    if (completed) *completed = 0;
    DeviceGuard dg(sv->device);
    int rc = ISO_OK;
    if (sv->tick_next >= sv->tick.size()) {       // the last tick is done: start one
        sv->tick.clear();
        sv->tick_next = 0;
        if (sv->queue.empty()) return ISO_OK;
        rc = start_tick(sv, &n);
    }
    if (rc == ISO_OK && sv->tick_next < sv->tick.size()) rc = emit_next(sv, &n);
    if (completed) *completed = n;
    return rc;
}

int iso_server_queued(const iso_server *sv, uint32_t *queued) {
    if (!sv || !queued) return ISO_ERR_INVALID_ARG;
    *queued = (uint32_t)(sv->queue.size() + (sv->tick.size() - std::min<size_t>(sv->tick_next, sv->tick.size())));
    return ISO_OK;
}

int iso_server_take(iso_server *sv, uint64_t ticket, iso_mesh *out) {
    if (!sv || !out) return ISO_ERR_INVALID_ARG;
    auto it = sv->done.find(ticket);
    if (it == sv->done.end()) {
        if (ticket == 0 || ticket >= sv->next_ticket) return ISO_ERR_INVALID_ARG;
        for (const Request &r : sv->queue)
            if (r.ticket == ticket) return ISO_PENDING;
        for (uint32_t j = sv->tick_next; j < sv->tick.size(); j++)
            if (sv->tick[j].ticket == ticket) return ISO_PENDING;
        return ISO_ERR_INVALID_ARG;       // already taken
    }
    *out = it->second.mesh;
    const int status = it->second.status;
    if (out->d_vertices) sv->held_bytes -= sv->tri_bytes * out->num_triangles;
    sv->done.erase(it);
    return status;
}

int iso_server_wait(iso_server *sv, uint64_t ticket, uint32_t timeout_ms, iso_mesh *out) {
    if (!sv || !out) return ISO_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const int rc = iso_server_take(sv, ticket, out);
        if (rc != ISO_PENDING) return rc;
        const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0);
        if ((uint64_t)ms.count() >= timeout_ms) return ISO_PENDING;
        uint32_t n = 0;
        const int src = iso_server_step(sv, &n);
        if (src != ISO_OK) return src;
    }
}

void iso_server_destroy(iso_server *sv) { free_server(sv); }

}  // extern "C"
