// Serving (C ABI in include/bcmc.h): isovalue requests on one resident
// volume, answered in ticks of up to max_batch requests (at most kMaxServe).
//   front of a tick (stream `front`)
//     serve_prep     clear the tick's counters and descriptors
//     serve_cull     one pass over the block ranges for all the tick's
//                    isovalues (Section 4.1): the union of their active sets
//                    and each request's own candidate list (a tick of one
//                    request without pins runs the single-volume range test)
//     cache update   Algorithm 1 and the decode (Section 4.2) on the union
//     front tail     the union's failures become every request's; each
//                    request gets its region of the stored-cases buffer
//   back of a tick (the server's stream, queued behind the front's event
//   without a host round trip)
//     count, scan    Sections 4.3-4.4 over all the tick's requests in one
//                    launch each: a request is a "view" of the volume (own
//                    control block, candidates, counts and offsets; shared
//                    cache), the views are the entries of a batch launch
//                    (they find no work if the union failed); on a volume
//                    with segment ranges one launch per request (per_view)
//     readback       every request's control block and the union's at once;
//                    the host checks the union (budget, timeouts) and
//                    allocates the meshes
//     emit           Section 4.5: at light load (a round of one or two
//                    requests, none waiting) or on a volume with segment
//                    ranges one launch per request, each finishing as its
//                    own emission ends; otherwise one launch for the round.
//                    Requests whose meshes would pass the vertex budget wait
//                    in the tick (their counts and lists kept) and emit in a
//                    later round once meshes are taken.
// Ticks are pipelined under load: once a tick's emission is queued and at
// least two requests wait, they are admitted as the next tick and its front
// runs on the second stream (at a lower priority) while the running tick
// emits; a lone waiting request is admitted when the running tick is done,
// and so is every tick on a volume with segment ranges or while the running
// tick's union takes more than half the cache (room_to_pin).  An overlapping
// front also counts the running tick's isovalues as active (pins), so the
// cache update it makes never evicts a block the running tick reads.  The
// two ticks use alternate halves of the request positions, so the new front
// never writes lists the running back reads.  Decoded blocks and all
// metadata stay resident between ticks.  If a union does not fit in the
// cache budget, its requests go back to the queue (an unpinned tick then
// takes half as many requests, down to one; a pinned one is simply retried
// without pins).
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
    uint32_t k_pin;                   // isovalues of the running tick: active, no candidates
    float iso[2 * kMaxServe];         // the requests' isovalues, then the pinned ones
    uint32_t *back_ctr;               // the work counters of this tick's batched launches
    Ctl *ctl[kMaxServe];              // per-request control blocks
    uint32_t *icand[kMaxServe];       // per-request candidate lists
    unsigned long long *desc_cand[kMaxServe];
    unsigned long long *desc_mc[kMaxServe];
    unsigned long long *desc_occ[kMaxServe];
    uint32_t cand_cap;                // room of each candidate list
    VolEntry *views;                  // the tick's views in device memory (the back's launch table)
    uint32_t single_cull;             // one request, no pins: the single-volume range test runs instead
    uint8_t *cases;                   // the server's stored-cases buffer (or null)
    unsigned long long case_cap;      // its room, in candidates (64 bytes each)
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
        if (a.single_cull) {                            // the single-volume range test reads them
            c->params.iso = a.iso[0];
            c->params.flags = 0;
        }
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
    if (tid < kNumLaunchCounters) a.back_ctr[tid] = 0;
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
// them or for a pinned isovalue (the running tick's); it is a candidate of
// request j when it is active for iso_j and its +group range contains
// iso_j (as in the single-volume cull).  Hits of the union are stamped with
// the epoch; the union's active and new lists feed the cache update.
template <int kR>
struct ServeCullSmem {
    TileScan<kR> ts;                          // union: active << 16 | new
    TileScan<kR> tc[kMaxServe];               // candidates of each request
    uint32_t bal[2 + kMaxServe][kR][8];       // union active, new, candidates
};

// kT: a power of two at least k + k_pin (the isovalue loop is unrolled to it);
// kSeg: the volume has segment ranges (and, like the single-volume range
// test, then takes tiles of 8192 blocks: 32 rounds)
template <int kT, bool kSeg>
__global__ void __launch_bounds__(kThreads) serve_cull_kernel(ServeArgs a) {
    constexpr int kR = kSeg ? 32 : kRounds;
    __shared__ ServeCullSmem<kR> sm;
    __shared__ uint32_t slot_x;
    constexpr uint32_t kTile = kR * kThreads;
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
        // groups of kHalf rounds; in each, every load (3x3x3 hull, +group
        // hull, slot) is issued before any of it is used, so a tile waits
        // for one memory round trip per group rather than one per round
        constexpr int kHalf = kR >= 16 ? 8 : kR / 2;
#pragma unroll
        for (int half = 0; half < kR / kHalf; half++) {
            // with segment ranges, a block's reads are skipped when its
            // segment's range holds none of the tick's isovalues
            uint32_t live = ~0u;
            if (kSeg) {
                float2 sh[kHalf];
#pragma unroll
                for (int i = 0; i < kHalf; i++) {
                    const uint32_t b = tile * kTile + (half * kHalf + i) * kThreads + threadIdx.x;
                    sh[i] = b < g.nb ? __ldg(s.seg + b / kSegBlocks) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < kHalf; i++) {
                    bool any = false;
#pragma unroll
                    for (int j = 0; j < kT; j++)
                        if (j < (int)(k + a.k_pin)) any = any || (sh[i].x < a.iso[j] && a.iso[j] <= sh[i].y);
                    if (!any) live &= ~(1u << i);
                }
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
                uint32_t am = 0, cm = 0;
                bool pin = false;
                if (b < g.nb) {
#pragma unroll
                    for (int j = 0; j < kT; j++) {
                        const bool in = h[i].x < a.iso[j] && a.iso[j] <= h[i].y;
                        if (j < (int)k) {
                            if (in) {
                                am |= 1u << j;
                                if (h8[i].x < a.iso[j] && a.iso[j] <= h8[i].y) cm |= 1u << j;
                            }
                        } else if (j < (int)(k + a.k_pin)) {
                            pin = pin || in;
                        }
                    }
                }
                const bool act = am != 0 || pin;
                const bool nw = act && sl[i] < 0;
                if (act && sl[i] >= 0) s.slast[sl[i]] = epoch;   // a hit: the slot's age resets
                const uint32_t ab = __ballot_sync(0xffffffffu, act);
                const uint32_t nbits = __ballot_sync(0xffffffffu, nw);
                if (lane == 0) {
                    sm.bal[0][r][warp] = ab;
                    sm.bal[1][r][warp] = nbits;
                    sm.ts.cnt[r][warp] = ((uint32_t)__popc(ab) << 16) | (uint32_t)__popc(nbits);
                    const uint32_t first = tile * kTile + r * kThreads + warp * 32;
                    if (first < g.nb) s.mactive[first >> 5] = ab;
                }
#pragma unroll
                for (int j = 0; j < (kT < kMaxServe ? kT : kMaxServe); j++) {
                    if (j >= (int)k) break;                         // k is uniform
                    const uint32_t cb = __ballot_sync(0xffffffffu, (cm >> j) & 1u);
                    if (lane == 0) {
                        sm.bal[2 + j][r][warp] = cb;
                        sm.tc[j].cnt[r][warp] = (uint32_t)__popc(cb);
                    }
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
        for (int r = 0; r < kR; r++) {
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

// The end of a tick's front (one thread: k <= 8).  The union's failures
// (budget, a timeout) become every request's, so the back finds no work;
// each request, in order, gets the next region of the stored-cases buffer
// while its candidates fit (a request without one has its cases
// classified again by the emission, which reads the same pointer).
__global__ void serve_front_tail_kernel(ServeArgs a) {
    if (threadIdx.x != 0) return;
    if (a.single_cull) a.ctl[0]->n_cand = a.base.s.ctl->n_cand;   // counted by the single-volume range test
    const uint32_t fail = a.base.s.ctl->status & (kStatusBudget | kStatusAnyTimeout);
    unsigned long long used = 0;
    for (uint32_t j = 0; j < a.k; j++) {
        Ctl *c = a.ctl[j];
        c->status |= fail;
        const unsigned long long n = c->n_cand;
        const bool fits = a.cases != nullptr && used + n <= a.case_cap;
        a.views[j].s.cases = fits ? a.cases + 64ull * used : nullptr;
        a.views[j].s.case_cap = fits ? n : 0ull;
        if (fits) used += n;
    }
}

// the tick's request control blocks, then the union's, for one readback
__global__ void serve_gather_kernel(ServeArgs a, Ctl *dst) {
    constexpr uint32_t kWords = sizeof(Ctl) / 4;
    for (uint32_t i = threadIdx.x; i < (a.k + 1) * kWords; i += blockDim.x) {
        const uint32_t j = i / kWords;
        const Ctl *src = j < a.k ? a.ctl[j] : a.base.s.ctl;
        reinterpret_cast<uint32_t *>(dst)[i] = reinterpret_cast<const uint32_t *>(src)[i % kWords];
    }
}

// Each request's output (mesh, capacity, format) into its control block; a
// request without a mesh in this emission round is skipped by it.
__global__ void serve_params_kernel(const VolEntry *__restrict__ views, const Params *__restrict__ p, uint32_t k) {
    const uint32_t j = threadIdx.x;
    if (j >= k) return;
    Ctl *c = views[j].s.ctl;
    c->params = p[j];
    c->status = p[j].out ? (c->status & ~(uint32_t)kStatusSkip) : (c->status | kStatusSkip);
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

struct Slot {                           // device state of one request position
    Ctl *ctl = nullptr;
    uint32_t *icand = nullptr, *counts = nullptr;
    unsigned long long *offsets = nullptr, *desc_cand = nullptr, *desc_mc = nullptr, *desc_occ = nullptr;
    uint32_t *iocc = nullptr;
};

enum Stage { kFront = 0, kCount = 1, kEmit = 2 };

struct Tick {                           // requests in flight on the GPU
    std::vector<Request> reqs;
    uint32_t parity = 0;                // which half of the request positions it uses
    bool pinned = false;                // its union also holds the previous tick's blocks
    Stage stage = kFront;
    bool checked = false;               // its union was checked (at the count readback)
    std::vector<float *> bufs;          // meshes (allocated round by round)
    std::vector<int> status;
    uint32_t emitted = 0;               // requests finished by earlier emission rounds
    uint32_t run_to = 0;                // the running round takes requests [emitted, run_to)
    ServeArgs args{};                   // its front's arguments (the back's gather reads them too)
};

constexpr uint64_t kMaxTickCaseBytes = 4ull << 30;   // stored cases of a tick, else emit classifies again

}  // namespace

struct iso_server {
    iso_volume *v = nullptr;
    int device = 0;
    cudaStream_t user = nullptr;        // the caller's stream (work before the server is ordered on it)
    cudaStream_t stream = nullptr;      // the backs: count, scan, emit (created here, high priority)
    cudaStream_t front = nullptr;       // the fronts: cull, cache update, decode (created here, low priority)
    uint32_t max_batch = 4, limit = 4;  // requests per tick; current limit after budget failures
    uint64_t vertex_budget = 0;         // 0 = none
    uint32_t format = kVertexFloat4;    // vertex format of the meshes
    uint64_t tri_bytes = 48;            // their bytes per triangle
    uint32_t cand_cap = 0;              // room of each request's candidate list
    uint64_t held_bytes = 0;            // finished meshes not yet taken
    Slot slots[2][kMaxServe];           // two halves: a tick's back and the next tick's front
    VolEntry views[2][kMaxServe];       // per-request views of the volume
    VolEntry *d_views[2] = {};          // the same in device memory (the back's launch tables)
    uint32_t *d_ctr[2] = {};            // work counters of each half's back launches
    Ctl *d_ctls[2] = {};                // control blocks gathered for one readback: k requests, then the union
    Params *d_params = nullptr;         // the requests' outputs, copied into their control blocks
    Ctl *h_ctls[2] = {};                // pinned mirrors of d_ctls
    Params *h_params = nullptr;
    uint8_t *cases = nullptr;           // stored cell cases of a tick's requests (count writes, emit reads)
    uint64_t case_cap = 0;              // its room in candidates
    bool blocked = false;               // the back waits for meshes to be taken (vertex budget)
    cudaEvent_t front_done[2] = {}, count_done = nullptr;
    cudaEvent_t emit_done[kMaxServe] = {};   // each request's emission in the running round
    Plan one_plan{}, back_plan{};       // launches over one view (kOne) or up to max_batch views
    uint64_t next_ticket = 1;
    std::deque<Request> queue;
    bool has_front = false, has_back = false;
    Tick front_tick, back_tick;         // a tick whose front runs, and one in its back
    uint32_t next_parity = 0;
    uint64_t ticks_finished = 0;        // backs completed (their requests finished or sent back)
    uint64_t rounds_finished = 0;       // emission rounds completed (every request of the round finished)
    std::map<uint64_t, Done> done;
};

namespace {

ServeArgs serve_args(const iso_server *sv, const Tick &t, const std::vector<Request> *pins) {
    ServeArgs a{};
    const iso_volume *v = sv->v;
    a.base = VolEntry{v->s, v->g, v->n_cull_desc, v->n_lru_desc};
    a.k = (uint32_t)t.reqs.size();
    const uint32_t p = t.parity;
    for (uint32_t j = 0; j < a.k; j++) {
        a.iso[j] = t.reqs[j].iso;
        a.ctl[j] = sv->slots[p][j].ctl;
        a.icand[j] = sv->slots[p][j].icand;
        a.desc_cand[j] = sv->slots[p][j].desc_cand;
        a.desc_mc[j] = sv->slots[p][j].desc_mc;
        a.desc_occ[j] = sv->slots[p][j].desc_occ;
    }
    a.k_pin = pins ? (uint32_t)pins->size() : 0u;
    for (uint32_t j = 0; j < a.k_pin; j++) a.iso[a.k + j] = (*pins)[j].iso;
    a.back_ctr = sv->d_ctr[p];
    a.cand_cap = sv->cand_cap;
    a.views = sv->d_views[p];
    a.cases = sv->cases;
    a.single_cull = (a.k == 1 && a.k_pin == 0) ? 1u : 0u;
    a.case_cap = sv->case_cap;
    return a;
}

void free_server(iso_server *sv) {
    if (!sv) return;
    DeviceGuard dg(sv->device);
    if (sv->front) cudaStreamSynchronize(sv->front);
    cudaStreamSynchronize(sv->stream);
    for (auto &kv : sv->done)
        if (kv.second.mesh.d_vertices) dfree_on(kv.second.mesh.d_vertices, sv->stream);
    if (sv->has_back)                     // a tick abandoned in flight
        for (float *b : sv->back_tick.bufs) dfree_on(b, sv->stream);
    for (auto &half : sv->slots)
        for (Slot &s : half) {
            void *p[] = {s.ctl, s.icand, s.counts, s.offsets, s.desc_cand, s.desc_mc, s.iocc};
            for (void *x : p) dfree_on(x, sv->stream);
        }
    void *q[] = {sv->d_views[0], sv->d_views[1], sv->d_ctr[0], sv->d_ctr[1], sv->d_ctls[0], sv->d_ctls[1],
                 sv->d_params, sv->cases};
    for (void *x : q) dfree_on(x, sv->stream);
    cudaStreamSynchronize(sv->stream);
    (void)cudaGetLastError();
    for (Ctl *h : {sv->h_ctls[0], sv->h_ctls[1]})
        if (h) cudaFreeHost(h);
    if (sv->h_params) cudaFreeHost(sv->h_params);
    for (cudaEvent_t e : {sv->front_done[0], sv->front_done[1], sv->count_done})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : sv->emit_done)
        if (e) cudaEventDestroy(e);
    if (sv->front) cudaStreamDestroy(sv->front);
    if (sv->stream) cudaStreamDestroy(sv->stream);
    (void)cudaGetLastError();
    delete sv;
}

void finish(iso_server *sv, const Request &r, int status, const Ctl *uni, const Ctl *c, float *buf) {
    Done d{};
    d.status = status;
    d.mesh.d_vertices = buf;
    if (c) {
        d.mesh.num_triangles = buf ? c->n_tri : 0;
        d.mesh.capacity_triangles = buf ? c->n_tri : 0;
        Ctl s = *uni;                   // the tick's cache figures, the request's own surface figures
        s.n_tri = c->n_tri;
        s.n_occ = c->n_occ;
        s.n_cand = c->n_cand;
        fill_stats(s, &d.mesh.stats, 0);
    }
    if (buf) sv->held_bytes += sv->tri_bytes * c->n_tri;
    sv->done[r.ticket] = d;
}

// requests back to the queue's front, in order
void requeue(iso_server *sv, const std::vector<Request> &reqs, size_t from) {
    for (size_t j = reqs.size(); j-- > from;) sv->queue.push_front(reqs[j]);
}

bool ready(cudaEvent_t e) {
    const cudaError_t r = cudaEventQuery(e);
    if (r == cudaErrorNotReady) return false;
    (void)cudaGetLastError();             // an error surfaces at the synchronisation that follows
    return true;
}

template <bool kSeg>
void launch_serve_cull(uint32_t kt, int ctas, const ServeArgs &a, cudaStream_t st) {
    if (kt <= 1) serve_cull_kernel<1, kSeg><<<ctas, kThreads, 0, st>>>(a);
    else if (kt <= 2) serve_cull_kernel<2, kSeg><<<ctas, kThreads, 0, st>>>(a);
    else if (kt <= 4) serve_cull_kernel<4, kSeg><<<ctas, kThreads, 0, st>>>(a);
    else if (kt <= 8) serve_cull_kernel<8, kSeg><<<ctas, kThreads, 0, st>>>(a);
    else serve_cull_kernel<16, kSeg><<<ctas, kThreads, 0, st>>>(a);
}

// Admit the queue's first requests as a tick and queue its front on the
// front stream (pins: the tick in its back, or null).
int launch_front(iso_server *sv, const std::vector<Request> *pins) {
    iso_volume *v = sv->v;
    Tick t;
    t.parity = sv->next_parity;
    t.pinned = pins && !pins->empty();
    const uint32_t k = std::min<uint32_t>(sv->limit, (uint32_t)sv->queue.size());
    for (uint32_t j = 0; j < k; j++) {
        t.reqs.push_back(sv->queue.front());
        sv->queue.pop_front();
    }
    const ServeArgs a = serve_args(sv, t, pins);
    const Launch single{nullptr, 1u, single_counters(v), a.base};
    cudaStream_t st = sv->front;
    serve_prep_kernel<<<v->plan.prep, kThreads, 0, st>>>(a);
    const uint32_t kt = a.k + a.k_pin;
    if (a.single_cull) {
        // one request and no pins: its active set is the union, so the
        // single-volume range test serves, writing the volume's lists and
        // the request's candidates (its counters in the volume's control
        // block, which the prep cleared)
        VolEntry view = a.base;
        view.s.icand = a.icand[0];
        view.s.desc_cand = a.desc_cand[0];
        launch_cull(Launch{nullptr, 1u, single_counters(v), view}, v->plan, st);
    } else if (v->seg) {
        launch_serve_cull<true>(kt, v->plan.cull, a, st);
    } else {
        launch_serve_cull<false>(kt, v->plan.cull, a, st);
    }
    launch_cache_update(single, v->plan, st);
    serve_front_tail_kernel<<<1, 32, 0, st>>>(a);
    cudaError_t e = cudaEventRecord(sv->front_done[t.parity], st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {               // the requests wait in the queue again
        (void)cudaGetLastError();
        requeue(sv, t.reqs, 0);
        return e == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA;
    }
    t.args = a;
    sv->front_tick = std::move(t);
    sv->has_front = true;
    sv->next_parity ^= 1u;
    return ISO_OK;
}

Launch back_launch(const iso_server *sv, const Tick &t) {
    const uint32_t k = (uint32_t)t.reqs.size();
    if (k == 1) return Launch{nullptr, 1u, sv->d_ctr[t.parity], sv->views[t.parity][0]};   // one view by value
    return Launch{sv->d_views[t.parity], k, sv->d_ctr[t.parity], VolEntry{}, sv->v->g.rate};
}

const Plan &back_plan(const iso_server *sv, const Tick &t) {
    return t.reqs.size() == 1 ? sv->one_plan : sv->back_plan;
}

// On a volume with segment ranges (the largest), a tick's count, scan and
// emission run one launch per request, each view by value with its own
// work counters and no stored cases: there a launch over one view is
// faster per view than one over the table (measured 3.8 against 5.0 ms of
// count per request of a 10240 x 7680 x 1536 volume), a launch's tail is
// negligible against its work, and stored cases gain nothing.
bool per_view(const iso_server *sv) { return sv->v->seg != nullptr; }

Launch view_launch(const iso_server *sv, const Tick &t, uint32_t j) {
    VolEntry view = sv->views[t.parity][j];
    view.s.cases = nullptr;
    view.s.case_cap = 0;
    uint32_t *ctr = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(view.s.ctl) + offsetof(Ctl, ctr));
    return Launch{nullptr, 1u, ctr, view};
}

// Queue the count and scan of the tick whose front was just queued (or is
// running) behind the front's event, then one readback of every request's
// control block and the union's.  Nothing waits on the host: the union is
// checked when the counts are back (a failed union leaves the back no work).
int queue_back(iso_server *sv) {
    cudaStream_t st = sv->stream;
    Tick t = std::move(sv->front_tick);
    sv->has_front = false;
    const uint32_t k = (uint32_t)t.reqs.size();
    auto failed = [&](cudaError_t e) {    // the requests wait in the queue again
        (void)cudaGetLastError();
        requeue(sv, t.reqs, 0);
        return e == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA;
    };
    cudaError_t e = cudaStreamWaitEvent(st, sv->front_done[t.parity], 0);
    if (e != cudaSuccess) return failed(e);
    if (per_view(sv)) {
        for (uint32_t j = 0; j < k; j++) {
            const Launch L = view_launch(sv, t, j);
            launch_mc_count(L, false, sv->one_plan, st);
            launch_mc_scan(L, sv->one_plan, st);
        }
    } else {
        const Launch L = back_launch(sv, t);
        const Plan &pl = back_plan(sv, t);
        launch_mc_count(L, false, pl, st);
        launch_mc_scan(L, pl, st);
    }
    serve_gather_kernel<<<1, 256, 0, st>>>(t.args, sv->d_ctls[t.parity]);
    e = cudaMemcpyAsync(sv->h_ctls[t.parity], sv->d_ctls[t.parity], (k + 1) * sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(sv->count_done, st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return failed(e);
    t.stage = kCount;
    sv->back_tick = std::move(t);
    sv->has_back = true;
    return ISO_OK;
}

// The tick's counts are back.  A failed union ends the tick (a timeout
// fails its requests; over the budget, its requests go back to the queue
// and an unpinned tick halves the tick size).  Otherwise start an emission
// round: allocate the meshes of the waiting requests, in order, while they
// fit the vertex budget (a mesh is always allowed when nothing is held),
// and queue one emission for them.  Returns kBlocked, with nothing queued,
// when the next mesh must wait for meshes to be taken.
constexpr int kBlocked = -1;
constexpr uint32_t kEachEmitMax = 2;   // light-load rounds of at most this many emit request by request

int start_emit(iso_server *sv, uint32_t *completed) {
    iso_volume *v = sv->v;
    cudaStream_t st = sv->stream;
    Tick &t = sv->back_tick;
    const uint32_t k = (uint32_t)t.reqs.size();
    const Ctl *c = sv->h_ctls[t.parity];
    if (!t.checked) {
        ISO_CK(cudaEventSynchronize(sv->count_done));
        const Ctl &uni = c[k];
        v->last_n_active = uni.n_active;
        v->last_n_new = uni.n_new;
        v->last_n_cand = 0;
        v->last_slots = uni.S;
        if (uni.status & (kStatusAnyTimeout | kStatusBudget)) {
            Tick done = std::move(sv->back_tick);   // not a finished back: a step goes on with the queue
            sv->has_back = false;
            if (uni.status & kStatusAnyTimeout) {
                status_to_error(v, uni.status);
                for (const Request &r : done.reqs) finish(sv, r, ISO_ERR_TIMEOUT, &uni, nullptr, nullptr);
                *completed += k;
            } else if (done.pinned || k > 1) {    // retry without the running tick's blocks, or with fewer requests
                requeue(sv, done.reqs, 0);
                if (!done.pinned) sv->limit = std::max(1u, k / 2);
            } else {
                finish(sv, done.reqs[0], ISO_ERR_BUDGET, &uni, nullptr, nullptr);
                *completed += 1;
            }
            return ISO_OK;
        }
        if (!t.pinned) sv->limit = std::min(sv->max_batch, sv->limit * 2);
        t.checked = true;
        t.bufs.assign(k, nullptr);
        t.status.assign(k, ISO_OK);
        t.emitted = 0;
        for (uint32_t j = 0; j < k; j++)
            if (c[j].status & (kStatusAnyTimeout | kStatusBounds))
                t.status[j] = (c[j].status & kStatusBounds) ? ISO_ERR_BOUNDS : ISO_ERR_TIMEOUT;
    }
    uint64_t held = sv->held_bytes;
    uint32_t j = t.emitted;
    for (; j < k; j++) {
        if (t.status[j] != ISO_OK) continue;  // fails without a mesh
        const uint64_t bytes = sv->tri_bytes * c[j].n_tri;
        if (sv->vertex_budget && held > 0 && held + bytes > sv->vertex_budget) break;
        if (c[j].n_tri && !t.bufs[j]) {   // (a round retried after an error keeps its meshes)
            const int rc = dalloc_on(&t.bufs[j], (size_t)c[j].n_tri * (sv->tri_bytes / 4), sv->device, st);
            if (rc) {
                t.status[j] = rc;
                continue;
            }
        }
        held += bytes;
    }
    if (j == t.emitted) {                     // the next mesh waits for meshes to be taken
        sv->blocked = true;
        return kBlocked;
    }
    sv->blocked = false;
    t.run_to = j;
    for (uint32_t i = 0; i < k; i++) {
        const bool out = i >= t.emitted && i < t.run_to && t.bufs[i];
        sv->h_params[i] = Params{t.reqs[i].iso, sv->format, 0u, 0u, 0u, 0u, out ? c[i].n_tri : 0ull,
                                 out ? (unsigned long long)(uintptr_t)t.bufs[i] : 0ull, 0ull, 0ull, 0ull};
    }
    ISO_CK(cudaMemcpyAsync(sv->d_params, sv->h_params, k * sizeof(Params), cudaMemcpyHostToDevice, st));
    serve_params_kernel<<<1, kMaxServe, 0, st>>>(sv->d_views[t.parity], sv->d_params, k);
    // At light load (a round of one or two requests and no request waiting):
    // one emission per request, its view by value, in order, so a request
    // finishes as soon as its own vertices are written.  Otherwise (a
    // backlog) one emission for all, whose single tail costs less than one
    // per request.  A view's stored cases are where the front's tail put
    // them (the same rule, on the host, from the same candidate counts).
    if (!per_view(sv) && (t.run_to - t.emitted > kEachEmitMax || !sv->queue.empty())) {
        launch_mc_emit(back_launch(sv, t), false, back_plan(sv, t), st);
        for (uint32_t i = t.emitted; i < t.run_to; i++) ISO_CK(cudaEventRecord(sv->emit_done[i], st));
        ISO_CK(cudaGetLastError());
        t.stage = kEmit;
        return ISO_OK;
    }
    uint64_t used = 0;
    for (uint32_t i = 0; i < k; i++) {
        VolEntry view = sv->views[t.parity][i];
        if (k > 1) {
            const uint64_t n = c[i].n_cand;
            const bool fits = sv->cases != nullptr && used + n <= sv->case_cap;
            view.s.cases = fits ? sv->cases + 64ull * used : nullptr;
            view.s.case_cap = fits ? n : 0ull;
            if (fits) used += n;
        }
        if (i < t.emitted || i >= t.run_to) continue;
        if (t.bufs[i]) {
            const Launch L = per_view(sv) ? view_launch(sv, t, i) : Launch{nullptr, 1u, sv->d_ctr[t.parity], view};
            launch_mc_emit(L, false, sv->one_plan, st);
        }
        ISO_CK(cudaEventRecord(sv->emit_done[i], st));
    }
    ISO_CK(cudaGetLastError());
    t.stage = kEmit;
    return ISO_OK;
}

// Requests of the running emission round whose emissions are done finish,
// in order (with `block`, waiting for the first of them).  The tick leaves
// the back once every request has; after a round, the next one waits for
// the budget.
int finish_round(iso_server *sv, bool block, uint32_t *completed) {
    Tick &t = sv->back_tick;
    const Ctl *c = sv->h_ctls[t.parity];
    const Ctl &uni = c[t.reqs.size()];
    while (t.emitted < t.run_to) {
        const uint32_t j = t.emitted;
        if (block) ISO_CK(cudaEventSynchronize(sv->emit_done[j]));
        else if (!ready(sv->emit_done[j])) break;
        block = false;
        finish(sv, t.reqs[j], t.status[j], &uni, &c[j], t.status[j] == ISO_OK ? t.bufs[j] : nullptr);
        if (t.status[j] != ISO_OK && t.bufs[j]) dfree_on(t.bufs[j], sv->stream);
        t.bufs[j] = nullptr;                  // the mesh is the finished request's now
        *completed += 1;
        t.emitted++;
    }
    if (t.emitted < t.run_to) return ISO_OK;  // the round goes on
    sv->rounds_finished++;
    if (t.emitted < t.reqs.size()) {
        t.stage = kCount;                     // counted, waiting for its next round
        return ISO_OK;
    }
    sv->has_back = false;
    sv->ticks_finished++;
    sv->back_tick = Tick{};
    return ISO_OK;
}

// A front may overlap the running tick (its isovalues pinned in the new
// union) only when that tick's union takes at most half the cache: a union
// with the pins is then likely to fit, while one that does not fit wastes
// the whole front (its cull reads the ranges for every pinned isovalue too)
// before going back to the queue.  Never on a volume with segment ranges:
// there a pinned front's union range test (two isovalues or more, few
// segments skipped) costs more than a one-request tick's single-volume one,
// and it shares the memory bandwidth with the running emission (measured:
// with overlap the served path sustained 13.9 against the plain path's
// 17.2 G triangles/s on a 10240 x 7680 x 1536 volume).
bool room_to_pin(const iso_server *sv) {
    if (per_view(sv)) return false;
    const Tick &t = sv->back_tick;
    return (uint64_t)sv->h_ctls[t.parity][t.reqs.size()].n_active * 2 <= sv->v->cap;
}

// One transition of the pipeline, the latest stage first: a finished
// emission completes its tick; returned counts start the emission; a
// finished front (with no tick in its back) starts the count; a free front
// admits the queue's next requests (pinned to the tick in its back, once
// that tick's emission is queued and at least two requests wait).
// Without `block` only transitions whose GPU work is done are taken;
// with it the first transition waits for its work.  Returns 1 if one was
// taken (or an error code as a negative number).
int advance(iso_server *sv, bool block, uint32_t *completed) {
    int rc = ISO_OK;
    if (sv->has_back && sv->back_tick.stage == kEmit) {
        if (!block && !ready(sv->emit_done[sv->back_tick.emitted])) goto admit;
        rc = finish_round(sv, block, completed);
        return rc ? -rc : 1;
    }
    if (sv->has_back && sv->back_tick.stage == kCount) {
        if (!block && !ready(sv->count_done)) goto admit;
        rc = start_emit(sv, completed);
        if (rc == kBlocked) return 0;              // nothing moves until meshes are taken
        return rc ? -rc : 1;
    }
    if (sv->has_front && !sv->has_back) {          // the back follows the front on the device
        rc = queue_back(sv);
        return rc ? -rc : 1;
    }
admit:
    // A front overlaps a back only when requests have piled up (at least two
    // wait), and only once the back's last kernel (the emission) is queued:
    // the front's persistent kernels, started earlier, would hold the SMs the
    // back's count or emission needs until they finish, and a lone request
    // gains nothing from overlapping (both halves keep the GPU busy) while
    // its front's memory traffic slows the running emission.
    if (!sv->has_front && !sv->queue.empty() &&
        (!sv->has_back || (sv->back_tick.stage == kEmit && sv->queue.size() >= 2 && room_to_pin(sv)))) {
        rc = launch_front(sv, sv->has_back ? &sv->back_tick.reqs : nullptr);
        return rc ? -rc : 1;
    }
    return 0;
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
    ISO_CK_RC(finish_upload(v));             // the server reads the bitstream on its own streams
    iso_server *sv = new (std::nothrow) iso_server();
    if (!sv) return ISO_ERR_OOM;
    sv->v = v;
    sv->device = v->device;
    sv->user = (cudaStream_t)o.stream;
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
    auto cuda_ok = [](cudaError_t e) { return e == cudaSuccess ? ISO_OK : ((void)cudaGetLastError(), ISO_ERR_CUDA); };
    // The backs (the latency of the requests in them) take precedence over
    // the next tick's front, which fills the SMs the back leaves idle (host
    // round trips, kernel tails).
    int prio_low = 0, prio_high = 0;
    TRY(cuda_ok(cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high)));
    TRY(cuda_ok(cudaStreamCreateWithPriority(&sv->stream, cudaStreamNonBlocking, prio_high)));
    TRY(cuda_ok(cudaStreamCreateWithPriority(&sv->front, cudaStreamNonBlocking, prio_low)));
    TRY(cuda_ok(cudaEventCreateWithFlags(&sv->count_done, cudaEventDisableTiming)));
    for (cudaEvent_t &e : sv->emit_done) TRY(cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)));
    for (int p = 0; p < 2; p++) {
        TRY(cuda_ok(cudaEventCreateWithFlags(&sv->front_done[p], cudaEventDisableTiming)));
        TRY(dalloc_on(&sv->d_views[p], kMaxServe, sv->device, sv->stream));
        TRY(dalloc_on(&sv->d_ctr[p], kNumLaunchCounters, sv->device, sv->stream));
        TRY(dalloc_on(&sv->d_ctls[p], kMaxServe + 1, sv->device, sv->stream));
        for (uint32_t j = 0; j < sv->max_batch; j++) {
            Slot &s = sv->slots[p][j];
            TRY(dalloc_on(&s.ctl, 1, sv->device, sv->stream));
            TRY(dalloc_on(&s.icand, cand, sv->device, sv->stream));
            TRY(dalloc_on(&s.counts, cand, sv->device, sv->stream));
            TRY(dalloc_on(&s.offsets, cand, sv->device, sv->stream));
            TRY(dalloc_on(&s.desc_cand, v->n_cull_desc, sv->device, sv->stream));
            TRY(dalloc_on(&s.desc_mc, 2 * n_mc_desc, sv->device, sv->stream));
            s.desc_occ = s.desc_mc + n_mc_desc;
            TRY(dalloc_on(&s.iocc, cand, sv->device, sv->stream));
            DevState d = v->s;            // the volume's cache and geometry, the request's own lists
            d.ctl = s.ctl;
            d.icand = s.icand;
            d.counts = s.counts;
            d.offsets = s.offsets;
            d.desc_cand = s.desc_cand;
            d.desc_mc = s.desc_mc;
            d.desc_occ = s.desc_occ;
            d.iocc = s.iocc;
            d.cases = nullptr;            // set below; a batch launch's per tick by the front
            d.case_cap = 0;
            d.cutw = nullptr;
            d.voff = nullptr;
            d.desc_vtx = nullptr;
            d.dbg_edges = nullptr;
            sv->views[p][j] = VolEntry{d, v->g, v->n_cull_desc, v->n_lru_desc};
        }
    }
    TRY(dalloc_on(&sv->d_params, kMaxServe, sv->device, sv->stream));
    // Stored cases (the count pass keeps each candidate's 64 cell cases for
    // the emission, as a volume does): by default for up to max_batch full
    // candidate lists, at most kMaxTickCaseBytes; without room the emission
    // classifies again.  A one-request tick's view (by value) holds the whole
    // buffer, a batch's views their regions (set by the front).
    {
        const uint64_t want = o.case_bytes ? o.case_bytes / 64 * 64
                                           : std::min<uint64_t>(kMaxTickCaseBytes, 64ull * cand * sv->max_batch);
        if (want && dalloc_on(&sv->cases, want, sv->device, sv->stream) == ISO_OK) sv->case_cap = want / 64;
        else sv->cases = nullptr;
        (void)cudaGetLastError();
        for (int p = 0; p < 2; p++) {
            sv->views[p][0].s.cases = sv->cases;
            sv->views[p][0].s.case_cap = sv->case_cap;
        }
    }
    if (cudaMallocHost((void **)&sv->h_ctls[0], (kMaxServe + 1) * sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&sv->h_ctls[1], (kMaxServe + 1) * sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void **)&sv->h_params, kMaxServe * sizeof(Params)) != cudaSuccess) {
        (void)cudaGetLastError();
        free_server(sv);
        return ISO_ERR_OOM;
    }
    cudaStream_t st = sv->stream;
    bool ok = cudaStreamSynchronize(v->stream) == cudaSuccess && cudaStreamSynchronize(sv->user) == cudaSuccess;
    for (int p = 0; ok && p < 2; p++) {
        ok = cudaMemcpyAsync(sv->d_views[p], sv->views[p], sv->max_batch * sizeof(VolEntry), cudaMemcpyHostToDevice,
                             st) == cudaSuccess;
        for (uint32_t j = 0; ok && j < sv->max_batch; j++) {
            ok = cudaMemsetAsync(sv->slots[p][j].ctl, 0, sizeof(Ctl), st) == cudaSuccess &&   // no field undefined
                 cudaMemsetAsync(sv->slots[p][j].icand, 0, cand * 4, st) == cudaSuccess &&
                 cudaMemsetAsync(sv->slots[p][j].desc_mc, 0, n_mc_desc * 16, st) == cudaSuccess;
        }
    }
    ok = ok && cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        free_server(sv);
        return ISO_ERR_CUDA;
    }
#undef TRY
    sv->one_plan = launch_plan(nullptr, sv->device, v->g.nb, cand, 1, true, v->g.rate);
    sv->back_plan = launch_plan(nullptr, sv->device, (uint64_t)v->g.nb * sv->max_batch,
                                (uint64_t)cand * sv->max_batch, sv->max_batch, false, v->g.rate);
    *out = sv;
    return ISO_OK;
}

int iso_server_submit(iso_server *sv, float isovalue, uint64_t *ticket) {
    if (!sv || !ticket || !std::isfinite(isovalue)) return ISO_ERR_INVALID_ARG;
    *ticket = sv->next_ticket++;
    sv->queue.push_back(Request{*ticket, isovalue});
    return ISO_OK;
}

int iso_server_poll(iso_server *sv, uint32_t *completed) {
    NvtxRange nvtx("iso_server_poll");
    if (!sv) return ISO_ERR_INVALID_ARG;
    uint32_t n = 0;
    DeviceGuard dg(sv->device);
    int r;
    while ((r = advance(sv, false, &n)) > 0) {
    }
    if (completed) *completed = n;
    return r < 0 ? -r : ISO_OK;
}

int iso_server_step(iso_server *sv, uint32_t *completed) {
    NvtxRange nvtx("iso_server_step");
    if (!sv) return ISO_ERR_INVALID_ARG;
    uint32_t n = 0;
    DeviceGuard dg(sv->device);
    const uint64_t ticks0 = sv->ticks_finished, rounds0 = sv->rounds_finished;
    int r = 0;
    for (;;) {
        r = advance(sv, false, &n);
        if (r > 0) continue;
        // an emission round finished, a tick ended otherwise (its requests
        // failed), a failure, the budget blocks, or nothing is in flight
        const bool mid_round = sv->has_back && sv->back_tick.stage == kEmit;
        if (r < 0 || sv->rounds_finished != rounds0 || sv->ticks_finished != ticks0 || (n > 0 && !mid_round) ||
            (!sv->has_front && !sv->has_back) || sv->blocked)
            break;
        r = advance(sv, true, &n);
        if (r < 0) break;
    }
    if (completed) *completed = n;
    return r < 0 ? -r : ISO_OK;
}

int iso_server_queued(const iso_server *sv, uint32_t *queued) {
    if (!sv || !queued) return ISO_ERR_INVALID_ARG;
    *queued = (uint32_t)(sv->queue.size() + (sv->has_front ? sv->front_tick.reqs.size() : 0) +
                         (sv->has_back ? sv->back_tick.reqs.size() - sv->back_tick.emitted : 0));
    return ISO_OK;
}

int iso_server_take(iso_server *sv, uint64_t ticket, iso_mesh *out) {
    if (!sv || !out) return ISO_ERR_INVALID_ARG;
    auto it = sv->done.find(ticket);
    if (it == sv->done.end()) {
        if (ticket == 0 || ticket >= sv->next_ticket) return ISO_ERR_INVALID_ARG;
        for (const Request &r : sv->queue)
            if (r.ticket == ticket) return ISO_PENDING;
        for (const Tick *t : {sv->has_front ? &sv->front_tick : nullptr, sv->has_back ? &sv->back_tick : nullptr})
            if (t)
                for (const Request &r : t->reqs)
                    if (r.ticket == ticket) return ISO_PENDING;
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
