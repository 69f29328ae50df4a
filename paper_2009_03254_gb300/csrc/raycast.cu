// Implicit isosurface ray casting over the block grid as a macrocell grid
// (the future work Section 4.6.2 proposes: the blocks as macrocells for
// space skipping, the isosurface of the trilinear interpolant found inside
// them), reading the decoded-block cache of Sections 4.1-4.2.
//
// iso_raycast runs the extraction's front for the isovalue (range test,
// cache update, decode: every block whose 2x2x2 group range holds the
// isovalue is active, and so is its whole group, so every sample a ray can
// need is cached), then one thread per pixel (16 x 16 pixel tiles per CTA)
// casts its ray:
//   - a slab test against the volume box gives the start; the block, then
//     the cell, holding the current point starts each level;
//   - each box's interval comes from its own slab test (not an
//     incremental update; the direction's reciprocal is taken once per
//     ray), and the next box is one step along the exit axis, so the
//     visited boxes and their intervals are fixed by the ray;
//   - a block is searched when its precomputed group range (hull8) holds
//     the isovalue; a cell when its 8 corners' range does: 5 samples of the
//     trilinear interpolant on its interval, then 12 bisection steps at the
//     first change of side;
//   - the hit is shaded from the interpolant's gradient (two-sided Lambert).
// Every float operation is one IEEE float32 operation (this file is built
// without multiply-add contraction), so the depths equal the CPU oracle's
// bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include "bcmc.h"
#include "volume.cuh"

namespace bcmc {

namespace {

constexpr int kTile = 16;                               // pixels per tile side (one CTA)

struct CastArgs {
    const int32_t *islot;
    const float *slots;
    const float2 *hull8;
    const Ctl *ctl;
    unsigned long long *hits;
    uint32_t *rgba;
    unsigned long long *nhit;
    uint32_t *err;
    uint32_t nx, ny, nz, nbx, nby, nbz;
    uint32_t width, height;
    float iso;
    float eye[3], fwd[3], right[3], up[3], light[3];
};

struct Ray {
    float o[3], d[3], inv[3];     // inv = 1 / d (0 where d == 0: unused)
};

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

// interval of the ray inside box [lo, hi]; false if an axis parallel to
// the ray misses it.  The exit axis is the first whose upper value is the
// interval's end (-1 if the ray is parallel to every axis).
__device__ __forceinline__ bool slab(const Ray &r, const float lo[3], const float hi[3], float &tin, float &tout,
                                     int &ax) {
    float a = -inf_f(), b = inf_f();
    ax = -1;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (r.d[k] == 0.0f) {
            if (r.o[k] < lo[k] || r.o[k] > hi[k]) return false;
            continue;
        }
        const float t0 = (lo[k] - r.o[k]) * r.inv[k], t1 = (hi[k] - r.o[k]) * r.inv[k];
        const float mn = t0 < t1 ? t0 : t1, mx = t0 < t1 ? t1 : t0;
        if (mn > a) a = mn;
        if (mx < b) {
            b = mx;
            ax = k;
        }
    }
    tin = a;
    tout = b;
    return true;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

__device__ __forceinline__ float trilinear(const float c[8], float fx, float fy, float fz) {
    const float c00 = c[0] + fx * (c[1] - c[0]), c10 = c[2] + fx * (c[3] - c[2]);
    const float c01 = c[4] + fx * (c[5] - c[4]), c11 = c[6] + fx * (c[7] - c[6]);
    const float c0 = c00 + fy * (c10 - c00), c1 = c01 + fy * (c11 - c01);
    return c0 + fz * (c1 - c0);
}

__device__ __forceinline__ float g_at(const Ray &r, const float c[8], const int cell[3], float iso, float t) {
    const float fx = clamp01(r.o[0] + t * r.d[0] - (float)cell[0]);
    const float fy = clamp01(r.o[1] + t * r.d[1] - (float)cell[1]);
    const float fz = clamp01(r.o[2] + t * r.d[2] - (float)cell[2]);
    return trilinear(c, fx, fy, fz) - iso;
}

__device__ bool cell_root(const Ray &r, const float c[8], const int cell[3], float iso, float a, float b,
                          float &thit) {
    const float h = (b - a) * 0.25f;
    float tk = a;
    bool sk = g_at(r, c, cell, iso, tk) < 0.0f;
    for (int k = 1; k <= 4; k++) {
        const float tn = k == 4 ? b : a + h * (float)k;
        const bool sn = g_at(r, c, cell, iso, tn) < 0.0f;
        if (sn != sk) {
            float lo = tk, hi = tn;
            for (int it = 0; it < 12; it++) {
                const float m = (lo + hi) * 0.5f;
                const bool sm = g_at(r, c, cell, iso, m) < 0.0f;
                if (sm == sk) lo = m;
                else hi = m;
            }
            thit = (lo + hi) * 0.5f;
            return true;
        }
        tk = tn;
        sk = sn;
    }
    return false;
}

// the first hit of the ray; the hit cell's corners in cv
__device__ bool cast(const CastArgs &a, const Ray &r, int32_t *gs, float &thit, int hc[3], int hb[3], float cv[8]) {
    const int n[3] = {(int)a.nx, (int)a.ny, (int)a.nz};
    int ncb[3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (n[k] < 2) return false;
        ncb[k] = (n[k] - 2) / 4 + 1;
    }
    const float vlo[3] = {0.0f, 0.0f, 0.0f};
    const float vhi[3] = {(float)(n[0] - 1), (float)(n[1] - 1), (float)(n[2] - 1)};
    float t0, t1;
    int ax;
    if (!slab(r, vlo, vhi, t0, t1, ax)) return false;
    if (t0 < 0.0f) t0 = 0.0f;
    if (!(t0 <= t1)) return false;
    int b[3];
#pragma unroll
    for (int k = 0; k < 3; k++) b[k] = clampi((int)floorf((r.o[k] + t0 * r.d[k]) * 0.25f), 0, ncb[k] - 1);
    float t = t0;
    const int stride = blockDim.x;                      // group slots of this thread: gs[k * stride]
    for (;;) {
        float blo[3], bhi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            blo[k] = (float)(4 * b[k]);
            const int h = 4 * b[k] + 4;
            bhi[k] = (float)(h < n[k] - 1 ? h : n[k] - 1);
        }
        float bin, bout;
        int bax;
        if (!slab(r, blo, bhi, bin, bout, bax) || bax < 0) return false;
        if (bin < t) bin = t;
        const uint32_t bid = (uint32_t)b[0] + a.nbx * ((uint32_t)b[1] + a.nby * (uint32_t)b[2]);
        const float2 hull = a.hull8[bid];
        if (bin <= bout && hull.x < a.iso && a.iso <= hull.y) {
            // cache slots of the block's group (-1 outside the volume)
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int gx = b[0] + (k & 1), gy = b[1] + ((k >> 1) & 1), gz = b[2] + (k >> 2);
                const bool in = gx < (int)a.nbx && gy < (int)a.nby && gz < (int)a.nbz;
                gs[k * stride] = in ? a.islot[(uint32_t)gx + a.nbx * ((uint32_t)gy + a.nby * (uint32_t)gz)] : -1;
            }
            int c[3];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const int last = 4 * b[k] + 3 < n[k] - 2 ? 4 * b[k] + 3 : n[k] - 2;
                c[k] = clampi((int)floorf(r.o[k] + bin * r.d[k]), 4 * b[k], last);
            }
            for (;;) {
                const float clo[3] = {(float)c[0], (float)c[1], (float)c[2]};
                const float chi[3] = {(float)(c[0] + 1), (float)(c[1] + 1), (float)(c[2] + 1)};
                float cin, cout;
                int cax;
                if (!slab(r, clo, chi, cin, cout, cax) || cax < 0) break;
                if (cin < bin) cin = bin;
                if (cin <= cout) {
                    float mn = inf_f(), mx = -inf_f();
#pragma unroll
                    for (int k = 0; k < 8; k++) {
                        const int x = c[0] + (k & 1), y = c[1] + ((k >> 1) & 1), z = c[2] + (k >> 2);
                        const int g = ((x >> 2) - b[0]) | (((y >> 2) - b[1]) << 1) | (((z >> 2) - b[2]) << 2);
                        const int32_t sl = gs[g * stride];
                        float v = 0.0f;
                        if (sl >= 0) v = a.slots[(size_t)sl * 64 + (x & 3) + 4 * (y & 3) + 16 * (z & 3)];
                        else atomicOr(a.err, 1u);       // never: every group member is cached
                        cv[k] = v;
                        mn = k == 0 ? v : (v < mn ? v : mn);
                        mx = k == 0 ? v : (v > mx ? v : mx);
                    }
                    if (mn < a.iso && a.iso <= mx && cell_root(r, cv, c, a.iso, cin, cout, thit)) {
#pragma unroll
                        for (int k = 0; k < 3; k++) {
                            hc[k] = c[k];
                            hb[k] = b[k];
                        }
                        return true;
                    }
                }
                // one step along the exit axis (selects, not an indexed array)
                bool out = false;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    if (k != cax) continue;
                    c[k] += r.d[k] > 0.0f ? 1 : -1;
                    const int last = 4 * b[k] + 3 < n[k] - 2 ? 4 * b[k] + 3 : n[k] - 2;
                    out = c[k] < 4 * b[k] || c[k] > last;
                }
                if (out) break;
            }
        }
        bool out = false;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (k != bax) continue;
            b[k] += r.d[k] > 0.0f ? 1 : -1;
            out = b[k] < 0 || b[k] >= ncb[k];
        }
        if (out) return false;
        t = bout;
    }
}

__global__ void __launch_bounds__(kTile * kTile) raycast_kernel(CastArgs a) {
    __shared__ int32_t gs[8 * kTile * kTile];
    if (a.ctl->status & (kStatusBudget | kStatusAnyTimeout)) return;   // the cache update failed
    const uint32_t tiles_x = (a.width + kTile - 1) / kTile;
    const int i = (int)((blockIdx.x % tiles_x) * kTile + (threadIdx.x % kTile));
    const int j = (int)((blockIdx.x / tiles_x) * kTile + (threadIdx.x / kTile));
    bool hit = false;
    if (i < (int)a.width && j < (int)a.height) {
        const float u = ((float)i + 0.5f) / (float)a.width * 2.0f - 1.0f;
        const float v = ((float)j + 0.5f) / (float)a.height * 2.0f - 1.0f;
        Ray r;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            r.o[k] = a.eye[k];
            r.d[k] = a.fwd[k] + u * a.right[k] + v * a.up[k];
            r.inv[k] = r.d[k] == 0.0f ? 0.0f : 1.0f / r.d[k];
        }
        const size_t px = (size_t)j * a.width + i;
        float t, cv[8];
        int c[3], b[3];
        hit = cast(a, r, gs + threadIdx.x, t, c, b, cv);
        if (!hit) {
            a.hits[px] = ~0ull;
            if (a.rgba) a.rgba[px] = 0u;
        } else {
            const uint32_t id = (uint32_t)b[0] + a.nbx * ((uint32_t)b[1] + a.nby * (uint32_t)b[2]);
            a.hits[px] = ((unsigned long long)__float_as_uint(t) << 32) | id;
            if (a.rgba) {
                const float base[3] = {0.85f, 0.75f, 0.55f};
                const float l2 = a.light[0] * a.light[0] + a.light[1] * a.light[1] + a.light[2] * a.light[2];
                const float linv = 1.0f / sqrtf(l2);
                const float L[3] = {a.light[0] * linv, a.light[1] * linv, a.light[2] * linv};
                const float fx = clamp01(r.o[0] + t * r.d[0] - (float)c[0]);
                const float fy = clamp01(r.o[1] + t * r.d[1] - (float)c[1]);
                const float fz = clamp01(r.o[2] + t * r.d[2] - (float)c[2]);
                const float gx = (1.0f - fz) * ((1.0f - fy) * (cv[1] - cv[0]) + fy * (cv[3] - cv[2])) +
                                 fz * ((1.0f - fy) * (cv[5] - cv[4]) + fy * (cv[7] - cv[6]));
                const float gy = (1.0f - fz) * ((1.0f - fx) * (cv[2] - cv[0]) + fx * (cv[3] - cv[1])) +
                                 fz * ((1.0f - fx) * (cv[6] - cv[4]) + fx * (cv[7] - cv[5]));
                const float gz = (1.0f - fy) * ((1.0f - fx) * (cv[4] - cv[0]) + fx * (cv[5] - cv[1])) +
                                 fy * ((1.0f - fx) * (cv[6] - cv[2]) + fx * (cv[7] - cv[3]));
                const float n2 = gx * gx + gy * gy + gz * gz;
                float inten = 0.2f;
                if (n2 > 0.0f) {
                    const float cth = fabsf(gx * L[0] + gy * L[1] + gz * L[2]) / sqrtf(n2);
                    inten = 0.2f + 0.8f * cth;
                    if (inten > 1.0f) inten = 1.0f;
                }
                uint32_t out = 255u << 24;
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const float x = inten * base[k] * 255.0f + 0.5f;
                    out |= ((uint32_t)x & 255u) << (8 * k);
                }
                a.rgba[px] = out;
            }
        }
    }
    const uint32_t nh = __reduce_add_sync(0xffffffffu, hit ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && nh) atomicAdd(a.nhit, (unsigned long long)nh);
}

}  // namespace

}  // namespace bcmc

extern "C" int iso_raycast(iso_volume *v, float isovalue, const iso_pinhole *cam, uint64_t *d_hits, uint32_t *d_rgba,
                           iso_raycast_stats *stats) {
    using namespace bcmc;
    using namespace bcmc_host;
    NvtxRange nvtx("iso_raycast");
    if (!v || !cam || !d_hits || !std::isfinite(isovalue) || cam->width == 0 || cam->height == 0 ||
        cam->width > 32768 || cam->height > 32768 || misaligned(d_hits, 8) || misaligned(d_rgba, 4))
        return ISO_ERR_INVALID_ARG;
    const float *vecs[5] = {cam->eye, cam->forward, cam->right, cam->up, cam->light};
    for (const float *p : vecs)
        for (int k = 0; k < 3; k++)
            if (!std::isfinite(p[k])) return ISO_ERR_INVALID_ARG;
    const double l2 = (double)cam->light[0] * cam->light[0] + (double)cam->light[1] * cam->light[1] +
                      (double)cam->light[2] * cam->light[2];
    if (!(l2 > 1e-30) || !(l2 < 1e30)) return ISO_ERR_INVALID_ARG;
    DeviceGuard dg(v->device);
    ISO_CK_RC(finish_upload(v));
    cudaStream_t st = v->stream;
    // the extraction's front for this isovalue: range test, cache update, decode
    *v->host_params = Params{isovalue, kVertexFloat4, 0u, 0u, 0u, 0u, 0ull, 0ull, 0ull, 0ull, 0ull};
    ISO_CK(cudaMemcpyAsync(&v->s.ctl->params, v->host_params, sizeof(Params), cudaMemcpyHostToDevice, st));
    const Launch L{nullptr, 1u, single_counters(v), VolEntry{v->s, v->g, v->n_cull_desc, v->n_lru_desc}};
    launch_front(L, v->plan, st, nullptr);
    void *scratch = nullptr;
    int rc = dalloc_bytes(&scratch, 16, v->device, st);
    if (rc) return rc;
    CastArgs a{};
    a.islot = v->s.islot;
    a.slots = v->s.slots;
    a.hull8 = v->s.hull8;
    a.ctl = v->s.ctl;
    a.hits = reinterpret_cast<unsigned long long *>(d_hits);
    a.rgba = d_rgba;
    a.nhit = static_cast<unsigned long long *>(scratch);
    a.err = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + 8);
    a.nx = v->g.nx;
    a.ny = v->g.ny;
    a.nz = v->g.nz;
    a.nbx = v->g.nbx;
    a.nby = v->g.nby;
    a.nbz = v->g.nbz;
    a.width = cam->width;
    a.height = cam->height;
    a.iso = isovalue;
    for (int k = 0; k < 3; k++) {
        a.eye[k] = cam->eye[k];
        a.fwd[k] = cam->forward[k];
        a.right[k] = cam->right[k];
        a.up[k] = cam->up[k];
        a.light[k] = cam->light[k];
    }
    unsigned long long counters[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(scratch, 0, 16, st);
    if (e == cudaSuccess) {
        const uint32_t tiles = ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
        raycast_kernel<<<tiles, kTile * kTile, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(v->host_ctl, v->s.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counters, scratch, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree_on(scratch, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA;
    }
    v->last_n_active = v->host_ctl->n_active;
    v->last_n_new = v->host_ctl->n_new;
    v->last_n_cand = v->host_ctl->n_cand;
    v->last_slots = v->host_ctl->S;
    v->last_tris = 0;
    rc = status_to_error(v, v->host_ctl->status);
    if (rc) return rc;
    if ((uint32_t)(counters[1] & 0xFFFFFFFFu)) return ISO_ERR_CUDA;
    if (stats) {
        stats->hits = counters[0];
        stats->n_active = v->host_ctl->n_active;
        stats->n_new = v->host_ctl->n_new;
        stats->n_slots = v->host_ctl->S;
    }
    return ISO_OK;
}
