// Rendering of an extracted surface (paper Section 4.6.2: the triangle soup,
// in the compressed vertex format of Section 4.5, is drawn directly; the
// block position comes from the block id and offsets the dequantised
// vertex).  CUDA kernels write headless device buffers: a fragment buffer
// of (depth bits << 32 | triangle) per pixel and an RGBA8 image.
//
// Rules (every float operation is a single IEEE operation: this file is
// compiled without FMA contraction):
//   world     block origin (4 bx, 4 by, 4 bz) + block-local position, or
//             + code * (4 / 1023) for compact vertices
//   clip      (X, Y, Z, W) = M (x, y, z, 1), each row summed left to right;
//             a triangle with a vertex at W <= 0 is not drawn
//   screen    r = 1 / W, sx = (X r * 0.5 + 0.5) * width, sy likewise (y up),
//             depth d = Z r * 0.5 + 0.5
//   edges     E(a, b; p) = (b.x - a.x)(p.y - a.y) - (b.y - a.y)(p.x - a.x),
//             evaluated with the endpoints in ascending (x, y) order and
//             negated when swapped (shared edges see opposite values, so a
//             mesh has no cracks and no double hits; the order and the
//             differences are taken once per triangle); counter-clockwise
//             orientation by swapping v1 and v2 when A = E(v0, v1; v2) < 0
//   coverage  pixel centres in the vertices' bounding box with all three
//             edge values >= 0, zero only on a top-left edge
//   depth     ((e0 d0 + e1 d1) + e2 d2) / A + 0, kept in [0, 1]
//   visible   the smallest (depth bits << 32 | triangle), by 64-bit atomicMin
//   shading   two-sided Lambert: 0.2 + 0.8 |n . L| / |n|, base colour
//             (0.85, 0.75, 0.55), rgb = floor(c * 255 + 0.5), alpha 255
//
// Triangles whose screen bounding box holds at most kSmallPixels pixel
// centres are covered by one thread; larger ones go to a list that one warp
// per triangle covers, lane by pixel.
#include <algorithm>
#include <cstdint>

#include "bcmc.h"
#include "volume.cuh"

namespace bcmc {

namespace {

constexpr uint32_t kSmallPixels = 32;
constexpr float kCodeScale = 0.0039100684f;          // 4 / 1023 rounded to float

struct RasterArgs {
    const void *verts;
    const uint32_t *idx;          // null: soup (vertex 3t + j)
    unsigned long long num_vtx;   // vertices in the buffer (indexed: a triangle reaching past them is not drawn)
    unsigned long long num_tri;
    unsigned long long *frag;
    uint32_t *big;                // triangles left for the warp kernel
    unsigned long long *ctr;      // [0] listed, [1] drawn, [2] big (as [0])
    uint32_t format;              // 0 float4, 1 compact
    uint32_t nbx, nby;
    unsigned long long inv_nbx, inv_nby;   // division magic (block id -> coordinates)
    uint32_t width, height;
    float m[16];
};

struct P2 {
    float x, y;
};

// An edge in canonical (ascending x, then y) endpoint order: its value at
// p is sign * (dx (p.y - a.y) - dy (p.x - a.x)), the same operations as
// evaluating it from the endpoints.
struct Edge {
    float ax, ay, dx, dy;
    bool neg;
    __device__ __forceinline__ void set(P2 a, P2 b) {
        neg = (b.x < a.x) || (b.x == a.x && b.y < a.y);
        if (neg) {
            const P2 t = a;
            a = b;
            b = t;
        }
        ax = a.x;
        ay = a.y;
        dx = b.x - a.x;
        dy = b.y - a.y;
    }
    __device__ __forceinline__ float at(float px, float py) const {
        const float e = dx * (py - ay) - dy * (px - ax);
        return neg ? -e : e;
    }
};

struct Tri {
    Edge e[3];                    // v1 -> v2, v2 -> v0, v0 -> v1 of the counter-clockwise triangle
    float d[3];
    float A;
    int i0, i1, j0, j1;
    bool tl[3];
};

__device__ __forceinline__ void world(const RasterArgs &a, unsigned long long k, float p[3]) {
    uint32_t id;
    float local[3];
    if (a.format == 0) {
        const float4 v = reinterpret_cast<const float4 *>(a.verts)[k];
        local[0] = v.x;
        local[1] = v.y;
        local[2] = v.z;
        id = __float_as_uint(v.w);
    } else {
        const uint2 v = reinterpret_cast<const uint2 *>(a.verts)[k];
#pragma unroll
        for (int c = 0; c < 3; c++) local[c] = (float)((v.x >> (10 * c)) & 1023u) * kCodeScale;
        id = v.y;
    }
    const uint32_t q = div_by(id, a.nbx, a.inv_nbx), bz = div_by(q, a.nby, a.inv_nby);
    const uint32_t bx = id - q * a.nbx, by = q - bz * a.nby;
    p[0] = (float)(4 * bx) + local[0];
    p[1] = (float)(4 * by) + local[1];
    p[2] = (float)(4 * bz) + local[2];
}

__device__ __forceinline__ unsigned long long vertex_index(const RasterArgs &a, unsigned long long t, int j) {
    return a.idx ? (unsigned long long)a.idx[3 * t + j] : 3 * t + j;
}

__device__ __forceinline__ float edge(P2 a, P2 b, float px, float py) {
    const bool swap = (b.x < a.x) || (b.x == a.x && b.y < a.y);
    if (swap) {
        const P2 t = a;
        a = b;
        b = t;
    }
    const float e = (b.x - a.x) * (py - a.y) - (b.y - a.y) * (px - a.x);
    return swap ? -e : e;
}

__device__ __forceinline__ bool top_left(P2 a, P2 b) {
    const float dx = b.x - a.x, dy = b.y - a.y;
    return dy < 0.0f || (dy == 0.0f && dx < 0.0f);
}

// projection, orientation and pixel range of triangle t; false: not drawn
__device__ bool setup(const RasterArgs &a, unsigned long long t, Tri &r) {
    if (a.idx) {                                       // indices past the vertex buffer: not drawn
#pragma unroll
        for (int j = 0; j < 3; j++)
            if (a.idx[3 * t + j] >= a.num_vtx) return false;
    }
    bool behind = false;
    P2 s[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        float p[3];
        world(a, vertex_index(a, t, j), p);
        const float *m = a.m;
        const float X = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
        const float Y = m[4] * p[0] + m[5] * p[1] + m[6] * p[2] + m[7];
        const float Z = m[8] * p[0] + m[9] * p[1] + m[10] * p[2] + m[11];
        const float W = m[12] * p[0] + m[13] * p[1] + m[14] * p[2] + m[15];
        if (!(W > 0.0f)) behind = true;
        const float rw = 1.0f / W;
        s[j].x = (X * rw * 0.5f + 0.5f) * (float)a.width;
        s[j].y = (Y * rw * 0.5f + 0.5f) * (float)a.height;
        r.d[j] = Z * rw * 0.5f + 0.5f;
    }
    if (behind) return false;
    float A = edge(s[0], s[1], s[2].x, s[2].y);
    if (A == 0.0f || A != A) return false;
    if (A < 0.0f) {
        const P2 ts = s[1];
        s[1] = s[2];
        s[2] = ts;
        const float td = r.d[1];
        r.d[1] = r.d[2];
        r.d[2] = td;
        A = edge(s[0], s[1], s[2].x, s[2].y);
        if (!(A > 0.0f)) return false;
    }
    r.A = A;
    const float xmin = fminf(fminf(s[0].x, s[1].x), s[2].x), xmax = fmaxf(fmaxf(s[0].x, s[1].x), s[2].x);
    const float ymin = fminf(fminf(s[0].y, s[1].y), s[2].y), ymax = fmaxf(fmaxf(s[0].y, s[1].y), s[2].y);
    const float fi0 = ceilf(xmin - 0.5f), fi1 = floorf(xmax - 0.5f);
    const float fj0 = ceilf(ymin - 0.5f), fj1 = floorf(ymax - 0.5f);
    const float wl = (float)(a.width - 1), hl = (float)(a.height - 1);
    if (fi1 < 0.0f || fj1 < 0.0f || fi0 > wl || fj0 > hl) return false;
    r.i0 = fi0 < 0.0f ? 0 : (int)fi0;
    r.i1 = fi1 > wl ? (int)a.width - 1 : (int)fi1;
    r.j0 = fj0 < 0.0f ? 0 : (int)fj0;
    r.j1 = fj1 > hl ? (int)a.height - 1 : (int)fj1;
    r.tl[0] = top_left(s[1], s[2]);
    r.tl[1] = top_left(s[2], s[0]);
    r.tl[2] = top_left(s[0], s[1]);
    r.e[0].set(s[1], s[2]);
    r.e[1].set(s[2], s[0]);
    r.e[2].set(s[0], s[1]);
    return true;
}

// test pixel (i, j) against triangle t and keep the nearer fragment
__device__ __forceinline__ void fragment(const RasterArgs &a, const Tri &r, uint32_t t, int i, int j) {
    const float px = (float)i + 0.5f, py = (float)j + 0.5f;
    const float e0 = r.e[0].at(px, py), e1 = r.e[1].at(px, py), e2 = r.e[2].at(px, py);
    if (e0 < 0.0f || e1 < 0.0f || e2 < 0.0f) return;
    if ((e0 == 0.0f && !r.tl[0]) || (e1 == 0.0f && !r.tl[1]) || (e2 == 0.0f && !r.tl[2])) return;
    const float dd = (e0 * r.d[0] + e1 * r.d[1] + e2 * r.d[2]) / r.A + 0.0f;
    if (!(dd >= 0.0f && dd <= 1.0f)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(dd) << 32) | t;
    unsigned long long *f = a.frag + (size_t)j * a.width + i;
    if (key < *f) atomicMin(f, key);                   // the read only skips atomics that cannot win
}

__global__ void __launch_bounds__(256) raster_small_kernel(RasterArgs a) {
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    uint32_t drawn = 0, big = 0;
    for (unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; t < a.num_tri;
         t += stride) {
        Tri r;
        if (!setup(a, t, r)) continue;
        drawn++;
        const uint32_t npx = (uint32_t)(r.i1 - r.i0 + 1) * (uint32_t)(r.j1 - r.j0 + 1);
        if (npx > kSmallPixels) {                      // the list holds every triangle
            big++;
            a.big[atomicAdd(&a.ctr[0], 1ull)] = (uint32_t)t;
            continue;
        }
        for (int j = r.j0; j <= r.j1; j++)
            for (int i = r.i0; i <= r.i1; i++) fragment(a, r, (uint32_t)t, i, j);
    }
    // per-warp totals
    const uint32_t d = __reduce_add_sync(0xffffffffu, drawn), b = __reduce_add_sync(0xffffffffu, big);
    if ((threadIdx.x & 31) == 0) {
        if (d) atomicAdd(&a.ctr[1], (unsigned long long)d);
        if (b) atomicAdd(&a.ctr[2], (unsigned long long)b);
    }
}

// one warp per listed triangle, lane by pixel of its bounding box
__global__ void __launch_bounds__(256) raster_big_kernel(RasterArgs a) {
    const unsigned long long n = a.ctr[0];
    const int lane = threadIdx.x & 31;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x / 32);
    for (unsigned long long w = (unsigned long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < n;
         w += warps) {
        const uint32_t t = a.big[w];
        Tri r;
        if (!setup(a, t, r)) continue;                  // warp-uniform
        const uint32_t bw = (uint32_t)(r.i1 - r.i0 + 1);
        const unsigned long long npx = (unsigned long long)bw * (uint32_t)(r.j1 - r.j0 + 1);
        for (unsigned long long k = lane; k < npx; k += 32)
            fragment(a, r, t, r.i0 + (int)(k % bw), r.j0 + (int)(k / bw));
    }
}

struct ShadeArgs {
    const void *verts;
    const uint32_t *idx;
    const unsigned long long *frag;
    uint32_t *rgba;
    unsigned long long pixels;
    uint32_t format, nbx, nby;
    float light[3];               // as given; normalised here
};

__global__ void __launch_bounds__(256) shade_kernel(ShadeArgs s) {
    RasterArgs a{};
    a.verts = s.verts;
    a.idx = s.idx;
    a.format = s.format;
    a.nbx = s.nbx;
    a.nby = s.nby;
    a.inv_nbx = div_magic(s.nbx);
    a.inv_nby = div_magic(s.nby);
    const float base[3] = {0.85f, 0.75f, 0.55f};
    const float l2 = s.light[0] * s.light[0] + s.light[1] * s.light[1] + s.light[2] * s.light[2];
    const float linv = 1.0f / sqrtf(l2);
    const float L[3] = {s.light[0] * linv, s.light[1] * linv, s.light[2] * linv};
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long k = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; k < s.pixels; k += stride) {
        const unsigned long long key = s.frag[k];
        if (key == ~0ull) {
            s.rgba[k] = 0u;
            continue;
        }
        const unsigned long long t = (uint32_t)key;
        float p[3][3];
#pragma unroll
        for (int j = 0; j < 3; j++) world(a, vertex_index(a, t, j), p[j]);
        const float u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
        const float v[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
        const float n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        const float n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        float inten = 0.2f;
        if (n2 > 0.0f) {
            const float c = fabsf(n[0] * L[0] + n[1] * L[1] + n[2] * L[2]) / sqrtf(n2);
            inten = 0.2f + 0.8f * c;
            if (inten > 1.0f) inten = 1.0f;
        }
        uint32_t out = 255u << 24;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float x = inten * base[c] * 255.0f + 0.5f;
            out |= ((uint32_t)x & 255u) << (8 * c);
        }
        s.rgba[k] = out;
    }
}

int grid_for(unsigned long long work, int device) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const unsigned long long want = (work + 255) / 256;
    const unsigned long long cap = (unsigned long long)std::max(1, sms) * 8;   // 2048 threads per SM
    return (int)std::max(1ull, std::min(want, cap));
}

}  // namespace

}  // namespace bcmc

extern "C" int iso_render(const void *d_vertices, int vertex_format, const uint32_t *d_indices,
                          uint64_t num_vertices, uint64_t num_triangles, uint32_t nx, uint32_t ny, uint32_t nz,
                          const iso_camera *camera, uint64_t *d_fragments, uint32_t *d_rgba,
                          iso_render_stats *stats, void *stream) {
    using namespace bcmc;
    using namespace bcmc_host;
    NvtxRange nvtx("iso_render");
    if (!camera || !d_fragments || camera->width == 0 || camera->height == 0 || camera->width > 32768 ||
        camera->height > 32768 || nx == 0 || ny == 0 || nz == 0 ||
        (vertex_format != ISO_VERTEX_FLOAT4 && vertex_format != ISO_VERTEX_PACKED) ||
        (num_triangles && !d_vertices) || num_triangles > 0xFFFFFFFFull ||
        (!d_indices && num_vertices < 3 * num_triangles) ||    // a soup needs its 3T vertices
        misaligned(d_vertices, vertex_format == ISO_VERTEX_FLOAT4 ? 16 : 8) || misaligned(d_indices, 4) ||
        misaligned(d_fragments, 8) || misaligned(d_rgba, 4))
        return ISO_ERR_INVALID_ARG;
    const float *L = camera->light;
    const double l2 = (double)L[0] * L[0] + (double)L[1] * L[1] + (double)L[2] * L[2];
    if (!(l2 > 1e-30) || !(l2 < 1e30)) return ISO_ERR_INVALID_ARG;
    for (int k = 0; k < 16; k++)
        if (!(camera->view_proj[k] == camera->view_proj[k])) return ISO_ERR_INVALID_ARG;
    int dev = 0;
    ISO_CK(cudaGetDevice(&dev));
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned long long pixels = (unsigned long long)camera->width * camera->height;
    ISO_CK(cudaMemsetAsync(d_fragments, 0xFF, pixels * 8, st));
    RasterArgs a{};
    a.verts = d_vertices;
    a.idx = d_indices;
    a.num_vtx = num_vertices;
    a.num_tri = num_triangles;
    a.frag = reinterpret_cast<unsigned long long *>(d_fragments);
    a.format = vertex_format == ISO_VERTEX_PACKED ? 1u : 0u;
    a.nbx = (nx + 3) / 4;
    a.nby = (ny + 3) / 4;
    a.inv_nbx = div_magic(a.nbx);
    a.inv_nby = div_magic(a.nby);
    a.width = camera->width;
    a.height = camera->height;
    for (int k = 0; k < 16; k++) a.m[k] = camera->view_proj[k];
    void *scratch = nullptr;                            // counters, then room to list every triangle
    const size_t ctr_bytes = 3 * sizeof(unsigned long long);
    int rc = dalloc_bytes(&scratch, ctr_bytes + (size_t)num_triangles * 4 + 16, dev, st);
    if (rc) return rc;
    a.ctr = static_cast<unsigned long long *>(scratch);
    a.big = reinterpret_cast<uint32_t *>(static_cast<char *>(scratch) + ctr_bytes);
    cudaError_t e = cudaMemsetAsync(a.ctr, 0, ctr_bytes, st);
    if (e == cudaSuccess && num_triangles) {
        raster_small_kernel<<<grid_for(num_triangles, dev), 256, 0, st>>>(a);
        // the list's length is known on the device only: a full grid, grid-stride
        raster_big_kernel<<<grid_for(~0ull >> 16, dev), 256, 0, st>>>(a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && d_rgba) {
        ShadeArgs s{};
        s.verts = d_vertices;
        s.idx = d_indices;
        s.frag = a.frag;
        s.rgba = d_rgba;
        s.pixels = pixels;
        s.format = a.format;
        s.nbx = a.nbx;
        s.nby = a.nby;
        s.light[0] = L[0];
        s.light[1] = L[1];
        s.light[2] = L[2];
        shade_kernel<<<grid_for(pixels, dev), 256, 0, st>>>(s);
        e = cudaGetLastError();
    }
    unsigned long long host_ctr[3] = {0, 0, 0};
    if (e == cudaSuccess && stats) {
        e = cudaMemcpyAsync(host_ctr, a.ctr, ctr_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    dfree_on(scratch, st);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? ISO_ERR_OOM : ISO_ERR_CUDA;
    }
    if (stats) {
        stats->drawn = host_ctr[1];
        stats->big = host_ctr[2];
    }
    return ISO_OK;
}
