/*
 * Oracle rasteriser for the rendering step of Section 4.6.2.  TEST
 * INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper draws the extracted triangle soup, in its compressed vertex
 * format, with WebGPU (Section 4.5: the block position comes from the
 * block id and offsets the dequantised vertex).  Here the image is defined
 * directly, with every float32 operation spelled out (this file is built
 * without FMA contraction), so that coverage and depth, which floating
 * point decides, can be compared exactly:
 *
 *   world position   block origin (4 bx, 4 by, 4 bz) of the vertex's block
 *                    id (x fastest) + its block-local position (float4
 *                    format), or + code * (4 / 1023) (compact format)
 *   clip             (X, Y, Z, W) = M (x, y, z, 1), M row-major, each row
 *                    summed left to right; a triangle with a vertex at
 *                    W <= 0 is not drawn (no clipping)
 *   screen           r = 1 / W, sx = (X r * 0.5 + 0.5) * width, sy likewise
 *                    with height (y up), depth d = Z r * 0.5 + 0.5
 *   edge function    E(a, b; p) = (b.x - a.x)(p.y - a.y) - (b.y - a.y)(p.x - a.x),
 *                    always evaluated with the endpoints in ascending
 *                    (x, then y) order and negated when swapped, so that two
 *                    triangles sharing an edge see exactly opposite values
 *   orientation      A = E(v0, v1; v2); A == 0: not drawn; A < 0: v1 and v2
 *                    swap and A is evaluated again (not drawn unless > 0)
 *   coverage         pixel (i, j), centre (i + 0.5, j + 0.5), inside the
 *                    bounding box of the screen vertices: i from
 *                    max(0, ceil(min sx - 0.5)) to min(width - 1,
 *                    floor(max sx - 0.5)), j likewise; covered when
 *                    e0 = E(v1, v2), e1 = E(v2, v0), e2 = E(v0, v1) are all
 *                    >= 0, a zero only on a top-left edge (dy < 0, or
 *                    dy == 0 and dx < 0, for the edge's direction in the
 *                    counter-clockwise triangle)
 *   depth            d = ((e0 d0 + e1 d1) + e2 d2) / A, + 0 (no negative
 *                    zero); fragments with d outside [0, 1] are dropped
 *   visibility       per pixel the smallest (depth bits << 32 | triangle)
 *   indexed input    a triangle with an index past the vertex count is not
 *                    drawn
 *   shading          n = (p1 - p0) x (p2 - p0) in world space;
 *                    intensity = 0.2 + 0.8 |n . L| / |n| (0.2 when |n| = 0,
 *                    L normalised), rgb = floor(intensity * base * 255 + 0.5)
 *                    with base (0.85, 0.75, 0.55), alpha 255; background 0
 */
#include "oracle.h"
#include <math.h>
#include <string.h>

#define BLOCK_CODE_SCALE 0.0039100684f      /* 4 / 1023 rounded to float */

typedef struct {
    float x, y;
} pt2;

static uint32_t fbits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* world position of vertex k (soup: 3t + j; indexed: idx[3t + j]) */
static void world(const void *verts, int format, int64_t k, int nx, int ny, float p[3])
{
    const int nbx = (nx + 3) / 4, nby = (ny + 3) / 4;
    uint32_t id;
    float local[3];
    if (format == 0) {
        const float *v = (const float *)verts + 4 * k;
        local[0] = v[0];
        local[1] = v[1];
        local[2] = v[2];
        id = fbits(v[3]);
    } else {
        const uint32_t *v = (const uint32_t *)verts + 2 * k;
        for (int a = 0; a < 3; a++) local[a] = (float)((v[0] >> (10 * a)) & 1023u) * BLOCK_CODE_SCALE;
        id = v[1];
    }
    const uint32_t bx = id % (uint32_t)nbx, by = (id / (uint32_t)nbx) % (uint32_t)nby,
                   bz = id / ((uint32_t)nbx * (uint32_t)nby);
    p[0] = (float)(4 * bx) + local[0];
    p[1] = (float)(4 * by) + local[1];
    p[2] = (float)(4 * bz) + local[2];
}

static float edge(pt2 a, pt2 b, float px, float py)
{
    int swap = (b.x < a.x) || (b.x == a.x && b.y < a.y);
    if (swap) {
        pt2 t = a;
        a = b;
        b = t;
    }
    float e = (b.x - a.x) * (py - a.y) - (b.y - a.y) * (px - a.x);
    return swap ? -e : e;
}

static int top_left(pt2 a, pt2 b)
{
    float dx = b.x - a.x, dy = b.y - a.y;
    return dy < 0.0f || (dy == 0.0f && dx < 0.0f);
}

static int64_t vertex_index(const uint32_t *idx, int64_t t, int j)
{
    return idx ? (int64_t)idx[3 * t + j] : 3 * t + j;
}

void orc_raster(const void *verts, int format, const uint32_t *idx, int64_t num_vtx, int64_t num_tri, int nx,
                int ny, int nz, const float m[16], int width, int height, uint64_t *frag)
{
    (void)nz;
    for (int64_t i = 0; i < (int64_t)width * height; i++) frag[i] = ~0ull;
    for (int64_t t = 0; t < num_tri; t++) {
        pt2 s[3];
        float d[3];
        int behind = 0;
        if (idx && (idx[3 * t] >= num_vtx || idx[3 * t + 1] >= num_vtx || idx[3 * t + 2] >= num_vtx))
            continue;                            /* an index past the vertex buffer: not drawn */
        for (int j = 0; j < 3; j++) {
            float p[3];
            world(verts, format, vertex_index(idx, t, j), nx, ny, p);
            float X = m[0] * p[0] + m[1] * p[1] + m[2] * p[2] + m[3];
            float Y = m[4] * p[0] + m[5] * p[1] + m[6] * p[2] + m[7];
            float Z = m[8] * p[0] + m[9] * p[1] + m[10] * p[2] + m[11];
            float W = m[12] * p[0] + m[13] * p[1] + m[14] * p[2] + m[15];
            if (!(W > 0.0f)) behind = 1;
            float rw = 1.0f / W;
            s[j].x = (X * rw * 0.5f + 0.5f) * (float)width;
            s[j].y = (Y * rw * 0.5f + 0.5f) * (float)height;
            d[j] = Z * rw * 0.5f + 0.5f;
        }
        if (behind) continue;
        float A = edge(s[0], s[1], s[2].x, s[2].y);
        if (A == 0.0f || A != A) continue;
        if (A < 0.0f) {
            pt2 ts = s[1];
            s[1] = s[2];
            s[2] = ts;
            float td = d[1];
            d[1] = d[2];
            d[2] = td;
            A = edge(s[0], s[1], s[2].x, s[2].y);
            if (!(A > 0.0f)) continue;
        }
        float xmin = fminf(fminf(s[0].x, s[1].x), s[2].x), xmax = fmaxf(fmaxf(s[0].x, s[1].x), s[2].x);
        float ymin = fminf(fminf(s[0].y, s[1].y), s[2].y), ymax = fmaxf(fmaxf(s[0].y, s[1].y), s[2].y);
        float fi0 = ceilf(xmin - 0.5f), fi1 = floorf(xmax - 0.5f);
        float fj0 = ceilf(ymin - 0.5f), fj1 = floorf(ymax - 0.5f);
        if (fi1 < 0.0f || fj1 < 0.0f || fi0 > (float)(width - 1) || fj0 > (float)(height - 1)) continue;
        int i0 = fi0 < 0.0f ? 0 : (int)fi0, i1 = fi1 > (float)(width - 1) ? width - 1 : (int)fi1;
        int j0 = fj0 < 0.0f ? 0 : (int)fj0, j1 = fj1 > (float)(height - 1) ? height - 1 : (int)fj1;
        int tl0 = top_left(s[1], s[2]), tl1 = top_left(s[2], s[0]), tl2 = top_left(s[0], s[1]);
        for (int j = j0; j <= j1; j++) {
            for (int i = i0; i <= i1; i++) {
                float px = (float)i + 0.5f, py = (float)j + 0.5f;
                float e0 = edge(s[1], s[2], px, py), e1 = edge(s[2], s[0], px, py), e2 = edge(s[0], s[1], px, py);
                if (e0 < 0.0f || e1 < 0.0f || e2 < 0.0f) continue;
                if ((e0 == 0.0f && !tl0) || (e1 == 0.0f && !tl1) || (e2 == 0.0f && !tl2)) continue;
                float dd = (e0 * d[0] + e1 * d[1] + e2 * d[2]) / A + 0.0f;
                if (!(dd >= 0.0f && dd <= 1.0f)) continue;
                uint64_t key = ((uint64_t)fbits(dd) << 32) | (uint64_t)(uint32_t)t;
                uint64_t *f = &frag[(int64_t)j * width + i];
                if (key < *f) *f = key;
            }
        }
    }
}

void orc_shade(const void *verts, int format, const uint32_t *idx, int nx, int ny, int nz, const float light[3],
               int width, int height, const uint64_t *frag, uint32_t *rgba)
{
    (void)nz;
    const float base[3] = {0.85f, 0.75f, 0.55f};
    float l2 = light[0] * light[0] + light[1] * light[1] + light[2] * light[2];
    float linv = 1.0f / sqrtf(l2);
    float L[3] = {light[0] * linv, light[1] * linv, light[2] * linv};
    for (int64_t k = 0; k < (int64_t)width * height; k++) {
        if (frag[k] == ~0ull) {
            rgba[k] = 0;
            continue;
        }
        int64_t t = (int64_t)(uint32_t)frag[k];
        float p[3][3];
        for (int j = 0; j < 3; j++) world(verts, format, vertex_index(idx, t, j), nx, ny, p[j]);
        float u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
        float v[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
        float n[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        float n2 = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
        float inten = 0.2f;
        if (n2 > 0.0f) {
            float c = fabsf(n[0] * L[0] + n[1] * L[1] + n[2] * L[2]) / sqrtf(n2);
            inten = 0.2f + 0.8f * c;
            if (inten > 1.0f) inten = 1.0f;
        }
        uint32_t out = 255u << 24;
        for (int a = 0; a < 3; a++) {
            float x = inten * base[a] * 255.0f + 0.5f;
            out |= ((uint32_t)x & 255u) << (8 * a);
        }
        rgba[k] = out;
    }
}
