/*
 * Oracle ray caster: implicit isosurface ray casting over the block grid
 * used as a macrocell grid (the future work Section 4.6.2 proposes: blocks
 * as macrocells for space skipping, the isosurface of the trilinear
 * interpolant found inside them).  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).  Every float operation is one IEEE float32 operation (built
 * without FMA contraction), so the GPU's hit depths can be compared
 * exactly.  The rules:
 *
 *   ray        pixel (i, j) of a width x height image: u = (i + 0.5) / width
 *              * 2 - 1, v likewise with j and height; origin = eye,
 *              direction d = forward + u * right + v * up, t >= 0
 *   slab       the interval of t inside a box [lo, hi] (per axis: if
 *              d_a == 0 the axis admits every t when lo_a <= o_a <= hi_a,
 *              none otherwise; else (lo_a - o_a) r_a and (hi_a - o_a) r_a,
 *              ordered, with r_a = 1 / d_a rounded once per ray); t_in = max
 *              over axes, t_out = min, the exit axis is the first axis whose
 *              upper value is t_out
 *   cells      the dual cells of the samples: cell (x, y, z), x in
 *              [0, nx - 2], covers [x, x + 1] x ...; block b holds the cells
 *              x in [4 bx, min(4 bx + 3, nx - 2)], its box [4 bx, min(4 bx + 4,
 *              nx - 1)] (blocks without cells are not visited)
 *   traversal  start at max(0, t_in of the volume box [0, n - 1]); the block
 *              and then the cell containing o + t d (floor, clamped to the
 *              grid and to the block); from a box, move one step along its
 *              exit axis (the sign of d); stop when leaving the grid
 *   macrocell  a block is searched only when the range of its 2x2x2 block
 *              group (itself and its +x, +y, +z neighbours' samples inside
 *              the volume) contains iso: lo < iso <= hi
 *   cell       a cell of a searched block is tested when the range of its 8
 *              corners contains iso; on its interval [a, b] (a raised to the
 *              block's entry and to the ray start) g(t) = trilinear(o + t d)
 *              - iso is sampled at a + k h, h = (b - a) * 0.25, k = 0..3, and
 *              at b; at the first k where (g < 0) changes, 12 bisection steps
 *              (m = (lo + hi) * 0.5, keep the half whose ends differ) and the
 *              hit is t = (lo + hi) * 0.5; local coordinates p - cell origin
 *              are clamped to [0, 1]; trilinear = lerp in x, then y, then z
 *   output     per pixel (t bits << 32 | block id) of the first hit, ~0 for
 *              none; shading as the rasteriser (two-sided Lambert, base
 *              colour (0.85, 0.75, 0.55)) with the normal the gradient of
 *              the trilinear interpolant at the hit
 */
#include "oracle.h"
#include <math.h>
#include <string.h>

typedef struct {
    float o[3], d[3], inv[3];   /* inv = 1 / d (0 where d == 0: unused) */
} ray_t;

static uint32_t fbits(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* slab interval of the ray in box [lo, hi]; returns 0 if some axis is empty */
static int slab(const ray_t *r, const float lo[3], const float hi[3], float *tin, float *tout, int *exit_axis)
{
    float a = -INFINITY, b = INFINITY;
    int ax = -1;
    for (int k = 0; k < 3; k++) {
        if (r->d[k] == 0.0f) {
            if (r->o[k] < lo[k] || r->o[k] > hi[k]) return 0;
            continue;
        }
        float t0 = (lo[k] - r->o[k]) * r->inv[k], t1 = (hi[k] - r->o[k]) * r->inv[k];
        float mn = t0 < t1 ? t0 : t1, mx = t0 < t1 ? t1 : t0;
        if (mn > a) a = mn;
        if (mx < b) {
            b = mx;
            ax = k;
        }
    }
    *tin = a;
    *tout = b;
    *exit_axis = ax;
    return 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static float at(const float *f, int nx, int ny, int x, int y, int z) { return f[(int64_t)x + nx * ((int64_t)y + (int64_t)ny * z)]; }

static float trilinear(const float c[8], float fx, float fy, float fz)
{
    float c00 = c[0] + fx * (c[1] - c[0]), c10 = c[2] + fx * (c[3] - c[2]);
    float c01 = c[4] + fx * (c[5] - c[4]), c11 = c[6] + fx * (c[7] - c[6]);
    float c0 = c00 + fy * (c10 - c00), c1 = c01 + fy * (c11 - c01);
    return c0 + fz * (c1 - c0);
}

static float clamp01(float x) { return fminf(fmaxf(x, 0.0f), 1.0f); }

static float g_at(const ray_t *r, const float c[8], const int cell[3], float iso, float t)
{
    float fx = clamp01(r->o[0] + t * r->d[0] - (float)cell[0]);
    float fy = clamp01(r->o[1] + t * r->d[1] - (float)cell[1]);
    float fz = clamp01(r->o[2] + t * r->d[2] - (float)cell[2]);
    return trilinear(c, fx, fy, fz) - iso;
}

/* first crossing of the cell on [a, b]; 1 and *thit when found */
static int cell_root(const ray_t *r, const float c[8], const int cell[3], float iso, float a, float b, float *thit)
{
    float h = (b - a) * 0.25f;
    float tk = a;
    int sk = g_at(r, c, cell, iso, tk) < 0.0f;
    for (int k = 1; k <= 4; k++) {
        float tn = k == 4 ? b : a + h * (float)k;
        int sn = g_at(r, c, cell, iso, tn) < 0.0f;
        if (sn != sk) {
            float lo = tk, hi = tn;
            for (int it = 0; it < 12; it++) {
                float m = (lo + hi) * 0.5f;
                int sm = g_at(r, c, cell, iso, m) < 0.0f;
                if (sm == sk) lo = m;
                else hi = m;
            }
            *thit = (lo + hi) * 0.5f;
            return 1;
        }
        tk = tn;
        sk = sn;
    }
    return 0;
}

static void corners(const float *f, int nx, int ny, const int cell[3], float c[8])
{
    for (int k = 0; k < 8; k++) c[k] = at(f, nx, ny, cell[0] + (k & 1), cell[1] + (k >> 1 & 1), cell[2] + (k >> 2 & 1));
}

/* range of the samples of block b's 2x2x2 group inside the volume */
static void group_range(const float *f, int nx, int ny, int nz, const int b[3], float *lo, float *hi)
{
    float mn = INFINITY, mx = -INFINITY;
    for (int z = 4 * b[2]; z < 4 * b[2] + 8 && z < nz; z++)
        for (int y = 4 * b[1]; y < 4 * b[1] + 8 && y < ny; y++)
            for (int x = 4 * b[0]; x < 4 * b[0] + 8 && x < nx; x++) {
                float v = at(f, nx, ny, x, y, z);
                if (v < mn) mn = v;
                if (v > mx) mx = v;
            }
    *lo = mn;
    *hi = mx;
}

static int cast(const float *f, int nx, int ny, int nz, float iso, const ray_t *r, float *thit, int hit_cell[3],
                int hit_block[3])
{
    const int n[3] = {nx, ny, nz};
    int ncb[3];                                  /* blocks holding cells */
    for (int k = 0; k < 3; k++) {
        if (n[k] < 2) return 0;
        ncb[k] = (n[k] - 2) / 4 + 1;
    }
    float vlo[3] = {0.0f, 0.0f, 0.0f}, vhi[3] = {(float)(nx - 1), (float)(ny - 1), (float)(nz - 1)};
    float t0, t1;
    int ax;
    if (!slab(r, vlo, vhi, &t0, &t1, &ax)) return 0;
    if (t0 < 0.0f) t0 = 0.0f;
    if (!(t0 <= t1)) return 0;
    int b[3];
    for (int k = 0; k < 3; k++) b[k] = clampi((int)floorf((r->o[k] + t0 * r->d[k]) * 0.25f), 0, ncb[k] - 1);
    float t = t0;
    for (;;) {
        float blo[3], bhi[3];
        for (int k = 0; k < 3; k++) {
            blo[k] = (float)(4 * b[k]);
            int h = 4 * b[k] + 4;
            bhi[k] = (float)(h < n[k] - 1 ? h : n[k] - 1);
        }
        float bin, bout;
        int bax;
        if (!slab(r, blo, bhi, &bin, &bout, &bax) || bax < 0) return 0;
        if (bin < t) bin = t;
        float glo, ghi;
        group_range(f, nx, ny, nz, b, &glo, &ghi);
        if (bin <= bout && glo < iso && iso <= ghi) {
            int c[3];
            for (int k = 0; k < 3; k++) {
                int last = 4 * b[k] + 3 < n[k] - 2 ? 4 * b[k] + 3 : n[k] - 2;
                c[k] = clampi((int)floorf(r->o[k] + bin * r->d[k]), 4 * b[k], last);
            }
            for (;;) {
                float clo[3] = {(float)c[0], (float)c[1], (float)c[2]};
                float chi[3] = {(float)(c[0] + 1), (float)(c[1] + 1), (float)(c[2] + 1)};
                float cin, cout;
                int cax;
                if (!slab(r, clo, chi, &cin, &cout, &cax) || cax < 0) break;
                if (cin < bin) cin = bin;
                if (cin <= cout) {
                    float cv[8];
                    corners(f, nx, ny, c, cv);
                    float mn = cv[0], mx = cv[0];
                    for (int k = 1; k < 8; k++) {
                        mn = cv[k] < mn ? cv[k] : mn;
                        mx = cv[k] > mx ? cv[k] : mx;
                    }
                    if (mn < iso && iso <= mx && cell_root(r, cv, c, iso, cin, cout, thit)) {
                        memcpy(hit_cell, c, sizeof c);
                        memcpy(hit_block, b, sizeof c);
                        return 1;
                    }
                }
                c[cax] += r->d[cax] > 0.0f ? 1 : -1;
                int last = 4 * b[cax] + 3 < n[cax] - 2 ? 4 * b[cax] + 3 : n[cax] - 2;
                if (c[cax] < 4 * b[cax] || c[cax] > last) break;
            }
        }
        b[bax] += r->d[bax] > 0.0f ? 1 : -1;
        if (b[bax] < 0 || b[bax] >= ncb[bax]) return 0;
        t = bout;
    }
}

void orc_raycast(const float *field, int nx, int ny, int nz, float iso, const float eye[3], const float fwd[3],
                 const float right[3], const float up[3], const float light[3], int width, int height,
                 uint64_t *hits, uint32_t *rgba)
{
    const float base[3] = {0.85f, 0.75f, 0.55f};
    float l2 = light[0] * light[0] + light[1] * light[1] + light[2] * light[2];
    float linv = 1.0f / sqrtf(l2);
    float L[3] = {light[0] * linv, light[1] * linv, light[2] * linv};
    const int nbx = (nx + 3) / 4, nby = (ny + 3) / 4;
    for (int j = 0; j < height; j++) {
        for (int i = 0; i < width; i++) {
            float u = ((float)i + 0.5f) / (float)width * 2.0f - 1.0f;
            float v = ((float)j + 0.5f) / (float)height * 2.0f - 1.0f;
            ray_t r;
            for (int k = 0; k < 3; k++) {
                r.o[k] = eye[k];
                r.d[k] = fwd[k] + u * right[k] + v * up[k];
                r.inv[k] = r.d[k] == 0.0f ? 0.0f : 1.0f / r.d[k];
            }
            int64_t px = (int64_t)j * width + i;
            float t;
            int c[3], b[3];
            if (!cast(field, nx, ny, nz, iso, &r, &t, c, b)) {
                hits[px] = ~0ull;
                if (rgba) rgba[px] = 0;
                continue;
            }
            uint32_t id = (uint32_t)b[0] + (uint32_t)nbx * ((uint32_t)b[1] + (uint32_t)nby * (uint32_t)b[2]);
            hits[px] = ((uint64_t)fbits(t) << 32) | id;
            if (!rgba) continue;
            float cv[8];
            corners(field, nx, ny, c, cv);
            float fx = clamp01(r.o[0] + t * r.d[0] - (float)c[0]);
            float fy = clamp01(r.o[1] + t * r.d[1] - (float)c[1]);
            float fz = clamp01(r.o[2] + t * r.d[2] - (float)c[2]);
            float gx = (1.0f - fz) * ((1.0f - fy) * (cv[1] - cv[0]) + fy * (cv[3] - cv[2])) +
                       fz * ((1.0f - fy) * (cv[5] - cv[4]) + fy * (cv[7] - cv[6]));
            float gy = (1.0f - fz) * ((1.0f - fx) * (cv[2] - cv[0]) + fx * (cv[3] - cv[1])) +
                       fz * ((1.0f - fx) * (cv[6] - cv[4]) + fx * (cv[7] - cv[5]));
            float gz = (1.0f - fy) * ((1.0f - fx) * (cv[4] - cv[0]) + fx * (cv[5] - cv[1])) +
                       fy * ((1.0f - fx) * (cv[6] - cv[2]) + fx * (cv[7] - cv[3]));
            float n2 = gx * gx + gy * gy + gz * gz;
            float inten = 0.2f;
            if (n2 > 0.0f) {
                float cth = fabsf(gx * L[0] + gy * L[1] + gz * L[2]) / sqrtf(n2);
                inten = 0.2f + 0.8f * cth;
                if (inten > 1.0f) inten = 1.0f;
            }
            uint32_t out = 255u << 24;
            for (int a = 0; a < 3; a++) {
                float x = inten * base[a] * 255.0f + 0.5f;
                out |= ((uint32_t)x & 255u) << (8 * a);
            }
            rgba[px] = out;
        }
    }
}
