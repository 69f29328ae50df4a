/*
 * Oracle marching cubes and block rules.  TEST INFRASTRUCTURE ONLY (see
 * oracle.h).
 *
 * Marching cubes (Lorensen and Cline 1987, cited by the paper in Sections
 * 2 and 3.3.3): each cell of the voxel grid gets an 8-bit case from which
 * corners lie below the isovalue; a case table lists the triangles, whose
 * vertices sit on cut cell edges at the linearly interpolated crossing.
 * The paper prints no table, so this file builds one from a rule:
 *   - on a face whose four edges are all cut (the diagonal pattern) the
 *     segments cut off each below-iso corner on its own, so two cells that
 *     share the face always agree;
 *   - segments are directed so that, seen from outside the cube, the
 *     below-iso corners lie to their right; linked through the cut edges
 *     they form disjoint cycles whose right-hand normal points toward the
 *     increasing field;
 *   - cycles are listed by their smallest edge number, each starts at its
 *     smallest edge and is fanned from it.
 * Edges 0-3 run along x, 4-7 along y, 8-11 along z; edge 4a+j has the
 * offsets (j&1, j>>1) on the two other axes taken in increasing order.
 */
#include "oracle.h"
#include <assert.h>
#include <string.h>

static void corner_pos(int c, int p[3]) { p[0] = c & 1; p[1] = c >> 1 & 1; p[2] = c >> 2 & 1; }

void orc_edge_info(int e, int *lo_corner, int *hi_corner, int *axis)
{
    int a = e / 4, j = e % 4;
    int p[3] = {0, 0, 0};
    int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;   /* the other two axes, increasing */
    p[o1] = j & 1;
    p[o2] = j >> 1;
    int lo = p[0] | p[1] << 1 | p[2] << 2;
    *lo_corner = lo;
    *hi_corner = lo | 1 << a;
    *axis = a;
}

static void edge_mid(int e, double m[3])
{
    int lo, hi, a, p[3];
    orc_edge_info(e, &lo, &hi, &a);
    corner_pos(lo, p);
    for (int i = 0; i < 3; i++) m[i] = p[i];
    m[a] += 0.5;
}

/* is point c to the right of the directed segment a->b, seen from the side
 * the normal n points to? */
static int right_of(const double a[3], const double b[3], const double c[3], const double n[3])
{
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double x[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    return x[0] * n[0] + x[1] * n[1] + x[2] * n[2] < 0.0;
}

int orc_mc_table(uint8_t num_tri[256], uint8_t tri_edges[256][3 * ORC_MAX_TRI])
{
    int max_tri = 0;
    memset(tri_edges, 0, 256 * 3 * ORC_MAX_TRI);
    for (int cs = 0; cs < 256; cs++) {
        int below[8], cut[12], next[12], indeg[12];
        for (int c = 0; c < 8; c++) below[c] = cs >> c & 1;
        for (int e = 0; e < 12; e++) {
            int lo, hi, a;
            orc_edge_info(e, &lo, &hi, &a);
            cut[e] = below[lo] != below[hi];
            next[e] = -1;
            indeg[e] = 0;
        }
        for (int a = 0; a < 3; a++)
            for (int s = 0; s < 2; s++) {
                double n[3] = {0, 0, 0};
                n[a] = 2 * s - 1;                     /* outward normal of the face */
                int fc[4], nfc = 0, fe[4], nfe = 0;
                for (int c = 0; c < 8; c++) {
                    int p[3];
                    corner_pos(c, p);
                    if (p[a] == s) fc[nfc++] = c;
                }
                for (int e = 0; e < 12; e++) {
                    int lo, hi, ea;
                    orc_edge_info(e, &lo, &hi, &ea);
                    int p[3];
                    corner_pos(lo, p);
                    if (ea != a && p[a] == s && cut[e]) fe[nfe++] = e;
                }
                assert(nfc == 4 && (nfe == 0 || nfe == 2 || nfe == 4));
                for (int i = 0; i < 4; i++) {
                    int c = fc[i];
                    if (!below[c]) continue;
                    int inc[2], ninc = 0;                 /* cut face edges at corner c */
                    for (int k = 0; k < nfe; k++) {
                        int lo, hi, ea;
                        orc_edge_info(fe[k], &lo, &hi, &ea);
                        if (lo == c || hi == c) inc[ninc++] = fe[k];
                    }
                    int ea, eb;
                    if (nfe == 4) {                        /* diagonal face: cut off corner c alone */
                        assert(ninc == 2);
                        ea = inc[0]; eb = inc[1];
                    } else if (nfe == 2 && ninc >= 1) {    /* one segment; c lies on its below side */
                        ea = fe[0]; eb = fe[1];
                    } else {
                        continue;
                    }
                    double pa[3], pb[3], pc[3];
                    edge_mid(ea, pa);
                    edge_mid(eb, pb);
                    int cp[3];
                    corner_pos(c, cp);
                    pc[0] = cp[0]; pc[1] = cp[1]; pc[2] = cp[2];
                    if (!right_of(pa, pb, pc, n)) { int t = ea; ea = eb; eb = t; }
                    if (next[ea] == -1) { next[ea] = eb; indeg[eb]++; }
                    else assert(next[ea] == eb);          /* same segment seen from another corner */
                }
            }
        int visited[12] = {0}, nt = 0;
        for (int e0 = 0; e0 < 12; e0++) {
            if (!cut[e0]) continue;
            assert(next[e0] >= 0 && indeg[e0] == 1);
            if (visited[e0]) continue;
            int cyc[12], len = 0, e = e0;
            do { visited[e] = 1; cyc[len++] = e; e = next[e]; } while (e != e0);
            for (int i = 1; i + 1 < len; i++) {
                tri_edges[cs][3 * nt + 0] = (uint8_t)cyc[0];
                tri_edges[cs][3 * nt + 1] = (uint8_t)cyc[i];
                tri_edges[cs][3 * nt + 2] = (uint8_t)cyc[i + 1];
                nt++;
            }
        }
        assert(nt <= ORC_MAX_TRI);
        num_tri[cs] = (uint8_t)nt;
        if (nt > max_tri) max_tri = nt;
    }
    return max_tri;
}

/* ---------------- plain marching cubes over the whole volume ---------------- */

static uint8_t g_num[256];
static uint8_t g_tri[256][3 * ORC_MAX_TRI];
static int g_ready = 0;

static void ensure_table(void)
{
    if (!g_ready) { orc_mc_table(g_num, g_tri); g_ready = 1; }
}

#define AT(f, x, y, z) (f)[(int64_t)(x) + (int64_t)nx * ((int64_t)(y) + (int64_t)ny * (int64_t)(z))]

static int case_of_cell(const float *f, int nx, int ny, int x, int y, int z, float iso)
{
    int cs = 0;
    for (int c = 0; c < 8; c++)
        if (AT(f, x + (c & 1), y + (c >> 1 & 1), z + (c >> 2 & 1)) < iso) cs |= 1 << c;
    return cs;
}

/* vertex on edge e of the cell with min corner (x,y,z): global edge id and
 * global position, the crossing interpolated in float64 */
static void edge_vertex(const float *f, int nx, int ny, int x, int y, int z, int e, float iso,
                        uint64_t *id, double pos[3])
{
    int lo, hi, a, p[3];
    orc_edge_info(e, &lo, &hi, &a);
    corner_pos(lo, p);
    int q[3] = {x + p[0], y + p[1], z + p[2]};
    int r[3] = {q[0], q[1], q[2]};
    r[a] += 1;
    double vlo = AT(f, q[0], q[1], q[2]), vhi = AT(f, r[0], r[1], r[2]);
    double t = ((double)iso - vlo) / (vhi - vlo);
    *id = 3 * ((uint64_t)q[0] + (uint64_t)nx * ((uint64_t)q[1] + (uint64_t)ny * (uint64_t)q[2])) + (uint64_t)a;
    pos[0] = q[0]; pos[1] = q[1]; pos[2] = q[2];
    pos[a] += t;
}

/* Every cell (x,y,z) with x <= nx-2, y <= ny-2, z <= nz-2, in z, y, x order.
 * Writes up to cap triangles (3 edge ids, 9 doubles and the linear index
 * of the cell's min corner each); returns the total count. */
int64_t orc_mc_full(const float *field, int nx, int ny, int nz, float iso,
                    uint64_t *edge_ids, double *pos, int64_t *cell_of_tri, int64_t cap)
{
    ensure_table();
    int64_t t = 0;
    for (int z = 0; z + 1 < nz; z++)
        for (int y = 0; y + 1 < ny; y++)
            for (int x = 0; x + 1 < nx; x++) {
                int cs = case_of_cell(field, nx, ny, x, y, z, iso);
                for (int k = 0; k < g_num[cs]; k++, t++) {
                    if (t >= cap) continue;
                    if (cell_of_tri) cell_of_tri[t] = x + (int64_t)nx * (y + (int64_t)ny * z);
                    for (int v = 0; v < 3; v++)
                        edge_vertex(field, nx, ny, x, y, z, g_tri[cs][3 * k + v], iso,
                                    edge_ids + 3 * t + v, pos + 9 * t + 3 * v);
                }
            }
    return t;
}

/* ---------------- block rules (Sections 4.1 - 4.5) ---------------- */

/* range [lo, hi] contains iso  <=>  lo < iso <= hi  (matches the case
 * convention: a corner equal to iso counts as not below) */
static int contains(float lo, float hi, float iso) { return lo < iso && iso <= hi; }

/* Section 4.1: a block is active if its own range, or the union of its
 * range with the range of any of its 26 neighbours inside the block grid,
 * contains the isovalue. */
void orc_active_blocks(const float *bmin, const float *bmax, int nbx, int nby, int nbz,
                       float iso, uint8_t *active)
{
    for (int bz = 0; bz < nbz; bz++)
        for (int by = 0; by < nby; by++)
            for (int bx = 0; bx < nbx; bx++) {
                int64_t b = bx + (int64_t)nbx * (by + (int64_t)nby * bz);
                int act = contains(bmin[b], bmax[b], iso);
                for (int dz = -1; dz <= 1 && !act; dz++)
                    for (int dy = -1; dy <= 1 && !act; dy++)
                        for (int dx = -1; dx <= 1 && !act; dx++) {
                            int x = bx + dx, y = by + dy, z = bz + dz;
                            if ((dx | dy | dz) == 0) continue;
                            if (x < 0 || y < 0 || z < 0 || x >= nbx || y >= nby || z >= nbz) continue;
                            int64_t n = x + (int64_t)nbx * (y + (int64_t)nby * z);
                            float lo = bmin[b] < bmin[n] ? bmin[b] : bmin[n];
                            float hi = bmax[b] > bmax[n] ? bmax[b] : bmax[n];
                            act = contains(lo, hi, iso);
                        }
                active[b] = (uint8_t)act;
            }
}

/* Sections 4.3-4.5 for the active blocks ids[0..n_ids) (ascending):
 * extents start at 5 along each axis where a +neighbour block exists and
 * drop back to 4 along the axes of any needed +neighbour (face, edge or
 * corner) that is not active; the block's dual cells inside those extents
 * and inside the volume are classified and counted; per-block triangle
 * counts are prefix-summed into output offsets; triangles are written in
 * block order, then cell order (x fastest), then table order.  Positions
 * are block-local: global minus 4 * block coordinates.
 * complete[i] = 1 when no extent was reset.  Returns the triangle total. */
int64_t orc_mc_blocks(const float *field, int nx, int ny, int nz, float iso,
                      const uint8_t *active, const uint32_t *ids, int64_t n_ids,
                      uint8_t *cell_case, uint8_t *cell_count, uint8_t *complete,
                      uint32_t *block_tri, uint64_t *block_off,
                      uint64_t *edge_ids, double *local_pos, uint32_t *tri_block, int64_t cap)
{
    ensure_table();
    int nbx = (nx + 3) / 4, nby = (ny + 3) / 4, nbz = (nz + 3) / 4;
    int64_t t = 0;
    for (int64_t i = 0; i < n_ids; i++) {
        uint32_t b = ids[i];
        int bc[3] = {(int)(b % nbx), (int)(b / nbx % nby), (int)(b / nbx / nby)};
        int nbd[3] = {nbx, nby, nbz};
        int ext[3];
        for (int a = 0; a < 3; a++) ext[a] = bc[a] + 1 < nbd[a] ? 5 : 4;
        int changed = 1, reset = 0;
        while (changed) {
            changed = 0;
            for (int o = 1; o < 8; o++) {
                int need = 1;
                for (int a = 0; a < 3; a++) if ((o >> a & 1) && ext[a] != 5) need = 0;
                if (!need) continue;
                int64_t n = (bc[0] + (o & 1)) + (int64_t)nbx * ((bc[1] + (o >> 1 & 1)) + (int64_t)nby * (bc[2] + (o >> 2 & 1)));
                if (!active[n]) {
                    for (int a = 0; a < 3; a++) if (o >> a & 1) ext[a] = 4;
                    changed = 1;
                    reset = 1;
                }
            }
        }
        complete[i] = (uint8_t)!reset;
        block_off[i] = (uint64_t)t;
        uint32_t cnt = 0;
        for (int c = 0; c < 64; c++) {
            int cx = c & 3, cy = c >> 2 & 3, cz = c >> 4;
            int x = 4 * bc[0] + cx, y = 4 * bc[1] + cy, z = 4 * bc[2] + cz;
            int inside = cx + 1 < ext[0] && cy + 1 < ext[1] && cz + 1 < ext[2] &&
                         x + 1 < nx && y + 1 < ny && z + 1 < nz;
            int cs = inside ? case_of_cell(field, nx, ny, x, y, z, iso) : 0;
            cell_case[64 * i + c] = (uint8_t)cs;
            cell_count[64 * i + c] = g_num[cs];
            for (int k = 0; k < g_num[cs]; k++, t++) {
                if (t >= cap) continue;
                tri_block[t] = b;
                for (int v = 0; v < 3; v++) {
                    double *p = local_pos + 9 * t + 3 * v;
                    edge_vertex(field, nx, ny, x, y, z, g_tri[cs][3 * k + v], iso, edge_ids + 3 * t + v, p);
                    p[0] -= 4 * bc[0]; p[1] -= 4 * bc[1]; p[2] -= 4 * bc[2];
                }
            }
            cnt += g_num[cs];
        }
        block_tri[i] = cnt;
    }
    return t;
}
