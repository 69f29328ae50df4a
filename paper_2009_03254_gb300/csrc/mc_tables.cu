// Marching-cubes case table of the library, built on the host when a
// volume is loaded.
//
// Marching cubes (Lorensen and Cline 1987, the per-cell step of paper
// Sections 4.4-4.5) needs, for each of the 256 below/above patterns of a
// cell's corners, the triangles to emit.  The paper prints no table; this
// one follows a rule chosen so that neighbouring cells always agree on a
// shared face:
//   walking a face's four corners counter-clockwise as seen from outside
//   the cell, every run of below-iso corners is cut off by one segment,
//   directed from the edge where the run starts to the edge where it ends
//   (a diagonal face therefore cuts off its two below corners separately);
//   the segments of the six faces link up through the cut edges into
//   closed cycles; cycles are taken in order of their smallest edge
//   number, each starting at that edge, and fanned from it.
// The resulting triangles have right-hand normals pointing toward the
// larger values.  Edges are numbered 4*axis + j, j giving the edge's
// offsets on the other two axes (in increasing axis order) as (j&1, j>>1).
#include <cstdint>
#include <cstring>

#include "mc_tables.cuh"

namespace bcmc {

namespace {

int edge_of(int c1, int c2) {
    const int d = c1 ^ c2;
    const int a = d == 1 ? 0 : (d == 2 ? 1 : 2);
    const int lo = c1 < c2 ? c1 : c2;
    int j = 0, bit = 0;
    for (int ax = 0; ax < 3; ax++) {
        if (ax == a) continue;
        j |= ((lo >> ax) & 1) << bit;
        bit++;
    }
    return 4 * a + j;
}

// the face's corners, counter-clockwise seen from outside
void face_ccw(int a, int s, int out[4]) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;      // (b, c, a) is right-handed
    static const int uv_pos[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};  // ccw seen from +a
    static const int uv_neg[4][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 0}};  // ccw seen from -a
    for (int i = 0; i < 4; i++) {
        const int *uv = s ? uv_pos[i] : uv_neg[i];
        out[i] = (s << a) | (uv[0] << b) | (uv[1] << c);
    }
}

}  // namespace

bool build_mc_tables(McTables *t) {
    std::memset(t, 0, sizeof(*t));
    for (int cs = 0; cs < 256; cs++) {
        int next[12], prev_count[12];
        for (int e = 0; e < 12; e++) { next[e] = -1; prev_count[e] = 0; }
        for (int a = 0; a < 3; a++)
            for (int s = 0; s < 2; s++) {
                int f[4];
                face_ccw(a, s, f);
                for (int i = 0; i < 4; i++) {
                    const int c0 = f[i], c1 = f[(i + 1) & 3];
                    if ((cs >> c0 & 1) || !(cs >> c1 & 1)) continue;   // not the start of a below run
                    int j = (i + 1) & 3;
                    while (cs >> f[(j + 1) & 3] & 1) j = (j + 1) & 3;  // walk to the run's last corner
                    const int e_in = edge_of(c0, c1), e_out = edge_of(f[j], f[(j + 1) & 3]);
                    if (next[e_in] != -1) return false;
                    next[e_in] = e_out;
                    prev_count[e_out]++;
                }
            }
        bool seen[12] = {};
        int nt = 0;
        for (int e0 = 0; e0 < 12; e0++) {
            if (next[e0] < 0 || seen[e0]) continue;
            if (prev_count[e0] != 1) return false;
            int cyc[12], len = 0, e = e0;
            do {
                if (len == 12 || next[e] < 0) return false;
                seen[e] = true;
                cyc[len++] = e;
                e = next[e];
            } while (e != e0);
            for (int k = 1; k + 1 < len; k++) {
                if (nt == kMaxTriPerCell) return false;
                t->tri_edges[cs][3 * nt + 0] = (uint8_t)cyc[0];
                t->tri_edges[cs][3 * nt + 1] = (uint8_t)cyc[k];
                t->tri_edges[cs][3 * nt + 2] = (uint8_t)cyc[k + 1];
                nt++;
            }
        }
        t->num_tri[cs] = (uint8_t)nt;
        if (nt > t->max_tri) t->max_tri = nt;
    }
    return true;
}

}  // namespace bcmc
