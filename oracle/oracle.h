/*
 * Plain CPU oracle for block-compressed isosurface extraction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this code: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no source with the CUDA library.
 *
 * Contents
 *   codec.c  fixed-rate 4x4x4 block codec in the style of ZFP's fixed-rate
 *            mode (paper Section 3.3.4 and Section 4.2.1; Lindstrom, "Fixed-
 *            rate compressed floating-point arrays", TVCG 2014), encoder and
 *            decoder, plus the per-block value ranges of Section 4.1.
 *   mc.c     marching-cubes case table built from a stated face rule, plain
 *            full-volume marching cubes, and the block-level rules of
 *            Sections 4.1-4.5 (active blocks, halo extents, occupied
 *            blocks, per-block counts and offsets, block-ordered output).
 *   raster.c the rendering step of Section 4.6.2 defined on the CPU:
 *            rasterisation of a triangle soup or indexed mesh in either
 *            vertex format to a depth | triangle-id buffer, and shading.
 *
 *   raycast.c implicit isosurface ray casting with the blocks as a
 *            macrocell grid (the future work of Section 4.6.2).
 *
 * Conventions
 *   voxel (x,y,z) of an nx*ny*nz volume sits at x + nx*(y + ny*z);
 *   block (bx,by,bz) has id bx + nbx*(by + nby*bz), nb* = ceil(n* / 4);
 *   voxel (i,j,k) inside a block sits at i + 4*j + 16*k;
 *   cell corner c has offset (c&1, (c>>1)&1, (c>>2)&1); case bit c is set
 *   iff the corner value is < iso.
 */
#ifndef BCMC_ORACLE_H
#define BCMC_ORACLE_H
#include <stdint.h>

#define ORC_PRECISION 27      /* block-floating-point integer precision */
#define ORC_MAX_TRI 12        /* upper bound on triangles per cell in the table */

/* ---- codec ---- */
void orc_encode_block(const float v[64], int rate, uint64_t *out);
void orc_decode_block(const uint64_t *in, int rate, float v[64]);
void orc_encode_volume(const float *field, int nx, int ny, int nz, int rate,
                       uint64_t *bits, float *bmin, float *bmax);
void orc_decode_volume(const uint64_t *bits, int nx, int ny, int nz, int rate, float *field);
void orc_decode_blocks(const uint64_t *bits, int rate, const uint32_t *ids, int64_t n, float *out);
void orc_coding_order(int perm[64]);
uint32_t orc_to_negabinary(int64_t x);
int32_t orc_from_negabinary(uint32_t u);
void orc_forward_lift(int64_t q[64]);
void orc_inverse_lift(int64_t q[64]);

/* ---- marching cubes ---- */
int orc_mc_table(uint8_t num_tri[256], uint8_t tri_edges[256][3 * ORC_MAX_TRI]);
void orc_edge_info(int e, int *lo_corner, int *hi_corner, int *axis);
int64_t orc_mc_full(const float *field, int nx, int ny, int nz, float iso,
                    uint64_t *edge_ids, double *pos, int64_t *cell_of_tri, int64_t cap);
void orc_active_blocks(const float *bmin, const float *bmax, int nbx, int nby, int nbz,
                       float iso, uint8_t *active);
int64_t orc_mc_blocks(const float *field, int nx, int ny, int nz, float iso,
                      const uint8_t *active, const uint32_t *ids, int64_t n_ids,
                      uint8_t *cell_case, uint8_t *cell_count, uint8_t *complete,
                      uint32_t *block_tri, uint64_t *block_off,
                      uint64_t *edge_ids, double *local_pos, uint32_t *tri_block, int64_t cap);

/* ---- rendering (raster.c) ---- */
void orc_raster(const void *verts, int format, const uint32_t *idx, int64_t num_vtx, int64_t num_tri, int nx,
                int ny, int nz, const float m[16], int width, int height, uint64_t *frag);
void orc_shade(const void *verts, int format, const uint32_t *idx, int nx, int ny, int nz, const float light[3],
               int width, int height, const uint64_t *frag, uint32_t *rgba);

/* ---- ray casting over the block macrocell grid (raycast.c) ---- */
void orc_raycast(const float *field, int nx, int ny, int nz, float iso, const float eye[3], const float fwd[3],
                 const float right[3], const float up[3], const float light[3], int width, int height,
                 uint64_t *hits, uint32_t *rgba);
#endif
