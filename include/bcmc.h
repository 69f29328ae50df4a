/*
 * bcmc.h -- C ABI of the GB300 block-compressed marching-cubes library.
 *
 * The library computes isosurfaces of a volume that is held on the GPU in
 * a fixed-rate block-compressed form, following the method of Usher and
 * Pascucci, "Interactive Visualization of Terascale Data in the Browser:
 * Fact or Fiction?" (arXiv 2009.03254), Section 4:
 *   - select the 4x4x4 blocks whose value range, or whose range joined
 *     with a neighbour's, contains the isovalue (Section 4.1);
 *   - find which of them are in a GPU-resident LRU cache of decoded
 *     blocks, give the others the least recently used free slots, and
 *     decode them into those slots (Section 4.2, Algorithm 1; 4.2.1);
 *   - run marching cubes over each active block and its +x/+y/+z halo
 *     (Section 4.3), count triangles per block and prefix-sum the counts
 *     into output offsets (Section 4.4), and write the triangles
 *     (Section 4.5).
 * Everything runs on the device; one small readback returns the counts.
 *
 * Conventions used throughout:
 *   - volumes are nx*ny*nz float32 samples, x fastest; the sample (x,y,z)
 *     is at x + nx*(y + ny*z);
 *   - blocks are 4x4x4 samples; nbx = ceil(nx/4) etc.; block (bx,by,bz)
 *     has id bx + nbx*(by + nby*bz); inside a block, sample (i,j,k) is at
 *     i + 4*j + 16*k; samples past the volume edge repeat the last one;
 *   - the compressed volume is nb = nbx*nby*nbz blocks of exactly
 *     rate*64 bits (rate 64-bit little-endian words) each, block b at word
 *     b*rate; the bit format is the library's ZFP-style fixed-rate format
 *     (block exponent, reversible integer lifting, sequency order,
 *     negabinary, group-tested bit planes), not libzfp's;
 *   - a cell is classified with bit c set iff its corner c =
 *     (c&1, (c>>1)&1, (c>>2)&1) is < iso; a value equal to iso is "above";
 *   - vertices are float4 {x, y, z, w}: x,y,z in [0,4] relative to the
 *     block origin 4*(bx,by,bz), w = the block id as uint32 bits; three
 *     consecutive vertices form one triangle whose right-hand normal
 *     points toward increasing values; triangles are ordered by block id,
 *     then cell (x fastest), then case-table order;
 *   - caller device buffers the library writes or reads as arrays must be
 *     aligned to their element: 16 bytes for float4 vertices, 8 for compact
 *     vertices, fragments and hits, 4 for indices and RGBA pixels; a
 *     misaligned one is refused with ISO_ERR_INVALID_ARG.
 *
 * Errors: every int-returning call returns ISO_OK or one of ISO_ERR_*;
 * no call throws or aborts.  A failed call leaves its outputs unspecified
 * and the volume usable, except ISO_ERR_CUDA, after which the CUDA context
 * may be unusable.
 *
 * Threads and streams: a volume is used by one host thread at a time.  All
 * of its device work is issued on the stream given at load (or set with
 * iso_set_stream).  Blocking calls synchronise that stream only.
 */
#ifndef BCMC_H
#define BCMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ISO_OK 0
#define ISO_ERR_INVALID_ARG 1  /* bad pointer, size, rate, dims or a non-finite isovalue */
#define ISO_ERR_OOM 2          /* a device or pinned-host allocation failed */
#define ISO_ERR_BUDGET 3       /* the active blocks do not fit in the cache budget */
#define ISO_ERR_CUDA 4         /* a CUDA runtime call failed */
#define ISO_ERR_TIMEOUT 5      /* a device-side wait gave up (bounded spin) */
#define ISO_ERR_CAPACITY 6     /* the caller's vertex buffer is too small */
#define ISO_PENDING 7          /* a served request is not finished yet (not an error) */
#define ISO_ERR_BOUNDS 9       /* checked builds only (BCMC_CHECKED): a device index fell outside its
                                  array; the access was skipped and the results are invalid (a
                                  library defect, reported instead of a memory fault) */
#define ISO_ERR_CORRUPT 8      /* the block ranges given at load are not ranges (NaN, or min > max);
                                  from iso_load_volume, or with ISO_ASYNC_UPLOAD from the calls on
                                  the volume */

/* iso_options.flags */
#define ISO_INPUT_ON_DEVICE 1u /* compressed/block_min/block_max are device pointers */
#define ISO_DEBUG 2u           /* keep per-stage debug copies (see iso_debug_get) */
#define ISO_ASYNC_UPLOAD 8u    /* host inputs: return once the load's work and the bitstream's copy
                                  are queued (the copy on a stream of the library's, after the
                                  ranges); the first extraction's range test and cache update
                                  overlap the copy and its decode waits for it.  The caller keeps
                                  `compressed` valid until the first call on the volume returns
                                  (pinned memory makes the copies asynchronous).  Ranges that are
                                  not ranges are then reported as ISO_ERR_CORRUPT by the first
                                  call on the volume, and by every call after it, instead of by
                                  iso_load_volume; iso_release still frees the volume */
#define ISO_NO_GRAPH 4u        /* launch each extraction's kernels one by one instead of
                                  replaying the CUDA graphs captured once a volume has been extracted 8 times */
#define ISO_SEGMENT_CULL 16u   /* keep a range per segment of 64 consecutive blocks (the hull of their
                                  3x3x3 ranges, 8 bytes per segment); the range test reads it first and
                                  skips the per-block reads of segments whose range cannot hold the
                                  isovalue (the same active set: a block's range lies within its
                                  segment's).  One more dependent read per tile: by default on only for
                                  volumes of at least 2^28 blocks, where most of the range test's time
                                  is those reads */
#define ISO_NO_SEGMENT_CULL 32u /* never keep segment ranges (ISO_SEGMENT_CULL wins if both are set) */

typedef struct iso_volume iso_volume;

typedef struct iso_options {
    uint32_t flags;            /* ISO_INPUT_ON_DEVICE | ISO_DEBUG | ISO_NO_GRAPH | ISO_ASYNC_UPLOAD |
                                  ISO_SEGMENT_CULL | ISO_NO_SEGMENT_CULL */
    uint32_t reserved;
    void *stream;              /* cudaStream_t for all device work; NULL = default stream */
    double initial_cache_fraction; /* initial slots as a fraction of nb; <= 0 means 0.1 (Section 4.2) */
    uint64_t cache_budget_bytes;   /* cap on decoded-block storage (256 B per slot); 0 = nb slots */
} iso_options;

typedef struct iso_stats {
    uint64_t num_triangles;    /* T: triangles of this surface */
    uint32_t n_active;         /* blocks selected by the range test (Section 4.1) */
    uint32_t n_new;            /* active blocks that were not cached and were decoded */
    uint32_t n_occupied;       /* active blocks that emit at least one triangle */
    uint32_t n_slots;          /* cache slots in use after growth */
    uint64_t cache_bytes;      /* n_slots * 256 */
    uint32_t epoch;            /* 1-based count of extractions on this volume */
    uint32_t reruns;           /* 1 if the output was produced twice to fit (only an over-budget
                                  iso_extract in waves whose first size guess was too small) */
    uint32_t n_candidates;     /* active blocks whose 2x2x2 +group range contains iso: the
                                  blocks the triangle stage visits */
    uint32_t waves;            /* passes: 1, or the number of waves of an extraction whose active
                                  blocks exceed the cache (see iso_extract) */
    uint64_t num_vertices;     /* vertices of an indexed mesh (iso_extract_indexed_into); else 0 */
} iso_stats;

typedef struct iso_mesh {
    float *d_vertices;         /* device float4[3 * num_triangles], owned by the library */
    uint64_t num_triangles;
    uint64_t capacity_triangles;
    iso_stats stats;
    void *priv;                /* library bookkeeping; do not touch */
} iso_mesh;

/* Device memory.  By default the library allocates from a stream-ordered
 * memory pool of its own per device, which keeps freed memory for reuse.
 * iso_set_allocator routes every later device allocation of the library
 * (volume state, meshes, scratch of batches, servers and renders) through
 * the caller: alloc(bytes, device, stream, ctx) returns memory usable in
 * the order of `stream` (NULL for failure: ISO_ERR_OOM), free(ptr, device,
 * stream, ctx) takes it back in that stream's order (a PyTorch caching
 * allocator fits both).  Each allocation is returned to the allocator that
 * made it, even after the hook changes.  alloc and free must both be set or
 * both be NULL (NULL: back to the pool).  Process-wide; call it while no
 * other thread is inside the library. */
typedef void *(*iso_alloc_fn)(size_t bytes, int device, void *stream, void *ctx);
typedef void (*iso_free_fn)(void *ptr, int device, void *stream, void *ctx);
int iso_set_allocator(iso_alloc_fn alloc, iso_free_fn free_fn, void *ctx);

/* Give the freed memory the library's pool keeps on `device` back to the
 * device, so that other allocators (a PyTorch caching allocator, cudaMalloc)
 * can use it; memory in use is untouched.  The small pinned host buffers
 * and the streams that released volumes left for later loads are freed
 * too.  Waits for all work on the device first (cudaDeviceSynchronize).  An allocation the pool cannot satisfy does
 * the same once by itself and retries before it reports ISO_ERR_OOM.
 * ISO_ERR_INVALID_ARG for a device without a pool of the library (nothing
 * was ever allocated there from it). */
int iso_release_cached_memory(int device);

/* Upload a compressed volume and set up its cache (Section 4: "uploading
 * the ZFP fixed-rate compressed data to the GPU"; Section 4.1: "precompute
 * and store the value range of each block when loading the data").
 *   compressed       nb*rate uint64 words (layout above), compressed_bytes
 *                    must equal nb*rate*8
 *   nx, ny, nz       volume size in samples, each >= 1
 *   rate_bits        bits per sample, 1..32
 *   block_min/max    per-block range over the block's in-volume samples AS
 *                    DECODED (nb floats each); the block method reproduces
 *                    full-volume marching cubes of the decoded field only
 *                    with ranges of the decoded values
 *   opt              may be NULL (defaults above)
 * Host inputs are copied; the caller keeps ownership.  With
 * ISO_INPUT_ON_DEVICE they are copied device-to-device.  On success *out
 * owns all device state until iso_release.  Blocks until the upload is done. */
int iso_load_volume(iso_volume **out, const void *compressed, size_t compressed_bytes,
                    uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate_bits,
                    const float *block_min, const float *block_max, const iso_options *opt);

/* Compute the isosurface at `isovalue` (Sections 4.1-4.5).  The vertex
 * buffer is allocated by the library (stream-ordered) and owned by
 * *out until iso_mesh_release.  Runs the stages up to the prefix sum,
 * waits for the triangle count, allocates the mesh at its exact size and
 * runs the emission (blocks until done).  isovalue must be finite.
 * Over budget (the paper always grows the cache; this library caps it):
 * when the surface's active blocks do not fit in the cache even at the
 * cap, the surface is extracted in waves of consecutive z-layers of blocks,
 * each wave's active blocks together with those of the layer after it
 * fitting in the cache; the triangles come out in the same order as from
 * one pass (stats.waves > 1; stats then sum over the waves, n_active
 * counting each block once; debug arrays describe the last wave).  Only if
 * one layer and the next do not fit together is ISO_ERR_BUDGET returned
 * (and then nothing of the cache changes).  The same holds for the _into
 * variants, except the all-blocks baseline. */
int iso_extract(iso_volume *v, float isovalue, iso_mesh *out);

/* As iso_extract, but writes into a caller-owned device buffer of
 * capacity_triangles triangles (float4[3 * capacity]).  If T exceeds it,
 * only the first `capacity` triangles are written, stats->num_triangles
 * holds T and ISO_ERR_CAPACITY is returned (the cache update stands). */
int iso_extract_into(iso_volume *v, float isovalue, float *d_vertices, uint64_t capacity_triangles,
                     iso_stats *stats);

/* As iso_extract_into, but each vertex is 8 bytes (the compact vertex
 * format of Section 4.5, 24 bytes per triangle): two uint32 words,
 * {qx | qy << 10 | qz << 20, block id}, where q = round(p / 4 * 1023) is
 * the 10-bit code of the block-local coordinate p in [0, 4] (decode as
 * q * 4 / 1023; within 2/1023 voxel of the float position).  p and q are
 * computed in IEEE float32: t = (iso - v_lo) / (v_hi - v_lo) with every
 * operation correctly rounded, p = lower corner + t, q = the nearest
 * integer (ties to even) to p * 255.75.  d_vertices holds
 * 6 * capacity_triangles uint32 words; same triangle order and errors as
 * iso_extract_into. */
int iso_extract_packed_into(iso_volume *v, float isovalue, uint32_t *d_vertices, uint64_t capacity_triangles,
                            iso_stats *stats);

/* Vertex formats of iso_extract_indexed_into */
#define ISO_VERTEX_FLOAT4 0    /* float4 {x, y, z block-local in [0, 4], w = block id bits}: 16 bytes */
#define ISO_VERTEX_PACKED 1    /* uint32 {qx | qy << 10 | qz << 20, block id}: 8 bytes (see
                                  iso_extract_packed_into for the codes) */

/* The indexed mesh Section 4.5 names as the alternative to the triangle
 * soup: vertices shared within each block (Flying Edges style, per block).
 * A block's vertices are the cut edges of its 5x5x5 sample window (edges
 * of its cells inside the volume whose two samples lie on opposite sides
 * of the isovalue), one vertex each; a vertex on a block face appears once
 * in every block whose cells use it.  Blocks come in ascending id (the
 * candidate order), a block's vertices in ascending global edge id
 * (3 * (x + nx*(y + ny*z)) + axis of the lower sample), and each vertex
 * holds the same position as the triangle soup's vertices on that edge
 * (bit for bit, in either format).  Triangles come in the soup's order, as
 * three uint32 indices into the vertex buffer, so that gathering the
 * vertices by index gives iso_extract_into's (or, packed,
 * iso_extract_packed_into's) output.
 *   d_vertices   capacity_vertices vertices of vertex_format (16 or 8 bytes)
 *   d_indices    3 * capacity_triangles uint32
 * Device pointers owned by the caller.  stats->num_vertices and
 * stats->num_triangles give V and T; if either buffer is too small, only
 * what fits is written and ISO_ERR_CAPACITY is returned (the cache update
 * stands), as also when V exceeds 2^32 - 1 (uint32 indices).  Waves as in
 * iso_extract: the waves' vertices and triangles are appended in order.
 * Same errors as iso_extract_into; ISO_ERR_INVALID_ARG for another
 * vertex_format. */
int iso_extract_indexed_into(iso_volume *v, float isovalue, int vertex_format, void *d_vertices,
                             uint64_t capacity_vertices, uint32_t *d_indices, uint64_t capacity_triangles,
                             iso_stats *stats);

/* ---- rendering (Section 4.6.2) ----
 * The paper draws the triangle soup, in its compressed vertex format, with
 * WebGPU; here CUDA kernels draw it into headless device buffers.  World
 * coordinates are voxel coordinates: a vertex is its block's origin
 * (4 bx, 4 by, 4 bz), from the block id (x fastest over ceil(n/4) blocks
 * per axis), plus its block-local position (float4) or code * 4/1023
 * (compact). */
typedef struct iso_camera {
    float view_proj[16];       /* row-major 4x4: clip (X, Y, Z, W) = M (x, y, z, 1) */
    float light[3];            /* direction towards the light (normalised by the library) */
    uint32_t width, height;    /* pixels, 1..32768 each */
} iso_camera;

typedef struct iso_render_stats {
    uint64_t drawn;            /* triangles in front of the camera with non-zero screen area
                                  whose bounding box meets the viewport */
    uint64_t big;              /* of them, covered one warp per triangle (bounding box over
                                  32 pixel centres) */
} iso_render_stats;

/* Rasterise num_triangles triangles (a soup: vertices 3t, 3t+1, 3t+2 when
 * d_indices is NULL, which needs num_vertices >= 3 * num_triangles; else
 * d_indices[3t + j], and a triangle with an index >= num_vertices is not
 * drawn) of vertex_format
 * (ISO_VERTEX_FLOAT4 / ISO_VERTEX_PACKED) from a volume of nx*ny*nz
 * samples.  Rules, every float operation a single IEEE float32 operation:
 * r = 1/W, sx = (X r * 0.5 + 0.5) * width, sy likewise (y up, row 0 at the
 * bottom), depth Z r * 0.5 + 0.5; triangles with a vertex at W <= 0 are not drawn
 * (no clipping); pixel centres (i + 0.5, j + 0.5) inside the triangle by
 * edge functions evaluated in a canonical endpoint order, with a top-left
 * rule on ties (a mesh is drawn without cracks or double hits); depth
 * interpolated by the edge values, fragments outside [0, 1] dropped.
 *   d_fragments  uint64[height * width] (row j at j * width): the smallest
 *                (depth bits << 32 | triangle) per pixel, ~0 where empty
 *   d_rgba       uint32[height * width] or NULL: r | g << 8 | b << 16 |
 *                a << 24, two-sided Lambert shading of the visible
 *                triangle, 0.2 + 0.8 |n.L| / |n| times (0.85, 0.75, 0.55),
 *                alpha 255; 0 where empty
 * Device buffers owned by the caller; queued on `stream`.  stats may be
 * NULL; when given, the call waits for the stream and fills it.
 * ISO_ERR_INVALID_ARG for a bad format, size, light (zero or not finite) or
 * a NaN in the matrix; ISO_ERR_OOM if the working list cannot be made. */
int iso_render(const void *d_vertices, int vertex_format, const uint32_t *d_indices, uint64_t num_vertices,
               uint64_t num_triangles, uint32_t nx, uint32_t ny, uint32_t nz, const iso_camera *camera,
               uint64_t *d_fragments, uint32_t *d_rgba, iso_render_stats *stats, void *stream);

/* ---- implicit isosurface ray casting (Section 4.6.2, future work) ----
 * The blocks serve as a macrocell grid for space skipping and the surface
 * is the isovalue set of the trilinear interpolant of the decoded samples,
 * read from the volume's block cache. */
typedef struct iso_pinhole {
    float eye[3];              /* ray origin, voxel coordinates */
    float forward[3];          /* direction through the image centre */
    float right[3], up[3];     /* image x and y at the image edge: the ray of pixel (i, j) has
                                  direction forward + u right + v up, u = (i + 0.5) / width * 2 - 1,
                                  v = (j + 0.5) / height * 2 - 1 (row 0 at the bottom) */
    float light[3];            /* direction towards the light (normalised by the library) */
    uint32_t width, height;    /* pixels, 1..32768 each */
} iso_pinhole;

typedef struct iso_raycast_stats {
    uint64_t hits;             /* pixels whose ray meets the surface */
    uint32_t n_active;         /* active blocks of the isovalue (Section 4.1) */
    uint32_t n_new;            /* of them, decoded into the cache by this call */
    uint32_t n_slots;          /* cache slots in use */
    uint32_t reserved;
} iso_raycast_stats;

/* Ray cast the isosurface at `isovalue` into headless device buffers.
 * First the extraction's front runs for the isovalue (range test, cache
 * update, decode: afterwards the cache holds what iso_extract would leave),
 * then one thread per pixel: rays start at t = 0 or where they enter the
 * volume box [0, n-1]^3 and visit blocks (the cells of block b span
 * [4b, min(4b + 4, n - 1)] per axis), then cells, in ray order, each box's
 * interval by its own slab test ((bound - origin) times the direction's
 * reciprocal, taken once per ray) and the next box one step along the exit
 * axis; a block is searched when its 2x2x2 group range holds the isovalue,
 * a cell when its 8 corners' range does (lo < iso <= hi, a sample equal to
 * iso counting as above); in a cell the interpolant is sampled at the ends
 * and 3 interior quarter points of the ray's interval, and 12 bisection
 * steps refine the first change of side.  Every float operation is one
 * IEEE float32 operation.
 *   d_hits  uint64[height * width]: (t bits << 32 | block id) of the first
 *           hit (t in units of the ray direction's length), ~0 for none
 *   d_rgba  uint32[height * width] or NULL: two-sided Lambert shading from
 *           the interpolant's gradient at the hit, as iso_render; 0 for none
 * Blocks until done.  ISO_ERR_BUDGET when the active blocks do not fit in
 * the cache (no waves here); other errors as iso_extract. */
int iso_raycast(iso_volume *v, float isovalue, const iso_pinhole *camera, uint64_t *d_hits, uint32_t *d_rgba,
                iso_raycast_stats *stats);

/* The full-volume baseline the paper measures against (the naive
 * data-parallel marching cubes of Section 3 over the whole decompressed
 * volume): the same pipeline with the range test switched off, so every
 * block is decoded into the cache and every cell is classified.  Because
 * the range test only skips blocks without crossings, the mesh is
 * identical to iso_extract_into's.  The cache must hold every block
 * (cache budget >= 256 * nb), else ISO_ERR_BUDGET. */
int iso_extract_all_blocks_into(iso_volume *v, float isovalue, float *d_vertices, uint64_t capacity_triangles,
                                iso_stats *stats);

/* Decode a whole compressed volume into a dense float32 field (nx*ny*nz,
 * x fastest; samples past the volume edge are dropped), one thread per
 * block (the full-volume decompression the paper times for ZFP).  Device
 * pointers; queued on `stream`, does not block. */
int iso_decode_volume(const uint64_t *d_bits, uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate_bits,
                      float *d_field, void *stream);

/* Naive data-parallel marching cubes over a dense field: the baseline of
 * Section 3.3.3 (Table "mc_naive_parallel_perf") that the block method is
 * measured against.  A pass over every cell classifies it and compacts the
 * cells the surface crosses (0 < case < 255) in ascending order; their
 * triangle counts (from the case table) are prefix-summed into output
 * offsets; a second pass over the crossing cells writes the triangles.  No
 * blocks, ranges or cache take part.
 *   d_field       device, nx*ny*nz float32 samples, x fastest (for instance
 *                 iso_decode_volume's output); 4-byte aligned
 *   d_vertices    device float4[3 * capacity_triangles], 16-byte aligned:
 *                 the triangle soup in full-volume marching-cubes order
 *                 (cells ascending, then table order), each vertex in the
 *                 format of iso_extract ({x, y, z} relative to the origin of
 *                 the 4x4x4 block holding the cell, w = that block's id), the
 *                 same bytes the block path writes for the same triangle
 *   d_edge_ids    optional (may be NULL) device uint64[3 * capacity]: the
 *                 global edge id 3*(x + nx*(y + ny*z)) + axis of each vertex
 *   stats         num_triangles and n_active_cells, filled also when the
 *                 triangles do not fit (ISO_ERR_CAPACITY: nothing written)
 * The volume may hold at most 2^32 - 1 cells.  Scratch (5 bytes per cell,
 * 8 per crossing cell) comes from the library's allocator.  Queued on
 * `stream`; the call blocks until it is done (it reads back two counts). */
typedef struct iso_dense_stats {
    uint64_t num_triangles;
    uint64_t n_active_cells;       /* cells the surface crosses */
} iso_dense_stats;
int iso_mc_dense(const float *d_field, uint32_t nx, uint32_t ny, uint32_t nz, float isovalue, float *d_vertices,
                 uint64_t capacity_triangles, uint64_t *d_edge_ids, iso_dense_stats *stats, void *stream);

/* Free a mesh's vertex buffer (stream-ordered on the volume's stream that
 * made it).  The volume must still be alive.  Safe on a zeroed mesh. */
int iso_mesh_release(iso_volume *v, iso_mesh *m);

/* Free every device and host resource of the volume (device memory goes
 * back to the library's pool; its small pinned host buffers and its upload
 * stream are kept, a few dozen at most, for the next load: see
 * iso_release_cached_memory).  NULL is a no-op. */
void iso_release(iso_volume *v);

/* Change the stream used by later calls on v (the previous stream is
 * synchronised first). */
int iso_set_stream(iso_volume *v, void *stream);

/* Drop every cached block (all slots empty, epoch kept): the next
 * extraction decodes all of its active blocks. */
int iso_cache_reset(iso_volume *v);

/* Test hook for the failure path of the device-side waits (the paper has no
 * counterpart).  With what = ISO_TEST_WITHHOLD_PREFIX, every later
 * extraction's range test (Section 4.1) runs with its first tile never
 * publishing its prefix sums, so each later tile's bounded wait gives up
 * after 1024 polls (about a millisecond); the extraction then returns
 * ISO_ERR_TIMEOUT and, as after any timeout, empties the cache.  what = 0
 * restores normal operation; the volume stays usable throughout.  It lets
 * a test drive a wait to its limit without hanging or faulting the GPU.
 * Any other value of `what` is ISO_ERR_INVALID_ARG. */
#define ISO_TEST_WITHHOLD_PREFIX 1u
int iso_set_test_fault(iso_volume *v, uint32_t what);

/* Per-stage timing.  With profiling on, each extraction records CUDA
 * events on the volume's stream between its kernels; iso_stage_times then
 * returns the last extraction's durations in milliseconds, in this order:
 *   0 prep (counters and descriptors), 1 cull (Section 4.1 and the
 *   hit/new split of Algorithm 1), 2 cache update (rest of Algorithm 1),
 *   3 decode (Section 4.2.1), 4 count (Sections 4.3-4.4: per-block
 *   triangle counts), 5 scan (Section 4.4: offsets), 6 emit (Section 4.5).
 * ms must hold n >= 7 floats.  Profiling off (the default) records
 * nothing. */
#define ISO_NUM_STAGES 7
int iso_set_profiling(iso_volume *v, int on);
int iso_stage_times(iso_volume *v, float *ms, int n);

/* Human-readable text for a status code (static storage). */
const char *iso_error_string(int status);

/* The library's marching-cubes case table (host-only, needs no GPU).  The
 * paper cites Lorensen and Cline's marching cubes without a table; this
 * one is generated by a face rule: on every cell face, each run of
 * below-iso corners (counter-clockwise, seen from outside) is cut off by
 * one segment, so a face with two diagonal below corners cuts them off
 * separately and adjacent cells always agree; the segments form cycles,
 * taken by smallest edge number and fanned from it.  num_tri receives 256
 * counts (at most 5); tri_edges receives 256 rows of 16 bytes, three edge
 * numbers per triangle.  Edge 4*a + j lies along axis a (0=x,1=y,2=z) at
 * offsets (j&1, j>>1) on the other two axes in increasing axis order. */
int iso_mc_case_table(uint8_t *num_tri, uint8_t *tri_edges);

/* Encode a device-resident float32 volume into the fixed-rate format on
 * the GPU (for producing test and benchmark inputs; the paper's method
 * itself only decodes).  d_field is nx*ny*nz floats (x fastest);
 * d_bits receives nb*rate words; d_bmin/d_bmax receive each block's range
 * over its decoded in-volume samples.  All pointers are device pointers;
 * the work is queued on `stream` and the call does not block.
 * Non-finite samples are not allowed (the output is then unspecified). */
int iso_encode_field(const float *d_field, uint32_t nx, uint32_t ny, uint32_t nz, uint32_t rate_bits,
                     uint64_t *d_bits, float *d_bmin, float *d_bmax, void *stream);

/* Decode blocks ids[0..n) of a device-resident compressed volume into
 * out (n*64 floats, block-local order), device pointers, queued on
 * `stream` (Section 4.2.1 applied to an explicit list). */
int iso_decode_blocks(const uint64_t *d_bits, uint32_t rate_bits, const uint32_t *d_ids, uint64_t n,
                      float *d_out, void *stream);

/* Active-block selection without any allocation.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * -- plug-ins inside an application whose allocator already owns the
 * device memory, and latency-critical loops that must not meet an
 * allocation's implicit synchronisation.
 * It performs the range test of the cull stage (a block is active when
 * lo < iso <= hi for the min/max of block_min/block_max over its 3x3x3
 * block neighbourhood) and writes the active block ids in ascending order,
 * like the ids iso_extract selects for the same ranges.
 *   d_bmin, d_bmax  device, nb floats each (ranges of the decoded samples)
 *   d_ids           device, room for `capacity` ids; ids past it are dropped
 *   d_count         device uint32, written after every id: the number of
 *                   active blocks (may exceed capacity), 0xFFFFFFFF if a
 *                   device-side wait timed out, or 0xFFFFFFFE if some
 *                   block's range is not a range (NaN, or min > max; the
 *                   ids are then unspecified)
 * All four buffers must be 4-byte aligned (else ISO_ERR_INVALID_ARG); the
 * call cannot check their lengths.  Its scratch is a fixed file-scope
 * device array of about 256 KiB, held by every GPU that loads the library
 * until the process exits; volumes of more than 2^26 blocks (2^32 samples)
 * are refused with ISO_ERR_INVALID_ARG.  The first call on a device looks
 * the array's address up with that device current: make that first call
 * before any stream capture.  All calls share the array and it keeps the
 * previous call's contents; each call clears what it needs, so calls that
 * overlap on the GPU (different streams at once) race and must be avoided.
 * The work is queued on `stream`; the call does not block. */
int iso_active_blocks_static(const float *d_bmin, const float *d_bmax, uint32_t nx, uint32_t ny, uint32_t nz,
                             float isovalue, uint32_t *d_ids, uint64_t capacity, uint32_t *d_count, void *stream);

/* ---- batches: many volumes in the same launches ---------------------
 * A batch extracts one surface from each of n loaded volumes, each at its
 * own isovalue, with every stage of Sections 4.1-4.5 running as ONE
 * persistent launch over all n volumes (work items numbered volume after
 * volume), the whole sequence replayed as one CUDA graph.  Each volume
 * keeps its own cache (Algorithm 1 runs per volume), so a volume's
 * surface, statistics and cache state after a batch extraction are
 * exactly those of extracting it alone at the same isovalue.
 *
 * The batch does not own its volumes: they must outlive it, must all live
 * on the current device, may not be loaded with ISO_DEBUG, may appear
 * only once, and may not be used by another call while a batch call runs
 * (batch calls block until they are done, so sequential use from one host
 * thread is safe).  Device work is issued on the batch's stream. */
typedef struct iso_batch iso_batch;

/* How the launches of a batch run.  For each persistent kernel: CTAs per
 * SM (0 = the kernel's occupancy limit, the default; larger values are
 * clamped to it) and, where the kernel has a choice, its tile size (0 =
 * default).  Every setting computes the same results. */
typedef struct iso_launch_shape {
    uint32_t cull_ctas;          /* Section 4.1 */
    uint32_t cull_tile;          /* block ranges per cull tile: 2048 or 4096 (default) */
    uint32_t cache_update_ctas;  /* Algorithm 1 (both cache-update kernels) */
    uint32_t decode_ctas;        /* Section 4.2.1 */
    uint32_t decode_tile;        /* new blocks per decode CTA: 64, 128 (default) or 256 */
    uint32_t count_ctas;         /* Section 4.4: per-block triangle counts */
    uint32_t count_tile;         /* candidate blocks per count CTA: 16, 32 (default) or 64 */
    uint32_t scan_ctas;          /* Section 4.4: offsets */
    uint32_t scan_tile;          /* counts per offset-scan tile: 1024, 2048 (default) or 4096 */
    uint32_t emit_ctas;          /* Section 4.5 */
    uint32_t emit_tile;          /* candidate blocks per emit CTA: 16, 32 (default) or 64 */
} iso_launch_shape;

/* The launch shape of a single volume's extractions (same fields and
 * rules as a batch's; every shape computes the same results).  Takes
 * effect from the next call; the volume's captured graphs are rebuilt.  A
 * volume starts with 4096-count scan tiles at one CTA per SM and 256-block
 * decode CTAs, the rest at the defaults (zeros in a shape passed here mean
 * the general defaults). */
int iso_set_shape(iso_volume *v, const iso_launch_shape *shape);
int iso_get_shape(const iso_volume *v, iso_launch_shape *shape);

/* volumes[0..n), 1 <= n <= 1024; stream: cudaStream_t (NULL = default). */
int iso_batch_create(iso_batch **out, iso_volume *const *volumes, uint32_t n, void *stream);

/* Extract surface i of volume i at isovalues[i] (host array, all finite).
 * Surfaces are written one after another into the caller's device buffer
 * d_vertices (float4[3 * capacity_triangles]): surface i occupies
 * triangles [tri_offsets[i], tri_offsets[i+1]).  tri_offsets (host,
 * n+1 entries) is always filled; if the total exceeds the capacity, only
 * triangles below it are written and ISO_ERR_CAPACITY is returned (the
 * caches are updated: calling again with a larger buffer repeats the same
 * surfaces from a warm cache).  stats (host, n entries) and status (host,
 * n entries: ISO_OK, ISO_ERR_BUDGET or ISO_ERR_TIMEOUT per volume) may be
 * NULL.  Returns the first volume error, else the capacity check's. */
int iso_batch_extract(iso_batch *b, const float *isovalues, float *d_vertices, uint64_t capacity_triangles,
                      uint64_t *tri_offsets, iso_stats *stats, int *status);

/* Set or read the batch's launch shape (the graph is re-captured).  A
 * tile size the kernels are not compiled for gives ISO_ERR_INVALID_ARG.
 * get_shape reports what runs: CTAs per SM after clamping, tile sizes. */
int iso_batch_set_shape(iso_batch *b, const iso_launch_shape *shape);
int iso_batch_get_shape(const iso_batch *b, iso_launch_shape *shape);

/* Autotune the launch shape on the given isovalues.  For each tile-size
 * variant i (0, 1, 2: the sizes listed above, smallest first; kernels
 * with fewer variants keep their last) and each k from 1 to the largest
 * occupancy limit, every kernel runs at variant i with min(k, its limit)
 * CTAs per SM; each setting is timed `trials` times (CUDA events between
 * the kernels, caches emptied before each run so that every run decodes
 * the same blocks) and each kernel keeps its fastest (tile, CTAs) pair.
 * The chosen shape is applied if the whole batch runs faster with it than
 * with the defaults, and returned in *best; best_ms[0] and best_ms[1] (may
 * be NULL) receive the cold-cache batch time of the default shape and of
 * the applied one.  The caches are left empty. */
int iso_batch_tune(iso_batch *b, const float *isovalues, float *d_vertices, uint64_t capacity_triangles,
                   int trials, iso_launch_shape *best, float *best_ms);

/* Free the batch (not its volumes).  NULL is a no-op. */
void iso_batch_release(iso_batch *b);

/* ---- serving: a request queue on one resident volume ----------------
 * Isovalue requests are queued with iso_server_submit and answered by
 * iso_server_step.  Requests are served in ticks of up to max_batch queued
 * requests (first come, first served).  A tick's front is one pass over the
 * block ranges that finds the union of its requests' active blocks
 * (Section 4.1) and each request's own candidates, then one cache update
 * and decode for the union (Section 4.2, Algorithm 1); its back counts and
 * scans all its requests (Sections 4.3-4.4) in one launch each, then, after
 * one readback of their triangle counts (the count follows the front on the
 * device, with no host round trip; the union's budget is checked at that
 * readback), emits them (Section 4.5) in one launch, or request by request
 * at light load (a round of one or two requests, none waiting) so that each
 * finishes as soon as its own emission does.  On a volume with segment
 * ranges every request's count, scan and emission is a launch of its own.  Under load ticks
 * overlap: when a tick's emission is queued and at least two requests wait,
 * they are admitted as the next tick and its front runs on a second stream
 * while the running tick emits (a lone waiting request is admitted when the
 * running tick is done; no overlap on volumes with segment ranges, see
 * ISO_SEGMENT_CULL, nor while the running tick's union takes more than half
 * the cache).  That front also counts the running
 * tick's isovalues as active, so its cache update evicts no block the
 * running tick reads; decoded blocks and all metadata stay resident between
 * ticks.
 * Admission: when a union's active blocks do not fit in the volume's cache
 * budget, its requests return to the queue: an overlapped tick is retried
 * once the running tick is done, otherwise later ticks take half as many
 * requests (down to one; a single request that does not fit finishes with
 * ISO_ERR_BUDGET).  Meshes are allocated when their sizes are known, in
 * request order: a tick emits in rounds, each taking the waiting requests
 * whose meshes fit together with the finished, not yet taken meshes under
 * vertex_budget_bytes (a mesh is always allowed when nothing is held); the
 * rest wait in the tick, their counts kept, until meshes are taken.  Every
 * served mesh is
 * identical, byte for byte, to iso_extract of the same isovalue on the
 * same data.  The server uses the volume's device state: do not extract
 * from the volume on another stream while a server call runs, and destroy
 * the server before the volume. */
typedef struct iso_server iso_server;

typedef struct iso_server_options {
    uint32_t max_batch;            /* requests per tick, 1..8; 0 = 4 */
    uint32_t vertex_format;        /* ISO_VERTEX_FLOAT4 (0, 48 bytes a triangle) or ISO_VERTEX_PACKED
                                      (24 bytes a triangle: the meshes' d_vertices then hold the compact
                                      uint32 pairs of iso_extract_packed_into) */
    uint64_t vertex_budget_bytes;  /* limit on held mesh bytes (48 or 24 per triangle); 0 = none */
    void *stream;                  /* cudaStream_t whose earlier work the server waits for at creation
                                      (NULL = default); the server runs on two streams of its own */
    uint64_t case_bytes;           /* room for the requests' stored cell cases, 64 bytes a candidate:
                                      0 = max_batch full candidate lists, at most 4 GiB; below 64 = none
                                      (every emission classifies again); the meshes are the same */
} iso_server_options;

/* v must not be loaded with ISO_DEBUG.  The server keeps 2 * max_batch
 * request positions (a running tick's and the next tick's), each with
 * candidate, count, offset and occupied-list arrays of min(cache slots, nb)
 * entries (20 bytes each), a buffer for the requests' stored cell cases
 * (case_bytes; a request whose cases do not fit is classified again by its
 * emission), and creates two streams: the backs run at the
 * device's highest stream priority, the fronts at its lowest, so a front
 * overlapping a back takes only the SMs the back leaves idle.  Meshes are
 * complete when a request finishes (the server waits for its emission). */
int iso_server_create(iso_server **out, iso_volume *v, const iso_server_options *opt);

/* Queue a request (host only, no device work); *ticket identifies it. */
int iso_server_submit(iso_server *s, float isovalue, uint64_t *ticket);

/* Advance the pipeline until requests finish (a tick's emission round is
 * done: every request of the round has finished), a union over the cache budget has gone back to the queue and
 * nothing else moved, the next mesh waits for meshes to be taken (vertex
 * budget: returns at once with none finished), or nothing is in flight (no
 * request waits); blocks while it waits for the GPU.  Ticks are
 * admitted on the way (the next one while the current one is in its back),
 * so work keeps running on the GPU when the call returns.  *completed (may
 * be NULL) receives the number of requests finished.  If queuing a tick's
 * work fails (ISO_ERR_CUDA, ISO_ERR_OOM), its requests return to the queue
 * and the call returns that error. */
int iso_server_step(iso_server *s, uint32_t *completed);

/* The same without blocking: take every transition whose GPU work is
 * already done (finish the requests whose emissions are done, start an
 * emission, start a count, admit the queued requests as the next tick) and
 * return at once.  A request loop
 * that polls between arrivals admits each arrival while the previous tick
 * is still on the GPU.  *completed (may be NULL) receives the number of
 * requests finished. */
int iso_server_poll(iso_server *s, uint32_t *completed);

/* Requests not finished yet (queued, or admitted into the next tick). */
int iso_server_queued(const iso_server *s, uint32_t *queued);

/* Hand a finished request's mesh to the caller (release it with
 * iso_mesh_release on the server's volume).  Returns ISO_PENDING if the
 * request is still queued, the request's own status if it finished
 * (ISO_OK, ISO_ERR_BUDGET, ISO_ERR_TIMEOUT, ISO_ERR_OOM, or ISO_ERR_BOUNDS
 * from the checked build; no mesh unless ISO_OK), ISO_ERR_INVALID_ARG for
 * an unknown or already taken ticket.
 * stats: n_active, n_new, n_slots, cache_bytes and epoch describe the
 * tick's union; num_triangles, n_occupied, n_candidates the request. */
int iso_server_take(iso_server *s, uint64_t ticket, iso_mesh *out);

/* Step the server until `ticket` is finished or timeout_ms milliseconds
 * have passed (0: look once, no step), then return as iso_server_take
 * (ISO_PENDING on timeout; a step's own error is returned as it comes). */
int iso_server_wait(iso_server *s, uint64_t ticket, uint32_t timeout_ms, iso_mesh *out);

/* Free the server, its queue and any finished meshes not taken. */
void iso_server_destroy(iso_server *s);

/* ---- debug and parity access (volumes loaded with ISO_DEBUG) ---------
 * Copies a per-stage array of the LAST extraction into host memory.
 * `bytes` is the size of host_dst; *count receives the number of elements
 * available (and copied, if they fit; otherwise ISO_ERR_CAPACITY). */
#define ISO_DBG_ACTIVE_IDS 1   /* uint32[n_active]  I_active, ascending (ISO_DEBUG volumes only) */
#define ISO_DBG_NEW_IDS 2      /* uint32[n_new]     I_new, ascending */
#define ISO_DBG_SLOT_OF_BLOCK 3 /* int32[nb]        I_slot (-1 = not cached) */
#define ISO_DBG_BLOCK_OF_SLOT 4 /* int32[n_slots]   S_block (-1 = empty) */
#define ISO_DBG_SLOT_LAST_USE 5 /* uint32[n_slots]  epoch of last use (0 = never) */
#define ISO_DBG_ACTIVE_MASK 6  /* uint32[ceil(nb/32)] M_active bitmask */
#define ISO_DBG_CELL_CASES 7   /* uint8[n_cand*64] case of each cell of each candidate block */
#define ISO_DBG_BLOCK_TRIS 8   /* uint32[n_cand]    triangles per candidate block (after an indexed
                                  extraction, bits 16-31 hold the block's vertices) */
#define ISO_DBG_BLOCK_OFFSETS 9 /* uint64[n_cand]   exclusive prefix of BLOCK_TRIS */
#define ISO_DBG_EDGE_IDS 10    /* uint64[3*T]       global edge id of each vertex:
                                  3*(x + nx*(y + ny*z)) + axis of its lower sample */
#define ISO_DBG_CANDIDATES 11  /* uint32[n_cand]    candidate block ids, ascending: the active
                                  blocks whose 2x2x2 +group range contains iso (the
                                  only blocks that can emit triangles) */
int iso_debug_get(iso_volume *v, int which, void *host_dst, size_t bytes, uint64_t *count);

/* Copy the decoded samples of cached blocks ids[0..n) (host array) to
 * host_out (n*64 floats).  Returns ISO_ERR_INVALID_ARG if a block is not
 * cached. */
int iso_debug_read_blocks(iso_volume *v, const uint32_t *ids, uint64_t n, float *host_out);

#ifdef __cplusplus
}
#endif
#endif /* BCMC_H */
