// Shared device-side definitions of the block-compressed marching-cubes
// library: volume geometry, the per-volume control block, the single-pass
// decoupled look-back scan used by every compaction, and small bit tools.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bcmc {

// ---------------------------------------------------------------- geometry

struct Geom {
    uint32_t nx, ny, nz;      // samples
    uint32_t nbx, nby, nbz;   // blocks per axis
    uint32_t nb;              // total blocks (< 2^31, checked at load)
    uint32_t rate;            // bits per sample = 64-bit words per block
    unsigned long long inv_nbx, inv_nby;   // floor(2^64 / d) + 1 (0 for d = 1): see block_coords
};

// Reciprocal for dividing 32-bit numbers by d with one 64-bit multiply:
// for n < 2^32, floor(n / d) = high 64 bits of n * (floor(2^64/d) + 1),
// since the error term n * (M - 2^64/d) / 2^64 < 2^-32 < 1/d cannot carry
// n/d past the next integer.
__host__ __device__ inline unsigned long long div_magic(uint32_t d) {
    // floor((2^64-1)/d) + 1: floor(2^64/d) + 1, or exactly 2^64/d when d is a
    // power of two (then the product is exact); both satisfy the bound above
    return d <= 1 ? 0ull : ~0ull / d + 1ull;
}

__device__ __forceinline__ uint32_t div_by(uint32_t n, uint32_t d, unsigned long long magic) {
    return d <= 1 ? n : (uint32_t)__umul64hi((unsigned long long)n, magic);
}

// block id -> (bx, by, bz)
__device__ __forceinline__ void block_coords(const Geom &g, uint32_t b, uint32_t &bx, uint32_t &by, uint32_t &bz) {
    const uint32_t q = div_by(b, g.nbx, g.inv_nbx);
    bx = b - q * g.nbx;
    bz = div_by(q, g.nby, g.inv_nby);
    by = q - bz * g.nby;
}

// ---------------------------------------------------------------- control block

// A bounded device wait that gives up sets the bit of its stage.  Each
// kernel sizes its work only from bits set before it starts, so all of
// its blocks agree on the sizes even when one of them times out.
enum Status : uint32_t {
    kStatusTimeout = 1u,      // cull look-back gave up
    kStatusBudget = 2u,       // new blocks do not fit in the slot cap
    kStatusTimeoutLru = 4u,   // cache-update look-back gave up
    kStatusTimeoutScan = 8u,  // triangle-offset look-back gave up
    kStatusCorrupt = 16u,     // a block range given at load is not a range (set by the hull kernel)
    kStatusBounds = 32u,      // checked builds: an index failed its bounds check (the access was skipped)
    kStatusSkip = 64u,        // serving: this request's emission is skipped (no mesh in this tick)
};
constexpr uint32_t kStatusAnyTimeout = kStatusTimeout | kStatusTimeoutLru | kStatusTimeoutScan;

// Checked builds (compiled with BCMC_CHECKED): an index is tested before
// the access it guards; a failed test sets kStatusBounds in the volume's
// status and the caller skips the access, so a defect surfaces as
// ISO_ERR_BOUNDS rather than as a memory fault.  In normal builds the test
// is compiled out (true).
#ifdef BCMC_CHECKED
__device__ __forceinline__ bool in_bounds(bool ok, uint32_t *status) {
    if (!ok) atomicOr(status, kStatusBounds);
    return ok;
}
#else
__device__ __forceinline__ bool in_bounds(bool, uint32_t *) { return true; }
#endif

// dynamic work counters of one launch sequence (tiles handed out in order)
enum LaunchCounter { kLcCull = 0, kLcLruA = 1, kLcLruB = 2, kLcScan = 3, kNumLaunchCounters = 4 };

// Per-extraction inputs, copied from pinned host memory by the first
// operation of each extraction (so a captured graph never changes).
enum VertexFormat : uint32_t {
    kVertexFloat4 = 0,            // float4 {x, y, z block-local, w = block id bits}: 16 B
    kVertexPacked = 1,            // uint2 {x | y << 10 | z << 20 (10-bit codes of p/4), block id}: 8 B
};

enum ParamFlags : uint32_t {
    kParamAllBlocks = 1u,         // no range test: every block is active and a candidate
    kParamWindow = 2u,            // a wave: only blocks with ids in [win_lo, win_act_hi) may be active,
                                  // only those in [win_lo, win_cand_hi) candidates
    kParamIndexed = 4u,           // indexed mesh: one vertex per cut edge of each block's window,
                                  // triangles as three uint32 vertex indices
    kParamTestWithhold = 8u,      // test hook: the range test's first tile never publishes its prefix,
                                  // and the other tiles wait kTestSpinLimit polls before giving up
};

struct Params {
    float iso;
    uint32_t format;              // VertexFormat
    uint32_t flags;               // ParamFlags
    uint32_t win_lo, win_cand_hi, win_act_hi;
    unsigned long long tri_cap;   // output capacity in triangles
    unsigned long long out;       // vertex buffer (float4 * or uint2 *)
    // indexed mesh only (kParamIndexed)
    unsigned long long idx_out;   // uint32 index buffer, 3 per triangle
    unsigned long long vert_cap;  // vertex buffer capacity in vertices
    unsigned long long vtx_base;  // added to every index (vertices of earlier waves)
};

// One per volume, in device memory.  Written only by the kernels of one
// extraction at a time (stream order), read back once per extraction.
struct Ctl {
    Params params;
    uint32_t epoch;           // extraction count; S_last values are epochs
    uint32_t n_active;        // |I_active|
    uint32_t n_new;           // |I_new|
    uint32_t n_cand;          // |I_cand|
    uint32_t n_assign;        // new blocks given a slot (n_new, or 0 on budget failure)
    uint32_t S;               // slots in the LRU
    uint32_t u;               // slots [0,u) have been used; [u,S) never
    uint32_t cap;             // physical slot capacity
    uint32_t lpar;            // which of the two list buffers holds the used-slot list
    uint32_t S_next, u_next;  // committed by the decode kernel
    uint32_t from_unused;     // assignments taken from [u, S_next)
    uint32_t from_used;       // assignments taken from the used list
    uint32_t keep_base;       // length of the surviving part of the used list
    uint32_t n_occ;           // occupied blocks
    uint32_t status;          // Status bits
    uint32_t mc_tiles;        // look-back descriptors the triangle kernel used (to clear)
    uint32_t lpar_next;       // the list buffer this update fills (lru_a sets it; the commit adopts it)
    uint32_t ctr[kNumLaunchCounters];   // work counters when the volume is extracted alone
    unsigned long long n_tri; // triangles of the surface
    unsigned long long n_vtx; // vertices of the indexed mesh (indexed extractions only)
};
static_assert(sizeof(Ctl) == 168, "the control block is read back every extraction: keep it at 168 bytes");

// ---------------------------------------------------------------- memory-model helpers

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------------------------- decoupled look-back
//
// Single-pass exclusive scan across tiles (Merrill and Garland's decoupled
// look-back).  A descriptor is 64 bits: the top two bits say whether the
// low 62 bits hold nothing yet (0), the tile's own aggregate (1) or the
// inclusive prefix through the tile (2).  Values are sums of non-negative
// counters, possibly two 31-bit counters packed side by side.
// Tiles are handed out in order by an atomic counter, so every tile that a
// waiter depends on belongs to a block that is already running; the wait
// is still bounded: after kSpinLimit polls the tile sets `timeout_bit` in
// Ctl::status and proceeds with what it has.

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPrefix = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr int kSpinLimit = 1 << 23;   // with at most 128 ns between polls: about a second
constexpr int kTestSpinLimit = 1 << 10;   // the test hook's shorter wait (kParamTestWithhold)

// Called by all 32 lanes of one warp.  Returns the exclusive prefix of
// `tile` (same value in every lane) and publishes the inclusive one.  Each
// poll reads a window of 32 x kLookbackPerLane predecessors (lane l reads
// the kLookbackPerLane nearest-first descriptors of its slice) and stops at
// the nearest inclusive prefix, summing the aggregates after it.
constexpr int kLookbackPerLane = 4;

__device__ __forceinline__ unsigned long long lookback_exclusive(unsigned long long *desc, uint32_t tile,
                                                                  unsigned long long aggregate,
                                                                  uint32_t *status, uint32_t timeout_bit,
                                                                  int spin_limit = kSpinLimit) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_relaxed(desc, kFlagPrefix | aggregate);
        return 0;
    }
    if (lane == 0) st_relaxed(desc + tile, kFlagAgg | aggregate);
    unsigned long long excl = 0;
    long long base = (long long)tile - 1;
    int spins = 0;
    unsigned sleep_ns = 16;
    while (true) {
        unsigned long long d[kLookbackPerLane];
#pragma unroll
        for (int k = 0; k < kLookbackPerLane; k++) {
            const long long idx = base - (long long)lane * kLookbackPerLane - k;
            d[k] = idx >= 0 ? ld_relaxed(desc + idx) : kFlagPrefix;
        }
        bool ready = true, has_prefix = false;
        unsigned long long v = 0;
#pragma unroll
        for (int k = 0; k < kLookbackPerLane; k++) {
            if (has_prefix) continue;
            const unsigned flag = (unsigned)(d[k] >> 62);
            if (flag == 0) ready = false;
            v += d[k] & kValueMask;
            if (flag == 2) has_prefix = true;
        }
        const unsigned rdy = __ballot_sync(0xffffffffu, ready);
        const unsigned pref = __ballot_sync(0xffffffffu, has_prefix && ready);
        const unsigned need = pref ? ((pref & (0u - pref)) << 1) - 1u : 0xffffffffu;   // lanes up to the first prefix
        if ((rdy & need) != need) {
            if (++spins > spin_limit) {
                // the status bit becomes visible before the (partial) prefix
                // published below, so a reader that sees the prefix and then
                // reads the status sees the bit too
                if (lane == 0) {
                    atomicOr(status, timeout_bit);
                    __threadfence();
                }
                break;
            }
            __nanosleep(sleep_ns);
            if (sleep_ns < 128) sleep_ns <<= 1;
            continue;
        }
        v = ((need >> lane) & 1u) ? v : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (pref) break;
        base -= 32 * kLookbackPerLane;
    }
    if (lane == 0) st_relaxed(desc + tile, kFlagPrefix | (excl + aggregate));
    return excl;
}

// ---------------------------------------------------------------- vertex interpolation

// t = (iso - v_lo) / (v_hi - v_lo) on a cut edge (iso lies between the two
// samples, so |iso - v_lo| <= |v_hi - v_lo|), each difference rounded once.
// The quotient goes through the reciprocal (kExact false: within 2 ulp for
// divisors in [2^-126, 2^126]) or is correctly rounded (kExact true).  A
// difference outside [2^-100, 2^125) -- samples near +-FLT_MAX, whose
// difference can even overflow, or samples so close that it is tiny -- is
// formed from the samples scaled by 2^-4 or 2^64: the scaling is exact up to
// underflow of samples far below the difference, the quotient stays the same
// real number, and the divisor lands inside the reciprocal's range.
template <bool kExact>
__device__ __forceinline__ float edge_fraction(float iso, float vlo, float vhi) {
    float a = __fsub_rn(iso, vlo), b = __fsub_rn(vhi, vlo);
    const float mb = fabsf(b);
    if (!(mb >= 0x1p-100f && mb < 0x1p125f)) {
        const float sc = mb >= 0x1p125f ? 0x1p-4f : 0x1p64f;
        const float slo = __fmul_rn(vlo, sc);
        a = __fsub_rn(__fmul_rn(iso, sc), slo);
        b = __fsub_rn(__fmul_rn(vhi, sc), slo);
    }
    return kExact ? __fdiv_rn(a, b) : __fdividef(a, b);
}

// ---------------------------------------------------------------- bit tools

// (x & ~m) | (y & m) as one three-input logic instruction
__device__ __forceinline__ uint32_t select_bits(uint32_t x, uint32_t y, uint32_t m) {
    uint32_t r;
    asm("lop3.b32 %0, %1, %2, %3, 0xD8;" : "=r"(r) : "r"(x), "r"(y), "r"(m));   // LUT of (c ? b : a): 0xD8
    return r;
}

// In-place transpose of a 32x32 bit matrix held in 32 words: afterwards
// bit j of a[i] is what bit i of a[j] was.  Five rounds of swapping the
// off-diagonal sub-blocks (16x16, 8x8, ..., 1x1); the 16- and 8-bit rounds
// move whole bytes, one byte permute per word.
__device__ __forceinline__ void transpose32(uint32_t (&a)[32]) {
#pragma unroll
    for (int j = 0; j < 16; j++) {        // (a, b) -> (a.lo16 | b.lo16 << 16, a.hi16 | b.hi16 << 16)
        const uint32_t x = a[j], y = a[j + 16];
        a[j] = __byte_perm(x, y, 0x5410);
        a[j + 16] = __byte_perm(x, y, 0x7632);
    }
#pragma unroll
    for (int j = 0; j < 32; j++) {        // bytes (a0 b0 a2 b2), (a1 b1 a3 b3)
        if (j & 8) continue;
        const uint32_t x = a[j], y = a[j + 8];
        a[j] = __byte_perm(x, y, 0x6240);
        a[j + 8] = __byte_perm(x, y, 0x7351);
    }
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 2; r < 5; r++) {
        const int s = 16 >> r;
        const uint32_t m = masks[r], mh = m << s;
#pragma unroll
        for (int j = 0; j < 32; j++) {
            if (j & s) continue;
            // swap the bits of a[j] under mh with those of a[j + s] under m,
            // each word as one shift and one three-input select
            const uint32_t x = a[j], y = a[j + s];
            a[j] = select_bits(x, y << s, mh);
            a[j + s] = select_bits(y, x >> s, m);
        }
    }
}

// ---------------------------------------------------------------- coefficient order
//
// Sequency of a transform coefficient along one axis: index 0 is the
// coarse average, 1 the coarse detail, 2 and 3 the fine details.  Codes
// list coefficients by the sum of the three sequencies, then by linear
// index (x fastest).
struct CodingOrder {
    int perm[64];             // perm[p] = linear index of the p-th coded coefficient
};

__host__ __device__ constexpr int axis_sequency(int i) { return i == 0 ? 0 : (i == 1 ? 1 : 2); }

__host__ __device__ constexpr CodingOrder make_coding_order() {
    CodingOrder o{};
    int n = 0;
    for (int level = 0; level <= 6; level++)
        for (int l = 0; l < 64; l++)
            if (axis_sequency(l & 3) + axis_sequency((l >> 2) & 3) + axis_sequency(l >> 4) == level) o.perm[n++] = l;
    return o;
}

// pos[l] = place of linear index l in the coded order (the inverse of perm)
struct CodingInverse {
    int pos[64];
};

__host__ __device__ constexpr CodingInverse make_coding_inverse(const CodingOrder &o) {
    CodingInverse v{};
    for (int p = 0; p < 64; p++) v.pos[o.perm[p]] = p;
    return v;
}

constexpr int kPrecision = 27;        // integer bits of the block-floating-point form
constexpr uint32_t kNegaMask = 0xAAAAAAAAu;

}  // namespace bcmc
