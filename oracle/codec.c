/*
 * Oracle codec: a fixed-rate coder for 4x4x4 blocks of float32 in the style
 * of ZFP's fixed-rate mode.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper decompresses ZFP fixed-rate blocks on the GPU, one thread per
 * block, into cache slots (Section 4.2.1, building on the ZFP port of
 * Section 3.3.4).  It relies on three properties of the fixed-rate mode:
 * 4^3 blocks, exactly rate*64 bits per block, and random access to any
 * block.  The format below has those properties and follows the steps of
 * Lindstrom (TVCG 2014): a common block exponent, conversion to integers,
 * a decorrelating integer transform, a reordering of the coefficients by
 * sequency, a negabinary mapping, and embedded coding of bit planes with
 * group tests, cut off at the bit budget.  It is not bit-compatible with
 * the ZFP library.
 *
 * Block format (64*rate bits, little-endian 64-bit words, bits LSB first):
 *   bit 0           1 if any value is non-zero, else the block is all zero
 *   bits 1..8       emax + 127, emax = max over non-zero values of the
 *                   frexp exponent, clamped below at -126
 *   then            bit planes 31..0 of the 64 negabinary coefficients
 * The integer transform is a two-level reversible S-transform (integer
 * Haar) along x, then y, then z.  Integers carry ORC_PRECISION = 27 bits so
 * that the transform's growth (one bit per axis) stays inside the range
 * that 32 negabinary digits represent.
 */
#include "oracle.h"
#include <math.h>
#include <string.h>
#include <assert.h>

/* ---------------- integer helpers ---------------- */

/* two's-complement wrap to 32 bits: the decoder's arithmetic is modulo 2^32 */
static int64_t wrap32(int64_t x)
{
    int64_t y = x & 0xffffffffLL;
    if (y >= 0x80000000LL) y -= 0x100000000LL;
    return y;
}

/* floor(x / 2) */
static int64_t floor_half(int64_t x)
{
    return x >= 0 ? x / 2 : -((-x + 1) / 2);
}

/* negabinary digits of x: x = sum_k d_k (-2)^k, d_k in {0,1} */
uint32_t orc_to_negabinary(int64_t x)
{
    uint32_t u = 0;
    int k = 0;
    while (x != 0) {
        assert(k < 32);
        int64_t r = x % -2;          /* remainder in {-1, 0, 1} */
        x /= -2;
        if (r < 0) { r += 2; x += 1; }
        if (r) u |= 1u << k;
        k++;
    }
    return u;
}

/* value of 32 negabinary digits, wrapped to int32 */
int32_t orc_from_negabinary(uint32_t u)
{
    int64_t v = 0, w = 1;
    for (int k = 0; k < 32; k++) {
        if (u >> k & 1u) v += w;
        w *= -2;
    }
    return (int32_t)wrap32(v);
}

/* ---------------- decorrelating transform ---------------- */

/* forward two-level S-transform of (a,b,c,d) -> (ll, hh, h0, h1) */
static void fwd4(int64_t *p, int s)
{
    int64_t a = p[0], b = p[s], c = p[2 * s], d = p[3 * s];
    int64_t h0 = wrap32(a - b), l0 = wrap32(b + floor_half(h0));
    int64_t h1 = wrap32(c - d), l1 = wrap32(d + floor_half(h1));
    int64_t hh = wrap32(l0 - l1), ll = wrap32(l1 + floor_half(hh));
    p[0] = ll; p[s] = hh; p[2 * s] = h0; p[3 * s] = h1;
}

/* exact inverse of fwd4 */
static void inv4(int64_t *p, int s)
{
    int64_t ll = p[0], hh = p[s], h0 = p[2 * s], h1 = p[3 * s];
    int64_t l1 = wrap32(ll - floor_half(hh));
    int64_t l0 = wrap32(hh + l1);
    int64_t b = wrap32(l0 - floor_half(h0));
    int64_t a = wrap32(h0 + b);
    int64_t d = wrap32(l1 - floor_half(h1));
    int64_t c = wrap32(h1 + d);
    p[0] = a; p[s] = b; p[2 * s] = c; p[3 * s] = d;
}

void orc_forward_lift(int64_t q[64])
{
    for (int z = 0; z < 4; z++) for (int y = 0; y < 4; y++) fwd4(q + 4 * y + 16 * z, 1);
    for (int z = 0; z < 4; z++) for (int x = 0; x < 4; x++) fwd4(q + x + 16 * z, 4);
    for (int y = 0; y < 4; y++) for (int x = 0; x < 4; x++) fwd4(q + x + 4 * y, 16);
}

void orc_inverse_lift(int64_t q[64])
{
    for (int y = 0; y < 4; y++) for (int x = 0; x < 4; x++) inv4(q + x + 4 * y, 16);
    for (int z = 0; z < 4; z++) for (int x = 0; x < 4; x++) inv4(q + x + 16 * z, 4);
    for (int z = 0; z < 4; z++) for (int y = 0; y < 4; y++) inv4(q + 4 * y + 16 * z, 1);
}

/* Coding order: coefficients sorted by total sequency s(i)+s(j)+s(k), with
 * s = {0,1,2,2} for (ll, hh, h0, h1), ties by linear index.  perm[p] is the
 * linear index of the p-th coded coefficient. */
void orc_coding_order(int perm[64])
{
    static const int seq[4] = {0, 1, 2, 2};
    int key[64];
    for (int n = 0; n < 64; n++) {
        perm[n] = n;
        key[n] = seq[n & 3] + seq[(n >> 2) & 3] + seq[n >> 4];
    }
    /* insertion sort, stable: keeps linear order inside a sequency level */
    for (int i = 1; i < 64; i++) {
        int v = perm[i], j = i - 1;
        while (j >= 0 && key[perm[j]] > key[v]) { perm[j + 1] = perm[j]; j--; }
        perm[j + 1] = v;
    }
}

/* ---------------- bit I/O with a hard budget ---------------- */

typedef struct { uint64_t *w; int pos, end; } writer;
typedef struct { const uint64_t *w; int pos, end; } reader;

static int w_room(const writer *s) { return s->pos < s->end; }
static void w_put(writer *s, int bit)
{
    assert(s->pos < s->end);
    if (bit) s->w[s->pos >> 6] |= 1ull << (s->pos & 63);
    s->pos++;
}
static int r_room(const reader *s) { return s->pos < s->end; }
static int r_get(reader *s)
{
    assert(s->pos < s->end);
    int b = (int)(s->w[s->pos >> 6] >> (s->pos & 63) & 1u);
    s->pos++;
    return b;
}

/* ---------------- block coder ---------------- */

void orc_encode_block(const float v[64], int rate, uint64_t *out)
{
    writer s = {out, 0, 64 * rate};
    memset(out, 0, (size_t)rate * 8);
    int nonzero = 0;
    for (int i = 0; i < 64; i++) if (v[i] != 0.0f) nonzero = 1;
    w_put(&s, nonzero);
    if (!nonzero) return;

    int emax = -126;
    for (int i = 0; i < 64; i++) {
        if (v[i] == 0.0f) continue;
        int e;
        frexp((double)v[i], &e);
        if (e > emax) emax = e;
    }
    for (int b = 0; b < 8; b++) w_put(&s, (emax + 127) >> b & 1);

    /* block floating point: q = trunc(v * 2^(P - emax)), exact in double */
    int64_t q[64];
    for (int i = 0; i < 64; i++) {
        q[i] = (int64_t)trunc(ldexp((double)v[i], ORC_PRECISION - emax));
        assert(q[i] < (1LL << ORC_PRECISION) && q[i] > -(1LL << ORC_PRECISION));
    }
    orc_forward_lift(q);

    int perm[64];
    orc_coding_order(perm);
    uint32_t u[64];
    for (int p = 0; p < 64; p++) u[p] = orc_to_negabinary(q[perm[p]]);

    /* embedded bit-plane coding, most significant plane first.  n counts
     * the coefficients already reached by the group tests; their bits are
     * sent verbatim.  A group test says whether any later coefficient has a
     * one in this plane; if so the later bits are sent one by one up to and
     * including that one (the last coefficient's one is implied). */
    int n = 0;
    for (int k = 31; k >= 0; k--) {
        for (int i = 0; i < n; i++) {
            if (!w_room(&s)) return;
            w_put(&s, u[i] >> k & 1u);
        }
        while (n < 64) {
            if (!w_room(&s)) return;
            int g = 0;
            for (int i = n; i < 64; i++) g |= (int)(u[i] >> k & 1u);
            w_put(&s, g);
            if (!g) break;
            for (;;) {
                if (n == 63) { n = 64; break; }
                if (!w_room(&s)) return;
                int b = (int)(u[n] >> k & 1u);
                w_put(&s, b);
                n++;
                if (b) break;
            }
        }
    }
}

void orc_decode_block(const uint64_t *in, int rate, float v[64])
{
    reader s = {in, 0, 64 * rate};
    if (!r_get(&s)) {
        for (int i = 0; i < 64; i++) v[i] = 0.0f;
        return;
    }
    int ebits = 0;
    for (int b = 0; b < 8; b++) ebits |= r_get(&s) << b;
    int emax = ebits - 127;

    uint32_t u[64];
    memset(u, 0, sizeof u);
    int n = 0;
    for (int k = 31; k >= 0; k--) {
        for (int i = 0; i < n; i++) {
            if (!r_room(&s)) goto done;
            if (r_get(&s)) u[i] |= 1u << k;
        }
        while (n < 64) {
            if (!r_room(&s)) goto done;
            if (!r_get(&s)) break;
            for (;;) {
                if (n == 63) { u[63] |= 1u << k; n = 64; break; }
                if (!r_room(&s)) goto done;
                int b = r_get(&s);
                if (b) u[n] |= 1u << k;
                n++;
                if (b) break;
            }
        }
    }
done:;
    int perm[64];
    orc_coding_order(perm);
    int64_t q[64];
    for (int p = 0; p < 64; p++) q[perm[p]] = orc_from_negabinary(u[p]);
    orc_inverse_lift(q);
    /* the integer becomes a float32 first (round to nearest even), then is
     * scaled by 2^(emax - P): exact while the result is normal, a second
     * rounding when it is subnormal (as ZFP dequantises) */
    for (int i = 0; i < 64; i++)
        v[i] = ldexpf((float)(int32_t)q[i], emax - ORC_PRECISION);
}

/* ---------------- volumes ---------------- */

static int imin(int a, int b) { return a < b ? a : b; }

/* gather block (bx,by,bz); voxels past the volume edge replicate the last
 * valid sample along each axis */
static void gather_block(const float *f, int nx, int ny, int nz, int bx, int by, int bz, float v[64])
{
    for (int k = 0; k < 4; k++)
        for (int j = 0; j < 4; j++)
            for (int i = 0; i < 4; i++) {
                int x = imin(4 * bx + i, nx - 1), y = imin(4 * by + j, ny - 1), z = imin(4 * bz + k, nz - 1);
                v[i + 4 * j + 16 * k] = f[(int64_t)x + (int64_t)nx * (y + (int64_t)ny * z)];
            }
}

/* Encode a volume.  bmin/bmax receive each block's range over its decoded,
 * in-volume voxels (the per-block ranges of Section 4.1; taken from the
 * decoded values so that the block method sees exactly the field it
 * triangulates). */
void orc_encode_volume(const float *field, int nx, int ny, int nz, int rate,
                       uint64_t *bits, float *bmin, float *bmax)
{
    int nbx = (nx + 3) / 4, nby = (ny + 3) / 4, nbz = (nz + 3) / 4;
    float v[64], d[64];
    for (int bz = 0; bz < nbz; bz++)
        for (int by = 0; by < nby; by++)
            for (int bx = 0; bx < nbx; bx++) {
                int64_t id = bx + (int64_t)nbx * (by + (int64_t)nby * bz);
                uint64_t *w = bits + id * rate;
                gather_block(field, nx, ny, nz, bx, by, bz, v);
                orc_encode_block(v, rate, w);
                orc_decode_block(w, rate, d);
                float lo = INFINITY, hi = -INFINITY;
                for (int k = 0; k < 4; k++)
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            if (4 * bx + i >= nx || 4 * by + j >= ny || 4 * bz + k >= nz) continue;
                            float x = d[i + 4 * j + 16 * k];
                            if (x < lo) lo = x;
                            if (x > hi) hi = x;
                        }
                bmin[id] = lo;
                bmax[id] = hi;
            }
}

void orc_decode_volume(const uint64_t *bits, int nx, int ny, int nz, int rate, float *field)
{
    int nbx = (nx + 3) / 4, nby = (ny + 3) / 4, nbz = (nz + 3) / 4;
    float d[64];
    for (int bz = 0; bz < nbz; bz++)
        for (int by = 0; by < nby; by++)
            for (int bx = 0; bx < nbx; bx++) {
                int64_t id = bx + (int64_t)nbx * (by + (int64_t)nby * bz);
                orc_decode_block(bits + id * rate, rate, d);
                for (int k = 0; k < 4; k++)
                    for (int j = 0; j < 4; j++)
                        for (int i = 0; i < 4; i++) {
                            int x = 4 * bx + i, y = 4 * by + j, z = 4 * bz + k;
                            if (x >= nx || y >= ny || z >= nz) continue;
                            field[(int64_t)x + (int64_t)nx * (y + (int64_t)ny * z)] = d[i + 4 * j + 16 * k];
                        }
            }
}

void orc_decode_blocks(const uint64_t *bits, int rate, const uint32_t *ids, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; i++) orc_decode_block(bits + (int64_t)ids[i] * rate, rate, out + 64 * i);
}
