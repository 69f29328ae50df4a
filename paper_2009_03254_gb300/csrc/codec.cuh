// Fixed-rate 4x4x4 block codec, device side (paper Section 4.2.1: each new
// block is decoded by one thread straight into its cache slot; the format
// follows ZFP's fixed-rate mode as summarised in Section 3.3.4).
//
// Block format, rate*64 bits in `rate` little-endian 64-bit words, bits
// taken LSB first:
//   bit 0      non-zero flag (0: all 64 samples are +0, the rest is padding)
//   bits 1..8  emax + 127, emax = largest binary exponent in the block
//              (frexp convention, at least -126)
//   then       the 32 bit planes, most significant first, of 64 negabinary
//              coefficients listed in sequency order.  In each plane, the
//              coefficients already reached are sent verbatim; then group
//              tests: a 1 means some later coefficient has a one in this
//              plane, followed by the later bits one by one up to and
//              including that one (a one in the last coefficient is not
//              sent); a 0 ends the plane.  Coding stops exactly when the
//              block's bits are used up; unread bits count as zero.
// Samples are q = trunc(v * 2^(27 - emax)) integers, decorrelated by a
// two-level integer S-transform along x, then y, then z; the decoder runs
// the exact inverse in 32-bit wrap-around arithmetic and returns
// (float)q * 2^(emax - 27), correctly rounded.
#pragma once

#include "common.cuh"

namespace bcmc {

__device__ __forceinline__ uint64_t low_mask(uint32_t n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// one word of the stream: through the read-only path unless the same kernel
// may have written it
template <bool kReadOnly>
__device__ __forceinline__ uint64_t load_word(const uint64_t *p) {
    if constexpr (kReadOnly) return __ldg(p);
    else return *p;
}

// A 128-bit window over a block's stream: bits [base, base+128) of the
// block in two words, refilled one word at a time, so each word of the
// block is loaded once.
template <bool kReadOnly>
struct BitWindow {
    const uint64_t *w;
    uint32_t nwords, next, base;
    uint64_t w0, w1;
    __device__ __forceinline__ void init(const uint64_t *words, uint32_t n) {
        w = words;
        nwords = n;
        w0 = load_word<kReadOnly>(w);
        w1 = n > 1 ? load_word<kReadOnly>(w + 1) : 0ull;
        next = 2;
        base = 0;
    }
    // 64 bits starting at pos (pos - base < 64 is kept by advance)
    __device__ __forceinline__ uint64_t peek(uint32_t pos) const {
        const uint32_t sh = pos - base;
        return sh ? (w0 >> sh) | (w1 << (64 - sh)) : w0;
    }
    // call after pos moved forward by at most 64 bits
    __device__ __forceinline__ void advance(uint32_t pos) {
        if (pos - base >= 64) {
            w0 = w1;
            w1 = next < nwords ? load_word<kReadOnly>(w + next) : 0ull;
            next++;
            base += 64;
        }
    }
};

// inverse of one two-level S-transform step on (ll, hh, h0, h1) -> (a, b, c, d)
__device__ __forceinline__ void inv_lift4(int32_t &p0, int32_t &p1, int32_t &p2, int32_t &p3) {
    const int32_t ll = p0, hh = p1, h0 = p2, h1 = p3;
    const int32_t l1 = (int32_t)((uint32_t)ll - (uint32_t)(hh >> 1));
    const int32_t l0 = (int32_t)((uint32_t)hh + (uint32_t)l1);
    const int32_t b = (int32_t)((uint32_t)l0 - (uint32_t)(h0 >> 1));
    const int32_t a = (int32_t)((uint32_t)h0 + (uint32_t)b);
    const int32_t d = (int32_t)((uint32_t)l1 - (uint32_t)(h1 >> 1));
    const int32_t c = (int32_t)((uint32_t)h1 + (uint32_t)d);
    p0 = a; p1 = b; p2 = c; p3 = d;
}

// forward step (a, b, c, d) -> (ll, hh, h0, h1); inputs |x| < 2^29
__device__ __forceinline__ void fwd_lift4(int32_t &p0, int32_t &p1, int32_t &p2, int32_t &p3) {
    const int32_t a = p0, b = p1, c = p2, d = p3;
    const int32_t h0 = a - b, l0 = b + (h0 >> 1);
    const int32_t h1 = c - d, l1 = d + (h1 >> 1);
    const int32_t hh = l0 - l1, ll = l1 + (hh >> 1);
    p0 = ll; p1 = hh; p2 = h0; p3 = h1;
}

// (float)q * 2^e with one rounding; e in [-154, 101]
__device__ __forceinline__ float scale_pow2(int32_t q, int e) {
    const float f = __int2float_rn(q);
    if (e >= -126) return __fmul_rn(f, __int_as_float((e + 127) << 23));   // exact unless it overflows
    // f * 2^(e+64) is exact and normal; the final multiply rounds once
    return __fmul_rn(__fmul_rn(f, __int_as_float((e + 64 + 127) << 23)), __int_as_float((127 - 64) << 23));
}

// Decode one block of `rate` words into out[64] (block-local order).
// `planes` is this thread's column of a shared-memory scratch area:
// plane k lives at planes[k * stride].
template <bool kReadOnly = true>
__device__ __forceinline__ void decode_block(const uint64_t *__restrict__ w, uint32_t rate, float (&out)[64],
                                             uint64_t *planes, uint32_t stride) {
    BitWindow<kReadOnly> bw;
    bw.init(w, rate);
    if (!(bw.w0 & 1ull)) {
#pragma unroll
        for (int i = 0; i < 64; i++) out[i] = 0.0f;
        return;
    }
    const int emax = (int)((bw.w0 >> 1) & 0xFFu) - 127;
    const uint32_t end = rate * 64u;
    uint32_t pos = 9;
    uint32_t n = 0;                        // coefficients reached by the group tests
    // Up to kTests group tests per iteration, preceded at the start of a
    // plane by the plane's verbatim bits (predicated, so every lane runs the
    // same instructions; a lane whose plane has ended sits out the rest of
    // the iteration).  Lanes of a warp decode different blocks; one loop of
    // uniform steps keeps them together even when their planes hold
    // different numbers of group tests, and several tests per step spread
    // the step's fixed cost.  Fixed-rate noise blocks at 8 bits/value code
    // about 16 planes with 1.6 group tests each on average: two tests per
    // step measured fastest (one: 4% slower, three: 1.5% slower).
    constexpr int kTests = 2;
    int k = 31;                            // plane number, most significant first
    uint64_t x = 0;
    bool opening = true;
    {
        // Until a coefficient is reached, a plane has no verbatim bits and a
        // 0 group test ends it: each 0 bit here is a whole empty plane.
        const uint64_t win = bw.peek(pos);
        uint32_t z = win ? (uint32_t)__ffsll((long long)win) - 1u : 64u;
        z = min(z, min(32u, end - pos));
        for (uint32_t j = 0; j < z; j++) planes[(uint32_t)(31 - (int)j) * stride] = 0ull;
        k -= (int)z;
        pos += z;
        bw.advance(pos);
    }
    while (k >= 0 && pos < end) {
        // the verbatim bits of the n coefficients reached so far
        const uint32_t m = opening ? min(n, end - pos) : 0u;
        const uint64_t pk = bw.peek(pos);
        x = opening ? (pk & low_mask(m)) : x;
        pos += m;
        bw.advance(pos);
        // a plane ends after its verbatim bits when every coefficient is
        // reached or the budget is spent (otherwise n < 64 and pos < end)
        bool plane_done = n >= 64 || pos >= end;
#pragma unroll
        for (int test = 0; test < kTests; test++) {
            if (plane_done) continue;
            const uint64_t win = bw.peek(pos);
            pos += 1;
            if (!(win & 1ull)) {           // no later coefficient has a one here
                plane_done = true;
            } else {
                const uint32_t limit = 63u - n;                 // bits that may be sent
                const uint32_t cnt = min(limit, end - pos);
                const uint64_t y = (win >> 1) & low_mask(cnt);
                if (y) {
                    const uint32_t z = (uint32_t)__ffsll((long long)y) - 1u;
                    pos += z + 1;
                    n += z;
                    x |= 1ull << n;
                    n += 1;
                } else if (cnt == limit) {
                    pos += limit;
                    x |= 1ull << 63;
                    n = 64;
                } else {
                    pos = end;             // the budget ran out inside the scan
                }
                plane_done = n >= 64 || pos >= end;
            }
            bw.advance(pos);
        }
        if (plane_done) {
            planes[(uint32_t)k * stride] = x;
            k--;
        }
        opening = plane_done;
    }
    for (; k >= 0; k--) planes[(uint32_t)k * stride] = 0ull;
    constexpr CodingOrder order = make_coding_order();
    int32_t q[64];
    uint32_t a[32];
#pragma unroll
    for (int j = 0; j < 32; j++) a[j] = (uint32_t)planes[(uint32_t)j * stride];
    transpose32(a);                        // a[i] = negabinary coefficient i
#pragma unroll
    for (int p = 0; p < 32; p++) q[order.perm[p]] = (int32_t)((a[p] ^ kNegaMask) - kNegaMask);
#pragma unroll
    for (int j = 0; j < 32; j++) a[j] = (uint32_t)(planes[(uint32_t)j * stride] >> 32);
    transpose32(a);                        // a[i] = coefficient 32 + i
#pragma unroll
    for (int p = 0; p < 32; p++) q[order.perm[32 + p]] = (int32_t)((a[p] ^ kNegaMask) - kNegaMask);
#pragma unroll
    for (int i = 0; i < 16; i++) inv_lift4(q[i], q[i + 16], q[i + 32], q[i + 48]);             // z
#pragma unroll
    for (int z = 0; z < 4; z++)
#pragma unroll
        for (int x = 0; x < 4; x++) inv_lift4(q[x + 16 * z], q[x + 4 + 16 * z], q[x + 8 + 16 * z], q[x + 12 + 16 * z]);  // y
#pragma unroll
    for (int i = 0; i < 16; i++) inv_lift4(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]);  // x
    const int e = emax - kPrecision;
#pragma unroll
    for (int i = 0; i < 64; i++) out[i] = scale_pow2(q[i], e);
}

// ---------------------------------------------------------------- encoder (input generation)

struct BitWriter {
    uint64_t *w;
    uint32_t nwords;
    uint32_t pos, end;
    uint64_t acc;                          // bits not yet stored, starting at word pos>>6
    __device__ void put(uint64_t bits, uint32_t count) {   // count <= 64, caller respects the budget
        while (count) {
            const uint32_t off = pos & 63;
            const uint32_t take = min(count, 64u - off);
            acc |= (bits & low_mask(take)) << off;
            bits = take < 64 ? bits >> take : 0;
            count -= take;
            pos += take;
            if ((pos & 63) == 0) { w[(pos >> 6) - 1] = acc; acc = 0; }
        }
    }
    __device__ uint32_t room() const { return end - pos; }
    __device__ void flush() {
        if (pos & 63) w[pos >> 6] = acc;
        for (uint32_t i = (pos + 63) >> 6; i < nwords; i++) w[i] = 0;
    }
};

// Encode v[64] into `rate` words at w.
__device__ __forceinline__ void encode_block(const float (&v)[64], uint32_t rate, uint64_t *w) {
    BitWriter bw{w, rate, 0, rate * 64u, 0};
    int maxe = 0;
    bool nonzero = false;
#pragma unroll
    for (int i = 0; i < 64; i++) {
        const uint32_t b = __float_as_uint(v[i]);
        nonzero |= (b & 0x7FFFFFFFu) != 0;
        maxe = max(maxe, (int)((b >> 23) & 0xFFu));
    }
    if (!nonzero) {
        bw.put(0, 1);
        bw.flush();
        return;
    }
    const int emax = maxe - 126;           // frexp exponent of the largest sample, >= -126
    bw.put(1u | ((uint32_t)(emax + 127) << 1), 9);
    int32_t q[64];
#pragma unroll
    for (int i = 0; i < 64; i++) {
        const uint32_t b = __float_as_uint(v[i]);
        const int E = (int)((b >> 23) & 0xFFu);
        const uint32_t M = E ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
        const int s = max(E, 1) - 150 + kPrecision - emax;   // |v| * 2^(P-emax) = M * 2^s
        uint32_t mag = s >= 0 ? (M << s) : (s > -32 ? (M >> -s) : 0u);
        q[i] = (b >> 31) ? -(int32_t)mag : (int32_t)mag;
    }
#pragma unroll
    for (int i = 0; i < 16; i++) fwd_lift4(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]);  // x
#pragma unroll
    for (int z = 0; z < 4; z++)
#pragma unroll
        for (int x = 0; x < 4; x++) fwd_lift4(q[x + 16 * z], q[x + 4 + 16 * z], q[x + 8 + 16 * z], q[x + 12 + 16 * z]);  // y
#pragma unroll
    for (int i = 0; i < 16; i++) fwd_lift4(q[i], q[i + 16], q[i + 32], q[i + 48]);             // z
    constexpr CodingOrder order = make_coding_order();
    uint32_t lo[32], hi[32];
#pragma unroll
    for (int p = 0; p < 64; p++) {
        const uint32_t u = ((uint32_t)q[order.perm[p]] + kNegaMask) ^ kNegaMask;
        if (p < 32) lo[p] = u; else hi[p - 32] = u;
    }
    transpose32(lo);                       // lo[k] = plane k of coefficients 0-31
    transpose32(hi);
    uint32_t n = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) {
        const int k = 31 - j;
        const uint64_t x = (uint64_t)lo[k] | ((uint64_t)hi[k] << 32);
        if (bw.room() == 0) break;
        {
            const uint32_t m = min(n, bw.room());
            if (m) bw.put(x, m);
            if (m < n) break;
        }
        bool out = false;
        while (n < 64) {
            if (bw.room() == 0) { out = true; break; }
            const uint64_t rest = x >> n;
            if (!rest) { bw.put(0, 1); break; }
            bw.put(1, 1);
            const uint32_t jpos = n + (uint32_t)__ffsll((long long)rest) - 1u;  // first one at or after n
            if (jpos < 63) {
                const uint32_t len = jpos - n + 1;          // zeros then the one
                const uint32_t r = bw.room();
                if (len > r) { bw.put(0, r); out = true; break; }
                bw.put(1ull << (len - 1), len);
                n = jpos + 1;
            } else {
                const uint32_t len = 63 - n;                // zeros up to coefficient 62; 63's one implied
                const uint32_t r = bw.room();
                if (len > r) { bw.put(0, r); out = true; break; }
                if (len) bw.put(0, len);
                n = 64;
            }
        }
        if (out) break;
    }
    bw.flush();
}

}  // namespace bcmc
