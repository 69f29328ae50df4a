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
// the exact inverse in 32-bit wrap-around arithmetic and returns the
// float32 of q (rounded to nearest even) times 2^(emax - 27): exact while
// the result is normal, rounded once more when it is subnormal.
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

// ---------------------------------------------------------------- staging
//
// A warp decodes up to 32 blocks at a time, one per lane (Section 4.2.1
// decodes one block per thread).  The blocks' words are first copied into
// a per-warp staging area of shared memory by coalesced loads: in each
// round consecutive lanes load consecutive 8-byte words, block after block,
// so a warp instruction reads 256 contiguous bytes of every block it
// touches.  Each lane then parses its own block from shared memory.
//
// A staged block takes 2R + 1 32-bit words (its 2R words, then a zero pad
// word; the odd stride spreads the lanes' reads over the banks), and the
// area ends with two more words, so a window may read up to two words past
// the block's last one (bits past the budget are never used).

__host__ __device__ constexpr uint32_t stage_words(uint32_t rate) { return 32u * (2u * rate + 1u) + 2u; }

// Copy block `id` of each lane that has one (`have`) into the warp's
// staging area `stage` (stage_words(rate) words).  Called by all 32 lanes.
template <bool kReadOnly>
__device__ __forceinline__ void stage_blocks(const uint64_t *__restrict__ bits, uint32_t rate, uint32_t id, bool have,
                                             uint32_t *stage) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t stride = 2u * rate + 1u;
    const uint32_t magic = (65535u + rate) / rate;          // ceil(2^16 / rate): j / rate = (j * magic) >> 16, j < 1024
    const uint32_t have_mask = __ballot_sync(0xffffffffu, have);
    // Rounds of kInFlight words per lane: every load of a round is issued
    // before the first shared store, so a lane waits for one memory latency
    // per round rather than one per word.  Round k of lane j copies word
    // j + 32k of the warp's 32 * rate, i.e. word w of block q.
    constexpr uint32_t kInFlight = 8;
    for (uint32_t k0 = 0; k0 < rate; k0 += kInFlight) {      // the same number of rounds in every lane
        uint64_t v[kInFlight];
#pragma unroll
        for (uint32_t k = 0; k < kInFlight; k++) {
            const uint32_t j = lane + 32u * (k0 + k);
            const uint32_t q = (j * magic) >> 16, w = j - q * rate;
            const uint32_t bq = __shfl_sync(0xffffffffu, id, (int)(q & 31u));
            v[k] = 0ull;
            if (k0 + k < rate && ((have_mask >> q) & 1u)) v[k] = load_word<kReadOnly>(bits + (size_t)bq * rate + w);
        }
#pragma unroll
        for (uint32_t k = 0; k < kInFlight; k++) {
            const uint32_t j = lane + 32u * (k0 + k);
            const uint32_t q = (j * magic) >> 16, w = j - q * rate;
            if (k0 + k < rate) {
                stage[q * stride + 2u * w] = (uint32_t)v[k];
                stage[q * stride + 2u * w + 1u] = (uint32_t)(v[k] >> 32);
            }
        }
    }
    stage[lane * stride + 2u * rate] = 0u;
    if (lane < 2) stage[32u * stride + lane] = 0u;
    __syncwarp();
}

// Shared-memory accesses by 32-bit shared-window address (the decoder's
// loops address the staging area and plane columns this way, so every
// access is a plain shared-memory load or store).
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_u64(uint32_t a, uint32_t lo, uint32_t hi) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(a), "r"(lo), "r"(hi));
}

// Bit windows over a staged block at shared address `w` (32-bit words).
struct StagedBits {
    uint32_t w;
    // 32 bits starting at bit pos
    __device__ __forceinline__ uint32_t win32(uint32_t pos) const {
        const uint32_t a = w + ((pos >> 5) << 2);
        return __funnelshift_r(lds_u32(a), lds_u32(a + 4), pos & 31u);
    }
    // 64 bits starting at bit pos, as two halves
    __device__ __forceinline__ void win64(uint32_t pos, uint32_t &lo, uint32_t &hi) const {
        const uint32_t a = w + ((pos >> 5) << 2), sh = pos & 31u;
        const uint32_t x = lds_u32(a), y = lds_u32(a + 4), z = lds_u32(a + 8);
        lo = __funnelshift_r(x, y, sh);
        hi = __funnelshift_r(y, z, sh);
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

// the same on two's-complement words held as uint32 (wrap-around arithmetic)
__device__ __forceinline__ void inv_lift4u(uint32_t &p0, uint32_t &p1, uint32_t &p2, uint32_t &p3) {
    const uint32_t ll = p0, hh = p1, h0 = p2, h1 = p3;
    const uint32_t l1 = ll - (uint32_t)((int32_t)hh >> 1);
    const uint32_t l0 = hh + l1;
    const uint32_t b = l0 - (uint32_t)((int32_t)h0 >> 1);
    const uint32_t a = h0 + b;
    const uint32_t d = l1 - (uint32_t)((int32_t)h1 >> 1);
    const uint32_t c = h1 + d;
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

// out[l] = float32(q[l]) * 2^e, e in [-154, 101]: the conversion rounds to
// nearest even; the scaling is exact while the result is normal and rounds
// once more when it is subnormal.  One branch per block (uniform in a warp
// unless some of its blocks have tiny exponents).
__device__ __forceinline__ void scale_block(const uint32_t (&q)[64], int e, float (&out)[64]) {
    if (e >= -126) {
        const float sc = __int_as_float((e + 127) << 23);
#pragma unroll
        for (int l = 0; l < 64; l++) out[l] = __fmul_rn(__int2float_rn((int32_t)q[l]), sc);
    } else {
        // f * 2^(e+64) is exact and normal; the final multiply rounds once
        const float sc = __int_as_float((e + 64 + 127) << 23), down = __int_as_float((127 - 64) << 23);
#pragma unroll
        for (int l = 0; l < 64; l++) out[l] = __fmul_rn(__fmul_rn(__int2float_rn((int32_t)q[l]), sc), down);
    }
}

// ---------------------------------------------------------------- group-test steps
//
// The group tests of a plane (after its verbatim bits) are read eight bits
// at a time through a 512-entry table: for a state (0: the next bit is a
// group test, 1: it is a run bit) and a byte of the stream, the entry holds
// what reading those bits one by one does --
//   bits 0-7    the run bits met, in order (coefficient n, n + 1, ...)
//   bits 8-11   how many run bits that is
//   bits 12-15  bits consumed (8, or fewer when a 0 test ends the plane)
//   bit 16      a 0 test ended the plane
//   bit 17      the state after the consumed bits
// A group test is a 1 followed by the run of later coefficients' bits up to
// and including the next one, or the 0 that ends the plane, so without the
// budget and coefficient 63's implied one the table step is exactly eight
// steps of that rule.  The decoder checks the two exceptions around it.
__host__ __device__ constexpr uint32_t group_step_entry(uint32_t state, uint32_t byte) {
    uint32_t runbits = 0, count = 0, consumed = 8, ended = 0;
    for (uint32_t i = 0; i < 8; i++) {
        const uint32_t bit = (byte >> i) & 1u;
        if (state == 0) {
            if (!bit) {
                ended = 1;
                consumed = i + 1;
                break;
            }
            state = 1;
        } else {
            runbits |= bit << count;
            count++;
            if (bit) state = 0;
        }
    }
    return runbits | (count << 8) | (consumed << 12) | (ended << 16) | (state << 17);
}

constexpr uint32_t kGroupTableEntries = 512;

// fill a block's copy of the table (all threads; the caller synchronises)
__device__ __forceinline__ void load_group_table(uint32_t *tab) {
    for (uint32_t i = threadIdx.x; i < kGroupTableEntries; i += blockDim.x) tab[i] = group_step_entry(i >> 8, i & 255u);
}

// One group-test event read bit by bit, with every rule: from state 0 a
// test bit (a 0 ends the plane), then (or from state 1) the rest of a run,
// at most 63 - n run bits (coefficient 63's one is implied) and no bit past
// the budget.  Updates pos, n, the plane (xlo, xhi) and `ended`.
__device__ __forceinline__ void group_event_exact(const StagedBits &st, uint32_t end, uint32_t &pos, uint32_t &n,
                                                  uint32_t &xlo, uint32_t &xhi, uint32_t state, bool &ended) {
    if (state == 0) {
        const uint32_t g = st.win32(pos);
        pos += 1;
        if (!(g & 1u)) {
            ended = true;
            return;
        }
    }
    const uint32_t lim = 63u - n;                // run bits that may be sent
    const uint32_t scan = min(lim, end - min(end, pos));   // of which the budget holds
    uint32_t z = 64u;                            // zeros before the run's one (64: none)
    for (uint32_t off = 0; off < scan; off += 32) {
        uint32_t w = st.win32(pos + off);
        if (scan - off < 32u) w &= (1u << (scan - off)) - 1u;
        if (w) {
            z = off + (uint32_t)__ffs(w) - 1u;
            break;
        }
    }
    if (z < 64u) {                               // z zeros, then coefficient n + z's one
        pos += z + 1;
        n += z;
        if (n < 32u) xlo |= 1u << n;
        else xhi |= 1u << (n - 32u);
        n += 1;
    } else if (scan == lim) {                    // zeros up to coefficient 62: 63's one is implied
        pos += lim;
        xhi |= 1u << 31;
        n = 64;
    } else {
        pos = end;                               // the budget ran out inside the run
    }
}

// Parse the bit planes of a staged block of `rate` words: plane k (most
// significant first) goes to shared address planes + k * stride as a 64-bit
// word whose bit i belongs to the i-th coded coefficient.  A zero block (flag bit 0: the
// rest is not read) has all planes zero.  Sets emax.
//
// The lanes of a warp parse different blocks.  One loop of uniform steps
// keeps them together: a step takes the plane's verbatim bits when it opens
// a plane, then up to kSteps table steps of its group tests, all
// predicated; a lane whose block is done sits the remaining steps out.
// Once every coefficient is reached (n = 64) a plane is its 64 verbatim
// bits, which a short loop of its own copies.
template <int kSteps = 2>
__device__ __forceinline__ void parse_planes(const StagedBits &st, uint32_t rate, uint32_t tab, uint32_t planes,
                                             uint32_t stride, int &emax) {
    const uint32_t head = lds_u32(st.w);
    emax = (int)((head >> 1) & 0xFFu) - 127;
    const uint32_t end = (head & 1u) ? rate * 64u : 0u;
    uint32_t pos = 9, n = 0;               // n: coefficients reached by the group tests
    int k = 31;                            // plane, most significant first
    if (end) {
        // Until a coefficient is reached, a plane has no verbatim bits and a
        // 0 group test ends it: each 0 bit here is a whole empty plane
        // (end - pos >= 55 at every rate, so the window is inside the budget).
        const uint32_t win = st.win32(pos);
        const uint32_t z = win ? (uint32_t)__ffs(win) - 1u : 32u;
        for (uint32_t j = 0; j < z; j++) sts_u64(planes + (31u - j) * stride, 0u, 0u);
        k -= (int)z;
        pos += z;
    }
    uint32_t xlo = 0u, xhi = 0u, state = 0u;
    bool opening = true, exact = false;    // exact: the next event is read bit by bit
    while (k >= 0 && pos < end && n < 64u) {
        if (opening) {                     // the verbatim bits of the n coefficients reached so far
            const uint32_t m = min(n, end - pos);
            uint32_t wlo, whi;
            st.win64(pos, wlo, whi);
            xlo = m >= 32u ? wlo : (wlo & ((1u << m) - 1u));
            xhi = m > 32u ? (whi & ((1u << (m - 32u)) - 1u)) : 0u;   // m < 64 here
            pos += m;
            state = 0u;
        }
        bool done = pos >= end;
        if (exact && !done) {              // the run reaches coefficient 63 inside the next byte
            bool ended = false;
            group_event_exact(st, end, pos, n, xlo, xhi, state, ended);
            state = 0u;
            exact = false;
            done = ended || pos >= end || n >= 64u;
        }
#pragma unroll
        for (int t = 0; t < kSteps; t++) {
            if (done || exact) continue;
            // bits past the budget read as zero: the staged block is followed
            // by a zero pad word, and a step reads at most 8 bits on
            const uint32_t byte = st.win32(pos) & 0xFFu;
            const uint32_t e = lds_u32(tab + (((state << 8) | byte) << 2));
            const uint32_t cnt = (e >> 8) & 15u;
            if (n + cnt > 63u) {           // a run bit for coefficient 63 or later: not a table step
                exact = true;
                continue;
            }
            const uint64_t bits = (uint64_t)(e & 0xFFu) << n;
            xlo |= (uint32_t)bits;
            xhi |= (uint32_t)(bits >> 32);
            n += cnt;
            pos += (e >> 12) & 15u;
            state = (e >> 17) & 1u;
            if (state && n == 63u && pos <= end) {   // the run reached coefficient 63: its one is implied
                xhi |= 1u << 31;
                n = 64;
                state = 0u;
            }
            done = ((e >> 16) & 1u) != 0u || pos >= end || n >= 64u;
        }
        if (done) {
            sts_u64(planes + (uint32_t)k * stride, xlo, xhi);
            k--;
        }
        opening = done;
    }
    // every coefficient reached: each remaining plane is the next 64 bits
    for (; k >= 0 && pos < end; k--) {
        const uint32_t m = min(64u, end - pos);
        uint32_t wlo, whi;
        st.win64(pos, wlo, whi);
        if (m < 64u) {
            wlo = m >= 32u ? wlo : (wlo & ((1u << m) - 1u));
            whi = m > 32u ? (whi & ((1u << (m - 32u)) - 1u)) : 0u;
        }
        sts_u64(planes + (uint32_t)k * stride, wlo, whi);
        pos += m;
    }
    for (; k >= 0; k--) sts_u64(planes + (uint32_t)k * stride, 0u, 0u);
}

// The second half of decoding a block, after parse_planes has written its
// bit planes (plane k at planes + k * stride bytes, shared-window address)
// and its exponent: two 32x32 bit transposes turn the planes into the 64
// negabinary coefficients, which are mapped back to integers, put in
// block order, inverse-lifted along z, y and x and scaled into out[64].
__device__ __forceinline__ void finish_planes(uint32_t pa, uint32_t ps, int emax, float (&out)[64]) {
    constexpr CodingOrder order = make_coding_order();
    uint32_t q[64];
    uint32_t a[32];
#pragma unroll
    for (int j = 0; j < 32; j++) a[j] = lds_u32(pa + (uint32_t)j * ps);
    transpose32(a);                        // a[p] = negabinary coefficient p (coded order)
#pragma unroll
    for (int p = 0; p < 32; p++) q[order.perm[p]] = (a[p] ^ kNegaMask) - kNegaMask;
#pragma unroll
    for (int j = 0; j < 32; j++) a[j] = lds_u32(pa + (uint32_t)j * ps + 4u);
    transpose32(a);                        // a[p] = coefficient 32 + p
#pragma unroll
    for (int p = 0; p < 32; p++) q[order.perm[32 + p]] = (a[p] ^ kNegaMask) - kNegaMask;
#pragma unroll
    for (int i = 0; i < 16; i++) inv_lift4u(q[i], q[i + 16], q[i + 32], q[i + 48]);             // z
#pragma unroll
    for (int z = 0; z < 4; z++)
#pragma unroll
        for (int x = 0; x < 4; x++) inv_lift4u(q[x + 16 * z], q[x + 4 + 16 * z], q[x + 8 + 16 * z], q[x + 12 + 16 * z]);  // y
#pragma unroll
    for (int i = 0; i < 16; i++) inv_lift4u(q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]);  // x
    scale_block(q, emax - kPrecision, out);
}

// Decode a staged block of `rate` words into out[64] (block-local order).
// `planes` is this thread's column of a shared-memory area: plane k lives at
// planes[k * stride].  A zero block decodes to 64 samples of +0.
__device__ __forceinline__ void decode_staged(const uint32_t *staged, uint32_t rate, const uint32_t *tab,
                                              float (&out)[64], uint64_t *planes, uint32_t stride) {
    int emax = 0;
    const uint32_t pa = smem_u32(planes), ps = stride * 8u;
    parse_planes(StagedBits{smem_u32(staged)}, rate, smem_u32(tab), pa, ps, emax);
    finish_planes(pa, ps, emax, out);
}

// Dynamic shared memory of a decoding kernel of `threads` threads: the
// plane columns (32 words of 8 bytes per thread), the group-step table, then
// one staging area per warp for blocks of up to `rate` words.
struct DecodeSmem {
    uint64_t *planes;
    uint32_t *tab;
    uint32_t *stage;          // this warp's staging area
};

__host__ __device__ constexpr size_t decode_smem_bytes(uint32_t threads, uint32_t rate) {
    return 32u * 8u * (size_t)threads + kGroupTableEntries * 4u + (size_t)(threads / 32u) * stage_words(rate) * 4u;
}

__device__ __forceinline__ DecodeSmem decode_smem_layout(uint64_t *base, uint32_t threads, uint32_t rate) {
    uint32_t *tab = reinterpret_cast<uint32_t *>(base + 32u * threads);
    return DecodeSmem{base, tab, tab + kGroupTableEntries + (threadIdx.x >> 5) * stage_words(rate)};
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
