"""Pins for the oracle's fixed-rate block codec (CPU only).

The paper fixes the codec's shape (ZFP fixed-rate mode, 4^3 blocks, one
block decodable on its own; Sections 3.3.4 and 4.2.1) but not its bits, so
the oracle codec is pinned by what holds for any such coder and by streams
worked out by hand from the format description in ``oracle/codec.c``.
"""
import math

import numpy as np
import pytest

import oracle
from synth import fields

RATES = (2, 4, 8, 16)


@pytest.mark.parametrize("rate", RATES)
@pytest.mark.parametrize("value", [1.0, -3.75, 0.1, 123456.789, -1e30, 3e-39, 2.0 ** -140, 1e-30])
def test_constant_block_is_exact(rate, value):
    # a constant block has only a DC coefficient, which costs about two bits
    # per plane: 9 + 2*32 bits fit in every rate >= 2
    v = np.full(64, value, np.float32)
    d = oracle.decode_block(oracle.encode_block(v, rate), rate)
    assert np.array_equal(d, v)


@pytest.mark.parametrize("rate", (1, 2, 8, 32))
def test_zero_block(rate):
    for v in (np.zeros(64, np.float32), np.full(64, -0.0, np.float32)):
        w = oracle.encode_block(v, rate)
        assert not w.any()                       # the zero flag is the only bit
        d = oracle.decode_block(w, rate)
        assert np.array_equal(d, np.zeros(64, np.float32)) and not np.signbit(d).any()


def test_hand_built_stream_for_one():
    # 1.0 = 0.5 * 2^1 -> emax = 1, biased 128; q = 2^(27-1) = 2^26 everywhere;
    # the transform leaves DC = 2^26 alone; 2^26 = (-2)^26 so its negabinary
    # code has only digit 26.  Planes 31..27: one group-test 0 each (bits
    # 9..13); plane 26: group test 1, DC bit 1, group test 0 (bits 14..16);
    # planes 25..0: DC bit 0 and group test 0.  69 bits, the rest zero.
    w = oracle.encode_block(np.ones(64, np.float32), 2)
    assert int(w[0]) == (1 | 1 << 8 | 1 << 14 | 1 << 15)
    assert int(w[1]) == 0
    assert np.array_equal(oracle.decode_block(w, 2), np.ones(64, np.float32))


def test_hand_built_stream_truncated():
    # the stream above cut after plane 26 (rate 1 keeps it whole): the
    # decoder must read exactly the DC and nothing else
    w = np.zeros(1, np.uint64)
    w[0] = 1 | 1 << 8 | 1 << 14 | 1 << 15
    assert np.array_equal(oracle.decode_block(w, 1), np.ones(64, np.float32))
    assert np.array_equal(oracle.encode_block(np.ones(64, np.float32), 1), w)


def test_header_fields():
    for value in (1.0, 3.0, -0.3, 1e-3, 5e4):
        w = int(oracle.encode_block(np.full(64, value, np.float32), 4)[0])
        assert w & 1 == 1
        assert (w >> 1) & 0xFF == math.frexp(value)[1] + 127


def test_negabinary_identity():
    # 32 negabinary digits <-> two's complement: u = (x + M) ^ M, M = 0xaaaaaaaa
    rng = np.random.default_rng(0)
    M = 0xAAAAAAAA
    for x in list(rng.integers(-(1 << 30), 1 << 30, 2000)) + [0, 1, -1, 2, -2, (1 << 30) - 1, -(1 << 30)]:
        x = int(x)
        u = oracle.to_negabinary(x)
        assert u == ((x + M) & 0xFFFFFFFF) ^ M
        assert oracle.from_negabinary(u) == x
        assert sum(((u >> k) & 1) * (-2) ** k for k in range(32)) == x
    for u in rng.integers(0, 1 << 32, 2000, dtype=np.uint64):
        u = int(u)
        want = (((u ^ M) - M + (1 << 31)) & 0xFFFFFFFF) - (1 << 31)
        assert oracle.from_negabinary(u) == want


def test_lift_hand_example():
    # one x-row (10, 9, 7, 8): h0 = 1, l0 = 9 + floor(1/2) = 9, h1 = -1,
    # l1 = 8 + floor(-1/2) = 7, hh = 2, ll = 7 + 1 = 8  ->  (8, 2, 1, -1).
    # A block made of 16 copies of that row is constant along y and z, so
    # the y and z passes leave only the first row.
    blk = np.tile(np.array([10, 9, 7, 8], np.int64), 16)
    c = oracle.forward_lift(blk)
    assert list(c[0:4]) == [8, 2, 1, -1]
    assert not c[4:].any()
    assert np.array_equal(oracle.inverse_lift(c), blk)


def test_lift_exact_inverse_and_range():
    rng = np.random.default_rng(1)
    for _ in range(300):
        q = rng.integers(-(1 << 27) + 1, 1 << 27, 64)
        c = oracle.forward_lift(q)
        assert np.abs(c).max() < (1 << 30)          # inside the negabinary range
        assert np.array_equal(oracle.inverse_lift(c), q)
    c = oracle.forward_lift(np.full(64, 12345, np.int64))
    assert c[0] == 12345 and not c[1:].any()         # constant -> DC only


def test_coding_order():
    perm = oracle.coding_order()
    assert sorted(perm) == list(range(64))
    seq = [0, 1, 2, 2]
    key = [seq[n & 3] + seq[(n >> 2) & 3] + seq[n >> 4] for n in perm]
    assert key == sorted(key)
    assert list(perm[:4]) == [0, 1, 4, 16]


def _errors(f, rate):
    bits, _, _ = oracle.encode_volume(f, rate)
    nz, ny, nx = f.shape
    d = oracle.decode_volume(bits, (nx, ny, nz), rate)
    e = d.astype(np.float64) - f
    return math.sqrt((e * e).mean()), np.abs(e).max(), d


@pytest.mark.parametrize("kind", ["noise", "sphere"])
def test_error_falls_with_rate(kind):
    f = fields.gradient_noise(32, 28, 24, 7) if kind == "noise" else fields.sphere_sdf(32, 28, 24, 9.0)
    errs = [_errors(f, r)[:2] for r in RATES]
    for (r0, m0), (r1, m1) in zip(errs, errs[1:]):
        assert r1 < r0 and m1 < m0


def test_rate16_error_bound():
    # measured on the oracle: the worst block error relative to the block's
    # largest magnitude is ~2e-5 (noise) and ~4e-6 (distance field) at 16
    # bits/value; 2^-10 leaves a wide margin
    for f in (fields.gradient_noise(32, 32, 32, 3), fields.sphere_sdf(32, 32, 32, 10.0)):
        _, _, d = _errors(f, 16)
        e = np.abs(d.astype(np.float64) - f).reshape(8, 4, 8, 4, 8, 4).max(axis=(1, 3, 5))
        m = np.abs(f).astype(np.float64).reshape(8, 4, 8, 4, 8, 4).max(axis=(1, 3, 5))
        assert (e / m).max() < 2.0 ** -10


def test_ranges_are_of_decoded_in_volume_voxels():
    f = fields.gradient_noise(13, 9, 6, 5)          # partial blocks on every axis
    bits, bmin, bmax = oracle.encode_volume(f, 4)
    d = oracle.decode_volume(bits, (13, 9, 6), 4)
    for bz in range(2):
        for by in range(3):
            for bx in range(4):
                b = bx + 4 * (by + 3 * bz)
                sub = d[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
                assert bmin[b] == sub.min() and bmax[b] == sub.max()


def test_blocks_decode_independently():
    f = fields.gradient_noise(20, 16, 12, 9)
    bits, _, _ = oracle.encode_volume(f, 8)
    full = oracle.decode_volume(bits, (20, 16, 12), 8)
    ids = np.array([0, 7, 14, 33, 59], np.uint32)
    blocks = oracle.decode_blocks(bits, 8, ids)
    for i, b in enumerate(ids):
        bx, by, bz = b % 5, b // 5 % 4, b // 20
        sub = full[4 * bz:4 * bz + 4, 4 * by:4 * by + 4, 4 * bx:4 * bx + 4]
        assert np.array_equal(blocks[i].reshape(4, 4, 4), sub)


def test_padding_replicates_last_sample():
    # a 1x1x1 volume is one block of 64 copies of its only value
    f = np.full((1, 1, 1), 2.5, np.float32)
    bits, bmin, bmax = oracle.encode_volume(f, 2)
    assert np.array_equal(oracle.decode_block(bits[0], 2), np.full(64, 2.5, np.float32))
    assert bmin[0] == bmax[0] == 2.5


def test_corrupt_stream_stays_in_bounds():
    rng = np.random.default_rng(3)
    for rate in (1, 2, 5, 8):
        for _ in range(200):
            w = rng.integers(0, 1 << 63, rate, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
            d = oracle.decode_block(w, rate)
            assert d.shape == (64,) and not np.isnan(d).any()


def _dc_only_stream(q, emax, rate):
    """A block whose only non-zero coefficient is the DC, q, written bit by bit
    from the format: the non-zero flag, emax + 127 in 8 bits, then for each
    plane k = 31..0 (n = coefficients reached so far): n verbatim bits, then
    group tests.  Before the DC is reached a plane is one test bit (its DC
    bit); the plane that reaches it is 1 (test), 1 (the DC's one), 0 (no
    later ones); every later plane is the DC's bit and a 0 test."""
    bits = [1] + [(emax + 127) >> b & 1 for b in range(8)]
    u = ((q + 0xAAAAAAAA) & 0xFFFFFFFF) ^ 0xAAAAAAAA      # negabinary digits of q
    reached = False
    for k in range(31, -1, -1):
        d = u >> k & 1
        if reached:
            bits += [d, 0]
        elif d:
            bits += [1, 1, 0]
            reached = True
        else:
            bits += [0]
    assert len(bits) <= 64 * rate
    w = np.zeros(rate, np.uint64)
    for i, b in enumerate(bits):
        w[i >> 6] |= np.uint64(b) << np.uint64(i & 63)
    return w


@pytest.mark.parametrize("q, emax, want", [
    # 2^26 + 9 becomes 2^26 + 8 as a float32 (spacing 8 there); times
    # 2^(-126-27) that is 2^22 + 0.5 subnormal steps of 2^-149, a tie, which
    # goes to the even 2^22: exactly 2^-127.  (Rounding the exact product
    # q * 2^-153 once would give 2^22 + 1 steps: the format's decoder rounds
    # the integer first, then scales, as ZFP's dequantisation does.)
    (2 ** 26 + 9, -126, 2.0 ** -127),
    (-(2 ** 26 + 9), -126, -(2.0 ** -127)),
    # 2^26 + 17 -> 2^26 + 16 as a float32, times 2^-153: 2^22 + 1 steps exactly
    (2 ** 26 + 17, -126, (2 ** 22 + 1) * 2.0 ** -149),
    # emax -110 and -100: the scaled value stays normal, the product is exact
    (2 ** 26 + 9, -110, (2 ** 26 + 8) * 2.0 ** -137),
    (2 ** 26 + 9, -100, (2 ** 26 + 8) * 2.0 ** -127),
    (12345, -120, 12345 * 2.0 ** -147),
])
def test_hand_built_stream_tiny_exponents(q, emax, want):
    # every sample of a DC-only block is the DC (the inverse transform of
    # (q, 0, ..., 0) is constant), so the decoder's last step, the int32 ->
    # float32 conversion and the scaling by 2^(emax - 27), is seen directly
    w = _dc_only_stream(q, emax, 2)
    d = oracle.decode_block(w, 2)
    assert np.array_equal(d, np.full(64, want, np.float32)), (d[0], want)
    assert np.float32(want) == want                          # the hand value is a float32
