"""Seeded synthetic scalar fields that stand in for the paper's volumes.

The paper benchmarks on CT/MRI scans and simulation outputs (Section 4.6,
Table "mc_benchmark_data") that are not available here.  These generators
produce float32 volumes with the same shapes and the two isosurface
topologies the paper distinguishes: nested surfaces (sphere distance field)
and turbulent sheets (band-limited gradient noise, and a channel-flow-like
spectral field).

This module holds no part of the isosurface method (no codec, no marching
cubes); it is shared by the CPU oracle and the GPU path only as a source of
inputs.  Every array is laid out C-order as (nz, ny, nx): x varies fastest.

All arithmetic is float64 using only +, -, *, / and sqrt in a fixed order, so
that the CUDA generator in ``synth/csrc/synth_fields.cu`` reproduces each
value bit for bit (it is compiled without FMA contraction).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1

# Perlin's "improved noise" gradient set: the 12 edge midpoints of a cube
# (K. Perlin, "Improving Noise", SIGGRAPH 2002).
GRADIENTS = np.array(
    [(1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0),
     (1, 0, 1), (-1, 0, 1), (1, 0, -1), (-1, 0, -1),
     (0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1)], dtype=np.float64)

# Scale that brings the 6-octave sum to roughly unit standard deviation (the
# unscaled sum measured 0.34 on a 256^3 window and 0.30 on another, seed 1).
# Fixed rather than measured per volume, so that any sub-window of a volume
# can be generated without whole-volume statistics.
NOISE_SCALE = 3.0


def _splitmix64(x):
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on uint64 numpy arrays."""
    x = (x + np.uint64(0x9E3779B97F4A7C15)) & np.uint64(MASK64)
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & np.uint64(MASK64)
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & np.uint64(MASK64)
    return x ^ (x >> np.uint64(31))


def lattice_hash(seed, octave, ix, iy, iz):
    """Counter-based hash of a lattice point: nested splitmix64 over
    (seed + octave, x, y, z).  Inputs broadcast; returns uint64."""
    with np.errstate(over="ignore"):
        h = _splitmix64(np.uint64(seed) + np.uint64(octave))
        h = _splitmix64(h + np.asarray(ix, dtype=np.int64).astype(np.uint64))
        h = _splitmix64(h + np.asarray(iy, dtype=np.int64).astype(np.uint64))
        h = _splitmix64(h + np.asarray(iz, dtype=np.int64).astype(np.uint64))
    return h


def _fade(t):
    # quintic 6t^5 - 15t^4 + 10t^3, evaluated as ((t*t)*t) * (t*(t*6 - 15) + 10)
    return ((t * t) * t) * ((t * ((t * 6.0) - 15.0)) + 10.0)


def gradient_noise(nx, ny, nz, seed, octaves=6, base_period=128, lacunarity=2,
                   gain=0.5, origin=(0, 0, 0), scale=NOISE_SCALE):
    """Sum of `octaves` octaves of lattice gradient noise, times `scale`.

    Octave o has lattice period base_period / lacunarity**o voxels (an
    integer >= 1) and amplitude gain**o.  `origin` = (x0, y0, z0) selects a
    window of the infinite field, so a sub-volume of a large volume can be
    produced exactly.  Returns float32 (nz, ny, nx).
    """
    x0, y0, z0 = origin
    out = np.zeros((nz, ny, nx), dtype=np.float64)
    for o in range(octaves):
        period = base_period // (lacunarity ** o)
        assert period >= 1 and period * (lacunarity ** o) == base_period
        amp = gain ** o
        inv = 1.0 / period                       # exact: period is a power of two
        xs = np.arange(x0, x0 + nx, dtype=np.int64)
        ys = np.arange(y0, y0 + ny, dtype=np.int64)
        zs = np.arange(z0, z0 + nz, dtype=np.int64)
        cx, cy, cz = xs // period, ys // period, zs // period
        fx = (xs - cx * period).astype(np.float64) * inv
        fy = (ys - cy * period).astype(np.float64) * inv
        fz = (zs - cz * period).astype(np.float64) * inv
        wx, wy, wz = _fade(fx), _fade(fy), _fade(fz)
        # gradients of the lattice points the window touches
        lx = np.arange(cx[0], cx[-1] + 2)
        ly = np.arange(cy[0], cy[-1] + 2)
        lz = np.arange(cz[0], cz[-1] + 2)
        h = lattice_hash(seed, o, lx[None, None, :], ly[None, :, None], lz[:, None, None])
        g = GRADIENTS[((h >> np.uint64(32)) % np.uint64(12)).astype(np.int64)]
        ix = (cx - lx[0])[None, None, :]
        iy = (cy - ly[0])[None, :, None]
        iz = (cz - lz[0])[:, None, None]
        dots = {}
        for k in (0, 1):
            for j in (0, 1):
                for i in (0, 1):
                    gg = g[iz + k, iy + j, ix + i]
                    dx = (fx - i)[None, None, :]
                    dy = (fy - j)[None, :, None]
                    dz = (fz - k)[:, None, None]
                    dots[(i, j, k)] = ((gg[..., 0] * dx) + (gg[..., 1] * dy)) + (gg[..., 2] * dz)
        wxb, wyb, wzb = wx[None, None, :], wy[None, :, None], wz[:, None, None]

        def lerp(a, b, w):
            return a + (w * (b - a))
        x00 = lerp(dots[(0, 0, 0)], dots[(1, 0, 0)], wxb)
        x10 = lerp(dots[(0, 1, 0)], dots[(1, 1, 0)], wxb)
        x01 = lerp(dots[(0, 0, 1)], dots[(1, 0, 1)], wxb)
        x11 = lerp(dots[(0, 1, 1)], dots[(1, 1, 1)], wxb)
        yz0 = lerp(x00, x10, wyb)
        yz1 = lerp(x01, x11, wyb)
        out = out + (amp * lerp(yz0, yz1, wzb))
    return (out * scale).astype(np.float32)


def sphere_sdf(nx, ny, nz, radius, center=None, origin=(0, 0, 0)):
    """f(p) = |p - c| - radius at integer voxel positions p (float32).

    The default centre is the grid centre ((n-1)/2 per axis)."""
    if center is None:
        center = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    x0, y0, z0 = origin
    dx = np.arange(x0, x0 + nx, dtype=np.float64) - center[0]
    dy = np.arange(y0, y0 + ny, dtype=np.float64) - center[1]
    dz = np.arange(z0, z0 + nz, dtype=np.float64) - center[2]
    s = ((dx * dx)[None, None, :] + (dy * dy)[None, :, None]) + (dz * dz)[:, None, None]
    return (np.sqrt(s) - radius).astype(np.float32)


def linear_ramp(nx, ny, nz, x0):
    """f(x, y, z) = x - x0: every isosurface is the plane x = x0 + iso."""
    f = np.arange(nx, dtype=np.float64) - x0
    return np.broadcast_to(f[None, None, :], (nz, ny, nx)).astype(np.float32)


# ---------------------------------------------------------------- channel-flow-like field
#
# A stand-in for the paper's DNS (a turbulent channel; Table
# "mc_benchmark_data"): u = U(zeta) + a(zeta) * u', zeta = z / (NZ - 1) the
# wall-normal coordinate, U(zeta) = tanh(zeta/d) tanh((1 - zeta)/d) with
# d = 0.08 the mean profile, a(zeta) = 0.3 (1 - U) + 0.1 the fluctuation
# envelope, and u' a sum of gradient-noise octaves whose amplitudes fall by
# 2^(-1/3) per halving of the period (energy per octave falling as
# k^(-2/3), the integral of a k^(-5/3) spectrum).  u' is evaluated in
# float32 (every dot product is exact; fades and lerps are single
# operations in a fixed order) so that a per-block GPU generator can
# reproduce it bit for bit at 10^11 samples.

CHANNEL_DELTA = 0.08
CHANNEL_GAIN = np.float32(2.0 ** (-1.0 / 3.0))
CHANNEL_SCALE = np.float32(3.0)
LN2 = 0.6931471805599453
INV_FACT = [1.0 / float(__import__("math").factorial(k)) for k in range(21)]


def exp_f64(y):
    """exp for float64 arrays by range reduction y = n ln2 + r and a
    degree-20 Taylor polynomial of exp(r) in Horner form (no fused
    operations), so the CUDA generator can repeat it exactly."""
    y = np.asarray(y, np.float64)
    n = np.rint(y / LN2)
    r = y - (n * LN2)
    p = np.full_like(r, INV_FACT[20])
    for k in range(19, -1, -1):
        p = (p * r) + INV_FACT[k]
    return np.ldexp(p, n.astype(np.int64))


def tanh_pos_f64(x):
    """tanh(x) for x >= 0 as (1 - e^(-2x)) / (1 + e^(-2x)) with exp_f64."""
    e = exp_f64(-2.0 * np.asarray(x, np.float64))
    return (1.0 - e) / (1.0 + e)


def channel_profile(nz_total, z):
    """(U, a) as float32 at the integer wall-normal positions z."""
    zeta = np.asarray(z, np.float64) / float(nz_total - 1)
    U = tanh_pos_f64(zeta / CHANNEL_DELTA) * tanh_pos_f64((1.0 - zeta) / CHANNEL_DELTA)
    a = (0.3 * (1.0 - U)) + 0.1
    return U.astype(np.float32), a.astype(np.float32)


def _noise_f32(xs, ys, zs, seed, octaves, base_period):
    """float32 gradient-noise octave sum at the grid xs x ys x zs (1-D int64 arrays)."""
    out = np.zeros((len(zs), len(ys), len(xs)), np.float32)
    amp = np.float32(1.0)
    f32 = np.float32
    for o in range(octaves):
        period = base_period >> o
        inv = f32(1.0 / period)
        cx, cy, cz = xs // period, ys // period, zs // period
        fx = (xs - cx * period).astype(f32) * inv
        fy = (ys - cy * period).astype(f32) * inv
        fz = (zs - cz * period).astype(f32) * inv
        fade = lambda t: ((t * t) * t) * ((t * ((t * f32(6.0)) - f32(15.0))) + f32(10.0))
        wx, wy, wz = fade(fx), fade(fy), fade(fz)
        lx = np.arange(cx.min(), cx.max() + 2)
        ly = np.arange(cy.min(), cy.max() + 2)
        lz = np.arange(cz.min(), cz.max() + 2)
        h = lattice_hash(seed, o, lx[None, None, :], ly[None, :, None], lz[:, None, None])
        g = GRADIENTS.astype(f32)[((h >> np.uint64(32)) % np.uint64(12)).astype(np.int64)]
        ix = (cx - lx[0])[None, None, :]
        iy = (cy - ly[0])[None, :, None]
        iz = (cz - lz[0])[:, None, None]
        d = {}
        for k in (0, 1):
            for j in (0, 1):
                for i in (0, 1):
                    gg = g[iz + k, iy + j, ix + i]
                    dx = (fx - f32(i))[None, None, :]
                    dy = (fy - f32(j))[None, :, None]
                    dz = (fz - f32(k))[:, None, None]
                    d[(i, j, k)] = ((gg[..., 0] * dx) + (gg[..., 1] * dy)) + (gg[..., 2] * dz)
        wxb, wyb, wzb = wx[None, None, :], wy[None, :, None], wz[:, None, None]

        def lerp(p, q, w):
            return p + (w * (q - p))
        x00 = lerp(d[(0, 0, 0)], d[(1, 0, 0)], wxb)
        x10 = lerp(d[(0, 1, 0)], d[(1, 1, 0)], wxb)
        x01 = lerp(d[(0, 0, 1)], d[(1, 0, 1)], wxb)
        x11 = lerp(d[(0, 1, 1)], d[(1, 1, 1)], wxb)
        val = lerp(lerp(x00, x10, wyb), lerp(x01, x11, wyb), wzb)
        out = out + (amp * val)
        amp = f32(amp * CHANNEL_GAIN)
    return out


def channel_field(nx, ny, nz, seed, nz_total=None, origin=(0, 0, 0), octaves=7, base_period=256):
    """Channel-flow-like field (see above) on a window, float32 (nz, ny, nx).
    nz_total is the full wall-normal extent (defaults to nz)."""
    nz_total = nz if nz_total is None else nz_total
    x0, y0, z0 = origin
    xs = np.arange(x0, x0 + nx, dtype=np.int64)
    ys = np.arange(y0, y0 + ny, dtype=np.int64)
    zs = np.arange(z0, z0 + nz, dtype=np.int64)
    U, a = channel_profile(nz_total, zs)
    n = _noise_f32(xs, ys, zs, seed, octaves, base_period)
    return U[:, None, None] + (a[:, None, None] * (n * CHANNEL_SCALE))


def channel_samples(points, seed, nz_total, octaves=7, base_period=256):
    """The channel field at arbitrary integer points (M, 3) as (x, y, z)."""
    pts = np.asarray(points, np.int64)
    out = np.empty(len(pts), np.float32)
    for i, (x, y, z) in enumerate(pts):
        out[i] = channel_field(1, 1, 1, seed, nz_total, origin=(int(x), int(y), int(z)),
                               octaves=octaves, base_period=base_period)[0, 0, 0]
    return out
