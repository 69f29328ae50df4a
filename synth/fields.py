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
