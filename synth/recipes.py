"""Workload recipes: volume shapes, code rates, isovalues and seeds.

Each recipe mirrors the shape of a workload in the paper's evaluation
(Section 4.6, Tables "mc_benchmark_data" and "mc_benchmark_table"):

* ``sphere64``   -- 64^3 sphere distance field, closed nested surface,
                    16 bits/value, isovalue 0 (correctness case).
* ``noise512``   -- 512^3 six-octave gradient noise (Plasma-sized volume),
                    8 bits/value, isovalues -1, -0.5, 0, 0.5, 1 in sequence.
* ``channel2k``  -- 2048 x 2048 x 1024 channel-flow-like spectral field,
                    4 bits/value, isovalue at the 70th percentile.
* ``batch64``    -- 64 volumes with per-axis sizes log-uniform in [32, 256].
* ``serve_dns``  -- 10240 x 7680 x 1536 DNS-shaped field at 2 bits/value
                    (coarser structure, so that one surface is 10^8-scale
                    triangles), the serving workload.

Channel isovalues are percentiles of the decoded data (``percentile``),
computed when the volume is built.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class VolumeRecipe:
    name: str
    dims: tuple          # (nx, ny, nz)
    rate: int            # bits per value of the fixed-rate code
    kind: str            # "sphere" | "noise" | "channel"
    seed: int
    isovalues: tuple
    radius: float = 0.0  # sphere only
    octaves: int = 7     # channel only: noise octaves and coarsest period (voxels)
    base_period: int = 256
    percentile: float = 0.0   # channel only: isovalue rank in the decoded data


SPHERE64 = VolumeRecipe("sphere64", (64, 64, 64), 16, "sphere", 0, (0.0,), radius=20.0)
NOISE512 = VolumeRecipe("noise512", (512, 512, 512), 8, "noise", 1, (-1.0, -0.5, 0.0, 0.5, 1.0))
CHANNEL2K = VolumeRecipe("channel2k", (2048, 2048, 1024), 4, "channel", 7, (), octaves=7, base_period=256,
                         percentile=0.7)
SERVE_DNS = VolumeRecipe("serve_dns", (10240, 7680, 1536), 2, "channel", 5, (), octaves=2, base_period=2048,
                         percentile=0.5)


def generate_cpu(recipe: VolumeRecipe, origin=(0, 0, 0), dims=None):
    """Generate (a window of) a recipe's field on the CPU as float32 (nz, ny, nx)."""
    from . import fields
    nx, ny, nz = dims if dims is not None else recipe.dims
    if recipe.kind == "sphere":
        gx, gy, gz = recipe.dims
        c = ((gx - 1) / 2.0, (gy - 1) / 2.0, (gz - 1) / 2.0)
        return fields.sphere_sdf(nx, ny, nz, recipe.radius, center=c, origin=origin)
    if recipe.kind == "noise":
        return fields.gradient_noise(nx, ny, nz, recipe.seed, origin=origin)
    if recipe.kind == "channel":
        return fields.channel_field(nx, ny, nz, recipe.seed, nz_total=recipe.dims[2], origin=origin,
                                    octaves=recipe.octaves, base_period=recipe.base_period)
    raise ValueError(f"no CPU generator for kind {recipe.kind!r}")


def batch64_recipes(seed=4, count=64, lo=32, hi=256):
    """The batched workload: `count` volumes whose per-axis sizes are drawn
    log-uniform in [lo, hi]; half sphere distance fields, half noise, each at
    an integer rate in 8..16 with its own isovalue."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dims = tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) for _ in range(3))
        rate = int(rng.integers(8, 17))
        if rng.random() < 0.5:
            r = 0.35 * min(dims)
            iso = float(rng.uniform(-0.1 * r, 0.1 * r))
            out.append(VolumeRecipe(f"batch{i}", dims, rate, "sphere", 0, (iso,), radius=r))
        else:
            iso = float(rng.uniform(-1.0, 1.0))
            out.append(VolumeRecipe(f"batch{i}", dims, rate, "noise", 1000 + i, (iso,)))
    return out
