"""Compressed volumes too large to hold as float32: generated and encoded
on the GPU in z-slabs of whole blocks, straight into one bitstream.

Blocks of a slab of whole block layers are consecutive in the volume's
block order (x fastest, then y, then z), so each slab's blocks, ranges and
bits land at a fixed offset of the full arrays; block contents depend only
on the samples of their own 4^3 cube, so the result equals encoding the
whole field at once.
"""
from __future__ import annotations

import numpy as np


def encode_recipe(recipe, slab=32, device="cuda"):
    """(bits int64 (nb, rate), bmin, bmax) device tensors of a recipe's field."""
    import torch
    import paper_2009_03254_gb300 as bc
    from . import gpu
    assert slab % 4 == 0
    nx, ny, nz = recipe.dims
    nbx, nby, nbz = bc.block_dims(recipe.dims)
    nb = nbx * nby * nbz
    bits = torch.empty((nb, recipe.rate), dtype=torch.int64, device=device)
    bmin = torch.empty(nb, dtype=torch.float32, device=device)
    bmax = torch.empty(nb, dtype=torch.float32, device=device)
    buf = torch.empty((min(slab, nz), ny, nx), dtype=torch.float32, device=device)
    layer = nbx * nby
    for z0 in range(0, nz, slab):
        h = min(slab, nz - z0)
        f = gpu.generate(recipe, origin=(0, 0, z0), dims=(nx, ny, h)) if recipe.kind != "channel" else \
            gpu.channel_field(nx, ny, h, recipe.seed, nz_total=nz, origin=(0, 0, z0), octaves=recipe.octaves,
                              base_period=recipe.base_period, out=buf[:h])
        b0, b1 = (z0 // 4) * layer, ((z0 + h + 3) // 4) * layer
        bc.encode_field(f, recipe.rate, out=(bits[b0:b1], bmin[b0:b1], bmax[b0:b1]))
    torch.cuda.synchronize()
    return bits, bmin, bmax


def percentile_isovalue(bits, dims, rate, p, m=1 << 24, seed=0):
    """The float32 value at rank floor(p * m) among m decoded samples: the
    64 samples of each of m / 64 blocks drawn uniformly (seeded) from the
    blocks that lie wholly inside the volume."""
    import torch
    import paper_2009_03254_gb300 as bc
    nbx, nby, nbz = bc.block_dims(dims)
    fx, fy, fz = dims[0] // 4, dims[1] // 4, dims[2] // 4          # whole blocks per axis
    rng = np.random.default_rng(seed)
    n = m // 64
    bx, by, bz = rng.integers(0, fx, n), rng.integers(0, fy, n), rng.integers(0, fz, n)
    ids = (bx + nbx * (by + nby * bz)).astype(np.uint32)
    vals = bc.decode_blocks(bits, rate, torch.from_numpy(ids.view(np.int32)).to(bits.device)).reshape(-1)
    k = int(np.floor(p * vals.numel()))
    k = min(max(k, 0), vals.numel() - 1)
    return float(torch.sort(vals).values[k].item())
