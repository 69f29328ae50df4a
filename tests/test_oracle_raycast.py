"""Pins for the oracle's ray caster over the block macrocell grid (the
future work of Section 4.6.2), CPU only.  The rules are stated in
oracle/raycast.c.  Checked against: closed-form hits on a plane and a
sphere; a fine float64 march along every ray over the trilinear
interpolant of the same samples (so no block or cell with a crossing is
skipped and misses are real); shading worked out by hand.
"""
import numpy as np
import pytest

import oracle
from synth import cameras, fields

NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


def ray_dirs(fwd, right, up, w, h):
    i = (np.arange(w, dtype=np.float32) + np.float32(0.5)) / np.float32(w) * np.float32(2) - np.float32(1)
    j = (np.arange(h, dtype=np.float32) + np.float32(0.5)) / np.float32(h) * np.float32(2) - np.float32(1)
    u, v = np.meshgrid(i, j)
    return (fwd[None, None, :].astype(np.float64) + u[..., None] * right.astype(np.float64) +
            v[..., None] * up.astype(np.float64))


def trilinear64(f, p):
    nz, ny, nx = f.shape
    x = np.clip(p[:, 0], 0, nx - 1 - 1e-9)
    y = np.clip(p[:, 1], 0, ny - 1 - 1e-9)
    z = np.clip(p[:, 2], 0, nz - 1 - 1e-9)
    x0, y0, z0 = np.floor(x).astype(int), np.floor(y).astype(int), np.floor(z).astype(int)
    fx, fy, fz = x - x0, y - y0, z - z0
    out = 0.0
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (fx if dx else 1 - fx) * (fy if dy else 1 - fy) * (fz if dz else 1 - fz)
                out = out + w * f[z0 + dz, y0 + dy, x0 + dx]
    return out


def march(f, iso, o, d, step=0.004):
    """First t where the trilinear interpolant crosses iso along o + t d
    inside the volume box, by fine float64 sampling (None if none)."""
    nz, ny, nx = f.shape
    hi = np.array([nx - 1, ny - 1, nz - 1], float)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = np.where(d != 0, (0 - o) / d, -np.inf)
        t1 = np.where(d != 0, (hi - o) / d, np.inf)
    a = max(0.0, np.max(np.minimum(t0, t1)))
    b = np.min(np.maximum(t0, t1))
    if not a < b:
        return None
    n = int((b - a) * np.linalg.norm(d) / step) + 2
    t = np.linspace(a, b, n)
    g = trilinear64(f, o[None, :] + t[:, None] * d[None, :]) - iso
    s = g < 0
    k = np.nonzero(s[1:] != s[:-1])[0]
    return None if len(k) == 0 else 0.5 * (t[k[0]] + t[k[0] + 1])


def unpack(hits):
    t = (hits >> np.uint64(32)).astype(np.uint32).view(np.float32)
    return np.where(hits == NONE, np.nan, t), (hits & np.uint64(0xFFFFFFFF)).astype(np.int64)


def test_plane_hits_at_the_closed_form():
    nx, ny, nz = 30, 21, 17
    f = fields.linear_ramp(nx, ny, nz, 9.25)                      # f = x - 9.25
    iso = 3.5
    eye, fwd, right, up = cameras.pinhole((-8.0, 10.0, 8.0), (20.0, 10.5, 8.5), 40.0, 1.0)
    hits, _ = oracle.raycast(f, iso, eye, fwd, right, up, (1, 0, 0), 24, 24)
    t, blk = unpack(hits)
    d = ray_dirs(fwd, right, up, 24, 24)
    p = eye.astype(np.float64) + t[..., None] * d
    ok = ~np.isnan(t)
    assert ok.sum() > 100
    assert np.abs(p[ok][:, 0] - (9.25 + iso)).max() < 2e-3          # on the plane x = 12.75
    bx = p[ok][:, 0] // 4
    nbx, nby, _ = oracle.block_dims((nx, ny, nz))
    assert np.all((blk[ok] % nbx == bx) | (blk[ok] % nbx == bx - 1))  # the block holding the hit cell


@pytest.mark.parametrize("seed", [0, 1])
def test_every_ray_against_a_fine_march(seed):
    dims = (26, 22, 19)
    f = fields.gradient_noise(*dims, seed, octaves=3, base_period=16)
    bits, _, _ = oracle.encode_volume(f, 12)
    d = oracle.decode_volume(bits, dims, 12)
    iso = float(np.quantile(d, 0.4))
    rng = np.random.default_rng(seed)
    for _ in range(2):
        az, el = rng.uniform(0, 360), rng.uniform(-60, 60)
        eye, fwd, right, up = cameras.pinhole_orbit(dims, az, el, distance_factor=0.8, fovy_deg=50, aspect=1.0)
        hits, _ = oracle.raycast(d, iso, eye, fwd, right, up, (0, 0, 1), 16, 16)
        t, _ = unpack(hits)
        dirs = ray_dirs(fwd, right, up, 16, 16)
        agree = missed = 0
        for j in range(16):
            for i in range(16):
                tr = march(d.astype(np.float64), iso, eye.astype(np.float64), dirs[j, i])
                if tr is None:
                    assert np.isnan(t[j, i]), (j, i)
                elif np.isnan(t[j, i]):
                    # sampling 4 points per cell misses only a pair of
                    # crossings closer than a quarter cell
                    missed += 1
                else:
                    assert abs(t[j, i] - tr) * np.linalg.norm(dirs[j, i]) < 0.02, (j, i)
                    agree += 1
        assert agree > 100 and missed <= 2


def test_sphere_silhouette_and_depth():
    n, r = 40, 12.0
    f = fields.sphere_sdf(n, n, n, r)
    c = np.array([(n - 1) / 2] * 3)                                    # the field's centre
    eye, fwd, right, up = cameras.pinhole(c + np.array([0.0, -60.0, 0.0]), c, 30.0, 1.0)
    hits, _ = oracle.raycast(f, 0.0, eye, fwd, right, up, (0, -1, 0), 32, 32)
    t, _ = unpack(hits)
    dirs = ray_dirs(fwd, right, up, 32, 32)
    o = eye.astype(np.float64) - c
    for j in range(32):
        for i in range(32):
            dd = dirs[j, i]
            a, b, cc = dd @ dd, 2 * o @ dd, o @ o - r * r
            disc = b * b - 4 * a * cc
            if disc < 0:
                # rays more than a voxel outside the silhouette miss
                dist = np.linalg.norm(np.cross(o, dd)) / np.linalg.norm(dd)
                if dist > r + 1:
                    assert np.isnan(t[j, i])
                continue
            tt = (-b - np.sqrt(disc)) / (2 * a)
            dist = np.linalg.norm(np.cross(o, dd)) / np.linalg.norm(dd)
            if dist < r - 1:
                assert abs(t[j, i] - tt) * np.sqrt(a) < 0.1              # trilinear sphere within 0.1 voxel


def test_shading_by_hand_and_no_surface():
    nx, ny, nz = 20, 16, 16
    f = fields.linear_ramp(nx, ny, nz, 8.0)                           # normal along x
    eye, fwd, right, up = cameras.pinhole((-5.0, 7.5, 7.5), (10.0, 7.5, 7.5), 20.0, 1.0)
    hits, lit = oracle.raycast(f, 0.5, eye, fwd, right, up, (-2.0, 0, 0), 8, 8)
    _, dim = oracle.raycast(f, 0.5, eye, fwd, right, up, (0, 1.0, 0), 8, 8)
    assert np.all(hits != NONE)
    assert np.all(lit == (217 | (191 << 8) | (140 << 16) | (255 << 24)))
    assert np.all(dim == (43 | (38 << 8) | (28 << 16) | (255 << 24)))
    hits, rgba = oracle.raycast(f, 100.0, eye, fwd, right, up, (1, 0, 0), 8, 8)
    assert np.all(hits == NONE) and np.all(rgba == 0)
