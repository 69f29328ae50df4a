"""GPU parity of the ray caster over the block macrocell grid (the future
work of Section 4.6.2) against the oracle's (oracle/raycast.c), bit for
bit: the first-hit depth and block of every pixel and the shaded RGBA8.
Both sides take every float32 operation in the same order.

The GPU reads the decoded samples from its block cache (filled by the
call's own range test, cache update and decode); the oracle reads the
decoded volume.  Cases: ragged noise volumes from outside, from inside and
along the axes (rays with zero direction components), a sphere, isovalues
without a surface, the cache afterwards, and a cache budget too small.
"""
import numpy as np
import pytest

import oracle
from synth import cameras, fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def pkg():
    import paper_2009_03254_gb300 as p
    return p


def check(vol, d, iso, cam, light, w, h):
    eye, fwd, right, up = cam
    hits, rgba, st = vol.raycast(iso, eye, fwd, right, up, light, w, h)
    got_h = hits.cpu().numpy().view(np.uint64)
    got_c = rgba.cpu().numpy().view(np.uint32)
    want_h, want_c = oracle.raycast(d, iso, eye, fwd, right, up, light, w, h)
    assert np.array_equal(got_h, want_h)
    assert np.array_equal(got_c, want_c)
    assert st["hits"] == int((want_h != np.uint64(0xFFFFFFFFFFFFFFFF)).sum())
    return st


@pytest.mark.parametrize("dims,rate,seed", [((37, 29, 23), 8, 1), ((48, 40, 36), 12, 2), ((21, 18, 9), 8, 3)])
def test_noise_volumes_match_oracle(dims, rate, seed):
    f = fields.gradient_noise(*dims, seed, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax)
    c = np.asarray(dims, float) / 2
    cams = [cameras.pinhole_orbit(dims, 35.0, 20.0, distance_factor=0.9, fovy_deg=50, aspect=1.4),
            cameras.pinhole_orbit(dims, 250.0, -40.0, distance_factor=1.2, fovy_deg=40, aspect=1.4),
            cameras.pinhole(c, c + np.array([10.0, 3.0, -2.0]), 80.0, 1.4),                  # inside
            (np.asarray([-5.0, c[1], c[2]], np.float32), np.asarray([1, 0, 0], np.float32),    # along +x
             np.asarray([0, 0.5, 0], np.float32), np.asarray([0, 0, 0.5], np.float32))]
    try:
        for iso in (float(np.median(d)), float(np.quantile(d, 0.25))):
            for cam in cams:
                st = check(vol, d, iso, cam, (0.3, -0.5, 0.8), 45, 33)    # odd sizes: zero components
                assert st["hits"] > 0
                assert st["n_active"] == int(oracle.active_blocks(bmin, bmax, oracle.block_dims(dims), iso).sum())
        st = check(vol, d, float(d.max()) + 1.0, cams[0], (0, 0, 1), 45, 33)
        assert st["hits"] == 0
        # the call leaves the cache as an extraction would: nothing new to decode
        iso = float(np.median(d))
        vol.raycast(iso, *cams[0], (0, 0, 1), 8, 8)
        m = vol.extract(iso)
        assert m.stats["n_new"] == 0
        m.release()
    finally:
        vol.release()


def test_sphere_matches_oracle():
    dims = (40, 40, 40)
    f = fields.sphere_sdf(*dims, 12.0)
    bits, bmin, bmax = oracle.encode_volume(f, 16)
    d = oracle.decode_volume(bits, dims, 16)
    vol = pkg().Volume(bits, dims, 16, bmin, bmax)
    try:
        c = np.array([19.5, 19.5, 19.5])
        for cam in (cameras.pinhole(c + np.array([0.0, -60.0, 0.0]), c, 30.0, 1.0),
                    cameras.pinhole(c + np.array([40.0, 35.0, 30.0]), c, 35.0, 1.25)):
            st = check(vol, d, 0.0, cam, (0, -1, 0), 40, 32)
            assert st["hits"] > 200
    finally:
        vol.release()


def test_over_budget_and_invalid():
    p = pkg()
    dims = (48, 40, 36)
    f = fields.gradient_noise(*dims, 7, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, 8)
    d = oracle.decode_volume(bits, dims, 8)
    small = p.Volume(bits, dims, 8, bmin, bmax, cache_budget_bytes=256 * 10)
    try:
        cam = cameras.pinhole_orbit(dims, 35.0, 20.0)
        with pytest.raises(p.IsoError) as e:
            small.raycast(float(np.median(d)), *cam, (0, 0, 1), 16, 16)
        assert e.value.code == p.ISO_ERR_BUDGET
        for kw in (dict(light=(0, 0, 0)), dict(width=0), dict(iso=float("nan"))):
            args = dict(iso=0.0, eye=cam[0], forward=cam[1], right=cam[2], up=cam[3], light=(0, 0, 1), width=8,
                        height=8)
            args.update(kw)
            with pytest.raises(p.IsoError) as e:
                small.raycast(**args)
            assert e.value.code == p.ISO_ERR_INVALID_ARG
    finally:
        small.release()


@pytest.mark.parametrize("dims", [(2, 2, 2), (5, 2, 3), (1, 6, 6), (4, 4, 4), (9, 3, 17)])
def test_degenerate_volumes_match_oracle(dims):
    # a single cell, thin and flat volumes (a dimension of 1: no cells, no
    # hits), exact multiples of 4
    rng = np.random.default_rng(3)
    f = rng.standard_normal((dims[2], dims[1], dims[0])).astype(np.float32)
    bits, bmin, bmax = oracle.encode_volume(f, 12)
    d = oracle.decode_volume(bits, dims, 12)
    vol = pkg().Volume(bits, dims, 12, bmin, bmax)
    try:
        c = (np.asarray(dims, float) - 1) / 2
        cam = cameras.pinhole(c + np.array([-3.0, -2.0, 4.0]) * max(dims), c, 40.0, 1.0)
        st = check(vol, d, float(np.median(d)), cam, (0.3, -0.5, 0.8), 21, 21)
        if 1 in dims:
            assert st["hits"] == 0
    finally:
        vol.release()
