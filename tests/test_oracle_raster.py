"""Pins for the oracle's rasteriser and shading (the rendering step of
Section 4.6.2), CPU only.

The rules are stated in oracle/raster.c.  These tests tie them to things
computed another way: hand-enumerated pixel sets, coverage counts of shared
edges (every pixel centre inside a tiled region is drawn exactly once),
depth order and ties, the closed-form depth of a plane under a perspective
projection, and colours of lit triangles worked out by hand.
"""
import numpy as np
import pytest

import oracle
from synth import cameras

DIMS = (64, 64, 64)
NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


def float4_vertices(points):
    """World points (n, 3) -> float4 block-local vertices + block id bits."""
    p = np.asarray(points, np.float64)
    nbx, nby, _ = oracle.block_dims(DIMS)
    b = np.minimum(np.floor(p / 4).astype(np.int64), np.array(oracle.block_dims(DIMS)) - 1)
    b = np.maximum(b, 0)
    local = (p - 4 * b).astype(np.float32)
    ids = (b[:, 0] + nbx * (b[:, 1] + nby * b[:, 2])).astype(np.uint32)
    out = np.zeros((len(p), 4), np.float32)
    out[:, :3] = local
    out[:, 3] = ids.view(np.float32)
    return out


def coverage(points, tris, width, height, m=None):
    """Per triangle: boolean (height, width) mask of the pixels it wins
    when drawn alone."""
    v = float4_vertices(points)
    masks = []
    for t in tris:
        soup = v[list(t)]
        f = oracle.raster(soup, None, 1, DIMS, cameras.orthographic(width, height) if m is None else m, width, height)
        masks.append(f != NONE)
    return masks


def test_right_triangle_hand_enumerated():
    # hypotenuse x + y = 8: centres with i + j = 7 lie on it; it is a
    # right edge (not top-left), so they are out; 28 pixels remain
    pts = [(0, 0, 1), (8, 0, 1), (0, 8, 1)]
    for order in ((0, 1, 2), (0, 2, 1)):                 # either winding
        (m,) = coverage(pts, [order], 8, 8)
        want = np.array([[i + j <= 6 for i in range(8)] for j in range(8)])
        assert np.array_equal(m, want)
    f = oracle.raster(float4_vertices(pts), None, 1, DIMS, cameras.orthographic(8, 8), 8, 8)
    d = (f[f != NONE] >> np.uint64(32)).astype(np.uint32).view(np.float32)
    assert np.all(d == np.float32(1.0 / 64.0))           # z = 1 of 64
    assert np.all((f[f != NONE] & np.uint64(0xFFFFFFFF)) == 0)


def test_top_and_left_edges_are_in():
    # all three edges pass through pixel centres: the left edge x = 0.5
    # (going down) and the top edge y = 6.5 (going left) keep theirs, the
    # diagonal y = x (going up, a right edge) does not: centres with j > i
    pts = [(0.5, 0.5, 1), (6.5, 6.5, 1), (0.5, 6.5, 1)]
    for order in ((0, 1, 2), (1, 0, 2)):
        (m,) = coverage(pts, [order], 8, 8)
        want = np.array([[i < j <= 6 for i in range(8)] for j in range(8)])
        assert np.array_equal(m, want) and m.sum() == 21


def test_square_split_on_its_diagonal_covers_each_pixel_once():
    pts = [(0, 0, 2), (8, 0, 2), (8, 8, 2), (0, 8, 2)]
    a, b = coverage(pts, [(0, 1, 2), (0, 2, 3)], 8, 8)
    assert np.array_equal(a.astype(int) + b.astype(int), np.ones((8, 8), int))
    assert a.sum() == 36 and b.sum() == 28                # the diagonal centres go to one side


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jittered_mesh_is_watertight(seed):
    # a grid of jittered points split into triangles with alternating
    # diagonals: every pixel centre inside it is drawn exactly once
    rng = np.random.default_rng(seed)
    n, cell, w = 9, 5.0, 40
    pts = []
    for j in range(n):
        for i in range(n):
            jit = rng.uniform(-1.2, 1.2, 2) if 0 < i < n - 1 and 0 < j < n - 1 else (0.0, 0.0)
            pts.append((i * cell + jit[0], j * cell + jit[1], 3.0 + rng.uniform(0, 1)))
    tris = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            tris += [(a, b, c), (a, c, d)] if (i + j) % 2 == 0 else [(a, b, d), (b, c, d)]
    masks = coverage(pts, tris, w, w)
    count = sum(m.astype(int) for m in masks)
    assert count.max() == 1
    assert np.all(count[:, :] == 1)                        # the grid spans the whole 40 x 40 viewport


def test_nearest_fragment_wins_and_ties_go_to_the_lower_id():
    v = float4_vertices([(0, 0, 10), (8, 0, 10), (0, 8, 10),       # t0 far
                         (0, 0, 5), (8, 0, 5), (0, 8, 5),          # t1 near
                         (0, 0, 5), (8, 0, 5), (0, 8, 5)])         # t2 = t1
    f = oracle.raster(v, None, 3, DIMS, cameras.orthographic(8, 8), 8, 8)
    drawn = f[f != NONE]
    assert len(drawn) == 28
    assert np.all((drawn & np.uint64(0xFFFFFFFF)) == 1)
    assert np.all((drawn >> np.uint64(32)).astype(np.uint32).view(np.float32) == np.float32(5.0 / 64.0))


def perspective(fovy_deg, aspect, near, far, eye, target):
    return cameras.look_at_perspective(fovy_deg, aspect, near, far, eye, target), (near, far)


def test_plane_depth_matches_the_projection():
    # camera on the z axis looking down -z at a square in the plane z = 10:
    # view depth 20, NDC z = (f + n)/(f - n) - 2 f n / ((f - n) 20)
    m, (n, fa) = perspective(60.0, 1.0, 1.0, 100.0, (32, 32, 30), (32, 32, 0))
    pts = [(24, 24, 10), (40, 24, 10), (40, 40, 10), (24, 40, 10)]
    v = float4_vertices(pts)[[0, 1, 2, 0, 2, 3]]
    f = oracle.raster(v, None, 2, DIMS, m, 64, 64)
    drawn = f[f != NONE]
    assert len(drawn) > 500
    d = (drawn >> np.uint64(32)).astype(np.uint32).view(np.float32).astype(np.float64)
    zn = (fa + n) / (fa - n) - 2 * fa * n / ((fa - n) * 20.0)
    assert np.abs(d - (0.5 * zn + 0.5)).max() < 2e-6
    # the square spans 16 of the 2 * 20 * tan(30 deg) world units across the view
    side = 16.0 / (2 * 20.0 * np.tan(np.radians(30))) * 64
    assert abs(len(drawn) - side * side) < 4 * side


def test_vertex_behind_the_camera_is_not_drawn():
    m, _ = perspective(60.0, 1.0, 1.0, 100.0, (32, 32, 30), (32, 32, 0))
    v = float4_vertices([(20, 20, 10), (44, 20, 10), (32, 40, 40)])      # z = 40 is behind the eye
    f = oracle.raster(v, None, 1, DIMS, m, 64, 64)
    assert np.all(f == NONE)


def test_compact_and_indexed_inputs_draw_the_same():
    rng = np.random.default_rng(5)
    codes = rng.integers(0, 1024, (30, 3)).astype(np.uint32)
    blocks = rng.integers(0, 16 ** 3, 30).astype(np.uint32)
    packed = np.stack([codes[:, 0] | (codes[:, 1] << 10) | (codes[:, 2] << 20), blocks], 1).astype(np.uint32)
    nbx = oracle.block_dims(DIMS)[0]
    b3 = np.stack([blocks % nbx, (blocks // nbx) % nbx, blocks // (nbx * nbx)], 1).astype(np.float32)
    local = codes.astype(np.float32) * np.float32(4.0 / 1023.0)
    f4 = np.zeros((30, 4), np.float32)
    f4[:, :3] = local
    f4[:, 3] = blocks.view(np.float32)
    idx = rng.integers(0, 30, (40, 3)).astype(np.uint32)
    m, _ = perspective(50.0, 1.25, 1.0, 300.0, (-20, -30, 110), (32, 32, 32))
    a = oracle.raster(packed, idx, 40, DIMS, m, 80, 64)
    b = oracle.raster(f4, idx, 40, DIMS, m, 80, 64)
    c = oracle.raster(f4[idx.reshape(-1)], None, 40, DIMS, m, 80, 64)
    assert (a != NONE).sum() > 100
    assert np.array_equal(a, b) and np.array_equal(b, c)
    assert np.all(4 * b3 + local >= 0)                                   # world = block origin + local


def test_shading_by_hand():
    pts = [(0, 0, 1), (8, 0, 1), (0, 8, 1)]                               # normal along +z
    v = float4_vertices(pts)
    f = oracle.raster(v, None, 1, DIMS, cameras.orthographic(8, 8), 8, 8)
    lit = oracle.shade(v, None, DIMS, (0.0, 0.0, 3.0), f)
    side = oracle.shade(v, None, DIMS, (1.0, 0.0, 0.0), f)
    back = oracle.shade(v, None, DIMS, (0.0, 0.0, -1.0), f)
    full = 217 | (191 << 8) | (140 << 16) | (255 << 24)                   # (0.85, 0.75, 0.55) * 255, rounded
    dim = 43 | (38 << 8) | (28 << 16) | (255 << 24)                       # 0.2 * the same
    assert np.all(lit[f != NONE] == full) and np.all(back[f != NONE] == full)   # two-sided
    assert np.all(side[f != NONE] == dim)
    assert np.all(lit[f == NONE] == 0)


def test_index_past_the_vertices_is_not_drawn():
    v = float4_vertices([(0, 0, 1), (8, 0, 1), (0, 8, 1)])
    good = np.array([[0, 1, 2]], np.uint32)
    bad = np.array([[0, 1, 3], [0, 1, 2]], np.uint32)        # the first reaches past the 3 vertices
    a = oracle.raster(v, good, 1, DIMS, cameras.orthographic(8, 8), 8, 8)
    b = oracle.raster(v, bad, 2, DIMS, cameras.orthographic(8, 8), 8, 8)
    assert (a != NONE).sum() == 28
    assert np.array_equal(b & np.uint64(0xFFFFFFFF00000000), a & np.uint64(0xFFFFFFFF00000000))
    assert np.all((b[b != NONE] & np.uint64(0xFFFFFFFF)) == 1)   # only triangle 1 is drawn
