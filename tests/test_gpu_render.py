"""GPU parity of the rasteriser (the rendering step of Section 4.6.2)
against the oracle's (oracle/raster.c), bit for bit: the fragment buffer
(depth bits and the visible triangle of every pixel) and the shaded RGBA8
image.  Both sides take every float32 operation in the same order, so the
coverage and depth decisions that floating point makes agree exactly.

Inputs come from the oracle: its block-ordered soup of a noise volume (as
float4 vertices, as compact 8-byte vertices, and as its indexed mesh),
hand-made meshes with shared edges and ties, and cameras from far (most
triangles under a pixel), close up (triangles over 32 pixel centres, drawn
by the warp kernel) and inside the volume (triangles behind the camera).
"""
import numpy as np
import pytest

import oracle
from synth import cameras, fields

pytestmark = pytest.mark.gpu

NONE = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def pkg():
    import paper_2009_03254_gb300 as p
    return p


def torch():
    import torch as t
    return t


def dev(a):
    t = torch()
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return t.from_numpy(a).cuda()


def gpu_render(verts, idx, n, dims, m, light, w, h):
    frag, rgba, st = pkg().render(dev(verts), n, dims, m, light, w, h,
                                  indices=None if idx is None else dev(idx), stats=True)
    return frag.cpu().numpy().view(np.uint64), rgba.cpu().numpy().view(np.uint32), st


def check(verts, idx, n, dims, m, light, w, h):
    f_gpu, c_gpu, st = gpu_render(verts, idx, n, dims, m, light, w, h)
    f_ref = oracle.raster(verts, idx, n, dims, m, w, h)
    c_ref = oracle.shade(verts, idx, dims, light, f_ref)
    assert np.array_equal(f_gpu, f_ref)
    assert np.array_equal(c_gpu, c_ref)
    return f_ref, st


@pytest.fixture(scope="module")
def surface():
    dims, rate = (48, 40, 36), 8
    f = fields.gradient_noise(*dims, 4, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    ref = oracle.extract(bits, dims, rate, bmin, bmax, float(np.median(d)))
    T = ref["num_triangles"]
    soup = np.zeros((3 * T, 4), np.float32)
    soup[:, :3] = ref["local_pos"].reshape(-1, 3).astype(np.float32)
    soup[:, 3] = np.repeat(ref["tri_block"], 3).view(np.float32)
    packed = oracle.quantized_vertices(ref["field"], float(np.median(d)), ref["edge_ids"], ref["tri_block"],
                                       dims).reshape(-1, 2)
    ix = oracle.indexed_mesh(ref["edge_ids"], ref["tri_block"], ref["local_pos"])
    iv = np.zeros((len(ix["vertex_edge"]), 4), np.float32)
    iv[:, :3] = ix["vertex_pos"].astype(np.float32)
    iv[:, 3] = ix["vertex_block"].view(np.float32)
    return dict(dims=dims, T=T, soup=soup, packed=packed, iv=iv, idx=ix["indices"].astype(np.uint32))


CAMERAS = {
    "far": lambda dims: cameras.orbit(dims, 30.0, 25.0, distance_factor=1.4, aspect=160 / 96),
    "side": lambda dims: cameras.orbit(dims, 200.0, -10.0, distance_factor=1.1, aspect=160 / 96),
    "close": lambda dims: cameras.look_at_perspective(40.0, 160 / 96, 0.5, 200.0, (20, 18, 30), (24, 20, 18)),
    "inside": lambda dims: cameras.look_at_perspective(70.0, 160 / 96, 0.5, 200.0, (24, 20, 18), (48, 40, 0)),
}


@pytest.mark.parametrize("cam", list(CAMERAS))
@pytest.mark.parametrize("kind", ["float4", "packed", "indexed"])
def test_surface_matches_oracle(surface, kind, cam):
    s = surface
    m = CAMERAS[cam](s["dims"])
    light = (0.3, -0.5, 0.8)
    if kind == "float4":
        f, st = check(s["soup"], None, s["T"], s["dims"], m, light, 160, 96)
    elif kind == "packed":
        f, st = check(s["packed"], None, s["T"], s["dims"], m, light, 160, 96)
    else:
        f, st = check(s["iv"], s["idx"], s["T"], s["dims"], m, light, 160, 96)
    assert (f != NONE).sum() > 200                     # the surface is on screen
    assert 0 < st["drawn"] <= s["T"]
    if cam == "close":
        assert st["big"] > 0                           # the warp kernel's path ran
    if cam == "far":
        assert st["big"] == 0


def test_hand_meshes_and_ties():
    dims = (64, 64, 64)

    def f4(points):
        p = np.asarray(points, np.float64)
        b = np.clip(np.floor(p / 4).astype(np.int64), 0, 15)
        out = np.zeros((len(p), 4), np.float32)
        out[:, :3] = (p - 4 * b).astype(np.float32)
        out[:, 3] = (b[:, 0] + 16 * (b[:, 1] + 16 * b[:, 2])).astype(np.uint32).view(np.float32)
        return out

    rng = np.random.default_rng(2)
    n, cell = 9, 5.0
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
    v = f4(pts)[np.array(tris).reshape(-1)]
    # the same mesh twice (ties go to the lower id) and a far copy under it
    under = v.copy()
    under[:, 2] += 0.5
    allv = np.concatenate([v, v, under])
    f, _ = check(allv, None, len(allv) // 3, dims, cameras.orthographic(40, 40), (0, 0, 1), 40, 40)
    assert np.all(f != NONE)
    assert np.all((f & np.uint64(0xFFFFFFFF)) < len(tris))        # the first copy wins everywhere
    # a big triangle over the whole viewport, both windings
    big = f4([(0, 0, 2), (80, 0, 2), (0, 80, 2), (0, 0, 2), (0, 80, 2), (80, 0, 2)])
    f, st = check(big, None, 2, dims, cameras.orthographic(40, 40), (1, 1, 1), 40, 40)
    assert st["big"] == 2 and np.all((f & np.uint64(0xFFFFFFFF)) == 0)


def test_index_past_the_vertices_is_not_drawn(surface):
    s = surface
    idx = s["idx"].copy()
    rng = np.random.default_rng(6)
    bad = rng.choice(len(idx), 50, replace=False)
    idx[bad, rng.integers(0, 3, 50)] = len(s["iv"]) + rng.integers(0, 1 << 30, 50).astype(np.uint32)
    m = CAMERAS["far"](s["dims"])
    f, st = check(s["iv"], idx, s["T"], s["dims"], m, (0.3, -0.5, 0.8), 160, 96)
    assert st["drawn"] <= s["T"] - 50
    assert not np.isin((f[f != NONE] & np.uint64(0xFFFFFFFF)).astype(np.int64), bad).any()


def test_empty_and_invalid():
    p = pkg()
    t = torch()
    dims = (16, 16, 16)
    m = cameras.orthographic(16, 16)
    v = t.zeros((3, 4), dtype=t.float32, device="cuda")
    frag, rgba, st = p.render(v, 0, dims, m, (0, 0, 1), 16, 8, stats=True)
    assert (frag == -1).all() and (rgba == 0).all() and st == {"drawn": 0, "big": 0}
    for kw in (dict(light=(0, 0, 0)), dict(width=0), dict(view_proj=np.full(16, np.nan, np.float32)),
               dict(num_triangles=2)):                  # a soup of 2 triangles needs 6 vertices
        args = dict(vertices=v, num_triangles=1, dims=dims, view_proj=m, light=(0, 0, 1), width=16, height=8)
        args.update(kw)
        with pytest.raises(p.IsoError) as e:
            p.render(**args)
        assert e.value.code == p.ISO_ERR_INVALID_ARG
