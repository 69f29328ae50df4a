"""Pins for the oracle's within-block indexed mesh (CPU only).

Section 4.5 names an indexed mesh with vertices shared inside each block
as the alternative to the triangle soup.  The oracle builds it from the
block-ordered soup by its plain definition (a block's vertices are the
distinct edges its triangles use, by axis, then lower sample).  These
tests tie it to
things outside that definition: gathering by index gives the soup back
exactly; a block's vertices are the cut edges of its 5x5x5 window found by
brute force over its cells; and with the blocks' vertices welded by edge,
a sphere is still a closed surface of Euler characteristic 2.
"""
import numpy as np
import pytest

import oracle
from synth import fields


def extract(field, iso, rate=16):
    nz, ny, nx = field.shape
    bits, bmin, bmax = oracle.encode_volume(field, rate)
    ref = oracle.extract(bits, (nx, ny, nz), rate, bmin, bmax, iso)
    return ref, oracle.indexed_mesh(ref["edge_ids"], ref["tri_block"], ref["local_pos"])


CASES = [
    ("sphere", lambda: fields.sphere_sdf(24, 20, 18, 6.5), 0.0),
    ("noise_ragged", lambda: fields.gradient_noise(33, 29, 21, 5, octaves=3, base_period=12), 0.05),
    ("noise_thin", lambda: fields.gradient_noise(41, 17, 9, 8, octaves=3, base_period=8), -0.1),
]


@pytest.mark.parametrize("name,make,iso", CASES, ids=[c[0] for c in CASES])
def test_gather_gives_the_soup(name, make, iso):
    ref, ix = extract(make(), iso)
    assert ref["num_triangles"] > 0
    idx = ix["indices"]
    assert idx.shape == (ref["num_triangles"], 3)
    assert idx.min() >= 0 and idx.max() < len(ix["vertex_edge"])
    assert np.array_equal(ix["vertex_edge"][idx], ref["edge_ids"])
    assert np.array_equal(ix["vertex_pos"][idx], ref["local_pos"])          # exact: same edge, same position
    assert np.array_equal(ix["vertex_block"][idx], np.repeat(ref["tri_block"][:, None], 3, 1))
    # every vertex is used, blocks ascend, a block's edges ascend strictly by
    # (axis, lower sample)
    assert len(np.unique(idx)) == len(ix["vertex_edge"])
    vb, ve = ix["vertex_block"].astype(np.int64), ix["vertex_edge"]
    assert np.all(np.diff(vb) >= 0)
    same = np.diff(vb) == 0
    key = (ve % 3) * (1 << 40) + ve // 3
    assert np.all(key[1:][same] > key[:-1][same])
    # a triangle's three corners are three different vertices
    assert np.all((idx[:, 0] != idx[:, 1]) & (idx[:, 1] != idx[:, 2]) & (idx[:, 0] != idx[:, 2]))


def window_cut_edges(field, iso, dims, b):
    """Brute force: global ids of the cut edges of block b's cells inside
    the volume (the block's indexed-mesh vertices), by axis, then id."""
    nx, ny, nz = dims
    nbx, nby, _ = oracle.block_dims(dims)
    bx, by, bz = b % nbx, (b // nbx) % nby, b // (nbx * nby)
    found = set()
    steps = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
    for cz in range(4 * bz, min(4 * bz + 4, nz - 1)):
        for cy in range(4 * by, min(4 * by + 4, ny - 1)):
            for cx in range(4 * bx, min(4 * bx + 4, nx - 1)):
                for ox in (0, 1):
                    for oy in (0, 1):
                        for oz in (0, 1):
                            x, y, z = cx + ox, cy + oy, cz + oz
                            for a, (dx, dy, dz) in enumerate(steps):
                                x2, y2, z2 = x + dx, y + dy, z + dz
                                # the edge must be one of the cell's own twelve
                                if x2 > cx + 1 or y2 > cy + 1 or z2 > cz + 1:
                                    continue
                                if (field[z, y, x] < iso) != (field[z2, y2, x2] < iso):
                                    found.add(3 * (x + nx * (y + ny * z)) + a)
    return sorted(found, key=lambda e: (e % 3, e))


@pytest.mark.parametrize("name,make,iso", CASES, ids=[c[0] for c in CASES])
def test_block_vertices_are_window_cut_edges(name, make, iso):
    f = make()
    nz, ny, nx = f.shape
    ref, ix = extract(f, iso)
    d = ref["field"]
    nb = int(np.prod(oracle.block_dims((nx, ny, nz))))
    vb, ve = ix["vertex_block"], ix["vertex_edge"]
    for b in range(nb):
        want = window_cut_edges(d, iso, (nx, ny, nz), b)
        got = ve[vb == b].tolist()
        assert got == want, b


def test_thin_last_block_layer_has_no_vertices():
    # nx = 4k + 1: the last block column holds one sample plane and no cells
    f = fields.gradient_noise(17, 12, 12, 2, octaves=2, base_period=6)
    ref, ix = extract(f, 0.0)
    nbx, _, _ = oracle.block_dims((17, 12, 12))
    assert ref["num_triangles"] > 0
    assert not np.any(ix["vertex_block"] % nbx == nbx - 1)


def welded_euler(ix):
    """Weld the blocks' copies of each edge's vertex, check every mesh edge
    has exactly two triangles on it, oppositely directed; return V - E + F."""
    tri = ix["vertex_edge"][ix["indices"]]
    directed = {}
    for t in tri:
        for i in range(3):
            d = (int(t[i]), int(t[(i + 1) % 3]))
            directed[d] = directed.get(d, 0) + 1
    for (a, b), k in directed.items():
        assert k == 1 and directed.get((b, a)) == 1
    V = len(np.unique(ix["vertex_edge"]))
    return V - len(directed) // 2 + len(tri)


@pytest.mark.parametrize("r", [4.5, 7.25])
def test_welded_sphere_is_closed(r):
    n = int(2 * r) + 9
    ref, ix = extract(fields.sphere_sdf(n, n + 3, n - 1, r), 0.0)
    assert welded_euler(ix) == 2
    # blocks share their face vertices: more vertices than the welded mesh
    assert len(ix["vertex_edge"]) > len(np.unique(ix["vertex_edge"]))


def test_empty_surface():
    f = fields.sphere_sdf(16, 16, 16, 5.0)
    ref, ix = extract(f, float(f.max()) + 1.0)
    assert ref["num_triangles"] == 0
    assert len(ix["vertex_edge"]) == 0 and ix["indices"].shape == (0, 3)
