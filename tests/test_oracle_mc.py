"""Pins for the oracle's marching cubes: case table, full-volume MC (CPU only).

The paper cites marching cubes (Lorensen and Cline 1987) without a table.
The oracle's table is generated from a stated face rule; these tests check
it by brute force over all 256 cases and the meshes it makes against closed
forms (plane, sphere area and volume) and topology (watertight, Euler
characteristic 2 on a sphere).
"""
import math

import numpy as np
import pytest

import oracle
from synth import fields

NUM, TRI, MAXT = oracle.mc_table()
EDGES = [oracle.edge_info(e) for e in range(12)]      # (lo corner, hi corner, axis)


def corner(c):
    return np.array([c & 1, c >> 1 & 1, c >> 2 & 1], float)


def mid(e):
    lo, hi, a = EDGES[e]
    return (corner(lo) + corner(hi)) / 2


def tris(cs):
    return [tuple(int(x) for x in TRI[cs][3 * k:3 * k + 3]) for k in range(NUM[cs])]


def face_segments(cs):
    """The rule, restated directly: per face, the cut edges; two cut edges
    make one segment; four make two segments that each cut off one
    below-iso corner.  Directed with the below corners on the right, seen
    from outside the cube."""
    below = [cs >> c & 1 for c in range(8)]
    segs = set()
    for a in range(3):
        for s in (0, 1):
            n = np.zeros(3)
            n[a] = 2 * s - 1
            cs_face = [c for c in range(8) if (c >> a & 1) == s]
            fe = [e for e in range(12) if EDGES[e][2] != a and (EDGES[e][0] >> a & 1) == s
                  and below[EDGES[e][0]] != below[EDGES[e][1]]]
            pairs = []
            if len(fe) == 2:
                c = next(c for c in cs_face if below[c])
                pairs.append((fe[0], fe[1], c))
            elif len(fe) == 4:
                for c in cs_face:
                    if below[c]:
                        inc = [e for e in fe if c in EDGES[e][:2]]
                        pairs.append((inc[0], inc[1], c))
            for ea, eb, c in pairs:
                u, v = mid(eb) - mid(ea), corner(c) - mid(ea)
                if np.dot(np.cross(u, v), n) > 0:     # c on the left: flip
                    ea, eb = eb, ea
                segs.add((ea, eb))
    return segs


def test_table_max_and_range():
    assert MAXT == 5 and NUM.max() == 5
    assert NUM[0] == 0 and NUM[255] == 0
    for cs in range(256):
        for t in tris(cs):
            assert all(0 <= e < 12 for e in t) and len(set(t)) == 3


@pytest.mark.parametrize("cs", range(256))
def test_case_brute_force(cs):
    below = [cs >> c & 1 for c in range(8)]
    cut = {e for e in range(12) if below[EDGES[e][0]] != below[EDGES[e][1]]}
    used = {e for t in tris(cs) for e in t}
    assert used == cut                                   # exactly the sign-change edges
    directed = {}
    for t in tris(cs):
        for i in range(3):
            d = (t[i], t[(i + 1) % 3])
            directed[d] = directed.get(d, 0) + 1
    segs = face_segments(cs)
    for d, k in directed.items():
        rev = (d[1], d[0])
        if d in segs:
            assert k == 1 and rev not in directed        # boundary segment, once
        else:
            assert k == 1 and directed.get(rev) == 1     # interior edge, paired opposite
    assert segs <= set(directed)                         # every face segment is used


@pytest.mark.parametrize("c", range(8))
def test_single_corner_normal_points_away(c):
    for cs, sign in ((1 << c, 1.0), (255 ^ (1 << c), -1.0)):
        (t,) = tris(cs)
        p = [mid(e) for e in t]
        nrm = np.cross(p[1] - p[0], p[2] - p[0])
        assert sign * np.dot(nrm, p[0] - corner(c)) > 0  # toward the larger values


def test_normals_follow_trilinear_gradient():
    # corner values -1 (below) / +1; at each triangle's centroid the normal
    # and the gradient of the trilinear interpolant agree in sign for all
    # cases without a diagonal face (where the interpolant is unambiguous)
    for cs in range(1, 255):
        below = [cs >> c & 1 for c in range(8)]
        diag = False
        for a in range(3):
            for s in (0, 1):
                fc = [c for c in range(8) if (c >> a & 1) == s]
                if sum(below[EDGES[e][0]] != below[EDGES[e][1]] for e in range(12)
                       if EDGES[e][2] != a and (EDGES[e][0] >> a & 1) == s) == 4:
                    diag = True
        if diag:
            continue
        val = [-1.0 if below[c] else 1.0 for c in range(8)]
        for t in tris(cs):
            p = [mid(e) for e in t]
            nrm = np.cross(p[1] - p[0], p[2] - p[0])
            x, y, z = sum(p) / 3
            g = np.zeros(3)
            for c in range(8):
                cx, cy, cz = corner(c)
                wx, wy, wz = (x if cx else 1 - x), (y if cy else 1 - y), (z if cz else 1 - z)
                g += val[c] * np.array([(1 if cx else -1) * wy * wz,
                                        (1 if cy else -1) * wx * wz,
                                        (1 if cz else -1) * wx * wy])
            assert np.dot(nrm, g) > 0, cs


def _area_volume(pos):
    a, b, c = pos[:, 0], pos[:, 1], pos[:, 2]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1).sum()
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    return area, vol


def test_plane_closed_form():
    nx, ny, nz = 24, 13, 10
    f = fields.linear_ramp(nx, ny, nz, 10.25)
    ids, pos = oracle.mc_full(f, 0.125)
    assert np.all(pos[:, :, 0] == 10.375)                 # x0 + iso, exactly
    area, _ = _area_volume(pos)
    assert abs(area - (ny - 1) * (nz - 1)) < 1e-9
    assert len(ids) == 2 * (ny - 1) * (nz - 1)


def _watertight(ids):
    edges = {}
    for t in ids:
        for i in range(3):
            d = (int(t[i]), int(t[(i + 1) % 3]))
            edges[d] = edges.get(d, 0) + 1
    for (a, b), k in edges.items():
        assert k == 1 and edges.get((b, a)) == 1
    V = len({int(v) for v in ids.ravel()})
    E = len(edges) // 2
    return V - E + len(ids)


@pytest.mark.parametrize("r", [5, 10, 20, 40])
def test_sphere_closed_surface(r):
    n = 2 * r + 8
    f = fields.sphere_sdf(n, n, n, float(r))
    ids, pos = oracle.mc_full(f, 0.0)
    assert _watertight(ids) == 2
    area, vol = _area_volume(pos)
    # measured on the oracle: area -1.3e-2, -3.1e-3, -7.9e-4, -2.0e-4 and
    # volume -2.4e-2, -6.0e-3, -1.5e-3, -3.7e-4 for r = 5..40, falling 4x per
    # doubling of r (second order); the bounds leave a 2x margin
    rel_a = abs(area / (4 * math.pi * r * r) - 1)
    rel_v = abs(vol / (4 / 3 * math.pi * r ** 3) - 1)
    assert vol > 0                                        # outward normals
    assert rel_a < {5: 0.026, 10: 0.0063, 20: 0.0016, 40: 0.0004}[r]
    assert rel_v < {5: 0.05, 10: 0.012, 20: 0.003, 40: 0.00075}[r]


def test_sphere_error_converges():
    errs = []
    for r in (5, 10, 20, 40):
        n = 2 * r + 8
        _, pos = oracle.mc_full(fields.sphere_sdf(n, n, n, float(r)), 0.0)
        area, _ = _area_volume(pos)
        errs.append(abs(area / (4 * math.pi * r * r) - 1))
    for e0, e1 in zip(errs, errs[1:]):
        assert e1 < e0 / 2


def test_compressed_sphere_is_watertight():
    f = fields.sphere_sdf(64, 64, 64, 20.0)
    bits, _, _ = oracle.encode_volume(f, 16)
    d = oracle.decode_volume(bits, (64, 64, 64), 16)
    ids, pos = oracle.mc_full(d, 0.0)
    assert _watertight(ids) == 2


@pytest.mark.parametrize("iso", [-1.0, 0.0, 2.0])
def test_constant_and_flat_fields(iso):
    f = np.full((6, 7, 5), 0.0, np.float32)
    ids, _ = oracle.mc_full(f, iso)
    assert len(ids) == 0                                  # no sign change anywhere


def test_iso_equal_to_voxels():
    # values exactly at iso count as not below: a 0/1 checker at iso 1 puts
    # 1-valued corners on the upper side; vertices land on grid points
    rng = np.random.default_rng(5)
    f = rng.integers(0, 2, (7, 6, 9)).astype(np.float32)
    ids, pos = oracle.mc_full(f, 1.0)
    assert len(ids) > 0
    assert np.all(pos == np.round(pos))
