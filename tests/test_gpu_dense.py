"""GPU parity of the naive data-parallel marching cubes over a dense field
(iso_mc_dense, the Section 3.3.3 baseline): against the oracle's plain
full-volume marching cubes, triangle for triangle in the same order (global
edge ids exact, positions within 1e-5 voxel of the oracle's float64
interpolation, each vertex tagged with the block holding its cell), and
against the block path's soup of the same decoded field (the same triangles
as a multiset, byte for byte)."""
import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu

POS_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def make_field(kind, dims, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return fields.gradient_noise(nx, ny, nz, seed + 1, octaves=4, base_period=16)
    if kind == "sphere":
        return fields.sphere_sdf(nx, ny, nz, 0.3 * min(dims))
    if kind == "random":
        return rng.standard_normal((nz, ny, nx)).astype(np.float32)
    if kind == "wide":
        vals = np.array([3e38, -3e38, 1e38, -1e38, 2e37, -5e36, 0.5, -0.25, 1e-39, -2e-39, 0.0], np.float32)
        return rng.choice(vals, size=(nz, ny, nx)).astype(np.float32)
    if kind == "checker":
        return rng.integers(0, 2, (nz, ny, nx)).astype(np.float32)
    raise ValueError(kind)


def check_dense(field, iso):
    import torch
    import paper_2009_03254_gb300 as pkg
    nz, ny, nx = field.shape
    verts, st, edges = pkg.mc_dense(torch.from_numpy(np.ascontiguousarray(field)).cuda(), iso, edge_ids=True)
    ids, pos, cells = oracle.mc_full(field, iso, return_cells=True)
    T = len(ids)
    assert st["num_triangles"] == T
    # crossing cells: 0 < case < 255, counted independently here
    if nx > 1 and ny > 1 and nz > 1:
        below = field < np.float32(iso)
        c = sum((below[dz:nz - 1 + dz, dy:ny - 1 + dy, dx:nx - 1 + dx].astype(np.int32) << (dx + 2 * dy + 4 * dz))
                for dz in (0, 1) for dy in (0, 1) for dx in (0, 1))
        assert st["n_active_cells"] == int(((c > 0) & (c < 255)).sum())
    if T == 0:
        return verts
    assert np.array_equal(edges.cpu().numpy().view(np.uint64), ids)
    v = verts.cpu().numpy()
    x, y, z = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    nbx, nby = (nx + 3) // 4, (ny + 3) // 4
    bx, by, bz = x // 4, y // 4, z // 4
    assert np.array_equal(v[:, 0, 3].view(np.uint32), (bx + nbx * (by + nby * bz)).astype(np.uint32))
    glob = v[:, :, :3].astype(np.float64) + 4.0 * np.stack([bx, by, bz], -1)[:, None, :]
    assert np.abs(glob - pos).max() < POS_TOL
    return verts


CASES = [("noise", (37, 21, 14), 8), ("sphere", (33, 2, 9), 8), ("random", (13, 9, 6), 4), ("wide", (18, 10, 9), 16),
         ("checker", (11, 9, 7), 8), ("sphere", (64, 64, 64), 16), ("random", (5, 5, 5), 3), ("noise", (1, 7, 9), 8)]


@pytest.mark.parametrize("kind,dims,rate", CASES)
def test_dense_mc_matches_full_volume_oracle(kind, dims, rate):
    f = make_field(kind, dims, 7)
    bits, _, _ = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    for iso in (0.0, float(np.median(d)), float(np.quantile(d, 0.2)), float(d.max()) + 1.0):
        check_dense(d, iso)


@pytest.mark.parametrize("kind,dims,rate", [("noise", (37, 21, 14), 8), ("sphere", (40, 33, 29), 12),
                                            ("random", (13, 9, 6), 4)])
def test_dense_mc_equals_block_path_soup(kind, dims, rate):
    # the decoded field on the device, then the same triangles as the block
    # path: the same 48 bytes per triangle, only in cell rather than block order
    import torch
    import paper_2009_03254_gb300 as pkg
    f = make_field(kind, dims, 3)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    dev_bits = torch.from_numpy(bits.view(np.int64)).cuda()
    field = pkg.decode_volume(dev_bits, dims, rate)
    vol = pkg.Volume(bits, dims, rate, bmin, bmax)
    try:
        for iso in (0.0, float(np.median(oracle.decode_volume(bits, dims, rate)))):
            verts, st, _ = pkg.mc_dense(field, iso)
            m = vol.extract(iso)
            assert st["num_triangles"] == m.num_triangles
            if m.num_triangles:
                a = np.ascontiguousarray(verts.cpu().numpy()).view(np.uint8).reshape(-1, 48)
                b = np.ascontiguousarray(m.vertices.cpu().numpy()).view(np.uint8).reshape(-1, 48)
                ka = np.lexsort(a.T[::-1])
                kb = np.lexsort(b.T[::-1])
                assert np.array_equal(a[ka], b[kb])
            m.release()
    finally:
        vol.release()


def test_dense_mc_capacity_and_arguments():
    import ctypes
    import torch
    import paper_2009_03254_gb300 as pkg
    f = make_field("sphere", (24, 20, 18), 0)
    dev = torch.from_numpy(f).cuda()
    _, st, _ = pkg.mc_dense(dev, 0.0)
    T = st["num_triangles"]
    assert T > 0
    small = torch.zeros((T - 1, 3, 4), dtype=torch.float32, device="cuda")
    s = pkg._DenseStats()
    rc = pkg.lib().iso_mc_dense(ctypes.c_void_p(dev.data_ptr()), 24, 20, 18, ctypes.c_float(0.0),
                                ctypes.c_void_p(small.data_ptr()), T - 1, None, ctypes.byref(s), None)
    assert rc == pkg.ISO_ERR_CAPACITY and s.num_triangles == T
    assert not small.any()                               # nothing written
    for args in ((0.0, 0, 20, 18), (float("nan"), 24, 20, 18)):
        rc = pkg.lib().iso_mc_dense(ctypes.c_void_p(dev.data_ptr()), *args[1:], ctypes.c_float(args[0]), None, 0,
                                    None, ctypes.byref(s), None)
        assert rc == pkg.ISO_ERR_INVALID_ARG
