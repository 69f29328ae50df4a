"""GPU parity of the within-block indexed mesh (Section 4.5's alternative
output: vertices shared inside each block) against the oracle's plain
definition (oracle.indexed_mesh over the oracle's own soup).

Indices, vertex counts, block ids and compact vertex codes must match bit
for bit; float positions within 1e-5 voxel (float32 against the oracle's
float64, as for the soup).  Gathering the GPU vertices by its indices must
also give the GPU's own soup byte for byte (same edge, same arithmetic).
Cases cover ragged volumes, blocks without cells (nx = 4k + 1), dense
random and checker fields (more than 96 vertices in a warp tile's four
blocks), empty surfaces, buffers too small, the captured graph alternating
with the soup, and waves under a small cache budget.
"""
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


def pkg():
    import paper_2009_03254_gb300 as p
    return p


def torch():
    import torch as t
    return t


def make_field(kind, dims, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return fields.gradient_noise(nx, ny, nz, seed + 1, octaves=4, base_period=16)
    if kind == "sphere":
        return fields.sphere_sdf(nx, ny, nz, 0.3 * min(dims))
    if kind == "random":
        return rng.standard_normal((nz, ny, nx)).astype(np.float32)
    if kind == "checker":
        return rng.integers(0, 2, (nz, ny, nx)).astype(np.float32)
    if kind == "wide":      # samples up to +-3e38: differences beyond 2^125 and past FLT_MAX, and tiny ones
        vals = np.array([3e38, -3e38, 1e38, -1e38, 2e37, -5e36, 0.5, -0.25, 1e-39, -2e-39, 0.0], np.float32)
        return rng.choice(vals, size=(nz, ny, nx)).astype(np.float32)
    raise ValueError(kind)


def oracle_indexed(bits, dims, rate, bmin, bmax, iso):
    ref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
    return ref, oracle.indexed_mesh(ref["edge_ids"], ref["tri_block"], ref["local_pos"])


def check_float(vol, ref, ix, iso):
    t = torch()
    V, T = len(ix["vertex_edge"]), ref["num_triangles"]
    verts = t.full((V + 5, 4), -7.0, dtype=t.float32, device="cuda")
    idx = t.full((T + 5, 3), -7, dtype=t.int32, device="cuda")
    st = vol.extract_indexed_into(iso, verts, idx)
    assert st["num_vertices"] == V and st["num_triangles"] == T
    gi = idx.cpu().numpy()
    gv = verts.cpu().numpy()
    assert np.array_equal(gi[:T].astype(np.int64), ix["indices"])
    assert (gi[T:] == -7).all() and (gv[V:] == -7.0).all()          # nothing past the mesh
    if V:
        assert np.abs(gv[:V, :3].astype(np.float64) - ix["vertex_pos"]).max() < POS_TOL
        assert np.array_equal(gv[:V, 3].view(np.uint32), ix["vertex_block"])
    return gv[:V], gi[:T]


def check_packed(vol, ref, ix, iso, dims):
    t = torch()
    V, T = len(ix["vertex_edge"]), ref["num_triangles"]
    verts = t.zeros((max(V, 1), 2), dtype=t.int32, device="cuda")
    idx = t.zeros((max(T, 1), 3), dtype=t.int32, device="cuda")
    st = vol.extract_indexed_into(iso, verts, idx)
    assert st["num_vertices"] == V and st["num_triangles"] == T
    assert np.array_equal(idx.cpu().numpy()[:T].astype(np.int64), ix["indices"])
    if V:
        # each vertex as a triangle with three equal corners in the soup's quantizer
        e3 = np.repeat(ix["vertex_edge"][:, None], 3, axis=1)
        want = oracle.quantized_vertices(ref["field"], iso, e3, ix["vertex_block"], dims)[:, 0, :]
        got = verts.cpu().numpy().view(np.uint32)[:V]
        assert np.array_equal(got, want)


@pytest.mark.parametrize("kind,dims,rate", [
    ("sphere", (24, 20, 18), 16), ("noise", (33, 29, 21), 8), ("noise", (41, 17, 9), 8),
    ("noise", (17, 12, 13), 12), ("random", (19, 14, 11), 8), ("checker", (11, 9, 7), 8),
    ("wide", (19, 14, 11), 16),
])
def test_indexed_matches_oracle(kind, dims, rate):
    t = torch()
    f = make_field(kind, dims, 3)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax)
    try:
        isos = [float(np.median(d)), float(np.quantile(d, 0.3)), float(d.max()) + 1.0]
        if kind == "sphere":
            isos = [0.0, 1.5] + isos
        if kind == "wide":
            isos = [0.0, 1e37, -1.5e38] + isos
        for iso in isos:
            ref, ix = oracle_indexed(bits, dims, rate, bmin, bmax, iso)
            gv, gi = check_float(vol, ref, ix, iso)
            # gathered by index: the soup, byte for byte
            T = ref["num_triangles"]
            soup = t.zeros((max(T, 1) * 3, 4), dtype=t.float32, device="cuda")
            vol.extract_into(iso, soup)
            if T:
                assert np.array_equal(gv[gi].reshape(-1, 4).view(np.uint32),
                                      soup.cpu().numpy()[:3 * T].view(np.uint32))
            check_packed(vol, ref, ix, iso, dims)
    finally:
        vol.release()


def test_indexed_graph_alternates_with_soup():
    # the captured graphs (one per output kind) keep giving the same meshes
    dims, rate = (40, 36, 28), 8
    f = make_field("noise", dims, 11)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax)
    try:
        isos = [float(x) for x in np.quantile(d, [0.4, 0.6, 0.5])]
        refs = [oracle_indexed(bits, dims, rate, bmin, bmax, x) for x in isos]
        for rnd in range(3):
            for x, (ref, ix) in zip(isos, refs):
                check_float(vol, ref, ix, x)
                m = vol.extract(x)
                assert m.num_triangles == ref["num_triangles"]
                m.release()
    finally:
        vol.release()


def test_indexed_capacity():
    t = torch()
    p = pkg()
    dims, rate = (33, 29, 21), 8
    f = make_field("noise", dims, 5)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    iso = float(np.median(oracle.decode_volume(bits, dims, rate)))
    ref, ix = oracle_indexed(bits, dims, rate, bmin, bmax, iso)
    V, T = len(ix["vertex_edge"]), ref["num_triangles"]
    assert V > 100 and T > 100
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        for vcap, tcap in ((V // 2, T + 1), (V, T // 3), (0, 0)):
            vb = t.full((V + 8, 4), -3.0, dtype=t.float32, device="cuda")
            ib = t.full((T + 8, 3), -3, dtype=t.int32, device="cuda")
            st = vol.extract_indexed_into(iso, vb[:vcap] if vcap else vb[:0], ib[:tcap] if tcap else ib[:0],
                                          check=False)
            assert st["status"] == p.ISO_ERR_CAPACITY
            assert st["num_vertices"] == V and st["num_triangles"] == T
            gv, gi = vb.cpu().numpy(), ib.cpu().numpy()
            assert (gv[vcap:] == -3.0).all() and (gi[tcap:] == -3).all()     # nothing past the buffers
            k = min(tcap, T)
            assert np.array_equal(gi[:k].astype(np.int64), ix["indices"][:k])
            if vcap:
                assert np.abs(gv[:vcap, :3] - ix["vertex_pos"][:vcap]).max() < POS_TOL
        v, i, st = vol.extract_indexed(iso, guess_triangles=16)     # grows to the exact size
        assert v.shape == (V, 4) and i.shape == (T, 3)
        assert np.array_equal(i.cpu().numpy().astype(np.int64), ix["indices"])
        with pytest.raises(p.IsoError):
            vol.extract_indexed_into(float("nan"), vb, ib)
    finally:
        vol.release()


def test_indexed_waves_under_small_cache():
    # a cache holding two block layers' active blocks but not the surface:
    # the waves' vertices and indices append to one mesh, equal to one pass
    dims, rate = (40, 36, 96), 8
    f = fields.gradient_noise(*dims, 6, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    iso = float(np.median(oracle.decode_volume(bits, dims, rate)))
    nbx, nby, nbz = oracle.block_dims(dims)
    act = oracle.active_blocks(bmin, bmax, (nbx, nby, nbz), iso).reshape(nbz, nby * nbx).sum(axis=1)
    budget = int(max(act[z] + (act[z + 1] if z + 1 < nbz else 0) for z in range(nbz))) + 5
    assert act.sum() > budget
    ref, ix = oracle_indexed(bits, dims, rate, bmin, bmax, iso)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * budget)
    try:
        for _ in range(2):
            gv, gi = check_float(vol, ref, ix, iso)
        t = torch()
        st = vol.extract_indexed_into(iso, t.zeros((len(gv), 2), dtype=t.int32, device="cuda"),
                                      t.zeros((len(gi), 3), dtype=t.int32, device="cuda"))
        assert st["waves"] > 1 and st["num_vertices"] == len(gv)
    finally:
        vol.release()


def test_indexed_debug_volume_edge_ids():
    # a debug volume (no graph) also records each soup corner's edge: the
    # edge of the indexed vertex it points at
    dims, rate = (26, 22, 19), 16
    f = make_field("sphere", dims, 0)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, debug=True)
    try:
        ref, ix = oracle_indexed(bits, dims, rate, bmin, bmax, 0.0)
        gv, gi = check_float(vol, ref, ix, 0.0)
        edges = vol.debug("edge_ids").reshape(-1, 3)
        assert np.array_equal(edges, ix["vertex_edge"][gi])
        cnt = vol.debug("block_tris")
        nv = (cnt >> 16).astype(np.int64)
        assert nv.sum() == len(gv)
        assert np.array_equal(cnt & 0xFFFF, np.bincount(np.searchsorted(vol.debug("candidates"), ref["tri_block"]),
                                                        minlength=len(cnt)))
    finally:
        vol.release()


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (5, 2, 3), (4, 4, 4), (9, 1, 9), (3, 3, 17)])
def test_indexed_degenerate_volumes(dims):
    # single samples, single cells, flat volumes (a dimension of 1: no cells)
    # and exact multiples of 4: same mesh as the oracle, empty where it is
    f = make_field("random", dims, 21)
    bits, bmin, bmax = oracle.encode_volume(f, 12)
    d = oracle.decode_volume(bits, dims, 12)
    vol = pkg().Volume(bits, dims, 12, bmin, bmax)
    try:
        iso = float(np.median(d))
        ref, ix = oracle_indexed(bits, dims, 12, bmin, bmax, iso)
        check_float(vol, ref, ix, iso)
        if 1 in dims:
            assert ref["num_triangles"] == 0 and len(ix["vertex_edge"]) == 0
    finally:
        vol.release()
