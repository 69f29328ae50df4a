"""GPU parity: every stage of the CUDA path against the CPU oracle.

Integer, index and bit results (decoded samples, bitstreams, active and new
block lists, cell cases, per-block counts and offsets, cache slot
assignment, triangle edge ids and their order) must match bit for bit.
Vertex positions must agree within 1e-5 voxel units: the oracle
interpolates in float64, the GPU in float32 with IEEE division; with
block-local coordinates in [0, 4] the float32 result is within a few ulp
of 4 (~1e-6), so 1e-5 is a bound with margin, not a fit.
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


def make_field(kind, dims, seed=0):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    if kind == "noise":
        return fields.gradient_noise(nx, ny, nz, seed + 1, octaves=4, base_period=16)
    if kind == "sphere":
        return fields.sphere_sdf(nx, ny, nz, 0.3 * min(dims))
    if kind == "random":
        return rng.standard_normal((nz, ny, nx)).astype(np.float32)
    if kind == "special":   # zeros of both signs, subnormals, huge and tiny magnitudes
        vals = np.array([0.0, -0.0, 1e-45, -3e-39, 1e-38, 1.5, -2.25, 1e30, -7e29, 3.4e-20, 65504.0], np.float32)
        f = rng.choice(vals, size=(nz, ny, nx)).astype(np.float32)
        f *= rng.choice(np.array([1.0, 0.5, 2.0], np.float32), size=f.shape)
        return f
    if kind == "checker":
        return rng.integers(0, 2, (nz, ny, nx)).astype(np.float32)
    if kind == "wide":      # samples up to +-3e38: differences beyond 2^125 and past FLT_MAX, and tiny ones
        vals = np.array([3e38, -3e38, 1e38, -1e38, 2e37, -5e36, 0.5, -0.25, 1e-39, -2e-39, 0.0], np.float32)
        return rng.choice(vals, size=(nz, ny, nx)).astype(np.float32)
    raise ValueError(kind)


def to_dev(a):
    t = torch()
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return t.from_numpy(a).cuda()


# ---------------------------------------------------------------- codec

DECODE_CASES = [("noise", (37, 21, 14)), ("sphere", (20, 20, 20)), ("random", (9, 13, 7)), ("special", (16, 12, 8))]


@pytest.mark.parametrize("rate", [1, 2, 3, 4, 8, 12, 16, 24, 32])
@pytest.mark.parametrize("kind,dims", DECODE_CASES)
def test_decode_blocks_bit_exact(kind, dims, rate):
    f = make_field(kind, dims, 3)
    bits, _, _ = oracle.encode_volume(f, rate)
    ids = np.arange(bits.shape[0], dtype=np.uint32)
    want = oracle.decode_blocks(bits, rate, ids)
    got = pkg().decode_blocks(to_dev(bits), rate, to_dev(ids)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("rate", [1, 2, 5, 8, 16])
def test_decode_corrupt_streams_bit_exact(rate):
    rng = np.random.default_rng(rate)
    bits = rng.integers(0, 1 << 63, (3000, rate), dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, (3000, rate), dtype=np.uint64)
    bits[::7, 0] |= np.uint64(1)
    ids = np.arange(3000, dtype=np.uint32)
    want = oracle.decode_blocks(bits, rate, ids)
    got = pkg().decode_blocks(to_dev(bits), rate, to_dev(ids)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("rate", [1, 2, 4, 7, 8, 16, 32])
@pytest.mark.parametrize("kind,dims", DECODE_CASES + [("sphere", (1, 1, 1)), ("noise", (5, 3, 2))])
def test_encode_field_bit_exact(kind, dims, rate):
    f = make_field(kind, dims, 5)
    want_bits, want_min, want_max = oracle.encode_volume(f, rate)
    bits, bmin, bmax = pkg().encode_field(to_dev(f), rate)
    torch().cuda.synchronize()
    assert np.array_equal(bits.cpu().numpy().view(np.uint64), want_bits)
    assert np.array_equal(bmin.cpu().numpy(), want_min)
    assert np.array_equal(bmax.cpu().numpy(), want_max)


def test_gpu_generators_match_numpy():
    import synth.gpu as sg
    sg.build()
    for dims, origin, seed in (((40, 24, 20), (0, 0, 0), 1), ((33, 17, 9), (100, 260, 31), 9)):
        want = fields.gradient_noise(*dims, seed, origin=origin)
        got = sg.gradient_noise(*dims, seed, origin=origin).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    want = fields.sphere_sdf(30, 26, 22, 9.5, center=(14.5, 12.0, 10.25), origin=(3, 4, 5))
    got = sg.sphere_sdf(30, 26, 22, 9.5, center=(14.5, 12.0, 10.25), origin=(3, 4, 5)).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    for dims, origin, nzt in (((37, 22, 18), (0, 0, 0), 18), ((24, 20, 30), (1024, 4096, 64), 1536)):
        want = fields.channel_field(*dims, 5, nz_total=nzt, origin=origin)
        got = sg.channel_field(*dims, 5, nz_total=nzt, origin=origin).cpu().numpy()
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


# ---------------------------------------------------------------- extraction

def plus_group_candidates(bmin, bmax, dims, iso, active):
    """Active blocks whose 2x2x2 +group (block and +x/+y/+z neighbours that
    exist) has a range containing iso: the only blocks that can emit."""
    nbx, nby, nbz = oracle.block_dims(dims)
    lo = bmin.reshape(nbz, nby, nbx).astype(np.float64)
    hi = bmax.reshape(nbz, nby, nbx).astype(np.float64)
    lo8, hi8 = lo.copy(), hi.copy()
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                sl = (slice(0, nbz - dz), slice(0, nby - dy), slice(0, nbx - dx))
                sh = (slice(dz, nbz), slice(dy, nby), slice(dx, nbx))
                lo8[sl] = np.minimum(lo8[sl], lo[sh])
                hi8[sl] = np.maximum(hi8[sl], hi[sh])
    return active & ((lo8 < iso) & (iso <= hi8)).ravel()


def check_surface(vol, bits, dims, rate, bmin, bmax, iso, mesh=None):
    p = pkg()
    if mesh is None:
        mesh = vol.extract(iso)
    ref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
    assert mesh.num_triangles == ref["num_triangles"]
    act = vol.debug("active_ids")
    assert np.array_equal(act, np.nonzero(ref["active"])[0].astype(np.uint32))
    mask = vol.debug("active_mask")
    bitsv = np.unpackbits(mask.view(np.uint8), bitorder="little")[:len(ref["active"])].astype(bool)
    assert np.array_equal(bitsv, ref["active"])
    # the triangle stage visits exactly the candidates; every block the
    # oracle finds occupied is one of them, and none of them needed an
    # extent reset
    cand_ids = vol.debug("candidates")
    want_cand = plus_group_candidates(bmin, bmax, dims, iso, ref["active"])
    assert np.array_equal(cand_ids, np.nonzero(want_cand)[0].astype(np.uint32))
    assert set(ref["ids"][ref["block_tri"] > 0].tolist()) <= set(cand_ids.tolist())
    cand = np.searchsorted(act, cand_ids)                  # positions in the active list
    assert ref["complete"][cand].all()
    cases = vol.debug("cell_cases").reshape(-1, 64)
    assert np.array_equal(cases, ref["cases"][cand])
    assert np.array_equal(vol.debug("block_tris"), ref["block_tri"][cand])
    assert np.array_equal(vol.debug("block_offsets"), ref["block_off"][cand])
    assert mesh.stats["n_occupied"] == int((ref["block_tri"] > 0).sum())
    assert mesh.stats["n_active"] == len(act)
    if len(act):
        got_blocks = vol.read_blocks(act)
        assert np.array_equal(got_blocks.view(np.uint32), oracle.decode_blocks(bits, rate, act).view(np.uint32))
    if ref["num_triangles"]:
        edges = vol.debug("edge_ids").reshape(-1, 3)
        assert np.array_equal(edges, ref["edge_ids"])
        v = mesh.vertices.cpu().numpy().reshape(-1, 3, 4)
        err = np.abs(v[:, :, :3].astype(np.float64) - ref["local_pos"]).max()
        assert err < POS_TOL, err
        assert np.array_equal(v[:, :, 3].view(np.uint32), np.repeat(ref["tri_block"][:, None], 3, axis=1))
        assert (v[:, :, :3] >= 0).all() and (v[:, :, :3] <= 4).all()
    mesh.release()
    return ref


EXTRACT_CASES = [("sphere", (64, 64, 64), 16), ("noise", (37, 21, 14), 8), ("random", (13, 9, 6), 4),
                 ("noise", (33, 20, 17), 12), ("random", (5, 5, 5), 3), ("random", (2, 3, 5), 8),
                 ("noise", (4, 4, 4), 2), ("random", (3, 2, 2), 16), ("sphere", (33, 2, 9), 8),
                 ("random", (1, 1, 1), 8), ("special", (18, 10, 9), 16), ("checker", (11, 9, 7), 8),
                 ("wide", (18, 10, 9), 16), ("wide", (13, 9, 6), 32)]


@pytest.mark.parametrize("kind,dims,rate", EXTRACT_CASES)
def test_extract_matches_oracle(kind, dims, rate):
    f = make_field(kind, dims, 7)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    isos = [0.0, float(np.median(d)), float(np.quantile(d, 0.2)), float(d.min()), float(d.max()), 1.0, -1e9, 1e9]
    if kind == "wide":
        assert np.isfinite(d).all()
        isos += [1e37, -1.5e38, 2e38]
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, debug=True)
    try:
        for iso in isos:
            check_surface(vol, bits, dims, rate, bmin, bmax, iso)
    finally:
        vol.release()


SEGMENT_CASES = [("sphere", (64, 64, 64), 16), ("noise", (96, 80, 72), 8), ("sphere", (130, 70, 36), 4),
                 ("special", (18, 10, 9), 16), ("wide", (13, 9, 6), 32), ("random", (2, 3, 5), 8)]


@pytest.mark.parametrize("kind,dims,rate", SEGMENT_CASES)
def test_segment_cull_matches_oracle(kind, dims, rate):
    # segment ranges forced on: the range test reads a segment's range first
    # and skips the blocks of segments that cannot hold the isovalue; the
    # active set, candidates and surface are the oracle's (the sphere and the
    # isovalues far in the tails leave most segments skipped)
    f = make_field(kind, dims, 7)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    isos = [0.0, float(np.median(d)), float(np.quantile(d, 0.02)), float(np.quantile(d, 0.98)), float(d.min()),
            float(d.max()), 1e9]
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, debug=True, segment_cull=True)
    try:
        for iso in isos:
            check_surface(vol, bits, dims, rate, bmin, bmax, iso)
    finally:
        vol.release()


def test_segment_cull_serving_and_batch_equal_plain():
    # the serving cull and a batch over segment-cull volumes give the plain
    # volume's meshes byte for byte
    p = pkg()
    dims, rate = (96, 80, 72), 8
    f = make_field("noise", dims, 11)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    isos = [float(x) for x in np.quantile(d, [0.05, 0.5, 0.95])]
    plain = p.Volume(bits, dims, rate, bmin, bmax, segment_cull=False)
    seg = p.Volume(bits, dims, rate, bmin, bmax, segment_cull=True)
    srv = p.Server(seg, max_batch=2)
    try:
        tickets = [srv.submit(x) for x in isos]
        while srv.queued():
            srv.step()
        for t, x in zip(tickets, isos):
            status, m = srv.take(t)
            assert status == p.ISO_OK
            ref = plain.extract(x)
            assert m.num_triangles == ref.num_triangles
            if ref.num_triangles:
                assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32),
                                      ref.vertices.cpu().numpy().view(np.uint32))
            m.release()
            ref.release()
        srv.release()
        srv = None
        batch = p.Batch([seg, plain])
        try:
            verts, offs, _ = batch.extract([isos[1], isos[1]])
            v = verts.cpu().numpy().view(np.uint32).reshape(-1, 3, 4)
            a, b = v[int(offs[0]):int(offs[1])], v[int(offs[1]):int(offs[2])]
            assert len(a) == len(b) > 0
            assert np.array_equal(a, b)
        finally:
            batch.release()
    finally:
        if srv is not None:
            srv.release()
        seg.release()
        plain.release()


def test_sphere64_closed_surface_on_gpu():
    # the 64^3 sphere distance field at 16 bits/value: watertight, genus 0
    f = fields.sphere_sdf(64, 64, 64, 20.0)
    bits, bmin, bmax = oracle.encode_volume(f, 16)
    vol = pkg().Volume(bits, (64, 64, 64), 16, bmin, bmax, debug=True)
    try:
        mesh = vol.extract(0.0)
        e = vol.debug("edge_ids").reshape(-1, 3)
        und = {}
        for t in e:
            for i in range(3):
                a, b = int(t[i]), int(t[(i + 1) % 3])
                und[(a, b)] = und.get((a, b), 0) + 1
        assert all(k == 1 and und.get((b, a)) == 1 for (a, b), k in und.items())
        V = len(set(e.ravel().tolist()))
        assert V - len(und) // 2 + len(e) == 2
        mesh.release()
    finally:
        vol.release()


@pytest.mark.parametrize("kind", ["random", "up", "down"])
def test_cache_matches_algorithm1(kind):
    dims, rate = (48, 40, 36), 8
    f = make_field("noise", dims, 11)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    nb = bits.shape[0]
    frac = 0.02
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, debug=True, initial_cache_fraction=frac)
    cache = oracle.LRUCache(nb, int(np.ceil(frac * nb)), nb)
    lo, hi = np.quantile(d, [0.05, 0.95])
    rng = np.random.default_rng(21)
    if kind == "random":
        isos = rng.uniform(lo, hi, 70)
    elif kind == "up":
        isos = np.linspace(lo, hi, 65)
    else:
        isos = np.linspace(hi, lo, 65)
    nbd = oracle.block_dims(dims)
    try:
        for iso in isos.astype(np.float32):
            mesh = vol.extract(float(iso))
            act = oracle.active_blocks(bmin, bmax, nbd, float(iso))
            I_new, _ = cache.update(act)
            assert np.array_equal(vol.debug("new_ids"), I_new.astype(np.uint32))
            assert mesh.stats["n_slots"] == cache.num_slots
            assert np.array_equal(vol.debug("slot_of_block"), cache.I_slot.astype(np.int32))
            assert np.array_equal(vol.debug("block_of_slot"), cache.S_block.astype(np.int32))
            assert np.array_equal(vol.debug("slot_last_use"), cache.last_use().astype(np.uint32))
            mesh.release()
        # the surface is still exact after all the evictions
        check_surface(vol, bits, dims, rate, bmin, bmax, float(np.median(d)))
    finally:
        vol.release()


def test_capped_cache_matches_algorithm1():
    # a budget of 1.25x the largest active set: the cache grows to its cap,
    # then every update evicts among the inactive slots; each step must
    # match the simulator of Algorithm 1 with the same cap
    dims, rate = (64, 64, 64), 8                 # spherical shells: the active set moves through the volume
    f = make_field("sphere", dims)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    nb = bits.shape[0]
    nbd = oracle.block_dims(dims)
    lo, hi = np.quantile(d, [0.05, 0.95])
    isos = np.random.default_rng(33).uniform(lo, hi, 60).astype(np.float32)
    acts = [oracle.active_blocks(bmin, bmax, nbd, float(x)) for x in isos]
    cap = int(np.ceil(1.25 * max(int(a.sum()) for a in acts)))
    assert cap < nb
    frac = 0.02
    vol = pkg().Volume(bits, dims, rate, bmin, bmax, debug=True, initial_cache_fraction=frac,
                       cache_budget_bytes=256 * cap)
    cache = oracle.LRUCache(nb, int(np.ceil(frac * nb)), cap)
    evicted = 0
    try:
        for iso, act in zip(isos, acts):
            before = cache.I_slot >= 0
            mesh = vol.extract(float(iso))
            I_new, _ = cache.update(act)
            evicted += int((before & (cache.I_slot < 0)).sum())
            assert np.array_equal(vol.debug("new_ids"), I_new.astype(np.uint32))
            assert mesh.stats["n_slots"] == cache.num_slots <= cap
            assert np.array_equal(vol.debug("slot_of_block"), cache.I_slot.astype(np.int32))
            assert np.array_equal(vol.debug("block_of_slot"), cache.S_block.astype(np.int32))
            assert np.array_equal(vol.debug("slot_last_use"), cache.last_use().astype(np.uint32))
            mesh.release()
        assert cache.num_slots == cap and evicted > 1000
        check_surface(vol, bits, dims, rate, bmin, bmax, float(np.median(d)))
    finally:
        vol.release()


def test_budget_exceeded_then_recovers():
    p = pkg()
    dims, rate = (40, 40, 40), 8
    f = make_field("noise", dims, 2)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = p.Volume(bits, dims, rate, bmin, bmax, debug=True, cache_budget_bytes=40 * 256)
    try:
        with pytest.raises(p.IsoError) as e:
            vol.extract(float(np.median(d)))
        assert e.value.code == p.ISO_ERR_BUDGET
        # a surface whose active set fits still comes out exact
        iso = float(d.max()) - 1e-3 * float(d.max() - d.min())
        ref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
        if ref["active"].sum() <= 40:
            check_surface(vol, bits, dims, rate, bmin, bmax, iso)
    finally:
        vol.release()


def test_extract_into_capacity_and_exact_allocation():
    p = pkg()
    t = torch()
    dims, rate = (32, 32, 32), 8
    f = fields.gradient_noise(*dims, 3, octaves=3, base_period=8)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    ref = oracle.extract(bits, dims, rate, bmin, bmax, 0.0)
    T = ref["num_triangles"]
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        # the library sizes the mesh from the count: exactly T, no second pass;
        # ten times (plain launches, then the captured count and emit graphs)
        for _ in range(10):
            mesh = vol.extract(0.0)
            assert mesh.stats["reruns"] == 0 and mesh.num_triangles == T
            v = mesh.vertices.cpu().numpy().reshape(-1, 3, 4)
            assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < POS_TOL
            mesh.release()
        other = oracle.extract(bits, dims, rate, bmin, bmax, 0.5)
        mesh = vol.extract(0.5)
        assert mesh.num_triangles == other["num_triangles"]
        assert np.abs(mesh.vertices.cpu().numpy().reshape(-1, 3, 4)[:, :, :3] - other["local_pos"]).max() < POS_TOL
        mesh.release()
        small = t.zeros((100, 3, 4), dtype=t.float32, device="cuda")
        with pytest.raises(p.IsoError) as e:
            vol.extract_into(0.0, small)
        assert e.value.code == p.ISO_ERR_CAPACITY
        st = vol.extract_into(0.0, small, check=False)
        assert st["num_triangles"] == T
        w = small.cpu().numpy()
        assert np.abs(w[:, :, :3] - ref["local_pos"][:100]).max() < POS_TOL
        big = t.zeros((T, 3, 4), dtype=t.float32, device="cuda")
        st = vol.extract_into(0.0, big)
        assert st["num_triangles"] == T and st["n_new"] == 0   # all hits the second time
        assert np.abs(big.cpu().numpy()[:, :, :3] - ref["local_pos"]).max() < POS_TOL
    finally:
        vol.release()


def test_cache_reset_and_side_stream():
    p = pkg()
    t = torch()
    dims, rate = (30, 26, 22), 8
    f = make_field("noise", dims, 4)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    s = t.cuda.Stream()
    with t.cuda.stream(s):
        vol = p.Volume(bits, dims, rate, bmin, bmax, debug=True)
        try:
            m = vol.extract(0.1)
            assert m.stats["n_new"] == m.stats["n_active"] > 0
            m.release()
            m = vol.extract(0.1)
            assert m.stats["n_new"] == 0
            m.release()
            vol.cache_reset()
            m = vol.extract(0.1)
            assert m.stats["n_new"] == m.stats["n_active"]
            m.release()
            check_surface(vol, bits, dims, rate, bmin, bmax, 0.1)
        finally:
            vol.release()


def test_invalid_arguments():
    p = pkg()
    dims, rate = (8, 8, 8), 4
    bits, bmin, bmax = oracle.encode_volume(make_field("noise", dims), rate)
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        for bad in (float("nan"), float("inf"), -float("inf")):
            with pytest.raises(p.IsoError) as e:
                vol.extract(bad)
            assert e.value.code == p.ISO_ERR_INVALID_ARG
    finally:
        vol.release()
    with pytest.raises(p.IsoError):
        p.Volume(bits, dims, 0, bmin, bmax)
    with pytest.raises(p.IsoError):
        p.Volume(bits[:-1], dims, rate, bmin, bmax)


def test_graph_and_plain_launches_agree():
    # the default path replays one captured CUDA graph per extraction; the
    # plain path launches the same kernels one by one: meshes, counts and
    # cache decisions must be identical
    p = pkg()
    dims, rate = (40, 36, 30), 8
    f = make_field("noise", dims, 8)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    a = p.Volume(bits, dims, rate, bmin, bmax, graph=True, initial_cache_fraction=0.05)
    b = p.Volume(bits, dims, rate, bmin, bmax, graph=False, initial_cache_fraction=0.05)
    t = torch()
    try:
        # two extractions per isovalue and volume (the exact-size and the
        # single-pass path): graphs are captured after eight, so the later
        # isovalues replay them
        for iso in (0.0, 0.3, -0.4, 0.3, 0.1, -0.2, 0.5, 0.0):
            ma, mb = a.extract(iso), b.extract(iso)
            assert ma.num_triangles == mb.num_triangles
            assert ma.stats == mb.stats
            va, vb = ma.vertices.cpu().numpy(), mb.vertices.cpu().numpy()
            assert np.array_equal(va.view(np.uint32), vb.view(np.uint32))
            oa = t.zeros((ma.num_triangles + 1, 3, 4), dtype=t.float32, device="cuda")
            ob = t.zeros_like(oa)
            sa, sb = a.extract_into(iso, oa), b.extract_into(iso, ob)
            assert sa == sb and sa["num_triangles"] == ma.num_triangles
            assert np.array_equal(oa.cpu().numpy().view(np.uint32), ob.cpu().numpy().view(np.uint32))
            ma.release()
            mb.release()
        ref = oracle.extract(bits, dims, rate, bmin, bmax, 0.1)
        m = a.extract(0.1)
        v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
        assert m.num_triangles == ref["num_triangles"]
        assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < POS_TOL
        m.release()
    finally:
        a.release()
        b.release()


# ---------------------------------------------------------------- compact vertices (Section 4.5)

@pytest.mark.parametrize("kind,dims,rate", [("sphere", (64, 64, 64), 16), ("noise", (37, 21, 14), 8),
                                            ("random", (13, 9, 6), 4), ("special", (18, 10, 9), 16),
                                            ("checker", (11, 9, 7), 8), ("wide", (18, 10, 9), 16)])
def test_packed_vertices_match_oracle(kind, dims, rate):
    t = torch()
    f = make_field(kind, dims, 7)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = pkg().Volume(bits, dims, rate, bmin, bmax)
    try:
        isos = [0.0, float(np.median(d)), float(np.quantile(d, 0.3)), 1.0]
        if kind == "wide":
            isos += [1e37, -1.5e38, 2e38]
        for iso in isos:
            ref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
            T = ref["num_triangles"]
            out = t.zeros((max(T, 1), 3, 2), dtype=t.int32, device="cuda")
            st = vol.extract_packed_into(iso, out)
            assert st["num_triangles"] == T
            if T:
                want = oracle.quantized_vertices(ref["field"], iso, ref["edge_ids"], ref["tri_block"], dims)
                got = out.cpu().numpy().view(np.uint32)[:T]
                assert np.array_equal(got, want)
            # the float format of the same surface afterwards is unchanged
            m = vol.extract(iso)
            assert m.num_triangles == T
            m.release()
    finally:
        vol.release()


# ---------------------------------------------------------------- full-volume baselines

@pytest.mark.parametrize("rate", [2, 8, 16])
@pytest.mark.parametrize("kind,dims", DECODE_CASES + [("sphere", (1, 1, 1)), ("noise", (5, 3, 2)),
                                                   ("random", (16, 12, 8))])
def test_decode_volume_matches_oracle(kind, dims, rate):
    f = make_field(kind, dims, 9)
    bits, _, _ = oracle.encode_volume(f, rate)
    want = oracle.decode_volume(bits, dims, rate)
    got = pkg().decode_volume(to_dev(bits), dims, rate).cpu().numpy()
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


@pytest.mark.parametrize("kind,dims,rate", [("noise", (37, 21, 14), 8), ("sphere", (33, 2, 9), 8),
                                            ("random", (13, 9, 6), 4), ("checker", (11, 9, 7), 8)])
def test_all_blocks_baseline_equals_extraction(kind, dims, rate):
    t = torch()
    f = make_field(kind, dims, 7)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    a = pkg().Volume(bits, dims, rate, bmin, bmax)
    b = pkg().Volume(bits, dims, rate, bmin, bmax)
    nb = bits.shape[0]
    try:
        for iso in (0.0, float(np.median(d)), float(np.quantile(d, 0.8))):
            m = a.extract(iso)
            T = m.num_triangles
            out = t.zeros((max(T, 1), 3, 4), dtype=t.float32, device="cuda")
            st = b.extract_all_blocks_into(iso, out)
            assert st["num_triangles"] == T and st["n_active"] == nb and st["n_candidates"] == nb
            if T:
                assert np.array_equal(out.cpu().numpy().reshape(-1, 4).view(np.uint32),
                                      m.vertices.cpu().numpy().view(np.uint32))
            m.release()
    finally:
        a.release()
        b.release()


# ---------------------------------------------------------------- over budget: waves

def test_over_budget_extraction_in_waves():
    p = pkg()
    t = torch()
    dims, rate = (40, 36, 96), 8
    f = fields.gradient_noise(*dims, 6, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    nbx, nby, nbz = oracle.block_dims(dims)
    iso = float(np.median(d))
    act = oracle.active_blocks(bmin, bmax, (nbx, nby, nbz), iso).reshape(nbz, nby * nbx).sum(axis=1)
    budget = int(max(act[z] + (act[z + 1] if z + 1 < nbz else 0) for z in range(nbz))) + 5
    assert act.sum() > budget                                    # one pass cannot hold the surface
    small = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * budget)
    full = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        ref = full.extract(iso)
        T = ref.num_triangles
        want = ref.vertices.cpu().numpy().view(np.uint32)
        out = t.zeros((T, 3, 4), dtype=t.float32, device="cuda")
        st = small.extract_into(iso, out)
        assert st["waves"] > 1 and st["num_triangles"] == T and st["n_active"] == int(act.sum())
        assert np.array_equal(out.cpu().numpy().reshape(-1, 4).view(np.uint32), want)
        # the library-allocated path, twice (its first guess is the last size)
        for _ in range(2):
            m = small.extract(iso)
            assert m.stats["waves"] > 1
            assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), want)
            m.release()
        # the oracle agrees too (positions, blocks, count)
        oref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
        assert oref["num_triangles"] == T
        v = out.cpu().numpy()
        assert np.abs(v[:, :, :3].astype(np.float64) - oref["local_pos"]).max() < POS_TOL
        # too small for one layer and the next: refused
        tiny = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * 10)
        with pytest.raises(p.IsoError) as e:
            tiny.extract(iso)
        assert e.value.code == p.ISO_ERR_BUDGET
        tiny.release()
        ref.release()
    finally:
        small.release()
        full.release()


def test_launch_shapes_agree():
    # every launch shape of a single volume computes the same bytes
    p = pkg()
    dims, rate = (37, 33, 29), 8
    f = make_field("noise", dims, 12)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        start = vol.get_shape()
        assert start["scan_tile"] == 4096 and start["decode_tile"] == 128
        ref = vol.extract(0.1)
        want = ref.vertices.cpu().numpy().view(np.uint32)
        ref.release()
        for shape in (dict(), dict(cull_tile=2048, decode_tile=64, count_tile=16, scan_tile=1024, emit_tile=16),
                      dict(count_tile=64, emit_tile=64, scan_ctas=1, emit_ctas=1, decode_ctas=2)):
            vol.set_shape(**shape)
            for _ in range(4):                      # plain launches, later the captured graphs
                vol.cache_reset()
                m = vol.extract(0.1)
                assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), want)
                m.release()
        with pytest.raises(p.IsoError):
            vol.set_shape(count_tile=48)
    finally:
        vol.release()


def test_async_upload():
    # the bitstream's copy overlaps the first extraction's front; every entry
    # point sees the whole volume (extraction, ray casting, batches, servers,
    # release before any use)
    import torch as t
    p = pkg()
    dims, rate = (44, 38, 31), 8
    f = make_field("noise", dims, 14)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    hb = t.from_numpy(bits.view(np.int64)).pin_memory()
    hmin, hmax = t.from_numpy(bmin).pin_memory(), t.from_numpy(bmax).pin_memory()
    sync = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        ref = sync.extract(0.05)
        want = ref.vertices.cpu().numpy().view(np.uint32)
        ref.release()
        for first in ("extract", "extract_into", "batch", "server", "release"):
            v = p.Volume(hb, dims, rate, hmin, hmax, async_upload=True)
            try:
                if first == "extract":
                    m = v.extract(0.05)
                    assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), want)
                    m.release()
                elif first == "extract_into":
                    out = t.zeros((len(want) // 3 + 1, 3, 4), dtype=t.float32, device="cuda")
                    st = v.extract_into(0.05, out)
                    got = out.cpu().numpy().reshape(-1, 4)[:3 * st["num_triangles"]].view(np.uint32)
                    assert np.array_equal(got, want)
                elif first == "batch":
                    b = p.Batch([v])
                    verts, offs, _ = b.extract(np.array([0.05], np.float32))
                    assert int(offs[1]) * 3 == len(want)
                    assert np.array_equal(verts.cpu().numpy().reshape(-1, 4).view(np.uint32)[:len(want)], want)
                    b.release()
                elif first == "server":
                    srv = p.Server(v)
                    status, m = srv.wait(srv.submit(0.05), timeout_ms=10000)
                    assert status == p.ISO_OK
                    assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), want)
                    m.release()
                    srv.release()
            finally:
                v.release()
    finally:
        sync.release()


def test_async_loads_double_buffered():
    # volumes streamed as the benchmark's end-to-end run does: volume i + 1 is
    # loaded (its bitstream still copying) before volume i's surfaces, and
    # three volumes of different sizes and rates are alive at once
    import torch as t
    p = pkg()
    cases = [((44, 38, 31), 8, 21), ((29, 33, 40), 12, 22), ((37, 21, 14), 4, 23)]
    data = []
    for dims, rate, seed in cases:
        f = make_field("noise", dims, seed)
        bits, bmin, bmax = oracle.encode_volume(f, rate)
        want = oracle.extract(bits, dims, rate, bmin, bmax, 0.0)
        data.append((dims, rate, t.from_numpy(bits.view(np.int64)).pin_memory(), t.from_numpy(bmin).pin_memory(),
                     t.from_numpy(bmax).pin_memory(), want))
    vols = []
    try:
        nxt = p.Volume(data[0][2], data[0][0], data[0][1], data[0][3], data[0][4], async_upload=True)
        for i, (dims, rate, _, _, _, want) in enumerate(data):
            cur = nxt
            vols.append(cur)
            if i + 1 < len(data):
                d = data[i + 1]
                nxt = p.Volume(d[2], d[0], d[1], d[3], d[4], async_upload=True)
            for iso in (0.0, -0.3):
                m = cur.extract(iso)
                if iso == 0.0:
                    assert m.num_triangles == want["num_triangles"]
                    v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
                    assert np.abs(v[:, :, :3].astype(np.float64) - want["local_pos"]).max() < POS_TOL
                    assert np.array_equal(v[:, :, 3].view(np.uint32),
                                          np.repeat(want["tri_block"][:, None], 3, axis=1))
                m.release()
    finally:
        for v in vols:
            v.release()
