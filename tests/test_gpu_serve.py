"""GPU parity of the serving path: requests answered in ticks on one
resident volume (one shared cull and cache update per tick, then one
batched count, scan and emit over the tick's requests; the next tick's
cull, cache update and decode overlapping the running tick's emission) must
give meshes identical, byte for byte, to extracting each isovalue alone;
admission splits ticks whose union of active blocks exceeds the cache
budget, defers meshes past the vertex budget, and a single request over
budget fails alone."""
import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def pkg():
    import paper_2009_03254_gb300 as p
    return p


def volume_pair(dims=(48, 40, 36), rate=8, seed=3, **kw):
    f = fields.gradient_noise(*dims, seed, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    p = pkg()
    return (bits, dims, rate, bmin, bmax, d), p.Volume(bits, dims, rate, bmin, bmax, **kw), \
        p.Volume(bits, dims, rate, bmin, bmax)


def same_mesh(m, ref):
    assert m.num_triangles == ref.num_triangles
    if m.num_triangles:
        assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), ref.vertices.cpu().numpy().view(np.uint32))


def drain(srv):
    while srv.queued():
        srv.step()


# room for the stored cell cases: the default (every request's), "one"
# (the largest request's candidates: the first requests of a tick only, and
# less than a full candidate list, so one-request ticks take the launch
# table), and none
CASE_ROOM = ["default", "one", "none"]


def case_bytes_for(room, alone, isos):
    if room == "default":
        return 0
    if room == "none":
        return 1
    most = 0
    for x in isos:
        m = alone.extract(float(x))
        most = max(most, m.stats["n_candidates"])
        m.release()
    return 64 * (most + 1)


@pytest.mark.parametrize("room", CASE_ROOM)
def test_served_meshes_equal_alone(room):
    # A step runs one tick: its requests' count, scan and emission as batched
    # launches; when at least two requests wait as that tick's emission is
    # queued they are admitted as the next tick, whose cull, cache update and
    # decode run on a second stream during this tick's emission, with this
    # tick's blocks pinned.  Every mesh must equal extracting its isovalue alone, whether
    # its tick ran alone or overlapped another, and whether its cases were
    # stored by the count pass or classified again by the emission.
    p = pkg()
    data, vol, alone = volume_pair()
    d = data[5]
    rng = np.random.default_rng(4)
    isos = list(rng.uniform(*np.quantile(d, [0.1, 0.9]), 13).astype(np.float32))
    isos += [isos[2], float(d.max()) + 1.0, float(d.min()) - 1.0]     # a repeat, two empty surfaces
    srv = p.Server(vol, max_batch=4, case_bytes=case_bytes_for(room, alone, isos))
    try:
        tickets = [srv.submit(float(x)) for x in isos[:6]]
        assert srv.step() == 4                                # the first tick, admitted at once
        assert srv.queued() == 2                              # the next tick's front is already queued
        tickets += [srv.submit(float(x)) for x in isos[6:]]   # arrivals while it runs
        finished = [4]
        while srv.queued():
            finished.append(srv.step())
        assert sum(finished) == len(isos) and max(finished) <= 4
        for t, x in zip(tickets, isos):
            status, m = srv.take(t)
            assert status == p.ISO_OK
            ref = alone.extract(float(x))
            same_mesh(m, ref)
            assert m.stats["n_candidates"] == ref.stats["n_candidates"]
            assert m.stats["n_occupied"] == ref.stats["n_occupied"]
            m.release()
            ref.release()
            with pytest.raises(p.IsoError):
                srv.take(t)                                   # already taken
    finally:
        srv.release()
        vol.release()
        alone.release()


@pytest.mark.parametrize("room", CASE_ROOM)
def test_one_request_ticks_equal_alone(room):
    # one request a tick: its view travels by value, or through the launch
    # table when a full candidate list does not fit the stored-cases room
    # (a smooth field: about 70% of the blocks active)
    p = pkg()
    dims, rate = (64, 48, 40), 8
    f = fields.gradient_noise(*dims, 5, octaves=3, base_period=48)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    alone = p.Volume(bits, dims, rate, bmin, bmax)
    isos = [float(x) for x in np.quantile(d, [0.3, 0.5, 0.7, 0.5])]
    case_bytes = case_bytes_for(room, alone, isos)
    assert room != "one" or case_bytes < 64 * int(np.prod(oracle.block_dims(dims)))
    srv = p.Server(vol, max_batch=1, case_bytes=case_bytes)
    try:
        tickets = [srv.submit(x) for x in isos]
        done = []
        while srv.queued():
            done.append(srv.step())
        assert sum(done) == len(isos) and max(done) == 1
        for t, x in zip(tickets, isos):
            status, m = srv.take(t)
            assert status == p.ISO_OK
            ref = alone.extract(x)
            same_mesh(m, ref)
            assert m.stats["n_candidates"] == ref.stats["n_candidates"]
            m.release()
            ref.release()
    finally:
        srv.release()
        vol.release()
        alone.release()


def test_overlapped_ticks_keep_the_running_ticks_blocks():
    # a cache too small for two distant isovalues' blocks at once: the second
    # tick's front, pinned to the first tick's blocks, cannot fit and waits
    # until the first tick is done (then runs unpinned); the meshes are
    # unaffected
    p = pkg()
    dims, rate = (48, 40, 36), 8
    f = fields.gradient_noise(*dims, 7, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    nbd = oracle.block_dims(dims)
    lo, hi = (float(x) for x in np.quantile(d, [0.2, 0.8]))
    a1 = oracle.active_blocks(bmin, bmax, nbd, lo)
    a2 = oracle.active_blocks(bmin, bmax, nbd, hi)
    budget = int(max(a1.sum(), a2.sum()))
    assert (a1 | a2).sum() > budget
    vol = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * budget, initial_cache_fraction=1.0)
    alone = p.Volume(bits, dims, rate, bmin, bmax)
    srv = p.Server(vol, max_batch=1)
    try:
        t1, t2, t3 = srv.submit(lo), srv.submit(hi), srv.submit(lo)
        done = []
        while srv.queued():
            done.append(srv.step())
        assert sum(done) == 3                                 # refused pinned fronts were retried
        for t, x in ((t1, lo), (t2, hi), (t3, lo)):
            status, m = srv.take(t)
            assert status == p.ISO_OK
            ref = alone.extract(x)
            same_mesh(m, ref)
            m.release()
            ref.release()
    finally:
        srv.release()
        vol.release()
        alone.release()


def test_union_over_budget_splits_the_tick():
    p = pkg()
    dims, rate = (48, 40, 36), 8
    f = fields.gradient_noise(*dims, 7, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    nbd = oracle.block_dims(dims)
    lo, hi = np.quantile(d, [0.25, 0.75])
    a1 = oracle.active_blocks(bmin, bmax, nbd, float(lo))
    a2 = oracle.active_blocks(bmin, bmax, nbd, float(hi))
    budget = int(max(a1.sum(), a2.sum()))
    assert (a1 | a2).sum() > budget                           # together they do not fit
    vol = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * budget, initial_cache_fraction=1.0)
    alone = p.Volume(bits, dims, rate, bmin, bmax)
    srv = p.Server(vol, max_batch=2)
    try:
        t1, t2 = srv.submit(float(lo)), srv.submit(float(hi))
        assert srv.step() == 1                                # the union was refused: one at a time
        drain(srv)
        for t, x in ((t1, lo), (t2, hi)):
            status, m = srv.take(t)
            assert status == p.ISO_OK
            ref = alone.extract(float(x))
            same_mesh(m, ref)
            m.release()
            ref.release()
        # one request that alone exceeds the budget fails by itself
        small = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=256 * 10)
        s2 = p.Server(small, max_batch=2)
        t = s2.submit(float(np.median(d)))
        s2.step()
        status, m = s2.take(t)
        assert status == p.ISO_ERR_BUDGET and m is None
        s2.release()
        small.release()
    finally:
        srv.release()
        vol.release()
        alone.release()


def test_vertex_budget_defers_until_meshes_are_taken():
    p = pkg()
    data, vol, alone = volume_pair(seed=5)
    d = data[5]
    isos = [float(x) for x in np.quantile(d, [0.3, 0.5, 0.7])]
    ref = [alone.extract(x) for x in isos]
    budget = 48 * max(r.num_triangles for r in ref) + 48      # room for about one mesh
    srv = p.Server(vol, max_batch=4, vertex_budget_bytes=budget)
    try:
        tickets = [srv.submit(x) for x in isos]
        assert srv.step() == 1                                # the first fits (nothing held)
        assert srv.queued() == 2                              # the other two wait in the tick, counted
        assert srv.step() == 0                                # the held mesh blocks the rest
        assert srv.step() == 0                                # (returning at once each time)
        st0, m0 = srv.take(tickets[0])
        assert st0 == p.ISO_OK
        same_mesh(m0, ref[0])
        m0.release()
        for i in (1, 2):
            assert srv.take(tickets[i])[0] == p.ISO_PENDING
            assert srv.step() == 1
            st, m = srv.take(tickets[i])
            assert st == p.ISO_OK
            same_mesh(m, ref[i])
            m.release()
    finally:
        for r in ref:
            r.release()
        srv.release()
        vol.release()
        alone.release()


def test_server_invalid_arguments():
    p = pkg()
    data, vol, alone = volume_pair(dims=(20, 20, 20))
    bits, dims, rate, bmin, bmax, _ = data
    dbg = p.Volume(bits, dims, rate, bmin, bmax, debug=True)
    try:
        for kw, v in ((dict(), dbg), (dict(max_batch=9), vol)):
            with pytest.raises(p.IsoError) as e:
                p.Server(v, **kw)
            assert e.value.code == p.ISO_ERR_INVALID_ARG
        srv = p.Server(vol)
        with pytest.raises(p.IsoError):
            srv.submit(float("nan"))
        with pytest.raises(p.IsoError):
            srv.take(12345)
        t = srv.submit(0.0)
        assert srv.take(t) == (p.ISO_PENDING, None)
        srv.step()
        st, m = srv.take(t)
        assert st == p.ISO_OK
        m.release()
        srv.release()
    finally:
        dbg.release()
        vol.release()
        alone.release()


def test_request_loop_against_plain_path():
    from paper_2009_03254_gb300 import serving
    p = pkg()
    data, vol, alone = volume_pair(dims=(64, 64, 48), seed=9)
    d = data[5]
    lo, hi = np.quantile(d, [0.05, 0.95])
    n = 60
    isos = serving.random_walk_isovalues(n, float(lo), float(hi), 5)
    arrivals = serving.poisson_arrivals(n, 2000.0, 1)
    srv = p.Server(vol, max_batch=8)
    try:
        res = serving.RequestLoop(srv, keep_meshes=True).run(arrivals, isos)
        plain = serving.RequestLoop(serving.PlainBackend(alone), keep_meshes=True).run(arrivals, isos)
        for a, b in zip(res, plain):
            assert a["status"] == b["status"] == p.ISO_OK
            same_mesh(a["mesh"], b["mesh"])
            a["mesh"].release()
            b["mesh"].release()
        assert serving.latency_summary(res)["served"] == n
    finally:
        srv.release()
        vol.release()
        alone.release()


def test_compact_vertices_served():
    # the compact 8-byte format: the same codes as extracting it alone, half
    # the bytes against the vertex budget
    import torch
    p = pkg()
    data, vol, alone = volume_pair(seed=11)
    d = data[5]
    isos = [float(x) for x in np.quantile(d, [0.3, 0.5, 0.7])]
    srv = p.Server(vol, max_batch=4, packed=True)
    try:
        tickets = [srv.submit(x) for x in isos]
        while srv.queued():
            srv.step()
        for t, x in zip(tickets, isos):
            status, m = srv.take(t)
            assert status == p.ISO_OK and m.packed
            T = m.num_triangles
            want = torch.zeros((max(T, 1), 3, 2), dtype=torch.int32, device="cuda")
            st = alone.extract_packed_into(x, want)
            assert st["num_triangles"] == T
            assert np.array_equal(m.vertices.cpu().numpy().reshape(-1, 3, 2), want.cpu().numpy()[:T])
            m.release()
    finally:
        srv.release()
        vol.release()
        alone.release()
    # a vertex format that is neither is refused
    import ctypes
    data2, v2, a2 = volume_pair(dims=(20, 20, 20))
    try:
        bad = p._ServerOptions()
        bad.vertex_format = 7
        h = ctypes.c_void_p()
        assert p.lib().iso_server_create(ctypes.byref(h), v2._h, ctypes.byref(bad)) == p.ISO_ERR_INVALID_ARG
    finally:
        v2.release()
        a2.release()
