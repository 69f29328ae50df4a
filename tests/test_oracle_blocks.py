"""Pins for the oracle's block rules and cache simulator (CPU only).

Section 4.1 marks a block active when its range, or its range joined with a
neighbour's, contains the isovalue; Sections 4.3-4.5 run marching cubes
block by block over the active blocks.  The block method must give exactly
the triangles of plain marching cubes over the decoded field, so the block
oracle is checked against the full-volume oracle, and the active set
against brute force over crossing cells.  The cache simulator of Algorithm
1 is checked against what an LRU cache must do.
"""
import numpy as np
import pytest

import oracle
from synth import fields


def canon(tri):
    """rotate each edge-id triple so its smallest id comes first (keeps orientation)"""
    t = np.asarray(tri, np.uint64)
    r = np.argmin(t, axis=1)
    idx = (r[:, None] + np.arange(3)[None, :]) % 3
    return np.take_along_axis(t, idx, axis=1)


def _volume(kind, dims, seed):
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.standard_normal((nz, ny, nx)).astype(np.float32)
    if kind == "noise":
        return fields.gradient_noise(nx, ny, nz, seed, octaves=4, base_period=16)
    return fields.sphere_sdf(nx, ny, nz, 0.3 * min(dims))


def _owner_and_cell(cells, dims):
    """owner block id and block-local cell index of each triangle's cell"""
    nx, ny, nz = dims
    cx, cy, cz = cells % nx, cells // nx % ny, cells // nx // ny
    nbx, nby = (nx + 3) // 4, (ny + 3) // 4
    owner = cx // 4 + nbx * (cy // 4 + nby * (cz // 4))
    cell = cx % 4 + 4 * (cy % 4) + 16 * (cz % 4)
    return owner, cell


CASES = [("random", (13, 9, 6)), ("random", (5, 5, 5)), ("noise", (33, 20, 17)), ("sphere", (24, 24, 24)),
         ("random", (2, 3, 5)), ("noise", (4, 4, 4)), ("random", (3, 2, 2)), ("sphere", (33, 2, 9))]


@pytest.mark.parametrize("kind,dims", CASES)
@pytest.mark.parametrize("rate", [4, 12])
def test_block_path_equals_full_mc(kind, dims, rate):
    f = _volume(kind, dims, 11)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d = oracle.decode_volume(bits, dims, rate)
    for iso in (float(np.median(d)), float(d.min()), float(np.quantile(d, 0.3)), 0.0):
        ids_full, pos_full, cells = oracle.mc_full(d, iso, return_cells=True)
        r = oracle.extract(bits, dims, rate, bmin, bmax, iso)
        assert r["num_triangles"] == len(ids_full)
        # same triangles; block order = stable sort of the plain order by (owner block, cell)
        owner, cell = _owner_and_cell(cells, dims)
        order = np.lexsort((cell, owner))
        assert np.array_equal(canon(r["edge_ids"]), canon(ids_full[order]))
        assert np.array_equal(r["edge_ids"], ids_full[order])
        assert np.array_equal(r["tri_block"], owner[order].astype(np.uint32))
        nbx, nby = (dims[0] + 3) // 4, (dims[1] + 3) // 4
        b = r["tri_block"].astype(np.int64)
        origin = np.stack([b % nbx, b // nbx % nby, b // nbx // nby], axis=1) * 4.0
        assert np.abs(r["local_pos"] + origin[:, None, :] - pos_full[order]).max(initial=0) < 1e-9
        # occupied blocks are exactly the owners of triangles
        occ = set(r["ids"][r["block_tri"] > 0].tolist())
        assert occ == set(owner.tolist())
        # offsets: sequential exclusive sum of the block counts
        run = 0
        for i, c in enumerate(r["block_tri"]):
            assert int(r["block_off"][i]) == run
            run += int(c)
        # counts per cell agree with the table, blocks with a reset emit nothing
        num, _, _ = oracle.mc_table()
        assert np.array_equal(num[r["cases"]], r["counts"])
        assert (r["block_tri"][~r["complete"]] == 0).all()


@pytest.mark.parametrize("kind,dims", CASES)
def test_active_covers_crossing_cells(kind, dims):
    f = _volume(kind, dims, 3)
    bits, bmin, bmax = oracle.encode_volume(f, 8)
    d = oracle.decode_volume(bits, dims, 8)
    nx, ny, nz = dims
    nbd = ((nx + 3) // 4, (ny + 3) // 4, (nz + 3) // 4)
    for iso in np.quantile(d, [0.1, 0.5, 0.9]):
        iso = float(iso)
        act = oracle.active_blocks(bmin, bmax, nbd, iso)
        need = np.zeros_like(act)
        below = d < iso
        for z in range(nz - 1):
            for y in range(ny - 1):
                for x in range(nx - 1):
                    c = below[z:z + 2, y:y + 2, x:x + 2]
                    if c.any() and not c.all():
                        for k in (0, 1):
                            for j in (0, 1):
                                for i in (0, 1):
                                    need[(x + i) // 4 + nbd[0] * ((y + j) // 4 + nbd[1] * ((z + k) // 4))] = True
        assert not (need & ~act).any()


def test_active_rule_literal_small():
    # 3 blocks in a row with ranges [0,1], [2,3], [5,6]: iso 4 is in no range;
    # the union of block 1 and block 2 is [2,6] -> both active; block 0's
    # unions reach [0,3] only -> inactive
    bmin = np.array([0, 2, 5], np.float32)
    bmax = np.array([1, 3, 6], np.float32)
    act = oracle.active_blocks(bmin, bmax, (3, 1, 1), 4.0)
    assert list(act) == [False, True, True]
    # "contains" is lo < iso <= hi
    assert list(oracle.active_blocks(np.array([1], np.float32), np.array([2], np.float32), (1, 1, 1), 1.0)) == [False]
    assert list(oracle.active_blocks(np.array([1], np.float32), np.array([2], np.float32), (1, 1, 1), 2.0)) == [True]


def test_all_above_and_all_below():
    f = fields.sphere_sdf(16, 16, 16, 5.0)
    bits, bmin, bmax = oracle.encode_volume(f, 8)
    for iso in (-1000.0, 1000.0):
        r = oracle.extract(bits, (16, 16, 16), 8, bmin, bmax, iso)
        assert r["num_triangles"] == 0 and not r["active"].any()


# ---------------------------------------------------------------- cache simulator

def _requests(kind, n_blocks, rng, count):
    out = []
    if kind == "random":
        for _ in range(count):
            m = np.zeros(n_blocks, bool)
            m[rng.choice(n_blocks, rng.integers(0, n_blocks // 3), replace=False)] = True
            out.append(m)
    else:
        centre = 0 if kind == "up" else n_blocks
        step = 3 if kind == "up" else -3
        for _ in range(count):
            m = np.zeros(n_blocks, bool)
            lo = max(0, centre - 20)
            m[lo:min(n_blocks, centre + 20)] = True
            out.append(m)
            centre += step
    return out


@pytest.mark.parametrize("kind", ["random", "up", "down"])
def test_lru_simulator_invariants(kind):
    rng = np.random.default_rng(7)
    nb = 400
    cache = oracle.LRUCache(nb, initial_slots=40, max_slots=nb)
    for m in _requests(kind, nb, rng, 200):
        last = cache.last_use().copy()
        S_before = cache.num_slots
        was_cached = cache.I_slot >= 0
        old_block = cache.S_block.copy()
        I_new, slots = cache.update(m)
        # every active block is cached, the maps are mutual inverses
        assert (cache.I_slot[m] >= 0).all()
        cached = np.nonzero(cache.I_slot >= 0)[0]
        assert np.array_equal(cache.S_block[cache.I_slot[cached]], cached)
        assert (np.sort(cache.S_block[cache.S_block >= 0]) == cached).all()
        # the new blocks are the active, previously uncached ones, ascending
        assert np.array_equal(I_new, np.nonzero(m & ~was_cached)[0])
        # evicted blocks are never active
        ev = old_block[slots[slots < S_before]]
        assert not m[ev[ev >= 0]].any()
        # LRU choice: the slots taken are the least recently used ones that
        # the request does not hold (ties by slot index; grown slots count as
        # never used)
        if len(I_new):
            held = set(cache.I_slot[m & was_cached].tolist())
            lu = np.concatenate([last, np.zeros(cache.num_slots - S_before, np.int64)])
            free = [s for s in range(cache.num_slots) if s not in held]
            want = sorted(free, key=lambda s: (lu[s], s))[:len(I_new)]
            assert list(slots) == want
        # the slot count only grows when the free slots run out
        if cache.num_slots > S_before:
            assert len(I_new) > S_before - int((m & was_cached).sum())


def test_lru_repeat_is_all_hits_and_budget():
    nb = 100
    m = np.zeros(nb, bool)
    m[10:50] = True
    c = oracle.LRUCache(nb, 10, 100)
    I_new, _ = c.update(m)
    assert len(I_new) == 40 and c.num_slots == 40          # max(2*10, 10 + 40 - 10)
    I_new, _ = c.update(m)
    assert len(I_new) == 0
    small = oracle.LRUCache(nb, 10, 30)
    with pytest.raises(oracle.OverBudget):
        small.update(m)


# ---------------------------------------------------------------- compact vertices (Section 4.5)

def test_quantized_vertices_within_half_a_step():
    from synth import fields
    dims = (21, 17, 13)
    f = fields.gradient_noise(*dims, 4, octaves=3, base_period=8)
    bits, bmin, bmax = oracle.encode_volume(f, 8)
    for iso in (-0.3, 0.0, 0.45):
        r = oracle.extract(bits, dims, 8, bmin, bmax, iso)
        q = oracle.quantized_vertices(r["field"], iso, r["edge_ids"], r["tri_block"], dims)
        assert q.shape == (r["num_triangles"], 3, 2)
        codes = q[..., 0]
        assert (codes >> 30 == 0).all()
        dec = np.stack([(codes >> (10 * k)) & 1023 for k in range(3)], -1) / 255.75
        # rounding to the nearest code, from a float32 position within ~5e-7 of the float64 one
        assert np.abs(dec - r["local_pos"]).max() <= 0.5 / 255.75 + 1e-6
        assert np.array_equal(q[..., 1], np.repeat(r["tri_block"][:, None], 3, axis=1).astype(np.uint32))


def test_quantized_vertices_hand_values():
    # samples 0 and 1 with iso 0.5: every vertex is at the middle of its edge,
    # t = 0.5 exactly, so a coordinate k + 0.5 has code round(255.75 * (k + 0.5))
    # = 128, 384, 639, 895 for k = 0..3 (127.875, 383.625, 639.375, 895.125)
    dims = (8, 8, 8)
    rng = np.random.default_rng(2)
    f = rng.integers(0, 2, (8, 8, 8)).astype(np.float32)
    ids, pos = oracle.mc_full(f, 0.5)
    owner = np.zeros(len(ids), np.int64)
    # owner block of each triangle: the block of its cell (any vertex's lower corner floor / 4 works
    # only inside a block, so take it from the edge of the first vertex's cell via the positions)
    cell = np.floor(pos.min(axis=1)).astype(np.int64)          # lower cell corner of each triangle
    bx, by, bz = cell[:, 0] // 4, cell[:, 1] // 4, cell[:, 2] // 4
    owner = bx + 2 * (by + 2 * bz)
    q = oracle.quantized_vertices(f, 0.5, ids, owner, dims)
    table = {0.5: 128, 1.5: 384, 2.5: 639, 3.5: 895, 0.0: 0, 1.0: 256, 2.0: 512, 3.0: 767, 4.0: 1023}
    local = pos - 4 * np.stack([bx, by, bz], -1)[:, None, :]
    want = np.vectorize(lambda v: table[v])(local).astype(np.uint32)
    got = np.stack([(q[..., 0] >> (10 * k)) & 1023 for k in range(3)], -1)
    assert np.array_equal(got, want)
