"""GPU parity of batched extraction: many volumes, each at its own isovalue,
through the same launches.

Each volume's surface from a batch must be bit-identical (vertex bytes and
order, counts, cache statistics) to extracting it alone, and both must
match the oracle (triangle count and block of every triangle exactly,
positions within 1e-5 voxel).  Every tile-size variant and launch shape
must give the same bytes, and the cache of every volume must follow
Algorithm 1 exactly as when extracted alone.
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
    if kind == "noise":
        return fields.gradient_noise(nx, ny, nz, seed + 1, octaves=4, base_period=16)
    if kind == "sphere":
        return fields.sphere_sdf(nx, ny, nz, 0.3 * min(dims))
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nz, ny, nx)).astype(np.float32)


# a mix of uneven sizes, ragged edges, tiny volumes and code rates
MIX = [("noise", (37, 21, 14), 8), ("sphere", (40, 36, 33), 12), ("random", (13, 9, 6), 4),
       ("noise", (64, 48, 40), 8), ("random", (1, 1, 1), 8), ("sphere", (33, 2, 9), 8),
       ("noise", (5, 3, 2), 2), ("random", (17, 30, 11), 16), ("noise", (24, 24, 24), 6)]


def load_mix(mix, seed=3, **kw):
    p = pkg()
    data, vols = [], []
    for i, (kind, dims, rate) in enumerate(mix):
        f = make_field(kind, dims, seed + i)
        bits, bmin, bmax = oracle.encode_volume(f, rate)
        d = oracle.decode_volume(bits, dims, rate)
        data.append((bits, dims, rate, bmin, bmax, d))
        vols.append(p.Volume(bits, dims, rate, bmin, bmax, **kw))
    return data, vols


def iso_rounds(data, n_rounds, seed):
    rng = np.random.default_rng(seed)
    rounds = []
    for r in range(n_rounds):
        isos = []
        for i, (_, _, _, _, _, d) in enumerate(data):
            lo, hi = np.quantile(d, [0.1, 0.9])
            x = float(rng.uniform(lo, hi)) if hi > lo else float(lo)
            if (r + i) % 7 == 3:
                x = float(d.max()) + 1.0          # empty surface
            isos.append(x)
        rounds.append(np.array(isos, np.float32))
    return rounds


def release(objs):
    for o in objs:
        o.release()


def test_batch_equals_alone_and_oracle():
    data, alone = load_mix(MIX)
    _, inbatch = load_mix(MIX)
    b = pkg().Batch(inbatch)
    cells = sum(int(np.prod(d[1])) for d in data)
    out = torch().empty((5 * cells + 16, 3, 4), dtype=torch().float32, device="cuda")   # <= 5 triangles a cell
    try:
        for isos in iso_rounds(data, 4, 11):
            r = b.extract_into(isos, out)
            offs, stats = r["offsets"], r["stats"]
            got = out.cpu().numpy().reshape(-1, 4)
            assert offs[0] == 0 and np.all(np.diff(offs.astype(np.int64)) >= 0)
            for i, vol in enumerate(alone):
                m = vol.extract(float(isos[i]))
                T = m.num_triangles
                assert offs[i + 1] - offs[i] == T
                mine = got[3 * int(offs[i]):3 * int(offs[i + 1])]
                if T:
                    assert np.array_equal(mine.view(np.uint32), m.vertices.cpu().numpy().view(np.uint32))
                for key in ("num_triangles", "n_active", "n_new", "n_occupied", "n_slots", "epoch", "n_candidates"):
                    assert stats[i][key] == m.stats[key], (i, key)
                m.release()
                bits, dims, rate, bmin, bmax, _ = data[i]
                ref = oracle.extract(bits, dims, rate, bmin, bmax, float(isos[i]))
                assert T == ref["num_triangles"]
                if T:
                    v = mine.reshape(-1, 3, 4)
                    assert np.abs(v[:, :, :3].astype(np.float64) - ref["local_pos"]).max() < POS_TOL
                    assert np.array_equal(v[:, :, 3].view(np.uint32),
                                          np.repeat(ref["tri_block"][:, None], 3, axis=1))
    finally:
        b.release()
        release(alone + inbatch)


def test_batch_cache_follows_algorithm1():
    mix = [("noise", (48, 40, 36), 8), ("noise", (30, 26, 22), 6), ("sphere", (44, 40, 38), 10)]
    data, vols = load_mix(mix, seed=5, initial_cache_fraction=0.02)
    caches = [oracle.LRUCache(bits.shape[0], int(np.ceil(0.02 * bits.shape[0])), bits.shape[0])
              for bits, *_ in data]
    b = pkg().Batch(vols)
    cells = sum(int(np.prod(d[1])) for d in data)
    out = torch().empty((5 * cells + 16, 3, 4), dtype=torch().float32, device="cuda")
    try:
        for isos in iso_rounds(data, 25, 17):
            stats = b.extract_into(isos, out)["stats"]
            for i, vol in enumerate(vols):
                bits, dims, rate, bmin, bmax, _ = data[i]
                act = oracle.active_blocks(bmin, bmax, oracle.block_dims(dims), float(isos[i]))
                I_new, _ = caches[i].update(act)
                assert np.array_equal(vol.debug("new_ids"), I_new.astype(np.uint32))
                assert stats[i]["n_slots"] == caches[i].num_slots
                assert np.array_equal(vol.debug("slot_of_block"), caches[i].I_slot.astype(np.int32))
                assert np.array_equal(vol.debug("block_of_slot"), caches[i].S_block.astype(np.int32))
                assert np.array_equal(vol.debug("slot_last_use"), caches[i].last_use().astype(np.uint32))
    finally:
        b.release()
        release(vols)


SHAPES = [dict(cull_tile=2048, decode_tile=64, count_tile=16, scan_tile=1024, emit_tile=16),
          dict(cull_tile=4096, decode_tile=256, count_tile=64, scan_tile=4096, emit_tile=64),
          dict(cull_tile=2048, decode_tile=128, count_tile=32, scan_tile=2048, emit_tile=32,
               cull_ctas=1, cache_update_ctas=1, decode_ctas=1, count_ctas=1, scan_ctas=1, emit_ctas=1),
          dict(decode_tile=256, count_tile=16, emit_tile=64, scan_tile=1024, count_ctas=2, emit_ctas=1)]


def test_batch_tile_variants_give_identical_bytes():
    data, vols = load_mix(MIX, seed=8)
    b = pkg().Batch(vols)
    isos = iso_rounds(data, 1, 23)[0]
    try:
        want, woffs, _ = b.extract(isos)
        want = want.cpu().numpy()
        for shape in SHAPES:
            for v in vols:
                v.cache_reset()
            b.set_shape(**shape)
            got_shape = b.shape
            for k, x in shape.items():
                if k.endswith("_tile"):
                    assert got_shape[k] == x
                else:
                    assert 1 <= got_shape[k] <= max(x, 1) or x == 0
            for rep in range(2):                       # cold, then warm
                got, offs, _ = b.extract(isos)
                assert np.array_equal(offs, woffs)
                assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
    finally:
        b.release()
        release(vols)


def test_batch_capacity_and_retry():
    p = pkg()
    t = torch()
    data, vols = load_mix(MIX[:4], seed=9)
    b = p.Batch(vols)
    isos = np.array([float(np.median(d[5])) for d in data], np.float32)
    try:
        full, offs, _ = b.extract(isos)
        total = int(offs[-1])
        assert total > 200
        small = t.zeros((100, 3, 4), dtype=t.float32, device="cuda")
        with pytest.raises(p.IsoError) as e:
            b.extract_into(isos, small)
        assert e.value.code == p.ISO_ERR_CAPACITY
        r = b.extract_into(isos, small, check=False)
        assert np.array_equal(r["offsets"], offs)
        assert np.array_equal(small.cpu().numpy().reshape(-1, 4).view(np.uint32),
                              full.cpu().numpy()[:300].view(np.uint32))
        assert all(st["n_new"] == 0 for st in r["stats"])   # warm caches
    finally:
        b.release()
        release(vols)


def test_batch_budget_failure_is_per_volume():
    p = pkg()
    data, vols = load_mix(MIX[:3], seed=10)
    bits, dims, rate, bmin, bmax, d = data[0]
    tight = p.Volume(bits, dims, rate, bmin, bmax, cache_budget_bytes=10 * 256)
    b = p.Batch([tight] + vols[1:])
    isos = np.array([float(np.median(x[5])) for x in data], np.float32)
    try:
        out = torch().zeros((200000, 3, 4), dtype=torch().float32, device="cuda")
        r = b.extract_into(isos, out, check=False)
        assert r["rc"] == p.ISO_ERR_BUDGET
        assert r["status"][0] == p.ISO_ERR_BUDGET and r["status"][1:] == [p.ISO_OK] * 2
        assert r["offsets"][1] == 0                    # the failed volume emits nothing
        for i in (1, 2):
            bits_i, dims_i, rate_i, bmin_i, bmax_i, _ = data[i]
            ref = oracle.extract(bits_i, dims_i, rate_i, bmin_i, bmax_i, float(isos[i]))
            assert r["offsets"][i + 1] - r["offsets"][i] == ref["num_triangles"]
    finally:
        b.release()
        release(vols + [tight])


def test_batch_invalid_arguments():
    p = pkg()
    data, vols = load_mix(MIX[:2], seed=12)
    bits, dims, rate, bmin, bmax, _ = data[0]
    dbg = p.Volume(bits, dims, rate, bmin, bmax, debug=True)
    try:
        for bad in ([vols[0], vols[0]], [vols[0], dbg], []):
            with pytest.raises(p.IsoError) as e:
                p.Batch(bad)
            assert e.value.code == p.ISO_ERR_INVALID_ARG
        b = p.Batch(vols)
        with pytest.raises(p.IsoError):
            b.extract(np.array([0.0, np.nan], np.float32))
        with pytest.raises(p.IsoError):
            b.set_shape(scan_tile=3000)
        with pytest.raises(ValueError):
            b.extract(np.zeros(3, np.float32))
        b.release()
    finally:
        release(vols + [dbg])


def test_batch_autotune_keeps_results():
    data, vols = load_mix(MIX, seed=13)
    b = pkg().Batch(vols)
    isos = iso_rounds(data, 1, 29)[0]
    try:
        want, woffs, _ = b.extract(isos)
        want = want.cpu().numpy()
        out = torch().empty((int(woffs[-1]) + 16, 3, 4), dtype=torch().float32, device="cuda")
        res = b.tune(isos, out, trials=1)
        sh = res["shape"]
        assert sh["cull_tile"] in (2048, 4096) and sh["decode_tile"] in (64, 128, 256)
        assert sh["count_tile"] in (16, 32, 64) and sh["emit_tile"] in (16, 32, 64)
        assert sh["scan_tile"] in (1024, 2048, 4096)
        assert 0 < res["tuned_ms"] <= res["default_ms"]
        got, offs, stats = b.extract(isos)             # caches were left empty: all new again
        assert np.array_equal(offs, woffs)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
        assert all(st["n_new"] == st["n_active"] for st in stats)
    finally:
        b.release()
        release(vols)


def test_batch64_workload_equals_alone():
    """The 64-volume workload (sizes log-uniform in [32, 256]) generated and
    encoded on the GPU, extracted as one batch in the configuration the
    benchmark times; every surface equals its volume extracted alone, and
    the smallest volumes are checked against the oracle in full."""
    import synth.gpu as sg
    from synth import recipes
    p = pkg()
    t = torch()
    sg.build()
    recs = recipes.batch64_recipes()
    alone, inbatch, isos, host = [], [], [], []
    order = np.argsort([np.prod(r.dims) for r in recs])
    small = set(order[:4].tolist())
    try:
        for i, r in enumerate(recs):
            f = sg.generate(r)
            bits, bmin, bmax = p.encode_field(f, r.rate)
            t.cuda.synchronize()
            alone.append(p.Volume(bits, r.dims, r.rate, bmin, bmax))
            inbatch.append(p.Volume(bits, r.dims, r.rate, bmin, bmax))
            isos.append(r.isovalues[0])
            if i in small:
                host.append((i, bits.cpu().numpy().view(np.uint64), bmin.cpu().numpy(), bmax.cpu().numpy()))
            del f
        b = p.Batch(inbatch)
        isos = np.array(isos, np.float32)
        for rep in range(2):                                  # cold, then warm
            verts, offs, _ = b.extract(isos)
            got = verts.cpu().numpy()
            assert int(offs[-1]) > 0
            for i, vol in enumerate(alone):
                m = vol.extract(float(isos[i]))
                assert offs[i + 1] - offs[i] == m.num_triangles
                if m.num_triangles:
                    assert np.array_equal(got[3 * int(offs[i]):3 * int(offs[i + 1])].view(np.uint32),
                                          m.vertices.cpu().numpy().view(np.uint32))
                m.release()
        for i, bits, bmin, bmax in host:
            r = recs[i]
            ref = oracle.extract(bits, r.dims, r.rate, bmin, bmax, float(isos[i]))
            mine = got[3 * int(offs[i]):3 * int(offs[i + 1])].reshape(-1, 3, 4)
            assert len(mine) == ref["num_triangles"]
            if len(mine):
                assert np.abs(mine[:, :, :3].astype(np.float64) - ref["local_pos"]).max() < POS_TOL
                assert np.array_equal(mine[:, :, 3].view(np.uint32), np.repeat(ref["tri_block"][:, None], 3, 1))
        b.release()
    finally:
        release(alone + inbatch)
