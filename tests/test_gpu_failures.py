"""Failure paths, driven without faulting or hanging the GPU.

* A device-side wait that runs out: the test hook ISO_TEST_WITHHOLD_PREFIX
  keeps the range test's first tile from publishing its prefix sums, so
  every later tile's bounded look-back wait (the decoupled look-back of the
  compaction, Section 4.1) gives up after a short limit.  The extraction
  must return ISO_ERR_TIMEOUT, and the volume must extract correctly again
  once the hook is off (plain launches and the captured graph alike).
* An allocation that fails: an allocator hook that refuses every request
  must turn into ISO_ERR_OOM from the load, from an extraction (its mesh)
  and from creating a server, and leave the library usable.
* Memory the library's pool keeps after a release goes back to the device
  with iso_release_cached_memory.
"""
import ctypes

import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _noise(dims, rate=8, seed=23):
    f = fields.gradient_noise(*dims, seed, octaves=4, base_period=32)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    return bits, bmin, bmax


def _check_against_oracle(pkg, vol, bits, dims, rate, bmin, bmax, iso):
    mesh = vol.extract(iso)
    ref = oracle.extract(bits, dims, rate, bmin, bmax, iso)
    try:
        assert mesh.num_triangles == ref["num_triangles"] > 0
        v = mesh.vertices.cpu().numpy().reshape(-1, 3, 4)
        assert np.array_equal(v[:, 0, 3].view(np.uint32), ref["tri_block"].astype(np.uint32))
        assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < 1e-5
    finally:
        mesh.release()


@pytest.mark.parametrize("graph", [False, True])
def test_wait_timeout_is_reported_and_the_volume_stays_usable(graph):
    import paper_2009_03254_gb300 as pkg

    dims, rate = (96, 88, 48), 8                 # 24 x 22 x 12 = 6336 blocks: two range-test tiles
    bits, bmin, bmax = _noise(dims, rate)
    vol = pkg.Volume(bits, dims, rate, bmin, bmax)
    try:
        if graph:                                # past the point where the extraction is a CUDA graph
            for _ in range(10):
                vol.extract(0.1).release()
        _check_against_oracle(pkg, vol, bits, dims, rate, bmin, bmax, 0.0)
        vol.set_test_fault(pkg.ISO_TEST_WITHHOLD_PREFIX)
        for iso in (0.0, 0.3):
            with pytest.raises(pkg.IsoError) as e:
                vol.extract(iso)
            assert e.value.code == pkg.ISO_ERR_TIMEOUT
        vol.set_test_fault(0)
        for iso in (0.0, 0.3):                   # the cache was emptied; everything is decoded again
            _check_against_oracle(pkg, vol, bits, dims, rate, bmin, bmax, iso)
        with pytest.raises(pkg.IsoError) as e:
            vol.set_test_fault(2)
        assert e.value.code == pkg.ISO_ERR_INVALID_ARG
    finally:
        vol.release()


def test_refused_allocations_are_reported_as_oom():
    import paper_2009_03254_gb300 as pkg

    dims, rate = (40, 36, 28), 8
    bits, bmin, bmax = _noise(dims, rate)
    vol = pkg.Volume(bits, dims, rate, bmin, bmax)
    refuse = pkg._ALLOC_FN(lambda nbytes, device, stream, ctx: None)
    never = pkg._FREE_FN(lambda ptr, device, stream, ctx: None)
    try:
        pkg._check(pkg.lib().iso_set_allocator(ctypes.cast(refuse, ctypes.c_void_p),
                                               ctypes.cast(never, ctypes.c_void_p), None), "iso_set_allocator")
        with pytest.raises(pkg.IsoError) as e:   # the load
            pkg.Volume(bits, dims, rate, bmin, bmax)
        assert e.value.code == pkg.ISO_ERR_OOM
        with pytest.raises(pkg.IsoError) as e:   # an extraction's mesh
            vol.extract(0.0)
        assert e.value.code == pkg.ISO_ERR_OOM
        with pytest.raises(pkg.IsoError) as e:   # a server's state
            pkg.Server(vol)
        assert e.value.code == pkg.ISO_ERR_OOM
    finally:
        pkg.use_pool_allocator()
    try:
        _check_against_oracle(pkg, vol, bits, dims, rate, bmin, bmax, 0.0)
    finally:
        vol.release()


def test_release_cached_memory_returns_the_pool():
    # a 512^3 volume of zero blocks at 2 bits/value reserves its whole slot
    # pool at load (2,097,152 slots, 537 MB); released, the memory stays in
    # the library's pool until iso_release_cached_memory gives it back
    import torch
    import paper_2009_03254_gb300 as pkg
    dims, rate = (512, 512, 512), 2
    nb = int(np.prod(oracle.block_dims(dims)))
    bits = torch.zeros(nb * rate, dtype=torch.int64, device="cuda")
    rng = torch.zeros(nb, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    vol = pkg.Volume(bits, dims, rate, rng, rng)
    m = vol.extract(0.5)                                      # nothing crosses: an empty mesh
    assert m.num_triangles == 0
    m.release()
    vol.release()
    torch.cuda.synchronize()
    kept = torch.cuda.mem_get_info()[0]
    assert pkg.release_cached_memory() is True
    freed = torch.cuda.mem_get_info()[0] - kept
    assert freed >= 500 * 10**6, freed
    # the library allocates again as before
    vol = pkg.Volume(bits, dims, rate, rng, rng)
    m = vol.extract(0.5)
    assert m.num_triangles == 0
    m.release()
    vol.release()
