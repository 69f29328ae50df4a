"""The allocation-free entry point, checked against the oracle and the pipeline.

iso_active_blocks_static serves callers that cannot allocate device memory
(a plug-in inside an application whose allocator owns the device memory, a
loop that must not stall on an allocation's implicit synchronisation): its
only scratch is a fixed array inside the library.  Two calls in a row must
select exactly the blocks of the oracle's active rule (block ids are
integers: the comparison is exact), which are also the ids iso_extract
selects.  This file is collected last so that a failure here cannot hide
any other test's result.
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


def _volume(dims=(70, 45, 38), rate=8, seed=17):
    f = fields.gradient_noise(*dims, seed, octaves=4, base_period=32)
    return oracle.encode_volume(f, rate)


def test_static_scratch_selection_matches_oracle_and_extract():
    import torch
    import paper_2009_03254_gb300 as pkg

    dims, rate = (70, 45, 38), 8
    bits, bmin, bmax = _volume(dims, rate)
    nbd = oracle.block_dims(dims)
    d_min, d_max = torch.from_numpy(bmin).cuda(), torch.from_numpy(bmax).cuda()
    vol = pkg.Volume(bits, dims, rate, bmin, bmax, debug=True)
    nb = bits.shape[0]
    ids = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        for iso in (0.0, 0.35):                       # two calls in a row share the scratch
            want = np.flatnonzero(oracle.active_blocks(bmin, bmax, nbd, iso)).astype(np.uint32)
            pkg.active_blocks_static(d_min, d_max, dims, iso, ids=ids, count=count)
            n = pkg.static_count(count)
            assert n == len(want) > 0
            assert np.array_equal(ids[:n].cpu().numpy().view(np.uint32), want)
            mesh = vol.extract(iso)                   # the pipeline's range test selects the same ids
            assert np.array_equal(vol.debug("active_ids"), want)
            mesh.release()
    finally:
        vol.release()


def test_static_scratch_short_capacity_keeps_the_full_count():
    import torch
    import paper_2009_03254_gb300 as pkg

    dims = (70, 45, 38)
    bits, bmin, bmax = _volume(dims)
    want = np.flatnonzero(oracle.active_blocks(bmin, bmax, oracle.block_dims(dims), 0.0)).astype(np.uint32)
    cap = len(want) // 2
    ids = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    _, count = pkg.active_blocks_static(torch.from_numpy(bmin).cuda(), torch.from_numpy(bmax).cuda(), dims, 0.0,
                                        ids=ids)
    assert pkg.static_count(count) == len(want)      # the ids past the capacity are dropped, not the count
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), want[:cap])


def test_static_scratch_reports_ranges_that_are_not_ranges():
    import torch
    import paper_2009_03254_gb300 as pkg

    dims = (40, 36, 20)
    _, bmin, bmax = _volume(dims)
    for bad in ("nan", "swap"):
        lo, hi = bmin.copy(), bmax.copy()
        if bad == "nan":
            lo[7] = np.nan
        else:
            lo[3], hi[3] = hi[3] + 1.0, lo[3]
        _, count = pkg.active_blocks_static(torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(), dims, 0.0)
        with pytest.raises(pkg.IsoError) as e:
            pkg.static_count(count)
        assert e.value.code == pkg.ISO_ERR_CORRUPT
    # the next call with good ranges is unaffected by the shared scratch
    want = np.flatnonzero(oracle.active_blocks(bmin, bmax, oracle.block_dims(dims), 0.0)).astype(np.uint32)
    ids, count = pkg.active_blocks_static(torch.from_numpy(bmin).cuda(), torch.from_numpy(bmax).cuda(), dims, 0.0)
    n = pkg.static_count(count)
    assert n == len(want) and np.array_equal(ids[:n].cpu().numpy().view(np.uint32), want)


def test_static_scratch_refuses_bad_buffers():
    import torch
    import paper_2009_03254_gb300 as pkg

    dims = (40, 36, 20)
    _, bmin, bmax = _volume(dims)
    d_min, d_max = torch.from_numpy(bmin).cuda(), torch.from_numpy(bmax).cuda()
    with pytest.raises(ValueError):                   # host memory
        pkg.active_blocks_static(torch.from_numpy(bmin), d_max, dims, 0.0)
    with pytest.raises(ValueError):                   # fewer ranges than blocks
        pkg.active_blocks_static(d_min[:-1], d_max, dims, 0.0)
    with pytest.raises(ValueError):                   # wrong dtype
        pkg.active_blocks_static(d_min.double(), d_max, dims, 0.0)
    with pytest.raises(ValueError):                   # no room for the count
        pkg.active_blocks_static(d_min, d_max, dims, 0.0, count=torch.zeros(0, dtype=torch.int32, device="cuda"))
    # the C entry point refuses misaligned device pointers before launching anything
    raw = torch.zeros(len(bmin) + 4, dtype=torch.float32, device="cuda")
    ids = torch.zeros(len(bmin), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = pkg.lib().iso_active_blocks_static(ctypes.c_void_p(raw.data_ptr() + 2), ctypes.c_void_p(d_max.data_ptr()),
                                            *dims, ctypes.c_float(0.0), ctypes.c_void_p(ids.data_ptr()), ids.numel(),
                                            ctypes.c_void_p(count.data_ptr()), None)
    assert rc == pkg.ISO_ERR_INVALID_ARG


def test_static_scratch_rejects_oversized_volume():
    import torch
    import paper_2009_03254_gb300 as pkg

    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.IsoError) as e:           # 2^26 + 1 blocks: more than the fixed scratch covers
        pkg._check(pkg.lib().iso_active_blocks_static(ctypes.c_void_p(dummy.data_ptr()),
                                                      ctypes.c_void_p(dummy.data_ptr()), 4 * 8193, 4 * 8192, 4,
                                                      ctypes.c_float(0.0), ctypes.c_void_p(ids.data_ptr()), 4,
                                                      ctypes.c_void_p(count.data_ptr()), None),
                   "iso_active_blocks_static")
    assert e.value.code == pkg.ISO_ERR_INVALID_ARG
