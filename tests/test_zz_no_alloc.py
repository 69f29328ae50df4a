"""The allocation-free entry point, checked against the regular pipeline.

iso_active_blocks_static serves callers that cannot allocate device memory
(a stream under graph capture, a plug-in inside an application that owns
the device memory, a loop that must not stall on an allocation): its only
scratch is a fixed array inside the library.  Two calls in a row must
select exactly the blocks that iso_extract selects for the same isovalues
(block ids are integers: the comparison is exact).  This file is collected
last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest

import oracle
from synth import fields

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_static_scratch_selection_matches_extract():
    import torch
    import paper_2009_03254_gb300 as pkg

    dims, rate = (70, 45, 38), 8
    f = fields.gradient_noise(*dims, 17, octaves=4, base_period=32)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    d_min, d_max = torch.from_numpy(bmin).cuda(), torch.from_numpy(bmax).cuda()
    vol = pkg.Volume(bits, dims, rate, bmin, bmax, debug=True)
    nb = bits.shape[0]
    ids = torch.full((nb,), -7, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    try:
        for iso in (0.0, 0.35):                       # two calls in a row share the scratch
            mesh = vol.extract(iso)
            want = vol.debug("active_ids")
            mesh.release()
            pkg.active_blocks_static(d_min, d_max, dims, iso, ids=ids, count=count)
            torch.cuda.synchronize()
            n = int(count.item())
            assert n == len(want) > 0
            assert np.array_equal(ids[:n].cpu().numpy().view(np.uint32), want)
    finally:
        vol.release()


def test_static_scratch_rejects_oversized_volume():
    import torch
    import paper_2009_03254_gb300 as pkg

    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    ids = torch.zeros(4, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(pkg.IsoError) as e:           # 2^26 + 1 blocks: more than the fixed scratch covers
        pkg.active_blocks_static(dummy, dummy, (4 * 8193, 4 * 8192, 4), 0.0, ids=ids, count=count)
    assert e.value.code == pkg.ISO_ERR_INVALID_ARG
