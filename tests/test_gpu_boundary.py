"""GPU tests of the boundary's remaining calls: the caller-supplied
allocator (PyTorch's caching allocator through iso_set_allocator), block
ranges that are not ranges (ISO_ERR_CORRUPT at load), and waiting on a
served request (iso_server_wait).  Meshes are checked against the oracle.
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


def volume_data(dims=(40, 36, 30), rate=8, seed=3):
    f = fields.gradient_noise(*dims, seed, octaves=4, base_period=16)
    bits, bmin, bmax = oracle.encode_volume(f, rate)
    return dims, rate, bits, bmin, bmax


def test_torch_allocator_serves_every_allocation():
    import torch
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data()
    ref = oracle.extract(bits, dims, rate, bmin, bmax, 0.0)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    p.use_torch_allocator()
    try:
        vol = p.Volume(bits, dims, rate, bmin, bmax)
        torch.cuda.synchronize()
        held = torch.cuda.memory_allocated() - base
        assert held >= bits.nbytes                    # the volume's state came from PyTorch
        m = vol.extract(0.0)
        assert m.num_triangles == ref["num_triangles"]
        v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
        assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < POS_TOL
        assert torch.cuda.memory_allocated() - base >= held + 48 * m.num_triangles
    finally:
        p.use_pool_allocator()
    # made under the hook, freed after switching back: still returned to PyTorch
    m.release()
    vol.release()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    # and the pool serves again
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    m = vol.extract(0.0)
    assert m.num_triangles == ref["num_triangles"]
    m.release()
    vol.release()
    assert torch.cuda.memory_allocated() == base
    # an allocation function without a free function is refused (and never called)
    import ctypes
    assert p.lib().iso_set_allocator(ctypes.c_void_p(1), None, None) == p.ISO_ERR_INVALID_ARG


def test_ranges_that_are_not_ranges_are_refused():
    import torch
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data(dims=(20, 20, 20))
    for broken in ("swap", "nan_min", "nan_max"):
        lo, hi = bmin.copy(), bmax.copy()
        k = 17
        if broken == "swap":
            lo[k], hi[k] = hi[k] + 1.0, lo[k]
        elif broken == "nan_min":
            lo[k] = np.nan
        else:
            hi[k] = np.nan
        for on_device in (False, True):
            args = (bits, lo, hi)
            if on_device:
                args = (torch.from_numpy(bits.view(np.int64)).cuda(), torch.from_numpy(lo).cuda(),
                        torch.from_numpy(hi).cuda())
            with pytest.raises(p.IsoError) as e:
                p.Volume(args[0], dims, rate, args[1], args[2])
            assert e.value.code == p.ISO_ERR_CORRUPT
    vol = p.Volume(bits, dims, rate, bmin, bmax)                   # the real ranges load
    vol.release()


def test_server_wait():
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data(seed=5)
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    alone = p.Volume(bits, dims, rate, bmin, bmax)
    srv = p.Server(vol, max_batch=4)
    try:
        isos = [-0.3, 0.0, 0.4]
        tickets = [srv.submit(x) for x in isos]
        assert srv.wait(tickets[2], timeout_ms=0) == (p.ISO_PENDING, None)    # look once, no step
        for t, x in zip(reversed(tickets), reversed(isos)):                   # the last one first
            status, m = srv.wait(t, timeout_ms=10000)
            assert status == p.ISO_OK
            ref = alone.extract(x)
            assert m.num_triangles == ref.num_triangles
            assert np.array_equal(m.vertices.cpu().numpy().view(np.uint32), ref.vertices.cpu().numpy().view(np.uint32))
            m.release()
            ref.release()
        with pytest.raises(p.IsoError):
            srv.wait(tickets[0], timeout_ms=10)                              # already taken
    finally:
        srv.release()
        vol.release()
        alone.release()


def test_misaligned_outputs_are_refused():
    # the checks run on the host before any launch: nothing is written
    import ctypes
    import torch
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data(dims=(20, 20, 20))
    vol = p.Volume(bits, dims, rate, bmin, bmax)
    try:
        buf = torch.zeros(20000 * 12 + 16, dtype=torch.float32, device="cuda")
        base = buf.data_ptr()
        st = p._Stats()
        L = p.lib()
        for off in (4, 8):
            ptr = ctypes.c_void_p(base + off)
            assert L.iso_extract_into(vol._h, ctypes.c_float(0.0), ptr, 4096, ctypes.byref(st)) == p.ISO_ERR_INVALID_ARG
            assert L.iso_extract_all_blocks_into(vol._h, ctypes.c_float(0.0), ptr, 4096,
                                                 ctypes.byref(st)) == p.ISO_ERR_INVALID_ARG
        ptr4 = ctypes.c_void_p(base + 4)
        assert L.iso_extract_packed_into(vol._h, ctypes.c_float(0.0), ptr4, 4096, ctypes.byref(st)) == \
            p.ISO_ERR_INVALID_ARG
        assert L.iso_extract_indexed_into(vol._h, ctypes.c_float(0.0), p.ISO_VERTEX_FLOAT4, ctypes.c_void_p(base + 8),
                                          1024, ctypes.c_void_p(base), 1024, ctypes.byref(st)) == p.ISO_ERR_INVALID_ARG
        assert L.iso_extract_indexed_into(vol._h, ctypes.c_float(0.0), p.ISO_VERTEX_PACKED, ctypes.c_void_p(base),
                                          1024, ctypes.c_void_p(base + 2), 1024, ctypes.byref(st)) == p.ISO_ERR_INVALID_ARG
        assert torch.count_nonzero(buf).item() == 0
        # the aligned pointer works
        assert L.iso_extract_into(vol._h, ctypes.c_float(0.0), ctypes.c_void_p(base + 16), 20000,
                                  ctypes.byref(st)) == p.ISO_OK
        assert st.num_triangles > 0
    finally:
        vol.release()


def test_async_load_reports_bad_ranges_on_first_call():
    # ISO_ASYNC_UPLOAD: the load returns at once; the range check's verdict
    # comes with the first call on the volume, and with every call after it
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data(dims=(20, 20, 20))
    lo, hi = bmin.copy(), bmax.copy()
    lo[5], hi[5] = hi[5] + 1.0, lo[5]
    vol = p.Volume(bits, dims, rate, lo, hi, async_upload=True)
    try:
        for _ in range(2):
            with pytest.raises(p.IsoError) as e:
                vol.extract(0.0)
            assert e.value.code == p.ISO_ERR_CORRUPT
    finally:
        vol.release()
    ref = oracle.extract(bits, dims, rate, bmin, bmax, 0.0)
    vol = p.Volume(bits, dims, rate, bmin, bmax, async_upload=True)     # the real ranges
    try:
        m = vol.extract(0.0)
        assert m.num_triangles == ref["num_triangles"]
        v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
        assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < POS_TOL
        m.release()
    finally:
        vol.release()


def test_load_release_cycles_reuse_host_mirrors_and_streams():
    # released volumes hand their pinned host mirrors and upload stream to
    # the next load: many volumes loaded and released in interleaved order
    # (more at once than one, fewer than the kept set, then more than it),
    # with asynchronous uploads on two caller streams, all extract the same
    # surface as the oracle
    import torch
    p = pkg()
    dims, rate, bits, bmin, bmax = volume_data(dims=(24, 20, 18))
    ref = oracle.extract(bits, dims, rate, bmin, bmax, 0.0)
    h_bits = torch.from_numpy(bits.view(np.int64)).pin_memory()
    h_min = torch.from_numpy(bmin).pin_memory()
    h_max = torch.from_numpy(bmax).pin_memory()
    lanes = [torch.cuda.Stream(), torch.cuda.Stream()]
    import ctypes

    def load(i):
        return p.Volume(h_bits, dims, rate, h_min, h_max, async_upload=True,
                        stream=ctypes.c_void_p(lanes[i % 2].cuda_stream))

    def check(vol):
        m = vol.extract(0.0)
        assert m.num_triangles == ref["num_triangles"]
        if m.num_triangles:
            v = m.vertices.cpu().numpy().reshape(-1, 3, 4)
            assert np.abs(v[:, :, :3] - ref["local_pos"]).max() < POS_TOL
        m.release()

    live = []
    for i in range(40):
        live.append(load(i))
        check(live[-1])
        if len(live) > 3:                       # release out of load order
            live.pop(1 if i % 3 else 0).release()
    many = [load(i) for i in range(80)]         # more at once than are kept for reuse
    for vol in many[::7]:
        check(vol)
    for vol in many + live:
        vol.release()
