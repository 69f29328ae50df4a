"""GB300 block-compressed marching cubes.

Thin Python binding over the C ABI of ``libbcmc.so`` (declared in
``include/bcmc.h``).  It only marshals arguments: every step of the
isosurface pipeline runs in the library's CUDA kernels.  PyTorch supplies
device memory and streams.  There is no CPU fallback: if the compiled
library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# BCMC_CHECKED=1 loads the checked build (device-side bounds checks, see build.py)
LIB_PATH = os.path.join(HERE, "_lib_checked" if os.environ.get("BCMC_CHECKED") == "1" else "_lib", "libbcmc.so")

ISO_OK = 0
ISO_ERR_INVALID_ARG = 1
ISO_ERR_OOM = 2
ISO_ERR_BUDGET = 3
ISO_ERR_CUDA = 4
ISO_ERR_TIMEOUT = 5
ISO_ERR_CAPACITY = 6
ISO_PENDING = 7
ISO_ERR_CORRUPT = 8
ISO_ERR_BOUNDS = 9

ISO_INPUT_ON_DEVICE = 1
ISO_DEBUG = 2
ISO_NO_GRAPH = 4
ISO_ASYNC_UPLOAD = 8
ISO_SEGMENT_CULL = 16
ISO_NO_SEGMENT_CULL = 32
ISO_TEST_WITHHOLD_PREFIX = 1
ISO_VERTEX_FLOAT4 = 0
ISO_VERTEX_PACKED = 1

DBG = {
    "active_ids": (1, np.uint32), "new_ids": (2, np.uint32), "slot_of_block": (3, np.int32),
    "block_of_slot": (4, np.int32), "slot_last_use": (5, np.uint32), "active_mask": (6, np.uint32),
    "cell_cases": (7, np.uint8), "block_tris": (8, np.uint32), "block_offsets": (9, np.uint64),
    "edge_ids": (10, np.uint64), "candidates": (11, np.uint32),
}


class IsoError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {error_string(code)} (status {code})")


class _Options(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("initial_cache_fraction", ctypes.c_double), ("cache_budget_bytes", ctypes.c_uint64)]


class _Stats(ctypes.Structure):
    _fields_ = [("num_triangles", ctypes.c_uint64), ("n_active", ctypes.c_uint32), ("n_new", ctypes.c_uint32),
                ("n_occupied", ctypes.c_uint32), ("n_slots", ctypes.c_uint32), ("cache_bytes", ctypes.c_uint64),
                ("epoch", ctypes.c_uint32), ("reruns", ctypes.c_uint32), ("n_candidates", ctypes.c_uint32),
                ("waves", ctypes.c_uint32), ("num_vertices", ctypes.c_uint64)]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class _Shape(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint32) for name in (
        "cull_ctas", "cull_tile", "cache_update_ctas", "decode_ctas", "decode_tile", "count_ctas", "count_tile",
        "scan_ctas", "scan_tile", "emit_ctas", "emit_tile")]

    def as_dict(self):
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class _ServerOptions(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("vertex_format", ctypes.c_uint32),
                ("vertex_budget_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("case_bytes", ctypes.c_uint64)]


class _Camera(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("light", ctypes.c_float * 3), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32)]


class _RenderStats(ctypes.Structure):
    _fields_ = [("drawn", ctypes.c_uint64), ("big", ctypes.c_uint64)]


class _Pinhole(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("forward", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("light", ctypes.c_float * 3), ("width", ctypes.c_uint32),
                ("height", ctypes.c_uint32)]


class _CastStats(ctypes.Structure):
    _fields_ = [("hits", ctypes.c_uint64), ("n_active", ctypes.c_uint32), ("n_new", ctypes.c_uint32),
                ("n_slots", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class _DenseStats(ctypes.Structure):
    _fields_ = [("num_triangles", ctypes.c_uint64), ("n_active_cells", ctypes.c_uint64)]


class _Mesh(ctypes.Structure):
    _fields_ = [("d_vertices", ctypes.c_void_p), ("num_triangles", ctypes.c_uint64),
                ("capacity_triangles", ctypes.c_uint64), ("stats", _Stats), ("priv", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libbcmc.so (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t
        i32 = ctypes.c_int
        sig = {
            "iso_load_volume": (i32, [ctypes.POINTER(P), P, sz, u32, u32, u32, u32, P, P, ctypes.POINTER(_Options)]),
            "iso_extract": (i32, [P, ctypes.c_float, ctypes.POINTER(_Mesh)]),
            "iso_extract_into": (i32, [P, ctypes.c_float, P, u64, ctypes.POINTER(_Stats)]),
            "iso_extract_packed_into": (i32, [P, ctypes.c_float, P, u64, ctypes.POINTER(_Stats)]),
            "iso_extract_all_blocks_into": (i32, [P, ctypes.c_float, P, u64, ctypes.POINTER(_Stats)]),
            "iso_extract_indexed_into": (i32, [P, ctypes.c_float, i32, P, u64, P, u64, ctypes.POINTER(_Stats)]),
            "iso_render": (i32, [P, i32, P, u64, u64, u32, u32, u32, ctypes.POINTER(_Camera), P, P,
                                 ctypes.POINTER(_RenderStats), P]),
            "iso_raycast": (i32, [P, ctypes.c_float, ctypes.POINTER(_Pinhole), P, P, ctypes.POINTER(_CastStats)]),
            "iso_decode_volume": (i32, [P, u32, u32, u32, u32, P, P]),
            "iso_mc_dense": (i32, [P, u32, u32, u32, ctypes.c_float, P, u64, P, ctypes.POINTER(_DenseStats), P]),
            "iso_mesh_release": (i32, [P, ctypes.POINTER(_Mesh)]),
            "iso_release": (None, [P]),
            "iso_set_stream": (i32, [P, P]),
            "iso_cache_reset": (i32, [P]),
            "iso_set_test_fault": (i32, [P, u32]),
            "iso_error_string": (ctypes.c_char_p, [i32]),
            "iso_mc_case_table": (i32, [P, P]),
            "iso_encode_field": (i32, [P, u32, u32, u32, u32, P, P, P, P]),
            "iso_decode_blocks": (i32, [P, u32, P, u64, P, P]),
            "iso_debug_get": (i32, [P, i32, P, sz, ctypes.POINTER(u64)]),
            "iso_debug_read_blocks": (i32, [P, P, u64, P]),
            "iso_set_profiling": (i32, [P, i32]),
            "iso_active_blocks_static": (i32, [P, P, u32, u32, u32, ctypes.c_float, P, u64, P, P]),
            "iso_stage_times": (i32, [P, ctypes.POINTER(ctypes.c_float), i32]),
            "iso_batch_create": (i32, [ctypes.POINTER(P), P, u32, P]),
            "iso_batch_extract": (i32, [P, P, P, u64, P, P, P]),
            "iso_batch_set_shape": (i32, [P, ctypes.POINTER(_Shape)]),
            "iso_set_shape": (i32, [P, ctypes.POINTER(_Shape)]),
            "iso_get_shape": (i32, [P, ctypes.POINTER(_Shape)]),
            "iso_batch_get_shape": (i32, [P, ctypes.POINTER(_Shape)]),
            "iso_batch_tune": (i32, [P, P, P, u64, i32, ctypes.POINTER(_Shape), P]),
            "iso_batch_release": (None, [P]),
            "iso_server_create": (i32, [ctypes.POINTER(P), P, ctypes.POINTER(_ServerOptions)]),
            "iso_server_submit": (i32, [P, ctypes.c_float, ctypes.POINTER(u64)]),
            "iso_server_step": (i32, [P, ctypes.POINTER(u32)]),
            "iso_server_poll": (i32, [P, ctypes.POINTER(u32)]),
            "iso_server_queued": (i32, [P, ctypes.POINTER(u32)]),
            "iso_server_take": (i32, [P, u64, ctypes.POINTER(_Mesh)]),
            "iso_server_wait": (i32, [P, u64, u32, ctypes.POINTER(_Mesh)]),
            "iso_set_allocator": (i32, [P, P, P]),
            "iso_release_cached_memory": (i32, [i32]),
            "iso_server_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def error_string(code):
    return lib().iso_error_string(int(code)).decode()


def _check(rc, where):
    if rc != ISO_OK:
        raise IsoError(rc, where)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    """device pointer of a torch tensor, host pointer of a numpy array"""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())


def block_dims(dims):
    nx, ny, nz = dims
    return (nx + 3) // 4, (ny + 3) // 4, (nz + 3) // 4


def mc_case_table():
    """The library's 256-case table: (num_tri uint8[256], tri_edges uint8[256, 16])."""
    num = np.zeros(256, np.uint8)
    tri = np.zeros((256, 16), np.uint8)
    _check(lib().iso_mc_case_table(_ptr(num), _ptr(tri)), "iso_mc_case_table")
    return num, tri


class _DeviceArray:
    """CUDA array interface over library-owned memory (no copy)."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


class Mesh:
    """A surface computed by Volume.extract (or served).  `vertices` is a
    (3T, 4) float32 CUDA tensor, or for compact meshes a (3T, 2) int32 one,
    viewing library-owned memory: valid until release()."""

    def __init__(self, volume, m, packed=False):
        self._volume = volume
        self._m = m
        self.packed = bool(packed)
        self.num_triangles = int(m.num_triangles)
        self.stats = m.stats.as_dict()

    @property
    def vertices(self):
        import torch
        width, typestr, dt = (2, "<i4", torch.int32) if self.packed else (4, "<f4", torch.float32)
        if not self._m.d_vertices:
            return torch.zeros((0, width), dtype=dt, device="cuda")
        arr = _DeviceArray(int(self._m.d_vertices), (3 * self.num_triangles, width), typestr)
        return torch.as_tensor(arr, device="cuda")

    def release(self):
        if self._m is not None and self._m.d_vertices:
            _check(lib().iso_mesh_release(self._volume._h, ctypes.byref(self._m)), "iso_mesh_release")
        self._m = None

    def __del__(self):
        try:
            if self._volume is not None and self._volume._h:
                self.release()
        except Exception:
            pass


class Volume:
    """A compressed volume resident on the GPU with its decoded-block cache.

    bits       uint64 words (nb*rate), numpy (host) or a CUDA tensor
    dims       (nx, ny, nz)
    rate       bits per sample
    bmin/bmax  per-block ranges of the decoded samples (nb floats each)
    segment_cull  None: segment ranges for volumes of 2^28 blocks or more;
               True / False: always / never (ISO_SEGMENT_CULL, ISO_NO_SEGMENT_CULL)
    """

    def __init__(self, bits, dims, rate, bmin, bmax, *, stream=None, debug=False, initial_cache_fraction=0.1,
                 cache_budget_bytes=0, graph=True, async_upload=False, segment_cull=None):
        self._h = None
        on_device = not isinstance(bits, np.ndarray) and bool(getattr(bits, "is_cuda", False))
        if not isinstance(bits, np.ndarray) and not on_device:       # CPU (e.g. pinned) torch tensors
            bits, bmin, bmax = bits.contiguous(), bmin.contiguous(), bmax.contiguous()
        elif not on_device:
            bits = np.ascontiguousarray(bits, np.uint64)
            bmin = np.ascontiguousarray(bmin, np.float32)
            bmax = np.ascontiguousarray(bmax, np.float32)
        self.dims = tuple(int(d) for d in dims)
        self.rate = int(rate)
        self.nb = int(np.prod(block_dims(self.dims)))
        opt = _Options()
        opt.flags = (ISO_INPUT_ON_DEVICE if on_device else 0) | (ISO_DEBUG if debug else 0) | \
            (0 if graph else ISO_NO_GRAPH) | (ISO_ASYNC_UPLOAD if async_upload else 0) | \
            ({None: 0, True: ISO_SEGMENT_CULL, False: ISO_NO_SEGMENT_CULL}[segment_cull])
        # with async_upload the bitstream is copied after this returns: keep it alive
        self._upload_source = bits if async_upload else None
        opt.stream = stream if stream is not None else _current_stream()
        opt.initial_cache_fraction = float(initial_cache_fraction)
        opt.cache_budget_bytes = int(cache_budget_bytes)
        nbytes = bits.nbytes if isinstance(bits, np.ndarray) else bits.numel() * bits.element_size()
        h = ctypes.c_void_p()
        nx, ny, nz = self.dims
        _check(lib().iso_load_volume(ctypes.byref(h), _ptr(bits), nbytes, nx, ny, nz, self.rate,
                                     _ptr(bmin), _ptr(bmax), ctypes.byref(opt)), "iso_load_volume")
        self._h = h
        self.debug_enabled = bool(debug)

    def extract(self, iso):
        m = _Mesh()
        _check(lib().iso_extract(self._h, ctypes.c_float(iso), ctypes.byref(m)), "iso_extract")
        return Mesh(self, m)

    def extract_into(self, iso, out, check=True):
        """Write the surface into `out`, a CUDA float32 tensor of shape (3C, 4)
        or (C, 3, 4) for C triangles.  Returns the stats dict."""
        cap = out.numel() // 12
        st = _Stats()
        rc = lib().iso_extract_into(self._h, ctypes.c_float(iso), _ptr(out), cap, ctypes.byref(st))
        if check:
            _check(rc, "iso_extract_into")
        d = st.as_dict()
        d["status"] = rc
        return d

    def extract_all_blocks_into(self, iso, out, check=True):
        """The full-volume baseline: every block decoded and visited (no range
        test); same mesh as extract_into.  Returns the stats dict."""
        cap = out.numel() // 12
        st = _Stats()
        rc = lib().iso_extract_all_blocks_into(self._h, ctypes.c_float(iso), _ptr(out), cap, ctypes.byref(st))
        if check:
            _check(rc, "iso_extract_all_blocks_into")
        d = st.as_dict()
        d["status"] = rc
        return d

    def extract_packed_into(self, iso, out, check=True):
        """The compact 8-byte vertices (two uint32 words: 10-bit codes of the
        block-local coordinates, block id) into `out`, a CUDA int32/uint32
        tensor of shape (C, 3, 2) for C triangles.  Returns the stats dict."""
        cap = out.numel() // 6
        st = _Stats()
        rc = lib().iso_extract_packed_into(self._h, ctypes.c_float(iso), _ptr(out), cap, ctypes.byref(st))
        if check:
            _check(rc, "iso_extract_packed_into")
        d = st.as_dict()
        d["status"] = rc
        return d

    def extract_indexed_into(self, iso, vertices, indices, check=True):
        """The indexed mesh (vertices shared within each block) into CUDA
        tensors: `vertices` float32 (V, 4) {x, y, z block-local, block id
        bits} or int32/uint32 (V, 2) compact vertices (the format follows the
        tensor), `indices` int32/uint32 (C, 3) for C triangles.  Gathering
        the vertices by index gives the triangle soup of extract_into (or
        extract_packed_into).  Returns the stats dict (num_vertices,
        num_triangles, status)."""
        import torch
        packed = vertices.dtype != torch.float32
        width = 2 if packed else 4
        assert vertices.is_cuda and vertices.is_contiguous() and vertices.numel() % width == 0
        assert indices.is_cuda and indices.is_contiguous() and indices.element_size() == 4
        st = _Stats()
        rc = lib().iso_extract_indexed_into(self._h, ctypes.c_float(iso),
                                            ISO_VERTEX_PACKED if packed else ISO_VERTEX_FLOAT4,
                                            _ptr(vertices), vertices.numel() // width, _ptr(indices),
                                            indices.numel() // 3, ctypes.byref(st))
        if check:
            _check(rc, "iso_extract_indexed_into")
        d = st.as_dict()
        d["status"] = rc
        return d

    def extract_indexed(self, iso, packed=False, guess_triangles=1 << 16):
        """The indexed mesh in buffers of its exact size: (vertices (V, 4)
        float32 or (V, 2) int32, indices (T, 3) int32, stats).  A first
        extraction into buffers of `guess_triangles` tells the sizes; when
        they were too small the extraction runs again into exact ones."""
        import torch
        width, dt = (2, torch.int32) if packed else (4, torch.float32)
        cap = max(1, int(guess_triangles))
        verts = torch.empty((cap, width), dtype=dt, device="cuda")
        idx = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
        st = self.extract_indexed_into(iso, verts, idx, check=False)
        if st["status"] == ISO_ERR_CAPACITY and st["num_vertices"] <= 0xFFFFFFFF:
            nv, nt = max(1, st["num_vertices"]), max(1, st["num_triangles"])
            verts = torch.empty((nv, width), dtype=dt, device="cuda")
            idx = torch.empty((nt, 3), dtype=torch.int32, device="cuda")
            st = self.extract_indexed_into(iso, verts, idx, check=False)
        _check(st["status"], "iso_extract_indexed_into")
        return verts[:st["num_vertices"]], idx[:st["num_triangles"]], st

    def raycast(self, iso, eye, forward, right, up, light, width, height, hits=None, rgba=None):
        """Ray cast the isosurface (rules in iso_raycast) into CUDA buffers:
        returns (hits int64 (height, width): t bits << 32 | block id, -1 for
        none; rgba int32 (height, width) or None with rgba=False; stats)."""
        import torch
        if hits is None:
            hits = torch.empty((height, width), dtype=torch.int64, device="cuda")
        if rgba is None:
            rgba = torch.empty((height, width), dtype=torch.int32, device="cuda")
        cam = _Pinhole()
        for name, vec in (("eye", eye), ("forward", forward), ("right", right), ("up", up), ("light", light)):
            arr = getattr(cam, name)
            for k in range(3):
                arr[k] = float(vec[k])
        cam.width, cam.height = int(width), int(height)
        st = _CastStats()
        _check(lib().iso_raycast(self._h, ctypes.c_float(iso), ctypes.byref(cam), _ptr(hits),
                                 _ptr(rgba) if rgba is not False else None, ctypes.byref(st)), "iso_raycast")
        return hits, (rgba if rgba is not False else None), {
            "hits": int(st.hits), "n_active": int(st.n_active), "n_new": int(st.n_new), "n_slots": int(st.n_slots)}

    def set_shape(self, **shape):
        """The launch shape of this volume's extractions (iso_set_shape):
        keyword fields of iso_launch_shape, the rest 0 (defaults)."""
        sh = _Shape()
        for k, val in shape.items():
            setattr(sh, k, int(val))
        _check(lib().iso_set_shape(self._h, ctypes.byref(sh)), "iso_set_shape")

    def get_shape(self):
        sh = _Shape()
        _check(lib().iso_get_shape(self._h, ctypes.byref(sh)), "iso_get_shape")
        return sh.as_dict()

    STAGES = ("prep", "cull", "cache_update", "decode", "count", "scan", "emit")

    def set_profiling(self, on=True):
        _check(lib().iso_set_profiling(self._h, 1 if on else 0), "iso_set_profiling")

    def stage_times(self):
        """ms per stage of the last extraction (profiling on)"""
        n = len(self.STAGES)
        buf = (ctypes.c_float * n)()
        _check(lib().iso_stage_times(self._h, buf, n), "iso_stage_times")
        return dict(zip(self.STAGES, [float(x) for x in buf]))

    def cache_reset(self):
        _check(lib().iso_cache_reset(self._h), "iso_cache_reset")

    def set_test_fault(self, what):
        """Test hook (iso_set_test_fault): ISO_TEST_WITHHOLD_PREFIX makes every
        later extraction's range-test wait run out and return ISO_ERR_TIMEOUT;
        0 restores normal operation."""
        _check(lib().iso_set_test_fault(self._h, what), "iso_set_test_fault")

    def set_stream(self, stream):
        _check(lib().iso_set_stream(self._h, stream), "iso_set_stream")

    def debug(self, name):
        which, dtype = DBG[name]
        cnt = ctypes.c_uint64()
        rc = lib().iso_debug_get(self._h, which, None, 0, ctypes.byref(cnt))
        if rc not in (ISO_OK, ISO_ERR_CAPACITY):
            _check(rc, "iso_debug_get")
        out = np.zeros(int(cnt.value), dtype)
        if out.size:
            _check(lib().iso_debug_get(self._h, which, _ptr(out), out.nbytes, ctypes.byref(cnt)), "iso_debug_get")
        return out

    def read_blocks(self, ids):
        ids = np.ascontiguousarray(ids, np.uint32)
        out = np.zeros((len(ids), 64), np.float32)
        _check(lib().iso_debug_read_blocks(self._h, _ptr(ids), len(ids), _ptr(out)), "iso_debug_read_blocks")
        return out

    def release(self):
        if self._h:
            lib().iso_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Batch:
    """Several loaded volumes extracted together, each at its own isovalue,
    with one launch per stage for all of them (replayed as a CUDA graph).
    Each volume keeps its own cache; its surface equals extracting it alone.
    The volumes must outlive the batch and be on the current device."""

    def __init__(self, volumes, *, stream=None):
        self._h = None
        self.volumes = list(volumes)
        n = len(self.volumes)
        arr = (ctypes.c_void_p * max(n, 1))(*[v._h.value if v._h else None for v in self.volumes])
        h = ctypes.c_void_p()
        _check(lib().iso_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), n,
                                      stream if stream is not None else _current_stream()), "iso_batch_create")
        self._h = h
        self.n = n
        self._last_total = 0

    def extract_into(self, isos, out, check=True):
        """Write the surfaces into `out` (CUDA float32, 12 floats per triangle).
        Returns a dict: offsets (uint64[n+1], surface i = triangles
        offsets[i]:offsets[i+1]), stats (list of dicts), status (list), rc."""
        isos = np.ascontiguousarray(isos, np.float32)
        if isos.shape != (self.n,):
            raise ValueError(f"need {self.n} isovalues")
        cap = out.numel() // 12 if out is not None else 0
        offsets = np.zeros(self.n + 1, np.uint64)
        stats = (_Stats * self.n)()
        status = np.zeros(self.n, np.int32)
        rc = lib().iso_batch_extract(self._h, _ptr(isos), _ptr(out) if cap else None, cap, _ptr(offsets),
                                     ctypes.cast(stats, ctypes.c_void_p), _ptr(status))
        if check:
            _check(rc, "iso_batch_extract")
        self._last_total = int(offsets[-1])
        return {"offsets": offsets, "stats": [st.as_dict() for st in stats], "status": status.tolist(), "rc": rc}

    def extract(self, isos):
        """Surfaces into a new CUDA tensor.  Returns (vertices (3T, 4) tensor,
        offsets uint64[n+1], stats list).  A first guess too small is
        retried once with the exact size (from a warm cache)."""
        import torch
        guess = self._last_total + self._last_total // 4 + 4096 if self._last_total else \
            sum(2 * v.nb for v in self.volumes) + 4096
        out = torch.empty((3 * guess, 4), dtype=torch.float32, device="cuda")
        r = self.extract_into(isos, out, check=False)
        if r["rc"] == ISO_ERR_CAPACITY:
            total = int(r["offsets"][-1])
            out = torch.empty((3 * max(total, 1), 4), dtype=torch.float32, device="cuda")
            r = self.extract_into(isos, out, check=False)
        _check(r["rc"], "iso_batch_extract")
        total = int(r["offsets"][-1])
        return out[:3 * total], r["offsets"], r["stats"]

    @property
    def shape(self):
        sh = _Shape()
        _check(lib().iso_batch_get_shape(self._h, ctypes.byref(sh)), "iso_batch_get_shape")
        return sh.as_dict()

    def set_shape(self, **shape):
        """CTAs per SM (``*_ctas``) and tile sizes (``*_tile``) per kernel; 0 or
        absent = default.  See iso_launch_shape in include/bcmc.h."""
        sh = _Shape(**{k: int(v) for k, v in shape.items()})
        _check(lib().iso_batch_set_shape(self._h, ctypes.byref(sh)), "iso_batch_set_shape")

    def tune(self, isos, out, trials=3):
        """Autotune each kernel's tile size and CTAs per SM on these isovalues
        (caches are emptied before each timed run and left empty).  Returns a
        dict with the applied shape and the cold batch time (ms) of the
        default shape and of the applied one."""
        isos = np.ascontiguousarray(isos, np.float32)
        sh = _Shape()
        ms = np.zeros(2, np.float32)
        _check(lib().iso_batch_tune(self._h, _ptr(isos), _ptr(out), out.numel() // 12, int(trials),
                                    ctypes.byref(sh), _ptr(ms)), "iso_batch_tune")
        return {"shape": sh.as_dict(), "default_ms": float(ms[0]), "tuned_ms": float(ms[1])}

    def release(self):
        if self._h:
            lib().iso_batch_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Server:
    """Isovalue requests on one resident volume, answered in ticks: each
    tick runs up to `max_batch` queued requests together (one cull pass for
    all, one cache update for their union, one launch per triangle stage),
    and the next tick's cull, cache update and decode overlap the running
    tick's emission.  See iso_server_* in include/bcmc.h.  The volume must
    outlive the server."""

    def __init__(self, volume, *, max_batch=4, vertex_budget_bytes=0, stream=None, packed=False, case_bytes=0):
        self._h = None
        self.volume = volume
        self.packed = bool(packed)
        opt = _ServerOptions()
        opt.max_batch = int(max_batch)
        opt.vertex_format = ISO_VERTEX_PACKED if packed else ISO_VERTEX_FLOAT4
        opt.vertex_budget_bytes = int(vertex_budget_bytes)
        opt.stream = stream if stream is not None else _current_stream()
        opt.case_bytes = int(case_bytes)
        h = ctypes.c_void_p()
        _check(lib().iso_server_create(ctypes.byref(h), volume._h, ctypes.byref(opt)), "iso_server_create")
        self._h = h

    def submit(self, iso):
        t = ctypes.c_uint64()
        _check(lib().iso_server_submit(self._h, ctypes.c_float(iso), ctypes.byref(t)), "iso_server_submit")
        return int(t.value)

    def step(self):
        """Advance until a tick is done (blocking); returns the requests finished."""
        n = ctypes.c_uint32()
        _check(lib().iso_server_step(self._h, ctypes.byref(n)), "iso_server_step")
        return int(n.value)

    def poll(self):
        """Take every transition whose GPU work is done, without blocking;
        returns the requests finished."""
        n = ctypes.c_uint32()
        _check(lib().iso_server_poll(self._h, ctypes.byref(n)), "iso_server_poll")
        return int(n.value)

    def queued(self):
        n = ctypes.c_uint32()
        _check(lib().iso_server_queued(self._h, ctypes.byref(n)), "iso_server_queued")
        return int(n.value)

    def take(self, ticket):
        """(status, Mesh or None): ISO_PENDING while queued; the mesh belongs
        to the caller (release it) when status is ISO_OK."""
        m = _Mesh()
        rc = lib().iso_server_take(self._h, int(ticket), ctypes.byref(m))
        if rc == ISO_ERR_INVALID_ARG:
            raise IsoError(rc, "iso_server_take")
        if rc != ISO_OK:
            return rc, None
        return rc, Mesh(self.volume, m, self.packed)

    def wait(self, ticket, timeout_ms=1000):
        """Step until the ticket is done or the timeout passes: (status, Mesh
        or None) as take (ISO_PENDING on timeout)."""
        m = _Mesh()
        rc = lib().iso_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(m))
        if rc == ISO_ERR_INVALID_ARG:
            raise IsoError(rc, "iso_server_wait")
        if rc != ISO_OK:
            return rc, None
        return rc, Mesh(self.volume, m, self.packed)

    def release(self):
        if self._h:
            lib().iso_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)
_hooks = []                           # the installed callbacks (kept alive)


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (iso_set_allocator), in the order of the stream each is made
    on."""
    import torch

    def alloc(nbytes, device, stream, ctx):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=int(stream or 0)))
        except RuntimeError:
            return None

    def free(ptr, device, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_FN(alloc), _FREE_FN(free)
    _check(lib().iso_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None),
           "iso_set_allocator")
    _hooks.append((a, f))


def use_pool_allocator():
    """Back to the library's own stream-ordered memory pool (allocations
    made through an earlier hook still go back to it)."""
    _check(lib().iso_set_allocator(None, None, None), "iso_set_allocator")


def release_cached_memory(device=None):
    """Give the freed memory the library's pool keeps on `device` (default:
    the current CUDA device) back to the device (iso_release_cached_memory);
    waits for the device first.  False if the library never allocated from
    its pool there."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    rc = lib().iso_release_cached_memory(dev)
    if rc == ISO_ERR_INVALID_ARG:
        return False
    _check(rc, "iso_release_cached_memory")
    return True


def render(vertices, num_triangles, dims, view_proj, light, width, height, indices=None, fragments=None,
           rgba=None, stream=None, stats=False):
    """Rasterise a soup (vertices 3t..3t+2) or, with `indices` (uint32/int32
    CUDA tensor (T, 3)), an indexed mesh into headless CUDA buffers (rules in
    iso_render).  `vertices`: CUDA float32 (V, 4) or int32 (V, 2) compact.
    Returns (fragments int64 (height, width): depth bits << 32 | triangle,
    -1 where empty; rgba int32 (height, width): r | g << 8 | b << 16 | a << 24;
    stats dict or None).  Pass `rgba=False` to skip shading."""
    import torch
    assert vertices.is_cuda and vertices.is_contiguous()
    fmt = ISO_VERTEX_FLOAT4 if vertices.dtype == torch.float32 else ISO_VERTEX_PACKED
    if fragments is None:
        fragments = torch.empty((height, width), dtype=torch.int64, device=vertices.device)
    if rgba is None:
        rgba = torch.empty((height, width), dtype=torch.int32, device=vertices.device)
    cam = _Camera()
    m = np.ascontiguousarray(view_proj, np.float32).reshape(16)
    for k in range(16):
        cam.view_proj[k] = float(m[k])
    for k in range(3):
        cam.light[k] = float(light[k])
    cam.width, cam.height = int(width), int(height)
    st = _RenderStats()
    nx, ny, nz = dims
    nv = vertices.numel() // (4 if fmt == ISO_VERTEX_FLOAT4 else 2)
    rc = lib().iso_render(_ptr(vertices), fmt, _ptr(indices) if indices is not None else None, nv,
                          int(num_triangles), nx, ny, nz, ctypes.byref(cam), _ptr(fragments), _ptr(rgba) if rgba is not False else None,
                          ctypes.byref(st) if stats else None,
                          stream if stream is not None else _current_stream())
    _check(rc, "iso_render")
    return fragments, (rgba if rgba is not False else None), ({"drawn": st.drawn, "big": st.big} if stats else None)


def encode_field(field, rate, stream=None, out=None):
    """Encode a CUDA float32 tensor of shape (nz, ny, nx) on the GPU.
    Returns (bits uint64-as-int64 tensor (nb, rate), bmin, bmax) on the same
    device, written into `out` = (bits, bmin, bmax) when given (contiguous,
    of those shapes)."""
    import torch
    assert field.is_cuda and field.dtype == torch.float32 and field.is_contiguous()
    nz, ny, nx = field.shape
    nb = int(np.prod(block_dims((nx, ny, nz))))
    if out is not None:
        bits, bmin, bmax = out
        assert bits.shape == (nb, rate) and bmin.numel() == nb and bmax.numel() == nb
        assert bits.is_contiguous() and bmin.is_contiguous() and bmax.is_contiguous()
    else:
        bits = torch.empty((nb, rate), dtype=torch.int64, device=field.device)
        bmin = torch.empty(nb, dtype=torch.float32, device=field.device)
        bmax = torch.empty(nb, dtype=torch.float32, device=field.device)
    _check(lib().iso_encode_field(_ptr(field), nx, ny, nz, rate, _ptr(bits), _ptr(bmin), _ptr(bmax),
                                  stream if stream is not None else _current_stream()), "iso_encode_field")
    return bits, bmin, bmax


def active_blocks_static(bmin, bmax, dims, iso, ids=None, count=None, stream=None):
    """Active block ids for `iso` from device ranges, through the entry point
    that allocates nothing (iso_active_blocks_static: its scratch is a fixed
    device array inside the library).

    bmin, bmax  CUDA float32 tensors, contiguous, one value per block (at least
                nb = prod(block_dims(dims)) each), on the current device
    ids         CUDA int32 tensor, contiguous: room for ids.numel() ids (ids past
                that are dropped, while count still counts them)
    count       CUDA int32 tensor of at least one element

    When ids or count are omitted they are made here by torch, outside the
    library call.  Returns (ids, count).  After the stream has run, count[0]
    holds the number of active blocks (it may exceed ids.numel()), or -1
    (0xFFFFFFFF) when a device-side wait timed out, or -2 (0xFFFFFFFE) when a
    range is not a range (NaN, or min > max); ``static_count`` reads it and
    raises IsoError for the two failures.  The buffers are checked here
    because the C call cannot check lengths: a short or host buffer would be
    read or written out of bounds on the device."""
    import torch
    nx, ny, nz = dims
    nb = int(np.prod(block_dims(dims)))
    dev = torch.device("cuda", torch.cuda.current_device())
    if ids is None:
        ids = torch.empty(max(nb, 1), dtype=torch.int32, device=dev)
    if count is None:
        count = torch.empty(1, dtype=torch.int32, device=dev)
    for name, t, dtypes, need in (("bmin", bmin, (torch.float32,), nb), ("bmax", bmax, (torch.float32,), nb),
                                  ("ids", ids, (torch.int32,), 0), ("count", count, (torch.int32,), 1)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device != dev:
            raise ValueError(f"{name} must be a CUDA tensor on the current device")
        if not t.is_contiguous() or t.dtype not in dtypes:
            raise ValueError(f"{name} must be contiguous with dtype {dtypes[0]}")
        if t.numel() < need:
            raise ValueError(f"{name} holds {t.numel()} elements, needs {need}")
    _check(lib().iso_active_blocks_static(_ptr(bmin), _ptr(bmax), nx, ny, nz, ctypes.c_float(iso), _ptr(ids),
                                          ids.numel(), _ptr(count),
                                          stream if stream is not None else _current_stream()),
           "iso_active_blocks_static")
    return ids, count


STATIC_COUNT_TIMEOUT = 0xFFFFFFFF
STATIC_COUNT_CORRUPT = 0xFFFFFFFE


def static_count(count):
    """The block count an active_blocks_static call wrote (waits for its
    stream); IsoError(ISO_ERR_TIMEOUT) or IsoError(ISO_ERR_CORRUPT) for the
    two failure codes."""
    n = int(count[0].item()) & 0xFFFFFFFF
    if n == STATIC_COUNT_TIMEOUT:
        raise IsoError(ISO_ERR_TIMEOUT, "iso_active_blocks_static")
    if n == STATIC_COUNT_CORRUPT:
        raise IsoError(ISO_ERR_CORRUPT, "iso_active_blocks_static")
    return n


def decode_volume(bits, dims, rate, out=None, stream=None):
    """Decode a whole CUDA bitstream tensor into a dense float32 (nz, ny, nx) tensor."""
    import torch
    nx, ny, nz = dims
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=bits.device)
    _check(lib().iso_decode_volume(_ptr(bits), nx, ny, nz, rate, _ptr(out),
                                   stream if stream is not None else _current_stream()), "iso_decode_volume")
    return out


def mc_dense(field, iso, out=None, edge_ids=False, stream=None):
    """Naive data-parallel marching cubes over a dense CUDA float32 field of
    shape (nz, ny, nx) (iso_mc_dense).  Returns (vertices, stats, edges):
    vertices a (T, 3, 4) float32 view (of `out` when it is given and large
    enough, else a new tensor), stats a dict, edges the (T, 3) global edge ids
    (int64 tensor) when edge_ids is set, else None."""
    import torch
    nz, ny, nx = field.shape
    st = _DenseStats()
    strm = stream if stream is not None else _current_stream()

    def call(buf, cap, ebuf):
        return lib().iso_mc_dense(_ptr(field), nx, ny, nz, ctypes.c_float(iso), _ptr(buf), cap, _ptr(ebuf),
                                  ctypes.byref(st), strm)

    cap = 0 if out is None else out.numel() // 12
    ebuf = torch.empty((max(cap, 1), 3), dtype=torch.int64, device=field.device) if edge_ids else None
    rc = call(out if cap else None, cap, ebuf if cap else None)
    if rc == ISO_ERR_CAPACITY:
        cap = int(st.num_triangles)
        out = torch.empty((cap, 3, 4), dtype=torch.float32, device=field.device)
        ebuf = torch.empty((cap, 3), dtype=torch.int64, device=field.device) if edge_ids else None
        rc = call(out, cap, ebuf)
    _check(rc, "iso_mc_dense")
    T = int(st.num_triangles)
    verts = out.reshape(-1)[:12 * T].view(T, 3, 4) if T else torch.empty((0, 3, 4), device=field.device)
    edges = ebuf[:T] if (edge_ids and T) else (torch.empty((0, 3), dtype=torch.int64) if edge_ids else None)
    return verts, {"num_triangles": T, "n_active_cells": int(st.n_active_cells)}, edges


def decode_blocks(bits, rate, ids, stream=None):
    """Decode blocks `ids` (CUDA uint32-as-int32 tensor) of a CUDA bitstream tensor.
    Returns a (n, 64) float32 CUDA tensor."""
    import torch
    n = ids.numel()
    out = torch.empty((n, 64), dtype=torch.float32, device=bits.device)
    _check(lib().iso_decode_blocks(_ptr(bits), rate, _ptr(ids), n, _ptr(out),
                                   stream if stream is not None else _current_stream()), "iso_decode_blocks")
    return out
