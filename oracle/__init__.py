"""Plain, slow, CPU-only oracle for the isosurface method.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product library.  It shares
no code with the CUDA path.

The numerical parts are plain C (``oracle/codec.c``, ``oracle/mc.c``) loaded
through ctypes; the cache simulator below is NumPy and follows Algorithm 1
of the paper (Section 4.2) step by step, including the sort by age.

Parity status of each function (what pins it, see ``tests/test_oracle_*``):
  codec       constant blocks exact, zero blocks exact, error falls with
              rate, transform and negabinary identities, hand-built streams
  mc_table    brute force over all 256 cases (cut edges, face rule,
              pairing of interior edges, orientation)
  mc_full     plane closed form, sphere area and volume convergence,
              watertightness and Euler characteristic
  active      brute force: every block touched by a crossing cell is active
  mc_blocks   equals mc_full reordered by block
  raster      hand-enumerated coverage of small triangles (top-left rule
              on the shared and boundary edges), quads and fans covered
              exactly once, nearer and lower-id fragments win, a plane's
              depth equals the projection's closed form, points behind the
              camera dropped; shade: normal along / across the light
  raycast     hits on a plane and a sphere against the closed forms, every
              hit and miss against a fine float64 march over the trilinear
              interpolant (no block or cell skipped wrongly), shading by hand
  indexed_mesh  gathers back to the soup exactly; a block's vertices are
              the cut edges of its window found by brute force; welded over
              blocks, a sphere stays closed with Euler characteristic 2
  LRUCache    invariants of the cache on random and sweep sequences
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None
MAX_TRI = 12


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int, ctypes.c_int64
        L.orc_encode_block.argtypes = [P, i32, P]
        L.orc_decode_block.argtypes = [P, i32, P]
        L.orc_encode_volume.argtypes = [P, i32, i32, i32, i32, P, P, P]
        L.orc_decode_volume.argtypes = [P, i32, i32, i32, i32, P]
        L.orc_decode_blocks.argtypes = [P, i32, P, i64, P]
        L.orc_coding_order.argtypes = [P]
        L.orc_to_negabinary.argtypes = [i64]
        L.orc_to_negabinary.restype = ctypes.c_uint32
        L.orc_from_negabinary.argtypes = [ctypes.c_uint32]
        L.orc_from_negabinary.restype = ctypes.c_int32
        L.orc_forward_lift.argtypes = [P]
        L.orc_inverse_lift.argtypes = [P]
        L.orc_mc_table.argtypes = [P, P]
        L.orc_mc_table.restype = i32
        L.orc_edge_info.argtypes = [i32, P, P, P]
        L.orc_mc_full.argtypes = [P, i32, i32, i32, ctypes.c_float, P, P, P, i64]
        L.orc_mc_full.restype = i64
        L.orc_active_blocks.argtypes = [P, P, i32, i32, i32, ctypes.c_float, P]
        L.orc_mc_blocks.argtypes = [P, i32, i32, i32, ctypes.c_float, P, P, i64,
                                    P, P, P, P, P, P, P, P, i64]
        L.orc_mc_blocks.restype = i64
        L.orc_raster.argtypes = [P, i32, P, i64, i64, i32, i32, i32, P, i32, i32, P]
        L.orc_shade.argtypes = [P, i32, P, i32, i32, i32, P, i32, i32, P, P]
        L.orc_raycast.argtypes = [P, i32, i32, i32, ctypes.c_float, P, P, P, P, P, i32, i32, P, P]
        _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def block_dims(dims):
    nx, ny, nz = dims
    return (nx + 3) // 4, (ny + 3) // 4, (nz + 3) // 4


# ---------------------------------------------------------------- codec

def encode_block(values, rate):
    v = np.ascontiguousarray(values, dtype=np.float32).reshape(64)
    out = np.zeros(rate, dtype=np.uint64)
    lib().orc_encode_block(_p(v), rate, _p(out))
    return out


def decode_block(words, rate):
    w = np.ascontiguousarray(words, dtype=np.uint64).reshape(rate)
    out = np.zeros(64, dtype=np.float32)
    lib().orc_decode_block(_p(w), rate, _p(out))
    return out


def encode_volume(field, rate):
    """field: float32 (nz, ny, nx).  Returns (bits uint64 (nb, rate), bmin, bmax)."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    nb = int(np.prod(block_dims((nx, ny, nz))))
    bits = np.zeros((nb, rate), dtype=np.uint64)
    bmin = np.zeros(nb, dtype=np.float32)
    bmax = np.zeros(nb, dtype=np.float32)
    lib().orc_encode_volume(_p(f), nx, ny, nz, rate, _p(bits), _p(bmin), _p(bmax))
    return bits, bmin, bmax


def decode_volume(bits, dims, rate):
    nx, ny, nz = dims
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    out = np.zeros((nz, ny, nx), dtype=np.float32)
    lib().orc_decode_volume(_p(b), nx, ny, nz, rate, _p(out))
    return out


def decode_blocks(bits, rate, ids):
    b = np.ascontiguousarray(bits, dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint32)
    out = np.zeros((len(ids), 64), dtype=np.float32)
    lib().orc_decode_blocks(_p(b), rate, _p(ids), len(ids), _p(out))
    return out


def coding_order():
    perm = np.zeros(64, dtype=np.int32)
    lib().orc_coding_order(_p(perm))
    return perm


def to_negabinary(x):
    return int(lib().orc_to_negabinary(int(x)))


def from_negabinary(u):
    return int(lib().orc_from_negabinary(int(u) & 0xFFFFFFFF))


def forward_lift(q):
    a = np.ascontiguousarray(q, dtype=np.int64).reshape(64).copy()
    lib().orc_forward_lift(_p(a))
    return a


def inverse_lift(q):
    a = np.ascontiguousarray(q, dtype=np.int64).reshape(64).copy()
    lib().orc_inverse_lift(_p(a))
    return a


# ---------------------------------------------------------------- marching cubes

def mc_table():
    num = np.zeros(256, dtype=np.uint8)
    tri = np.zeros((256, 3 * MAX_TRI), dtype=np.uint8)
    m = lib().orc_mc_table(_p(num), _p(tri))
    return num, tri, int(m)


def edge_info(e):
    lo, hi, a = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    lib().orc_edge_info(e, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(a))
    return lo.value, hi.value, a.value


def mc_full(field, iso, return_cells=False):
    """Plain marching cubes over every cell (z, y, x order).
    Returns (edge_ids uint64 (T, 3), positions float64 (T, 3, 3) global)
    and, if asked, the linear index of each triangle's cell."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    L = lib()
    t = L.orc_mc_full(_p(f), nx, ny, nz, float(iso), None, None, None, 0)
    ids = np.zeros((t, 3), dtype=np.uint64)
    pos = np.zeros((t, 3, 3), dtype=np.float64)
    cells = np.zeros(t, dtype=np.int64)
    L.orc_mc_full(_p(f), nx, ny, nz, float(iso), _p(ids), _p(pos), _p(cells), t)
    return (ids, pos, cells) if return_cells else (ids, pos)


def active_blocks(bmin, bmax, nbdims, iso):
    nbx, nby, nbz = nbdims
    out = np.zeros(nbx * nby * nbz, dtype=np.uint8)
    lib().orc_active_blocks(_p(np.ascontiguousarray(bmin, np.float32)),
                            _p(np.ascontiguousarray(bmax, np.float32)), nbx, nby, nbz, float(iso), _p(out))
    return out.astype(bool)


def mc_blocks(field, iso, active):
    """Block-ordered marching cubes over the active blocks (Sections 4.3-4.5)."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    nz, ny, nx = f.shape
    act = np.ascontiguousarray(active, dtype=np.uint8)
    ids = np.nonzero(act)[0].astype(np.uint32)
    n = len(ids)
    cases = np.zeros((n, 64), np.uint8)
    counts = np.zeros((n, 64), np.uint8)
    complete = np.zeros(n, np.uint8)
    btri = np.zeros(n, np.uint32)
    boff = np.zeros(n, np.uint64)
    L = lib()
    args = [_p(f), nx, ny, nz, float(iso), _p(act), _p(ids), n, _p(cases), _p(counts), _p(complete),
            _p(btri), _p(boff)]
    t = L.orc_mc_blocks(*args, None, None, None, 0)
    eids = np.zeros((t, 3), np.uint64)
    lpos = np.zeros((t, 3, 3), np.float64)
    tblk = np.zeros(t, np.uint32)
    L.orc_mc_blocks(*args, _p(eids), _p(lpos), _p(tblk), t)
    return dict(ids=ids, cases=cases, counts=counts, complete=complete.astype(bool),
                block_tri=btri, block_off=boff, edge_ids=eids, local_pos=lpos, tri_block=tblk,
                num_triangles=int(t))


def extract(bits, dims, rate, bmin, bmax, iso):
    """The whole method on the CPU: decode every block, select active blocks
    by the block ranges, then block-ordered marching cubes."""
    field = decode_volume(bits, dims, rate)
    act = active_blocks(bmin, bmax, block_dims(dims), iso)
    out = mc_blocks(field, iso, act)
    out["active"] = act
    out["field"] = field
    return out


def quantized_vertices(field, iso, edge_ids, tri_block, dims):
    """The compact vertex format (Section 4.5, 8 bytes a vertex): for every
    vertex of the block-ordered triangles, the 10-bit codes of its block-local
    coordinates and its block id, packed as (qx | qy << 10 | qz << 20, id).

    Each vertex lies on the cut edge given by its global edge id
    (3 * (x + nx*(y + ny*z)) + axis of the lower sample).  The code of a
    coordinate p in [0, 4] is round(p / 4 * 1023); because rounding decides
    an integer, the position is taken in float32 with one IEEE rounding per
    operation: t = (iso - v_lo) / (v_hi - v_lo), p = lower corner + t, and
    q = the nearest integer (ties to even) to p * 255.75.  When
    |v_hi - v_lo| is 2^125 or more (samples near +-FLT_MAX, where the float32
    difference can overflow to infinity), both differences are taken of the
    samples times 2^-4, which leaves the quotient's real value unchanged
    (scaling samples that small differences is exact, and the tiny ones it
    rounds are far below the difference)."""
    f = np.ascontiguousarray(field, np.float32)
    nx, ny, nz = dims
    e = np.asarray(edge_ids, np.uint64).reshape(-1)
    axis = (e % 3).astype(np.int64)
    lin = (e // 3).astype(np.int64)
    x, y, z = lin % nx, (lin // nx) % ny, lin // (nx * ny)
    vlo = f[z, y, x]
    vhi = f[z + (axis == 2), y + (axis == 1), x + (axis == 0)]
    iso32 = np.float32(iso)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        a, b = iso32 - vlo, vhi - vlo                      # float32 operations
        big = ~(np.abs(b) < np.float32(2.0 ** 125))        # includes an overflow to infinity
        s = np.float32(2.0 ** -4)
        a = np.where(big, iso32 * s - vlo * s, a).astype(np.float32)
        b = np.where(big, vhi * s - vlo * s, b).astype(np.float32)
        t = a / b
    blk = np.repeat(np.asarray(tri_block, np.int64), 3)
    nbx, nby, _ = block_dims(dims)
    bx, by, bz = blk % nbx, (blk // nbx) % nby, blk // (nbx * nby)
    codes = np.zeros(len(e), np.uint32)
    for k, (c, b) in enumerate(((x, bx), (y, by), (z, bz))):
        p = (c - 4 * b).astype(np.float32)                 # block-local lower corner (exact)
        p = np.where(axis == k, p + t, p).astype(np.float32)
        q = np.rint(p * np.float32(255.75)).astype(np.uint32)
        codes |= q << np.uint32(10 * k)
    out = np.stack([codes, blk.astype(np.uint32)], axis=1)
    return out.reshape(-1, 3, 2)


def indexed_mesh(edge_ids, tri_block, local_pos):
    """The within-block indexed mesh (Section 4.5 names it as the
    alternative to the triangle soup: vertices shared inside each block) of
    a block-ordered soup.

    A block's vertices are the distinct edges its triangles use, ordered by
    axis (x-edges, then y-, then z-edges) and, within an axis, by the
    edge's lower sample (x fastest); blocks follow the soup's (ascending)
    block order; a triangle corner becomes the index of its (block, edge)
    vertex.  Global edge id = 3 * (x + nx*(y + ny*z)) + axis.  Returns a
    dict: vertex_edge (V,) uint64, vertex_block (V,) uint32, vertex_pos
    (V, 3) float64 block-local (the position of the vertex's first corner
    in the soup), indices (T, 3) int64."""
    e = np.asarray(edge_ids, np.uint64).reshape(-1)
    blk = np.repeat(np.asarray(tri_block, np.uint64), 3)
    pos = np.asarray(local_pos, np.float64).reshape(-1, 3)
    if len(e) == 0:
        return dict(vertex_edge=np.zeros(0, np.uint64), vertex_block=np.zeros(0, np.uint32),
                    vertex_pos=np.zeros((0, 3)), indices=np.zeros((0, 3), np.int64))
    keys = np.stack([blk, e % np.uint64(3), e // np.uint64(3)], axis=1)     # sorted lexicographically
    uniq, first, inv = np.unique(keys, axis=0, return_index=True, return_inverse=True)
    return dict(vertex_edge=uniq[:, 2] * np.uint64(3) + uniq[:, 1], vertex_block=uniq[:, 0].astype(np.uint32),
                vertex_pos=pos[first], indices=inv.reshape(-1, 3).astype(np.int64))


# ---------------------------------------------------------------- rendering (Section 4.6.2)

def _vertex_buffer(vertices):
    """(array, format): float32 (V, 4) -> format 0; uint32/int32 (V, 2) -> 1."""
    v = np.ascontiguousarray(vertices)
    if v.dtype == np.float32:
        return v.reshape(-1, 4), 0
    return v.view(np.uint32).reshape(-1, 2), 1


def raster(vertices, indices, num_triangles, dims, view_proj, width, height):
    """Visible fragment of every pixel (oracle/raster.c states the rules):
    uint64 (height, width), (depth bits << 32) | triangle, all ones where
    nothing is drawn.  `vertices` float32 (V, 4) block-local + block id bits
    or uint32 (V, 2) compact; `indices` None for a soup (vertex 3t + j) or
    uint32 (T, 3) (a triangle with an index past the vertices is not
    drawn); view_proj row-major 4x4 float32."""
    v, fmt = _vertex_buffer(vertices)
    idx = None if indices is None else np.ascontiguousarray(indices, np.uint32)
    m = np.ascontiguousarray(view_proj, np.float32).reshape(16)
    out = np.zeros((height, width), np.uint64)
    nx, ny, nz = dims
    lib().orc_raster(_p(v), fmt, _p(idx), len(v), int(num_triangles), nx, ny, nz, _p(m), width, height, _p(out))
    return out


def shade(vertices, indices, dims, light, frag):
    """RGBA8 (as uint32, r in the low byte) of each pixel of a fragment
    buffer from raster()."""
    v, fmt = _vertex_buffer(vertices)
    idx = None if indices is None else np.ascontiguousarray(indices, np.uint32)
    f = np.ascontiguousarray(frag, np.uint64)
    h, w = f.shape
    out = np.zeros((h, w), np.uint32)
    l3 = np.ascontiguousarray(light, np.float32).reshape(3)
    nx, ny, nz = dims
    lib().orc_shade(_p(v), fmt, _p(idx), nx, ny, nz, _p(l3), w, h, _p(f), _p(out))
    return out


def raycast(field, iso, eye, forward, right, up, light, width, height):
    """Implicit isosurface ray casting over the block macrocell grid
    (oracle/raycast.c states the rules).  field float32 (nz, ny, nx), the
    decoded volume.  Returns (hits uint64 (height, width): t bits << 32 |
    block id of the first hit, all ones for none; rgba uint32 (height,
    width))."""
    f = np.ascontiguousarray(field, np.float32)
    nz, ny, nx = f.shape
    vec = [np.ascontiguousarray(x, np.float32).reshape(3) for x in (eye, forward, right, up, light)]
    hits = np.zeros((height, width), np.uint64)
    rgba = np.zeros((height, width), np.uint32)
    lib().orc_raycast(_p(f), nx, ny, nz, float(iso), *[_p(x) for x in vec], width, height, _p(hits), _p(rgba))
    return hits, rgba


# ---------------------------------------------------------------- cache (Algorithm 1)

class OverBudget(RuntimeError):
    pass


class LRUCache:
    """GPU-driven LRU block cache of Section 4.2, simulated on the CPU.

    State as in the paper: S_age, S_block (-1 = empty), I_slot (-1 = not
    cached) and the persistent availability mask M_avail.  `update` runs
    the steps of Algorithm 1 in order.  Readings of points the paper leaves
    open: slots start available with age 0 and age once per update, so a
    never-used slot is as old as the number of updates so far; slots added
    by growth get that same age ("a high age"); the sort by age is stable,
    so equal ages keep ascending slot order; growth is to
    max(2S, S + n_new - n_avail), capped at `max_slots`.
    """

    def __init__(self, n_blocks, initial_slots, max_slots):
        self.max_slots = int(max_slots)
        s = int(min(initial_slots, max_slots))
        self.S_age = np.zeros(s, np.int64)
        self.S_block = np.full(s, -1, np.int64)
        self.M_avail = np.ones(s, bool)
        self.I_slot = np.full(n_blocks, -1, np.int64)
        self.updates = 0

    @property
    def num_slots(self):
        return len(self.S_age)

    def update(self, M_active):
        M_active = np.asarray(M_active, bool)
        self.updates += 1
        # IncrementSlotAge
        self.S_age += 1
        # MarkNewBlocks
        cached = self.I_slot >= 0
        hit = M_active & cached
        M_new = M_active & ~cached
        self.S_age[self.I_slot[hit]] = 0
        self.M_avail[self.I_slot[hit]] = False
        self.M_avail[self.I_slot[cached & ~M_active]] = True
        # PrefixSum over M_new and M_avail
        n_new = int(M_new.sum())
        n_avail = int(self.M_avail.sum())
        if n_new == 0:
            return np.zeros(0, np.int64), np.zeros(0, np.int64)
        if n_new > n_avail:
            S = self.num_slots
            grow_to = min(self.max_slots, max(2 * S, S + n_new - n_avail))
            if n_new > n_avail + grow_to - S:
                raise OverBudget(f"{n_new} new blocks, {n_avail} free slots, cap {self.max_slots}")
            extra = grow_to - S
            self.S_age = np.concatenate([self.S_age, np.full(extra, self.updates, np.int64)])
            self.S_block = np.concatenate([self.S_block, np.full(extra, -1, np.int64)])
            self.M_avail = np.concatenate([self.M_avail, np.ones(extra, bool)])
        # StreamCompactIDs / StreamCompact
        I_new = np.nonzero(M_new)[0]
        I_avail = np.nonzero(self.M_avail)[0]
        K_age = self.S_age[I_avail]
        # SortByKey: descending age
        I_avail = I_avail[np.argsort(-K_age, kind="stable")]
        # AssignSlots
        s = I_avail[:n_new]
        evicted = self.S_block[s]
        self.I_slot[evicted[evicted >= 0]] = -1
        self.S_block[s] = I_new
        self.I_slot[I_new] = s
        self.M_avail[s] = False
        self.S_age[s] = 0
        return I_new, s

    def last_use(self):
        """Update index at which each slot was last used (0 = never)."""
        return self.updates - self.S_age
