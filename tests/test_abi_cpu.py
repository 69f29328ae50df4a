"""CPU-side checks of the C ABI: the library builds, loads without a GPU,
exports every function include/bcmc.h declares, and its host-built case
table equals the oracle's table (two independent generators of the same
face rule)."""
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2009_03254_gb300 import build
    build.build()
    import paper_2009_03254_gb300 as pkg
    return pkg.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "bcmc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(iso_[a-z_]+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    names = declared_functions()
    for required in ("iso_load_volume", "iso_extract", "iso_release"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_error_strings(L):
    import paper_2009_03254_gb300 as pkg
    assert pkg.error_string(0) == "ok"
    codes = (pkg.ISO_ERR_INVALID_ARG, pkg.ISO_ERR_OOM, pkg.ISO_ERR_BUDGET, pkg.ISO_ERR_CUDA, pkg.ISO_ERR_TIMEOUT,
             pkg.ISO_ERR_CAPACITY, pkg.ISO_PENDING, pkg.ISO_ERR_CORRUPT, pkg.ISO_ERR_BOUNDS)
    texts = [pkg.error_string(code) for code in codes]
    assert all(t not in ("ok", "unknown status") for t in texts)
    assert len(set(texts)) == len(texts)                 # each code has its own message
    assert pkg.error_string(99) == "unknown status"
    # the binding's constants are the header's
    header = open(os.path.join(ROOT, "include", "bcmc.h")).read()
    for name in ("ISO_ERR_INVALID_ARG", "ISO_ERR_OOM", "ISO_ERR_BUDGET", "ISO_ERR_CUDA", "ISO_ERR_TIMEOUT",
                 "ISO_ERR_CAPACITY", "ISO_PENDING", "ISO_ERR_CORRUPT", "ISO_ERR_BOUNDS"):
        assert f"#define {name} {getattr(pkg, name)} " in header, name


def test_library_table_equals_oracle_table(L):
    import paper_2009_03254_gb300 as pkg
    num, tri = pkg.mc_case_table()
    onum, otri, omax = oracle.mc_table()
    assert omax == 5
    assert np.array_equal(num, onum)
    for cs in range(256):
        n = int(num[cs])
        assert np.array_equal(tri[cs, :3 * n], otri[cs, :3 * n]), cs


def test_checked_build_compiles_and_exports_the_same_calls():
    # the bounds-checked variant of the library (BCMC_CHECKED) keeps building
    # and exports every call the header declares
    import ctypes
    from paper_2009_03254_gb300 import build
    lib = build.build(checked=True)
    assert os.path.exists(lib) and "_lib_checked" in lib
    L = ctypes.CDLL(lib)
    for name in declared_functions():
        assert hasattr(L, name), name


def test_arguments_refused_before_any_device_work(L):
    # argument rules of the boundary that need no GPU: every case below is
    # refused by host arithmetic before the first CUDA call, so it runs on
    # any machine (and never allocates)
    import ctypes
    import paper_2009_03254_gb300 as pkg
    bad = pkg.ISO_ERR_INVALID_ARG
    dummy = np.zeros(64, dtype=np.uint64)
    rng = np.zeros(64, dtype=np.float32)
    p_bits, p_rng = ctypes.c_void_p(dummy.ctypes.data), ctypes.c_void_p(rng.ctypes.data)

    def load(dims, rate, nbytes, bits=p_bits, lo=p_rng, hi=p_rng, out=True):
        h = ctypes.c_void_p()
        return L.iso_load_volume(ctypes.byref(h) if out else None, bits, nbytes, *dims, rate, lo, hi, None)

    def size_of(dims, rate):
        nb = ((dims[0] + 3) // 4) * ((dims[1] + 3) // 4) * ((dims[2] + 3) // 4)
        return nb * rate * 8

    ok_dims = (8, 8, 8)
    for rate in (0, 33, 64):                                     # rate_bits outside [1, 32]
        assert load(ok_dims, rate, size_of(ok_dims, 4)) == bad
    for dims in ((0, 8, 8), (8, 0, 8), (8, 8, 0)):               # a dimension of 0
        assert load(dims, 4, 0) == bad
    # 2^31 blocks (2048 x 1024 x 1024): ids and packed counters are 31-bit
    big = (4 * 2048, 4 * 1024, 4 * 1024)
    assert load(big, 1, size_of(big, 1)) == bad
    big_ragged = (4 * 2048 - 3, 4 * 1024 - 3, 4 * 1024 - 3)     # the same block grid, partial blocks
    assert load(big_ragged, 1, size_of(big_ragged, 1)) == bad
    # a bitstream whose size is not nb * R * 8 bytes
    for nbytes in (size_of(ok_dims, 4) - 8, size_of(ok_dims, 4) + 8, 0):
        assert load(ok_dims, 4, nbytes) == bad
    # missing pointers
    n = size_of(ok_dims, 4)
    assert load(ok_dims, 4, n, bits=None) == bad
    assert load(ok_dims, 4, n, lo=None) == bad
    assert load(ok_dims, 4, n, hi=None) == bad
    assert load(ok_dims, 4, n, out=False) == bad
    # calls on no volume
    m = pkg._Mesh()
    assert L.iso_extract(None, ctypes.c_float(0.0), ctypes.byref(m)) == bad
    st = pkg._Stats()
    assert L.iso_extract_into(None, ctypes.c_float(0.0), None, 0, ctypes.byref(st)) == bad
    # the dense decoder: no input, or a block grid past 2^31 blocks
    assert L.iso_decode_volume(None, 8, 8, 8, 4, p_bits, None) == bad
    assert L.iso_decode_volume(p_bits, *big, 1, p_bits, None) == bad
