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
