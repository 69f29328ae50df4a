"""The checked build runs the parity tests clean.

The checked build (BCMC_CHECKED, `build(checked=True)`) tests on the device
every guarded index of the hot path before its access: block ids against
the block count, slots against the slot capacity, list positions against
the list capacity (the +group slot lookups, the halo staging, the decode's
block and slot, the cache update's assignments and lists, the cases, cut
words and compacted occupied list).  A failed test skips the access and
the call returns ISO_ERR_BOUNDS, so an indexing defect shows up as an error
instead of a memory fault.  Here a child process loads that library
(BCMC_CHECKED=1) and runs a cross-section of the GPU parity tests: every
result must still match the oracle and no check may fail.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_parity_clean():
    sys.path.insert(0, ROOT)
    from paper_2009_03254_gb300 import build
    lib = build.build(checked=True)
    assert lib.endswith(os.path.join("_lib_checked", "libbcmc.so"))
    env = dict(os.environ, BCMC_CHECKED="1")
    probe = subprocess.run([sys.executable, "-c", "import paper_2009_03254_gb300 as p; p.lib(); print(p.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0, probe.stderr[-2000:]
    assert "_lib_checked" in probe.stdout
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "-k",
           "extract_matches_oracle or cache_matches_algorithm1 or capped_cache or over_budget or launch_shapes "
           "or packed_vertices or decode_blocks_bit_exact",
           "tests/test_gpu_indexed.py", "tests/test_gpu_batch.py", "tests/test_gpu_serve.py"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
