"""The GPU suite against the checked build of the library.

compute-sanitizer is not available where these tests run, so the library
has a checked build (paper_2603_19764_b300.build(checked=True), compiled
with -DSPH_BOUNDS_CHECK): before every access whose index comes from data --
cell ranges, sort positions, the candidate lists and their overflow region,
the permutation, the active-particle list -- the index is tested against its
array, and a failed test is latched in the status word and reported as
SPH_E_INTERNAL by the synchronising call (the access is redirected to index
0, so nothing faults). Every other GPU test runs here once more in a child
process that loads the checked build (SPH_CHECKED=1): all of them passing
means that no such index left its array on any of their inputs (tiny,
ragged, coincident, periodic, batched, hierarchical, full-size)."""
import os
import subprocess
import sys

import pytest

from paper_2603_19764_b300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_suite_passes_on_the_checked_build():
    lib = build.build(checked=True)
    env = dict(os.environ, SPH_CHECKED="1")
    which = subprocess.run([sys.executable, "-c",
                            "from paper_2603_19764_b300 import sph; print(sph.LIB_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert which.stdout.strip() == lib
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-q", "-x",
                        "-k", "not checked_build and not fma_peak"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "SPH_E_INTERNAL" not in r.stdout, tail
