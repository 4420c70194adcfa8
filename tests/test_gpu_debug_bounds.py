"""The FE_DEBUG_BOUNDS build (libfe_dbg.so) on valid inputs.

In that build the kernels check their indirect indices -- SpMV and V-cycle
columns, restriction and prolongation indices, the residual gather lists,
the tangent scatter map -- and an index outside its array raises a device
flag that every call turns into FE_ERR_DEVICE_FLAG (the access is redirected
to entry 0, so nothing outside the arrays is touched).  A part of the
parity suite runs against that build in a child process: every call must
succeed, i.e. no check fires on the library's own valid inputs.  No test
feeds an out-of-range index to a kernel.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SUBSET = [
    "tests/test_gpu_parity.py::test_residual_and_energy",
    "tests/test_gpu_parity.py::test_tangent_fp64",
    "tests/test_gpu_parity.py::test_gmres",
    "tests/test_gpu_parity.py::test_nl_solve_fp64",
    "tests/test_gpu_amg.py::test_vcycle_matches_the_oracle",
    "tests/test_gpu_amg.py::test_nl_solve_with_amg",
]


def test_debug_bounds_build_runs_the_parity_subset_clean():
    pytest.importorskip("torch")
    from paper_2203_05610_gb300 import build as B
    so = B.build(debug_bounds=True)
    env = dict(os.environ, FE_LIB_VARIANT="debug_bounds")
    probe = subprocess.run([sys.executable, "-c", "import paper_2203_05610_gb300 as fe; print(fe.SO_PATH)"],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert probe.returncode == 0 and probe.stdout.strip() == so, probe.stdout + probe.stderr
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", *SUBSET],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "failed" not in r.stdout
