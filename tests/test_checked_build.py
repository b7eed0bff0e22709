"""The bounds-checked debug build (libh3dgs_check.so, compiled with -DH3DGS_CHECK) on the small parity
cases: the forward and adjoint tests of the tiny scenes run in a child process that loads that build.

Every index the cut, preprocess, sort, blend and adjoint kernels take from data (parent and cut ids,
list entries, radix staging slots and scatter destinations, work items) is range-checked there before
its access; a failure skips the access, never traps, and sets bit 7 of the device flags, which the
parity helpers assert clear (tests/gpu_path.py, tests/test_parity_backward.py).  This stands in for a
memory checker, which does not run on these GPUs.  The child's results must also still match the
oracle, since the checked build runs the same arithmetic.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_loaded_library_reports_its_build():
    """In the child (H3DGS_LIB set) the checked build is loaded; in a plain run the default build."""
    from paper_2406_12080_b300 import build, h3dgs
    want_checked = os.environ.get("H3DGS_LIB") == build.LIB_CHECK
    assert h3dgs.h3dgs_build_flags() == (1 if want_checked else 0)


def test_small_parity_cases_under_the_checked_build():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_12080_b300 import build
    lib = build.build(check=True)
    env = {**os.environ, "H3DGS_LIB": lib}
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
           "tests/test_checked_build.py::test_loaded_library_reports_its_build",
           "tests/test_parity_forward.py", "tests/test_parity_backward.py",
           "-k", "not full_size and not twenty_thousand and not under_the_checked_build"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and "failed" not in r.stdout, tail
