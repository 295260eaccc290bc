"""The bounds-checked build (QMCSPL_DEBUG_BOUNDS, a stand-in for a memory sanitizer, which is
not available for these runs): every table load and every position index of
the kernels is range checked, a bad one is recorded in the error word and skipped.  The GPU
parity suites run again against that build in a subprocess; their sync() calls would report
any flagged access as QMCSPL_ERR_DEVICE."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SUITES = ["tests/test_parity_bspline.py", "tests/test_parity_variants.py", "tests/test_parity_limits.py",
          "tests/test_parity_bloch.py", "tests/test_parity_general.py", "tests/test_parity_separate_grad.py",
          "tests/test_parity_order_batched.py", "tests/test_parity_backward.py", "tests/test_parity_staged.py"]


def test_parity_suites_under_the_bounds_checked_build():
    from paper_1309_6250_gb300 import build
    lib = build.build(debug_bounds=True)
    env = dict(os.environ, QMCSPL_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu",
                        "-p", "no:cacheprovider", *SUITES], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=1800)
    tail = "\n".join(r.stdout.strip().splitlines()[-15:])
    assert r.returncode == 0, tail
    assert " passed" in tail
