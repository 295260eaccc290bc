"""The library's general B-spline basis (csrc/general_basis.cuh, the weights of the degree-n and
graded-grid kernels and of their adjoint) compiled for the host: every derivative order up to
the third equals central differences of the order below, on uniform and on graded knots, and
the non-uniform routine on evenly spaced knots equals the uniform one (derivatives scaled by
the grid size).  Pins the third-derivative weights the adjoint uses without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_basis_derivatives_on_the_host(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "basis_probe")
    src = os.path.join(ROOT, "tests", "basis_probe.cpp")
    inc = os.path.join(ROOT, "paper_1309_6250_gb300", "csrc")
    subprocess.run([gxx, "-std=c++17", "-O2", "-Wno-unknown-pragmas", "-I", inc, src, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    rows = [list(map(float, line.split())) for line in out if line.strip()]
    assert [int(r[0]) for r in rows] == [1, 3, 5, 7]
    for deg, u1, u2, u3, n1, n2, n3, same, d3scale in rows:
        assert u1 < 1e-8 and u2 < 1e-8 and u3 < 1e-8, (deg, u1, u2, u3)
        assert n1 < 1e-6 and n2 < 1e-6 and n3 < 1e-6, (deg, n1, n2, n3)
        assert same < 1e-9, (deg, same)
        if deg >= 3:
            assert d3scale > 0.1          # the third derivative is not identically zero
        else:
            assert d3scale == 0.0
