"""GPU parity of the Lagrange and pp-spline variants against the FP64 oracle, and the
paper's statement that interpolating B-splines and pp-splines give identical values."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, gpu_eval, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("n_orb", [1, 5, 24])
def test_lagrange_ragged_nonorthogonal(storage, n_orb):
    """Eq. (lagrangeinterpolation3) over the five tables of Sec. III C."""
    dims = (9, 10, 12)
    lat, mil, coef = inputs.random_cell(300 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="lagrange", storage=storage)
    tabs = oracle.lagrange_tables(lat, mil, coef, dims)
    for k in range(5):
        tol = {"f64": 1e-13, "f32": 1e-7, "bf16": 8e-3}[storage]
        assert oracle.relative_error(spl.get_table(k), tabs[k]) <= tol
    pos = np.vstack([inputs.positions(lat, 257, 1), inputs.positions(lat, 40, 2, -2.0, 3.0)])
    ref = oracle.lagrange_eval(rounded(tabs, storage), lat, pos)
    assert_parity(gpu_eval(spl, pos), ref, TOL[storage], "lagrange/%s/O=%d" % (storage, n_orb))


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("n_orb", [1, 5, 24])
def test_pp_ragged_nonorthogonal(storage, n_orb):
    """Eq. (pp-splineinterpolation3): 8 coefficients per grid point, 2x2x2 corners."""
    dims = (9, 10, 12)
    lat, mil, coef = inputs.random_cell(400 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="pp", storage=storage)
    sig = oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims))
    for e in range(8):
        tol = {"f64": 1e-12, "f32": 1e-7, "bf16": 8e-3}[storage]
        assert oracle.relative_error(spl.get_table(e), sig[e]) <= tol, e
    info = spl.info()
    assert info["entries_per_point"] == 8 and info["rows_z"] == dims[2] + 1
    pos = np.vstack([inputs.positions(lat, 257, 3), inputs.positions(lat, 40, 4, -2.0, 3.0)])
    ref = oracle.pp_eval(rounded(sig, storage), lat, pos)
    assert_parity(gpu_eval(spl, pos), ref, TOL[storage], "pp/%s/O=%d" % (storage, n_orb))


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_c2_variants_same_inputs(storage):
    """The Si-like 48^3 cell with Lagrange and pp on the same coefficients (2048 of the
    1024 x 32 positions)."""
    w = inputs.make_workload("c2", n_pos=2048)
    dims = w.cell.grid
    lg = splines(w.lattice, dims, w.miller, w.coef, method="lagrange", storage=storage)
    ref = oracle.lagrange_eval(rounded(oracle.lagrange_tables(w.lattice, w.miller, w.coef, dims), storage),
                               w.lattice, w.pos)
    assert_parity(gpu_eval(lg, w.pos), ref, TOL[storage], "c2 lagrange")
    pp = splines(w.lattice, dims, w.miller, w.coef, method="pp", storage=storage)
    sig = oracle.pp_tables(oracle.grid_values(w.lattice, w.miller, w.coef, dims))
    assert_parity(gpu_eval(pp, w.pos), oracle.pp_eval(rounded(sig, storage), w.lattice, w.pos),
                  TOL[storage], "c2 pp")


def test_interpolating_bspline_equals_pp_on_gpu():
    """Sec. II / III A: interpolating B-splines and pp-splines yield identical functions."""
    dims = (10, 11, 12)
    lat, mil, coef = inputs.random_cell(9, dims, 6, 6.0, 5.0, NONORTHO)
    pos = inputs.positions(lat, 500, 5, -1, 2)
    b = gpu_eval(splines(lat, dims, mil, coef, method="interp", storage="f64", separate_lap=False), pos)
    p = gpu_eval(splines(lat, dims, mil, coef, method="pp", storage="f64"), pos)
    assert_parity(p, b, 1e-11, "interp vs pp")
