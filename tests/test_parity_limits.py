"""GPU path at the limits of its index arithmetic and at the degenerate inputs of the method,
against the oracle: a grid axis of the maximum 512 points, positions exactly on grid points
and cell faces and just below s = 1 (where N s rounds up to N and the cell index must wrap),
a large ragged orbital count, a constant orbital (a single G = 0 planewave), and the same
positions through input order, cell order, every storage type and the record/no-record
paths."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, oracle_tables, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def boundary_positions(lat, dims):
    """Grid points, cell faces, s = 1 - 2^-53 and s = -0.0, in crystal coordinates."""
    rng = np.random.default_rng(1500)
    s = []
    for _ in range(40):
        idx = rng.integers(0, dims)
        s.append(idx / np.array(dims, dtype=float))                       # grid points
    one_minus = np.nextafter(1.0, 0.0)
    s += [[one_minus, one_minus, one_minus], [0.0, one_minus, 0.5], [-0.0, 0.25, one_minus],
          [1.0, 2.0, -3.0], [0.5 / dims[0], 0.5, 0.5]]
    s = np.array(s)
    return np.ascontiguousarray(s @ np.asarray(lat).T)


@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
def test_maximum_grid_axis_and_boundary_positions(storage):
    dims = (512, 5, 4)
    lat = np.diag([40.0, 3.0, 2.5])
    mil = inputs.miller_set(lat, 3.5)
    mil = mil[np.all(np.abs(mil[:, 1:]) <= 1, axis=1)]             # keep the short axes resolved
    coef = inputs.pw_coefficients(lat, mil, 3, 6.0, 1501)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    beta, blap = oracle_tables(lat, mil, coef, dims, "smooth", storage, True)
    pos = boundary_positions(lat, dims)
    got = gpu_eval(spl, pos)
    ref = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
    assert_parity(got, ref, TOL[storage], "512 axis " + storage)
    # the same positions with records (>= 8192 positions) and in cell order
    many = np.concatenate([pos] * 200)
    for order in ("input", "cell"):
        spl.set_order(order)
        v, g, l = gpu_eval(spl, many)
        assert_parity((v[:pos.shape[0]], g[:pos.shape[0]], l[:pos.shape[0]]), ref, TOL[storage],
                      "512 axis records/%s/%s" % (order, storage))
    spl.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_large_ragged_orbital_count(storage):
    """301 orbitals: 76 FP32 chunks (or 38 BF16 chunks) split over lanes and tiles with a
    ragged last chunk."""
    dims = (10, 11, 12)
    lat, mil, coef = inputs.random_cell(1502, dims, 301, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=False)
    inf = spl.info()
    assert inf["n_orb_padded"] > 301
    pos = inputs.positions(lat, 200, 1503, -1, 2)
    got = gpu_eval(spl, pos)
    beta, _ = oracle_tables(lat, mil, coef, dims, "smooth", storage, False)
    ref = oracle.bspline_eval(beta, lat, pos)
    assert_parity(got, ref, TOL[storage], "301 orbitals " + storage)


@pytest.mark.parametrize("method", ["smooth", "interp", "lagrange", "pp"])
def test_constant_orbital(method):
    """A single G = 0 planewave is a constant orbital: every method reproduces the constant
    with zero gradient and Laplacian (the smoothing spline exactly, since gamma_0 = 27/8 and
    the weights sum to (3/2)^3)."""
    dims = (6, 7, 8)
    lat = NONORTHO
    mil = np.zeros((1, 3), dtype=np.int32)
    coef = np.array([[2.5 + 0.0j]])
    spl = splines(lat, dims, mil, coef, method=method, storage="f64", separate_lap=True)
    pos = inputs.positions(lat, 50, 1504, -2, 3)
    v, g, l = gpu_eval(spl, pos)
    assert np.abs(v - 2.5).max() < 1e-13
    assert np.abs(g).max() < 1e-12 and np.abs(l).max() < 1e-11


@pytest.mark.parametrize("dims", [(4, 4, 4), (5, 6, 7)])
@pytest.mark.parametrize("method,storage,sep", [("smooth", "f64", True), ("smooth", "f32", False),
                                                ("interp", "bf16", True), ("interp", "df64", False),
                                                ("lagrange", "f32", True), ("pp", "f64", False)])
def test_tiny_grids_every_method(dims, method, storage, sep):
    """The smallest grids accepted (4 points per axis), where every stencil wraps and the
    ghost planes repeat the same planes; positions inside and far outside the cell, with
    and without records and cell order."""
    lat, mil, coef = inputs.random_cell(1510, dims, 5, 2.0, 3.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=sep)
    tabs = oracle_tables(lat, mil, coef, dims, method, storage, sep)
    pos = inputs.positions(lat, 60, 1511, -3, 4)
    if method in ("smooth", "interp"):
        ref = oracle.bspline_eval(tabs[0], lat, pos, beta_lap=tabs[1])
    elif method == "lagrange":
        ref = oracle.lagrange_eval(tabs, lat, pos)
    else:
        ref = oracle.pp_eval(tabs, lat, pos)
    assert_parity(gpu_eval(spl, pos), ref, TOL[storage], "tiny %s %s/%s" % (dims, method, storage))
    many = np.concatenate([pos] * 150)
    spl.set_order("cell")
    v, g, l = gpu_eval(spl, many)
    assert_parity((v[:60], g[:60], l[:60]), ref, TOL[storage], "tiny cell order")
    spl.close()


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_far_positions_take_the_fp64_reduction(storage):
    """Float and bfloat16 tables reduce coordinates in double-float arithmetic within 1024 lattice
    vectors of the origin (|s| < 1024) and in FP64 beyond: positions up to 3,000 lattice vectors
    away, on both sides of that limit, through the no-record path (< 8192 positions) and the
    record path in input and cell order, against the oracle and bit for bit against each other."""
    dims = (12, 13, 14)
    lat, mil, coef = inputs.random_cell(2470, dims, 8, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    rng = np.random.default_rng(2471)
    frac = rng.uniform(0.0, 1.0, size=(600, 3))
    # lattice shifts: well inside the double-float range, straddling |s| = 1024, and far beyond
    # it, in every octant
    shifts = np.concatenate([rng.integers(-5, 6, size=(200, 3)),
                             rng.choice([-1, 1], size=(200, 3)) * rng.integers(1000, 1050, size=(200, 3)),
                             rng.integers(-3000, 3001, size=(200, 3))])
    pos = np.ascontiguousarray((frac + shifts) @ lat.T)
    beta, blap = oracle_tables(lat, mil, coef, dims, "smooth", storage, True)
    ref = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
    few = gpu_eval(spl, pos)                          # no records
    assert_parity(few, ref, TOL[storage], "far positions, no records " + storage)
    many = np.concatenate([pos] * 14)                 # 8,400 positions: records
    outs = {}
    for order in ("input", "cell"):
        spl.set_order(order)
        outs[order] = gpu_eval(spl, many)
        for a, b in zip(outs[order], few):
            assert np.array_equal(a[:pos.shape[0]], b), order
    spl.close()
