"""GPU interpolating B-splines of degree 1, 5, 7 on uniform grids and of degree 1, 3, 5, 7 on
graded (non-uniform) grids (qmcspl_create_grid) against the oracle's recurrence-based
definition."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, oracle_tables, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TTOL = {"f64": 1e-12, "f32": 1e-7, "bf16": 8e-3}


def graded(dims):
    return tuple(inputs.graded_knots(d, 0.5, 0.17 * a) for a, d in enumerate(dims))


CASES = ([(deg, False, st, sep) for deg in (1, 5, 7) for st in ("f64", "f32", "bf16") for sep in (False, True)] +
         [(deg, True, st, sep) for deg in (1, 3, 5, 7) for st in ("f64", "f32", "bf16") for sep in (False, True)])


@pytest.mark.parametrize("degree,nonuni,storage,sep", CASES)
def test_general_tables_and_outputs_match_oracle(degree, nonuni, storage, sep):
    dims = (11, 12, 13)
    lat, mil, coef = inputs.random_cell(1400 + degree, dims, 5, 5.0, 4.0, NONORTHO)
    knots = graded(dims) if nonuni else None
    spl = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=sep, degree=degree,
                  knots=knots)
    inf = spl.info()
    assert inf["degree"] == degree and inf["nonuniform"] == int(nonuni)
    kk = knots if nonuni else (None,) * 3
    rb, rl = oracle.general_interp_tables(lat, mil, coef, dims, degree, kk, laplacian=sep)
    assert oracle.relative_error(spl.get_table(0), rb) < TTOL[storage]
    if sep:
        assert oracle.relative_error(spl.get_table(1), rl) < TTOL[storage]
    pos = inputs.positions(lat, 60, 1401, -1, 2)
    got = gpu_eval(spl, pos)
    ob, ol = oracle_tables(lat, mil, coef, dims, "interp", storage, sep, degree=degree, knots=knots)
    ref = oracle.general_eval(ob, lat, pos, degree, kk, beta_lap=ol)
    assert_parity(got, ref, TOL[storage], "degree %d nonuni=%d %s sep=%d" % (degree, nonuni, storage, sep))
    spl.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_uniform_points_through_the_general_kernel_equal_the_cubic_path(storage):
    """A 'non-uniform' grid whose points are l/N runs the general kernel and the axis solves;
    it must give the paper's cubic interpolating spline of the tuned path."""
    dims = (10, 12, 14)
    lat, mil, coef = inputs.random_cell(1410, dims, 7, 5.0, 4.0, NONORTHO)
    knots = tuple(np.arange(d) / d for d in dims)
    gen = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=True, knots=knots)
    std = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=True)
    pos = inputs.positions(lat, 3000, 1411, -1, 2)
    tol = {"f64": 1e-12, "f32": 2e-6}[storage]
    assert oracle.relative_error(gen.get_table(0), std.get_table(0)) < (1e-12 if storage == "f64" else 1e-6)
    assert_parity(gpu_eval(gen, pos), gpu_eval(std, pos), tol, "uniform points")


def test_bloch_on_a_graded_grid():
    kp = inputs.KPOINTS["generic"]
    dims = (11, 12, 13)
    lat, mil, coef = inputs.random_bloch_cell(1420, 3, 5.0, 4.0, kp, NONORTHO)
    knots = graded(dims)
    spl = splines(lat, dims, mil, coef, method="interp", storage="f64", separate_lap=True, knots=knots, kpoint=kp)
    rb, rl = oracle.general_interp_tables(lat, mil, coef, dims, 3, knots, laplacian=True, kpoint=kp)
    assert oracle.relative_error(spl.get_table(0), rb) < 1e-12
    pos = inputs.positions(lat, 40, 1421, -1, 2)
    v, g, l = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    spl.sync()
    got = tuple(x.cpu().numpy() for x in (v, g, l))
    u = oracle.general_eval(rb, lat, pos, 3, knots, beta_lap=rl)
    ref = oracle.bloch_combine(*u, lat, kp, pos, True, False)
    assert_parity(got, ref, 1e-11, "bloch graded")


def test_general_orders_noalloc_checkpoint_and_rejections(tmp_path):
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import OrbitalSplines, eval_batched
    dims = (14, 14, 14)
    lat, mil, coef = inputs.random_cell(1430, dims, 12, 6.0, 5.0, NONORTHO)
    for kw in (dict(degree=5), dict(knots=graded(dims)), dict(degree=7, knots=graded(dims))):
        spl = splines(lat, dims, mil, coef, method="interp", storage="f32", separate_lap=False, **kw)
        pos = torch.from_numpy(inputs.positions(lat, 10000, 1431, -1, 2)).to(dev())
        spl.set_order("input")
        ref = [o.clone() for o in spl.eval_vgl(pos)]
        spl.set_order("cell")
        out = spl.eval_vgl(pos)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(out, ref))
        lib = _lib.load()
        na = spl.alloc_outputs(pos.shape[0])
        _lib.check(lib.qmcspl_eval_vgl_noalloc(spl.handle, pos.data_ptr(), pos.shape[0], na[0].data_ptr(),
                                               na[1].data_ptr(), na[2].data_ptr(), None))
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(na, ref))
        path = tmp_path / "general.qmcspl"
        spl.save(str(path))
        back = OrbitalSplines.load(str(path), device=dev())
        assert back.info()["degree"] == spl.info()["degree"]
        assert back.info()["nonuniform"] == spl.info()["nonuniform"]
        out = back.eval_vgl(pos)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(out, ref))
        # the adjoint of the loaded handle equals the original's (up to the order of the FP32
        # partial sums of the orbital tiles, which meet in atomic adds)
        up = torch.ones_like(ref[0])
        d1, d0 = back.backward(pos, gv=up), spl.backward(pos, gv=up)
        assert oracle.relative_error(d1.cpu().numpy(), d0.cpu().numpy()) < 1e-6
        with pytest.raises(_lib.QmcsplError) as ei:
            eval_batched([spl], [pos])
        assert ei.value.code == _lib.ERR_UNSUPPORTED
        back.close()
        spl.close()
    # a non-uniform grid too coarse for the planewave band is refused
    with pytest.raises(_lib.QmcsplError) as ei:
        splines(lat, (6, 6, 6), mil, coef, method="interp", storage="f64", knots=graded((6, 6, 6)))
    assert ei.value.code == _lib.ERR_ARG


@pytest.mark.parametrize("degree,nonuni", [(1, False), (5, False), (7, False), (1, True), (3, True), (5, True),
                                           (7, True)])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_general_with_position_records_matches_oracle(degree, nonuni, storage):
    """From 8192 positions on, a per-position pass precomputes the cell and local coordinate
    (the offset from the interval's left grid point on graded grids) and the kernel builds the
    weights in the table's arithmetic type; sampled outputs against the oracle."""
    dims = (11, 12, 13)
    lat, mil, coef = inputs.random_cell(1440 + degree, dims, 6, 5.0, 4.0, NONORTHO)
    knots = graded(dims) if nonuni else None
    spl = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=False, degree=degree,
                  knots=knots)
    pos = inputs.positions(lat, 9000, 1441, -1, 2)
    v, g, l = gpu_eval(spl, pos)
    sample = np.arange(0, 9000, 211)
    kk = knots if nonuni else (None,) * 3
    ob, _ = oracle_tables(lat, mil, coef, dims, "interp", storage, False, degree=degree, knots=knots)
    ref = oracle.general_eval(ob, lat, pos[sample], degree, kk)
    assert_parity((v[sample], g[sample], l[sample]), ref, TOL[storage], "records deg %d %s" % (degree, storage))
    spl.close()


@pytest.mark.parametrize("degree", [1, 5, 7])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_smoothing_of_other_degrees_matches_oracle(degree, storage):
    """Smoothing B-splines of degree n (Eq. b-splinecoefficients with the degree-n gamma):
    tables and outputs against the oracle, with and without the Laplacian table."""
    dims = (11, 12, 13)
    lat, mil, coef = inputs.random_cell(1450 + degree, dims, 5, 5.0, 4.0, NONORTHO)
    rb, rl = oracle.smoothing_tables_degree(lat, mil, coef, dims, degree, laplacian=True)
    for sep in (False, True):
        spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=sep, degree=degree)
        assert oracle.relative_error(spl.get_table(0), rb) < TTOL[storage]
        if sep:
            assert oracle.relative_error(spl.get_table(1), rl) < TTOL[storage]
        pos = inputs.positions(lat, 50, 1451, -1, 2)
        got = gpu_eval(spl, pos)
        ob, ol = oracle_tables(lat, mil, coef, dims, "smooth", storage, sep, degree=degree)
        ref = oracle.general_eval(ob, lat, pos, degree, beta_lap=ol)
        assert_parity(got, ref, TOL[storage], "smoothing degree %d %s sep=%d" % (degree, storage, sep))
        spl.close()
