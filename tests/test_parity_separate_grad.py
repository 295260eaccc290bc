"""GPU B-splines with separate gradient tables (Sec. III C: separate approximations of
the gradient and the Laplacian, five tables) against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, oracle_tables, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["smooth", "interp"])
@pytest.mark.parametrize("storage", ["f64", "df64", "f32", "bf16"])
@pytest.mark.parametrize("n_orb", [3, 16])
def test_separate_gradient_tables_match_oracle(method, storage, n_orb):
    dims = (9, 10, 11)
    lat, mil, coef = inputs.random_cell(1200 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage=storage, separate_lap=True,
                  separate_grad=True)
    inf = spl.info()
    assert inf["n_tables"] == 5 and inf["separate_grad"] == 1
    ref_t = oracle.derivative_tables(method, lat, mil, coef, dims)
    ttol = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-7, "bf16": 8e-3}[storage]
    for i in range(5):
        assert oracle.relative_error(spl.get_table(i), ref_t[i]) < ttol
    tabs = oracle_tables(lat, mil, coef, dims, method, storage, True, True)
    pos = inputs.positions(lat, 400, 1201, -1, 2)
    got = gpu_eval(spl, pos)
    ref = oracle.bspline_eval_separate(tabs, lat, pos)
    assert_parity(got, ref, TOL[storage], "separate grad %s/%s" % (method, storage))
    # the separate approximations are closer to the planewave derivatives than the
    # derivatives of the value spline (Sec. III C, Fig. 1)
    if storage == "f64":
        pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
        _, dg, _ = oracle.bspline_eval(tabs[0], lat, pos)
        assert oracle.relative_mean_absolute_error(got[1], pg) < oracle.relative_mean_absolute_error(dg, pg)
    spl.close()


@pytest.mark.parametrize("storage", ["f64", "df64", "f32"])
def test_separate_gradient_tables_for_bloch_orbitals(storage):
    kp = inputs.KPOINTS["generic"]
    dims = (9, 10, 11)
    lat, mil, coef = inputs.random_bloch_cell(1210, 5, 6.0, 5.0, kp, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True,
                  separate_grad=True, kpoint=kp)
    ref_t = oracle.bloch_tables("smooth", lat, mil, coef, kp, dims, gradient=True)
    for i in range(5):
        assert oracle.relative_error(spl.get_table(i), ref_t[i]) < (1e-7 if storage == "f32" else 1e-12)
    tabs = oracle_tables(lat, mil, coef, dims, "smooth", storage, True, True, kpoint=kp)
    pos = inputs.positions(lat, 300, 1211, -1, 2)
    v, g, l = spl.eval_vgl(torch.from_numpy(pos).to(dev()))
    spl.sync()
    got = tuple(x.cpu().numpy().astype(np.complex128) for x in (v, g, l))
    ref = oracle.bloch_eval("smooth", tabs, lat, kp, pos)
    assert_parity(got, ref, TOL[storage], "bloch separate grad/" + storage)
    spl.close()


def test_separate_gradient_orders_noalloc_checkpoint_and_rejections(tmp_path):
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.api import OrbitalSplines, eval_batched
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_cell(1220, dims, 20, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="interp", storage="f32", separate_lap=True, separate_grad=True)
    pos = torch.from_numpy(inputs.positions(lat, 12000, 1221, -1, 2)).to(dev())
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
    path = tmp_path / "sg.qmcspl"
    spl.save(str(path))
    back = OrbitalSplines.load(str(path), device=dev())
    assert back.separate_grad and back.info()["n_tables"] == 5
    out = back.eval_vgl(pos)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(out, ref))
    with pytest.raises(_lib.QmcsplError) as ei:
        eval_batched([spl], [pos])
    assert ei.value.code == _lib.ERR_UNSUPPORTED
    back.close()
    spl.close()
