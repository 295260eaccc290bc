"""qmcspl_set_table and the autograd binding as an optimiser of the coefficients: a table read
with qmcspl_get_table and written back leaves the handle bit for bit as it was; a changed table
changes the outputs exactly as the oracle's evaluation of that table says; and SGD on beta
through torch.autograd follows the same steps taken with the oracle's forward and adjoint."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, assert_parity, dev, gpu_eval, oracle_tables, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def t(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev(), dtype=dtype)


ROUND_TRIP = [dict(method="smooth", storage=s, separate_lap=True) for s in ("f64", "df64", "f32", "bf16")] + \
             [dict(method="lagrange", storage="f32", separate_lap=True), dict(method="pp", storage="bf16"),
              dict(method="interp", storage="f32", separate_lap=True, separate_grad=True),
              dict(method="smooth", storage="f32", separate_lap=False, kpoint=(0.137, -0.291, 0.412)),
              dict(method="interp", storage="f64", separate_lap=True, degree=5)]


@pytest.mark.parametrize("kw", ROUND_TRIP, ids=lambda k: "-".join(str(v) for v in k.values()))
def test_round_trip_through_get_and_set_table_is_exact(kw):
    dims = (9, 10, 11)
    kw = dict(kw)
    if "kpoint" in kw:
        lat, mil, coef = inputs.random_bloch_cell(2300, 5, 6.0, 5.0, kw["kpoint"], NONORTHO)
    else:
        lat, mil, coef = inputs.random_cell(2300, dims, 5, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, **kw)
    inf = spl.info()
    n_tab = 8 if kw["method"] == "pp" else inf["n_tables"]
    pos = t(inputs.positions(lat, 9000, 2301, -1, 2))
    before = [x.clone() for x in spl.eval_vgl(pos)]
    tabs = [spl.get_table(i) for i in range(n_tab)]
    for i, tab in enumerate(tabs):
        # float32 sources for the reduced-precision tables, float64 otherwise
        spl.set_table(i, t(tab, spl.out_dtype))
    after = spl.eval_vgl(pos)
    spl.sync()
    assert all(torch.equal(a, b) for a, b in zip(before, after))
    assert all(np.array_equal(spl.get_table(i), tabs[i]) for i in range(n_tab))
    spl.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_a_changed_table_changes_the_outputs_as_the_oracle_says(storage):
    """New random tables (not planewave splines at all) written into a handle: its outputs are the
    oracle's evaluation of those tables, rounded as stored; the ghost planes follow (positions
    outside the cell, every stencil column wrapping somewhere)."""
    dims = (9, 10, 11)
    lat, mil, coef = inputs.random_cell(2310, dims, 7, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    rng = np.random.default_rng(2311)
    b = rng.standard_normal(dims + (7,))
    bl = rng.standard_normal(dims + (7,))
    spl.set_table(0, t(b))
    spl.set_table(1, t(bl, torch.float32))
    pos = inputs.positions(lat, 500, 2312, -2, 3)
    got = gpu_eval(spl, pos)
    ref = oracle.bspline_eval(rounded(b, storage), lat, pos,
                              beta_lap=rounded(bl.astype(np.float32).astype(np.float64), storage))
    assert_parity(got, ref, TOL[storage], "set_table " + storage)
    spl.close()


def test_set_table_rejects_bad_arguments():
    from paper_1309_6250_gb300 import _lib
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_cell(2320, dims, 3, 5.0, 4.0, np.eye(3) * 6.0)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f32", separate_lap=False)
    good = torch.zeros(spl.coef_shape(), dtype=torch.float32, device=dev())
    lib = _lib.load()
    assert lib.qmcspl_set_table(spl.handle, 1, good.data_ptr(), _lib.F32, None) == _lib.ERR_ARG   # no lap table
    assert lib.qmcspl_set_table(spl.handle, 0, good.data_ptr(), _lib.BF16, None) == _lib.ERR_ARG  # source dtype
    assert lib.qmcspl_set_table(spl.handle, 0, None, _lib.F32, None) == _lib.ERR_ARG
    with pytest.raises(ValueError):
        spl.set_table(0, torch.zeros((8, 8, 8, 4), dtype=torch.float32, device=dev()))
    spl.close()


@pytest.mark.parametrize("storage,tol", [("f64", 1e-11), ("f32", 2e-5)])
def test_sgd_on_beta_follows_the_oracle(storage, tol):
    """Five SGD steps on the value and Laplacian tables of a smoothing B-spline, driven by
    torch.autograd through the GPU forward and adjoint, reduce the loss
    L = sum (val - v*)^2 + sum (lap - l*)^2 towards another orbital set's outputs (v*, l*) and
    land where the same steps with the oracle's forward and adjoint land (FP64 tables: to FP64
    rounding; FP32 tables: the oracle steps take the FP32-rounded tables each step)."""
    from paper_1309_6250_gb300.autograd import evaluate
    dims = (10, 11, 12)
    lat, mil, coef = inputs.random_cell(2200, dims, 4, 5.0, 4.0, NONORTHO)
    _, mil2, coef2 = inputs.random_cell(2201, dims, 4, 5.0, 4.0, NONORTHO)
    b0, bl0 = oracle_tables(lat, mil, coef, dims, "smooth", "f64", True)
    tb, tbl = oracle_tables(lat, mil2, coef2, dims, "smooth", "f64", True)
    pos_np = inputs.positions(lat, 300, 2202, -1, 2)
    tv, _, tl = oracle.bspline_eval(tb, lat, pos_np, beta_lap=tbl)
    lr, steps = 0.05, 5
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=True)
    dt = spl.out_dtype
    beta = t(rounded(b0, storage), dt).requires_grad_(True)
    blap = t(rounded(bl0, storage), dt).requires_grad_(True)
    opt = torch.optim.SGD([beta, blap], lr=lr)
    pos, tv_d, tl_d = t(pos_np), t(tv, dt), t(tl, dt)
    losses = []
    for _ in range(steps):
        opt.zero_grad()
        v, g, l = evaluate(spl, pos, beta, blap)
        loss = ((v - tv_d) ** 2).sum() + ((l - tl_d) ** 2).sum()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    assert all(a > b for a, b in zip(losses, losses[1:])), losses
    # the oracle's steps
    b, bl = rounded(b0, storage), rounded(bl0, storage)
    rlosses = []
    for _ in range(steps):
        v, g, l = oracle.bspline_eval(b, lat, pos_np, beta_lap=bl)
        rlosses.append(float(np.sum((v - tv) ** 2) + np.sum((l - tl) ** 2)))
        db, dbl, _ = oracle.bspline_adjoint(b, lat, pos_np, 2 * (v - tv), np.zeros_like(g), 2 * (l - tl), beta_lap=bl)
        b, bl = b - lr * db, bl - lr * dbl
        if storage == "f32":
            b, bl = rounded(b, "f32"), rounded(bl, "f32")
    assert np.allclose(losses, rlosses, rtol=tol, atol=0), (losses, rlosses)
    assert oracle.relative_error(beta.detach().double().cpu().numpy(), b) < tol
    assert oracle.relative_error(blap.detach().double().cpu().numpy(), bl) < tol
    # the next forward uploads the optimised tables and evaluates them
    with torch.no_grad():
        got = tuple(x.double().cpu().numpy() for x in evaluate(spl, pos, beta, blap))
    ref = oracle.bspline_eval(rounded(b, storage), lat, pos_np, beta_lap=rounded(bl, storage))
    assert_parity(got, ref, max(TOL[storage], tol), "after SGD")
    # a tensor that did not change is not uploaded again; an in-place change is
    seen = dict(spl._uploaded)
    evaluate(spl, pos, beta, blap)
    assert spl._uploaded == seen
    with torch.no_grad():
        blap.mul_(0.5)
    v, g, l = evaluate(spl, pos, beta, blap)
    assert spl._uploaded[1] != seen[1] and spl._uploaded[0] == seen[0]
    ref_l = oracle.bspline_eval(rounded(b, storage), lat, pos_np, beta_lap=rounded(0.5 * bl, storage))[2]
    assert oracle.relative_error(l.detach().double().cpu().numpy(), ref_l) < max(TOL[storage], tol)
    spl.close()
