"""GPU adjoint (qmcspl_eval_vgl_backward and the autograd binding) against the FP64
oracle adjoint, an exact linearity identity and central finite differences."""
import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs
from gpu_helpers import NONORTHO, TOL, dev, oracle_tables, rounded, splines

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device=dev(), dtype=dtype)


def gpu_backward(spl, pos, gv, gg, gl):
    sep = bool(spl.info()["separate_lap"])
    dc = torch.zeros(spl.coef_shape(), dtype=spl.out_dtype, device=dev())
    dcl = torch.zeros_like(dc) if sep else None
    dpos = spl.backward(t(pos, torch.float64), t(gv, spl.out_dtype), t(gg, spl.out_dtype),
                        t(gl, spl.out_dtype), dcoef=dc, dcoef_lap=dcl)
    spl.sync()
    return dc.double().cpu().numpy(), None if dcl is None else dcl.double().cpu().numpy(), \
        dpos.cpu().numpy()


def away_from_planes(lat, dims, pos, margin):
    s = pos @ np.linalg.inv(lat).T * np.array(dims)
    f = s - np.floor(s)
    return np.all((f > margin) & (f < 1 - margin), axis=1)


@pytest.mark.parametrize("method", ["smooth", "interp"])
@pytest.mark.parametrize("sep", [False, True])
@pytest.mark.parametrize("n_orb", [3, 16])
def test_fp64_backward_matches_oracle(method, sep, n_orb):
    dims = (9, 10, 11)
    lat, mil, coef = inputs.random_cell(600 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage="f64", separate_lap=sep)
    beta, blap = oracle_tables(lat, mil, coef, dims, method, "f64", sep)
    pos = inputs.positions(lat, 300, 12, -1, 2)
    gv, gg, gl = inputs.upstream_weights(300, n_orb, 13)
    dc, dcl, dpos = gpu_backward(spl, pos, gv, gg, gl)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(beta, lat, pos, gv, gg, gl, beta_lap=blap)
    assert oracle.relative_error(dc, rdc) < 1e-12
    if sep:
        assert oracle.relative_error(dcl, rdcl) < 1e-12
    assert oracle.relative_error(dpos, rdpos) < 1e-12


@pytest.mark.parametrize("method", ["smooth", "interp"])
@pytest.mark.parametrize("sep", [False, True])
def test_df64_backward_matches_oracle(method, sep):
    """Double-float tables: the adjoint runs in FP64 on the stored pairs (hi + lo, the FP64
    table to about 2^-48), so it equals the oracle adjoint on the oracle's FP64 tables."""
    dims = (9, 10, 11)
    n_orb = 6
    lat, mil, coef = inputs.random_cell(640, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method=method, storage="df64", separate_lap=sep)
    assert spl.out_dtype == torch.float64
    beta, blap = oracle_tables(lat, mil, coef, dims, method, "df64", sep)
    pos = inputs.positions(lat, 300, 641, -1, 2)
    gv, gg, gl = inputs.upstream_weights(300, n_orb, 642)
    dc, dcl, dpos = gpu_backward(spl, pos, gv, gg, gl)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(beta, lat, pos, gv, gg, gl, beta_lap=blap)
    assert oracle.relative_error(dc, rdc) < 1e-12
    if sep:
        assert oracle.relative_error(dcl, rdcl) < 1e-12
    assert oracle.relative_error(dpos, rdpos) < 1e-12


def test_fp64_linearity_identity_and_position_fd():
    """L is linear in beta: sum(dL/dbeta * beta) = L(beta) with the GPU forward pass; and
    dL/dr against central differences of the GPU forward (h = 1e-4 bohr, FP64)."""
    dims = (12, 12, 12)
    lat, mil, coef = inputs.random_cell(700, dims, 8, 6.0, 5.0, NONORTHO)
    for sep in (False, True):
        spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=sep)
        pos = inputs.positions(lat, 200, 14)
        pos = pos[away_from_planes(lat, dims, pos, 0.01)]
        n = pos.shape[0]
        gv, gg, gl = inputs.upstream_weights(n, 8, 15)

        def loss(p):
            v, g, l = spl.eval_vgl(t(p, torch.float64))
            spl.sync()
            return (np.sum(gv * v.cpu().numpy()) + np.sum(gg * g.cpu().numpy()) +
                    np.sum(gl * l.cpu().numpy()))

        dc, dcl, dpos = gpu_backward(spl, pos, gv, gg, gl)
        lin = np.sum(dc * spl.get_table(0)) + (np.sum(dcl * spl.get_table(1)) if sep else 0.0)
        assert lin == pytest.approx(loss(pos), rel=1e-12)
        h = 1e-4
        fd = np.zeros_like(dpos)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            # per-position losses: perturb one coordinate of every position at once
            # (positions are independent, so the sum separates)
            lp = [None, None]
            for k, sgn in enumerate((1, -1)):
                v, g, l = spl.eval_vgl(t(pos + sgn * e, torch.float64))
                spl.sync()
                lp[k] = (np.sum(gv * v.cpu().numpy(), 1) + np.sum(gg * g.cpu().numpy(), (1, 2)) +
                         np.sum(gl * l.cpu().numpy(), 1))
            fd[:, a] = (lp[0] - lp[1]) / (2 * h)
        assert oracle.relative_error(dpos, fd) < 1e-6


def test_c5_si64_backward_fp32():
    """Si-like 64-atom cell, 128 orbitals on 72^3, FP32 tables with the Laplacian table,
    4096 positions, N(0,1) upstream weights on value, gradient and Laplacian: coefficient
    and position gradients against the oracle adjoint (FP64) on the oracle's tables rounded to
    FP32 as the GPU stores them."""
    w = inputs.make_workload("c5")
    dims = w.cell.grid
    spl = splines(w.lattice, dims, w.miller, w.coef, method="smooth", storage="f32", separate_lap=True)
    beta, blap = oracle_tables(w.lattice, w.miller, w.coef, dims, "smooth", "f32", True)
    n = w.pos.shape[0]
    gv, gg, gl = inputs.upstream_weights(n, w.coef.shape[0], 3005)
    gv32, gg32, gl32 = (x.astype(np.float32).astype(np.float64) for x in (gv, gg, gl))
    dc, dcl, dpos = gpu_backward(spl, w.pos, gv32, gg32, gl32)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(beta, w.lattice, w.pos, gv32, gg32, gl32, beta_lap=blap)
    e = [oracle.relative_error(dc, rdc), oracle.relative_error(dcl, rdcl), oracle.relative_error(dpos, rdpos)]
    print("c5 backward relative errors (dcoef, dcoef_lap, dpos): %s" % ["%.2e" % x for x in e])
    assert e[0] < TOL["f32"] and e[1] < TOL["f32"] and e[2] < TOL["f32"]
    # the stored tables are the oracle's within FP32 rounding
    assert oracle.relative_error(spl.get_table(0), beta) < 1e-7
    assert oracle.relative_error(spl.get_table(1), blap) < 1e-7


def test_autograd_function_positions_and_coefficients():
    from paper_1309_6250_gb300.autograd import evaluate
    dims = (10, 10, 12)
    lat, mil, coef = inputs.random_cell(800, dims, 6, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=True)
    beta, beta_lap = spl.coefficient_parameters()
    pos_np = inputs.positions(lat, 64, 16)
    pos = t(pos_np, torch.float64).requires_grad_(True)
    gv, gg, gl = inputs.upstream_weights(64, 6, 17)
    v, g, l = evaluate(spl, pos, beta, beta_lap)
    loss = (v * t(gv, torch.float64)).sum() + (g * t(gg, torch.float64)).sum() + \
        (l * t(gl, torch.float64)).sum()
    loss.backward()
    rb, rbl = oracle_tables(lat, mil, coef, dims, "smooth", "f64", True)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(rb, lat, pos_np, gv, gg, gl, beta_lap=rbl)
    assert oracle.relative_error(pos.grad.cpu().numpy(), rdpos) < 1e-12
    assert oracle.relative_error(beta.grad.cpu().numpy(), rdc) < 1e-12
    assert oracle.relative_error(beta_lap.grad.cpu().numpy(), rdcl) < 1e-12
    # only some outputs used: missing upstream gradients count as zero
    pos.grad = None
    v, g, l = evaluate(spl, pos)
    (v * t(gv, torch.float64)).sum().backward()
    z = np.zeros_like(gg), np.zeros_like(gl)
    _, _, rdpos_v = oracle.bspline_adjoint(rb, lat, pos_np, gv, z[0], z[1], beta_lap=rbl)
    assert oracle.relative_error(pos.grad.cpu().numpy(), rdpos_v) < 1e-12


def test_double_float_variants_are_rejected_at_creation():
    from paper_1309_6250_gb300 import _lib
    dims = (8, 8, 8)
    lat, mil, coef = inputs.random_cell(5, dims, 2, 5.0, 4.0, np.eye(3) * 6.0)
    pos = torch.zeros((4, 3), dtype=torch.float64, device=dev())
    for method in ("lagrange", "pp"):
        with pytest.raises(_lib.QmcsplError) as ei:
            splines(lat, dims, mil, coef, method=method, storage="df64")
        assert ei.value.code == _lib.ERR_UNSUPPORTED


# ---------------------------------------------------------------------------
# Bloch orbitals (complex outputs z = exp(i k.r) w): the adjoint of the bracket and of the phase
# ---------------------------------------------------------------------------

def complex_upstream(n, n_orb, seed):
    gv, gg, gl = inputs.upstream_weights(n, 2 * n_orb, seed)
    c = lambda a: a[..., 0::2] + 1j * a[..., 1::2]
    return c(gv), c(gg), c(gl)


def bloch_loss(z, g):
    """L = sum Re(conj(g) z) = sum (Re g Re z + Im g Im z): g is dL/dRe z + i dL/dIm z."""
    return float(sum(np.sum((np.conj(gi) * zi).real) for gi, zi in zip(g, z)))


def gpu_backward_complex(spl, pos, g):
    sep = bool(spl.info()["separate_lap"])
    cd = torch.complex128 if spl.out_dtype == torch.float64 else torch.complex64
    dc = torch.zeros(spl.coef_shape(), dtype=spl.out_dtype, device=dev())
    dcl = torch.zeros_like(dc) if sep else None
    dpos = spl.backward(t(pos, torch.float64), *(t(x, cd) for x in g), dcoef=dc, dcoef_lap=dcl)
    spl.sync()
    return dc.double().cpu().numpy(), None if dcl is None else dcl.double().cpu().numpy(), \
        dpos.cpu().numpy()


@pytest.mark.parametrize("storage,tol_lin,tol_fd", [("f64", 1e-11, 1e-6), ("df64", 1e-11, 1e-6),
                                                     ("f32", 2e-5, 3e-3)])
@pytest.mark.parametrize("sep", [False, True])
def test_bloch_backward_linearity_and_position_fd(storage, tol_lin, tol_fd, sep):
    """L is linear in the stored tables: sum(dL/dbeta * beta') = L(beta') for random tables
    beta' evaluated by the oracle (Bloch forward: spline of u, then the phase and the product
    rule); dL/dr against central differences of the oracle forward on the oracle's tables rounded
    as stored (h = 1e-4 bohr, positions away from grid planes)."""
    k = inputs.KPOINTS["generic"]
    dims = (10, 11, 12)
    n_orb = 3
    lat, mil, coef = inputs.random_bloch_cell(1700, n_orb, 5.0, 4.0, k, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=sep, kpoint=k)
    pos = inputs.positions(lat, 120, 1701, -1, 2)
    pos = pos[away_from_planes(lat, dims, pos, 0.02)]
    n = pos.shape[0]
    g = complex_upstream(n, n_orb, 1702)
    if storage == "f32":
        g = tuple((x.real.astype(np.float32) + 1j * x.imag.astype(np.float32)).astype(np.complex128) for x in g)
    dc, dcl, dpos = gpu_backward_complex(spl, pos, g)
    rng = np.random.default_rng(1703)
    for _ in range(2):
        b1 = rng.standard_normal(dims + (2 * n_orb,))
        b2 = rng.standard_normal(dims + (2 * n_orb,)) if sep else None
        z = oracle.bloch_eval("smooth", b1, lat, k, pos, tables_lap=b2)
        lin = np.sum(dc * b1) + (np.sum(dcl * b2) if sep else 0.0)
        ref = bloch_loss(z, g)
        assert abs(lin - ref) <= tol_lin * max(1.0, abs(ref)), (lin, ref)
    beta, blap = oracle_tables(lat, mil, coef, dims, "smooth", storage, sep, kpoint=k)
    h = 1e-4
    fd = np.zeros_like(dpos)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lp = []
        for sgn in (1, -1):
            z = oracle.bloch_eval("smooth", beta, lat, k, pos + sgn * e, tables_lap=blap)
            lp.append(sum(np.sum((np.conj(gi) * zi).real.reshape(n, -1), axis=1) for gi, zi in zip(g, z)))
        fd[:, a] = (lp[0] - lp[1]) / (2 * h)
    assert oracle.relative_error(dpos, fd) < tol_fd


def test_bloch_autograd_matches_the_direct_adjoint():
    """Complex outputs through torch.autograd: the gradient torch passes back for a real loss is
    dL/dRe z + i dL/dIm z, so positions and coefficients get exactly the direct adjoint."""
    from paper_1309_6250_gb300.autograd import evaluate
    k = inputs.KPOINTS["X"]
    dims = (10, 10, 12)
    lat, mil, coef = inputs.random_bloch_cell(1710, 4, 5.0, 4.0, k, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage="f64", separate_lap=True, kpoint=k)
    beta, beta_lap = spl.coefficient_parameters()
    assert tuple(beta.shape) == spl.coef_shape() == dims + (8,)
    pos_np = inputs.positions(lat, 64, 1711)
    pos = t(pos_np, torch.float64).requires_grad_(True)
    g = complex_upstream(64, 4, 1712)
    v, gr, l = evaluate(spl, pos, beta, beta_lap)
    assert v.dtype == torch.complex128
    loss = sum((torch.conj(t(gi, torch.complex128)) * zi).real.sum() for gi, zi in zip(g, (v, gr, l)))
    loss.backward()
    dc, dcl, dpos = gpu_backward_complex(spl, pos_np, g)
    assert oracle.relative_error(pos.grad.cpu().numpy(), dpos) < 1e-13
    assert oracle.relative_error(beta.grad.cpu().numpy(), dc) < 1e-13
    assert oracle.relative_error(beta_lap.grad.cpu().numpy(), dcl) < 1e-13


# ---------------------------------------------------------------------------
# five tables (Lagrange; B-splines with separate gradient tables): dcoef holds all five
# ---------------------------------------------------------------------------

FIVE = [dict(method="lagrange", separate_lap=True),
        dict(method="smooth", separate_lap=True, separate_grad=True),
        dict(method="interp", separate_lap=True, separate_grad=True),
        dict(method="pp", separate_lap=False)]


def five_forward(method, tabs, lat, pos, k=None):
    if k is not None:
        return oracle.bloch_eval(method, tabs, lat, k, pos)
    if method == "lagrange":
        return oracle.lagrange_eval(tabs, lat, pos)
    if method == "pp":
        return oracle.pp_eval(tabs, lat, pos)
    return oracle.bspline_eval_separate(tabs, lat, pos)


@pytest.mark.parametrize("kw", FIVE, ids=["lagrange", "smooth_sepgrad", "interp_sepgrad", "pp"])
@pytest.mark.parametrize("storage,tol_lin,tol_fd", [("f64", 1e-11, 1e-6), ("df64", 1e-11, 1e-6),
                                                     ("f32", 2e-5, 3e-3)])
@pytest.mark.parametrize("bloch", [False, True])
def test_five_table_backward_linearity_and_position_fd(kw, storage, tol_lin, tol_fd, bloch):
    """Five-table handles (the outputs are the values of five interpolants) and pp-splines
    (eight coefficient entries per grid point): the outputs are linear in the tables, so the
    coefficient adjoint is checked by sum(dL/dbeta * beta') = L(beta') with the oracle on random
    tables, and the position adjoint against central differences of the oracle forward
    (positions away from grid planes, where the Lagrange interpolant's derivatives jump)."""
    if storage == "df64" and not kw.get("separate_grad"):
        pytest.skip("double-float tables are for B-splines")
    dims = (10, 11, 12)
    n_orb = 3
    k = inputs.KPOINTS["generic"] if bloch else None
    if bloch:
        lat, mil, coef = inputs.random_bloch_cell(1800, n_orb, 5.0, 4.0, k, NONORTHO)
        spl = splines(lat, dims, mil, coef, storage=storage, kpoint=k, **kw)
    else:
        lat, mil, coef = inputs.random_cell(1800, dims, n_orb, 5.0, 4.0, NONORTHO)
        spl = splines(lat, dims, mil, coef, storage=storage, **kw)
    n_tab = 8 if kw["method"] == "pp" else 5
    assert spl.info()["n_tables"] == 5 or kw["method"] == "pp"
    nf = spl.coef_shape()[-1]
    pos = inputs.positions(lat, 120, 1801, -1, 2)
    pos = pos[away_from_planes(lat, dims, pos, 0.02)]
    n = pos.shape[0]
    if bloch:
        g = complex_upstream(n, n_orb, 1802)
        cd = torch.complex128 if storage in ("f64", "df64") else torch.complex64
    else:
        g = inputs.upstream_weights(n, n_orb, 1802)
        cd = spl.out_dtype
    if storage == "f32":
        r32 = lambda x: (x.real.astype(np.float32) + 1j * x.imag.astype(np.float32)) if bloch else \
            x.astype(np.float32).astype(np.float64)
        g = tuple(r32(x) for x in g)
    dc = torch.zeros((n_tab,) + spl.coef_shape(), dtype=spl.out_dtype, device=dev())
    dpos = spl.backward(t(pos, torch.float64), *(t(x, cd) for x in g), dcoef=dc)
    spl.sync()
    dc, dpos = dc.double().cpu().numpy(), dpos.cpu().numpy()
    loss = (lambda z: bloch_loss(z, g)) if bloch else \
        (lambda z: float(sum(np.sum(gi * zi) for gi, zi in zip(g, z))))
    rng = np.random.default_rng(1803)
    for _ in range(2):
        b5 = rng.standard_normal((n_tab,) + dims + (nf,))
        ref = loss(five_forward(kw["method"], b5, lat, pos, k))
        lin = np.sum(dc * b5)
        assert abs(lin - ref) <= tol_lin * max(1.0, abs(ref)), (lin, ref)
    tabs = oracle_tables(lat, mil, coef, dims, kw["method"], storage, kw["separate_lap"],
                         kw.get("separate_grad", False), kpoint=k)
    h = 1e-4
    fd = np.zeros_like(dpos)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lp = []
        for sgn in (1, -1):
            z = five_forward(kw["method"], tabs, lat, pos + sgn * e, k)
            if bloch:
                lp.append(sum(np.sum((np.conj(gi) * zi).real.reshape(n, -1), axis=1) for gi, zi in zip(g, z)))
            else:
                lp.append(sum(np.sum((gi * zi).reshape(n, -1), axis=1) for gi, zi in zip(g, z)))
        fd[:, a] = (lp[0] - lp[1]) / (2 * h)
    assert oracle.relative_error(dpos, fd) < tol_fd
    spl.close()


def test_five_table_autograd_and_argument_checks():
    from paper_1309_6250_gb300 import _lib
    from paper_1309_6250_gb300.autograd import evaluate
    dims = (10, 10, 12)
    lat, mil, coef = inputs.random_cell(1810, dims, 4, 5.0, 4.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="lagrange", storage="f64", separate_lap=True)
    beta, none = spl.coefficient_parameters()
    assert none is None and tuple(beta.shape) == (5,) + spl.coef_shape()
    pos_np = inputs.positions(lat, 64, 1811)
    pos = t(pos_np, torch.float64).requires_grad_(True)
    gv, gg, gl = inputs.upstream_weights(64, 4, 1812)
    v, g, l = evaluate(spl, pos, beta)
    loss = (v * t(gv, torch.float64)).sum() + (g * t(gg, torch.float64)).sum() + \
        (l * t(gl, torch.float64)).sum()
    loss.backward()
    dc = torch.zeros((5,) + spl.coef_shape(), dtype=torch.float64, device=dev())
    dpos = spl.backward(t(pos_np, torch.float64), t(gv, torch.float64), t(gg, torch.float64),
                        t(gl, torch.float64), dcoef=dc)
    spl.sync()
    assert oracle.relative_error(pos.grad.cpu().numpy(), dpos.cpu().numpy()) < 1e-13
    assert oracle.relative_error(beta.grad.cpu().numpy(), dc.cpu().numpy()) < 1e-13
    # all five tables go to dcoef: a separate dcoef_lap is refused
    with pytest.raises(_lib.QmcsplError) as ei:
        spl.backward(t(pos_np, torch.float64), t(gv, torch.float64), dcoef=dc, dcoef_lap=torch.zeros_like(dc))
    assert ei.value.code == _lib.ERR_ARG


# ---------------------------------------------------------------------------
# B-splines of other degrees and on graded grids (the general adjoint)
# ---------------------------------------------------------------------------

def graded(dims):
    return tuple(inputs.graded_knots(d, 0.45, 0.2 * a) for a, d in enumerate(dims))


# f64 for every degree and grid kind, f32 / bf16 on a few (their sums run in FP32: the
# tolerance allows for up to 512-term FP32 sums per output)
GENERAL = [(d, g, "f64", sep) for d, g in ((1, False), (5, False), (7, False), (1, True), (3, True), (5, True),
                                            (7, True)) for sep in (False, True)] + \
          [(5, False, "f32", True), (7, True, "f32", False), (1, True, "f32", True), (7, False, "bf16", True),
           (3, True, "bf16", False)]


@pytest.mark.parametrize("degree,grad,storage,sep", GENERAL)
def test_general_backward_matches_oracle(degree, grad, storage, sep):
    """Coefficient and position adjoints of degree-n B-splines (interpolating; graded grids)
    against the oracle's brute-force transpose of its evaluation, on the oracle's tables rounded
    as stored; ragged orbital count, positions outside the cell."""
    dims = (8, 9, 10)
    n_orb = 5
    knots = graded(dims) if grad else None
    lat, mil, coef = inputs.random_cell(1800 + degree, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="interp", storage=storage, separate_lap=sep, degree=degree,
                  knots=knots)
    beta, blap = oracle_tables(lat, mil, coef, dims, "interp", storage, sep, degree=degree, knots=knots)
    n = 60
    pos = inputs.positions(lat, n, 1801 + degree, -1, 2)
    gv, gg, gl = inputs.upstream_weights(n, n_orb, 1802)
    if storage != "f64":
        gv, gg, gl = (x.astype(np.float32).astype(np.float64) for x in (gv, gg, gl))
    dc, dcl, dpos = gpu_backward(spl, pos, gv, gg, gl)
    rdc, rdcl, rdpos = oracle.general_adjoint(beta, lat, pos, gv, gg, gl, degree=degree,
                                              knots=knots if grad else (None, None, None), beta_lap=blap)
    tol = 1e-11 if storage == "f64" else 1e-5
    assert oracle.relative_error(dc, rdc) < tol
    if sep:
        assert oracle.relative_error(dcl, rdcl) < tol
    assert oracle.relative_error(dpos, rdpos) < tol


def test_general_backward_bloch_on_a_graded_grid():
    """Bloch orbitals with quintic splines on a graded grid: the coefficient adjoint by
    linearity against the oracle's forward (general evaluation of u, then the phase and the
    product rule), the position adjoint against central differences of that forward."""
    k = inputs.KPOINTS["generic"]
    dims = (9, 10, 11)
    n_orb = 2
    knots = graded(dims)
    lat, mil, coef = inputs.random_bloch_cell(1810, n_orb, 5.0, 4.0, k, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="interp", storage="f64", separate_lap=True, kpoint=k,
                  degree=5, knots=knots)
    pos = inputs.positions(lat, 40, 1811, -1, 2)
    n = pos.shape[0]
    g = complex_upstream(n, n_orb, 1812)
    dc, dcl, dpos = gpu_backward_complex(spl, pos, g)

    def forward(b1, b2, p):
        u = oracle.general_eval(b1, lat, p, 5, knots, beta_lap=b2)
        return oracle.bloch_combine(*u, lat, k, p, True, False)

    rng = np.random.default_rng(1813)
    for _ in range(2):
        b1 = rng.standard_normal(dims + (2 * n_orb,))
        b2 = rng.standard_normal(dims + (2 * n_orb,))
        lin = np.sum(dc * b1) + np.sum(dcl * b2)
        ref = bloch_loss(forward(b1, b2, pos), g)
        assert abs(lin - ref) <= 1e-11 * max(1.0, abs(ref)), (lin, ref)
    beta, blap = oracle_tables(lat, mil, coef, dims, "interp", "f64", True, kpoint=k, degree=5, knots=knots)
    h = 1e-5
    fd = np.zeros_like(dpos)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lp = []
        for sgn in (1, -1):
            z = forward(beta, blap, pos + sgn * e)
            lp.append(sum(np.sum((np.conj(gi) * zi).real.reshape(n, -1), axis=1) for gi, zi in zip(g, z)))
        fd[:, a] = (lp[0] - lp[1]) / (2 * h)
    assert oracle.relative_error(dpos, fd) < 1e-6


def test_general_backward_nonfinite_position_and_empty_call():
    """A non-finite position gives NaN dL/dr for that position only and adds nothing to dbeta;
    an empty call is a no-op (degree 5 on a graded grid, FP64)."""
    dims = (8, 9, 10)
    lat, mil, coef = inputs.random_cell(1820, dims, 4, 6.0, 5.0, NONORTHO)
    knots = graded(dims)
    spl = splines(lat, dims, mil, coef, method="interp", storage="f64", separate_lap=False, degree=5,
                  knots=knots)
    pos = inputs.positions(lat, 12, 1821, -1, 2)
    gv, gg, gl = inputs.upstream_weights(12, 4, 1822)
    bad = pos.copy()
    bad[5] = np.nan
    from paper_1309_6250_gb300 import _lib
    dcb = torch.zeros(spl.coef_shape(), dtype=torch.float64, device=dev())
    dpb = spl.backward(t(bad, torch.float64), t(gv, torch.float64), t(gg, torch.float64), t(gl, torch.float64),
                       dcoef=dcb)
    with pytest.raises(_lib.QmcsplError) as ei:     # the non-finite position is reported
        spl.sync()
    assert ei.value.code == _lib.ERR_DEVICE
    dc_bad, dpos_bad = dcb.cpu().numpy(), dpb.cpu().numpy()
    keep = np.arange(12) != 5
    dc_ok, _, dpos_ok = gpu_backward(spl, pos[keep], gv[keep], gg[keep], gl[keep])
    assert np.all(np.isnan(dpos_bad[5])) and np.all(np.isfinite(dpos_bad[keep]))
    assert oracle.relative_error(dpos_bad[keep], dpos_ok) < 1e-13
    assert oracle.relative_error(dc_bad, dc_ok) < 1e-13
    empty = torch.zeros((0, 3), dtype=torch.float64, device=dev())
    dc = torch.zeros(spl.coef_shape(), dtype=torch.float64, device=dev())
    out = spl.backward(empty, dcoef=dc)
    spl.sync()
    assert out.shape == (0, 3) and float(dc.abs().sum()) == 0.0


# ---------------------------------------------------------------------------
# cell order (many walkers): the adjoint visits positions sorted by cell, coordinates from records
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
def test_cell_ordered_backward_matches_input_order_and_oracle(storage):
    """32,768 positions on the Si-like 8-atom cell (16 orbitals, 48^3, smoothing + Laplacian
    table): the cell-ordered adjoint against input order and
    against the oracle adjoint on the oracle's tables rounded as stored."""
    w = inputs.make_workload("c2")
    dims = w.cell.grid
    spl = splines(w.lattice, dims, w.miller, w.coef, method="smooth", storage=storage, separate_lap=True)
    n, o = w.pos.shape[0], w.coef.shape[0]
    gv, gg, gl = inputs.upstream_weights(n, o, 3100)
    if storage != "f64":
        gv, gg, gl = (x.astype(np.float32).astype(np.float64) for x in (gv, gg, gl))
    out = {}
    for order in ("input", "cell"):
        spl.set_order(order)
        out[order] = gpu_backward(spl, w.pos, gv, gg, gl)
    tol = TOL[storage] if storage != "bf16" else TOL["f32"]    # FP32 arithmetic on the stored tables
    for a, b in zip(out["cell"], out["input"]):
        assert oracle.relative_error(a, b) < (1e-13 if storage == "f64" else 1e-6)
    beta, blap = oracle_tables(w.lattice, w.miller, w.coef, dims, "smooth", storage, True)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(beta, w.lattice, w.pos, gv, gg, gl, beta_lap=blap)
    dc, dcl, dpos = out["cell"]
    for got, ref in ((dc, rdc), (dcl, rdcl), (dpos, rdpos)):
        assert oracle.relative_error(got, ref) < tol
    spl.close()


@pytest.mark.slow
def test_c3_mgo64_backward_full_size():
    """The many-walker adjoint at full size: 2048 x 256 positions, 128 orbitals on 96^3, FP32 tables
    with the Laplacian table, cell order.  dL/dr of every 1024th position against the oracle
    adjoint; the coefficient adjoint of the first 8 orbitals by the exact linearity identity
    sum(dL/dbeta * beta') = L(beta') with random tables beta' evaluated by the oracle at every
    position (beta' zero for the other orbitals)."""
    w = inputs.make_workload("c3")
    dims = w.cell.grid
    n, o = w.pos.shape[0], w.coef.shape[0]
    spl = splines(w.lattice, dims, w.miller, w.coef, method="smooth", storage="f32", separate_lap=True)
    rng = np.random.default_rng(3200)
    gv = rng.standard_normal((n, o), dtype=np.float32)
    gg = rng.standard_normal((n, 3, o), dtype=np.float32)
    gl = rng.standard_normal((n, o), dtype=np.float32)
    dc = torch.zeros(spl.coef_shape(), dtype=torch.float32, device=dev())
    dcl = torch.zeros_like(dc)
    dpos = spl.backward(t(w.pos, torch.float64), t(gv, torch.float32), t(gg, torch.float32), t(gl, torch.float32),
                        dcoef=dc, dcoef_lap=dcl)
    spl.sync()
    sample = np.arange(0, n, 1024)
    # dL/dr of a position involves every orbital: the oracle adjoint of the sample on all 128
    bfull, blfull = oracle_tables(w.lattice, w.miller, w.coef, dims, "smooth", "f32", True)
    up = [x[sample].astype(np.float64) for x in (gv, gg, gl)]
    _, _, rdpos = oracle.bspline_adjoint(bfull, w.lattice, w.pos[sample], *up, beta_lap=blfull)
    e_pos = oracle.relative_error(dpos.cpu().numpy()[sample], rdpos)
    b1 = rng.standard_normal(dims + (8,))
    b2 = rng.standard_normal(dims + (8,))
    v, g, l = oracle.bspline_eval(b1, w.lattice, w.pos, beta_lap=b2)
    ref = float(np.sum(gv[:, :8] * v) + np.sum(gg[:, :, :8] * g) + np.sum(gl[:, :8] * l))
    dcn, dcln = dc.double().cpu().numpy()[..., :8], dcl.double().cpu().numpy()[..., :8]
    lin = float(np.sum(dcn * b1) + np.sum(dcln * b2))
    scale = float(np.sum(np.abs(dcn) * np.abs(b1)) + np.sum(np.abs(dcln) * np.abs(b2)))
    print("c3 backward: dpos relative error %.2e, linearity %.3e vs %.3e (scale %.3e)" % (e_pos, lin, ref, scale))
    assert e_pos < TOL["f32"]
    assert abs(lin - ref) <= 2e-6 * scale
    spl.close()


@pytest.mark.parametrize("storage,n_orb,sep", [("f32", 150, True), ("f32", 40, False), ("f64", 70, True),
                                               ("bf16", 24, True)])
def test_gathered_adjoint_clustered_positions_and_ragged_slices(storage, n_orb, sep):
    """The coefficient adjoint gathered per 4^3-cell bin: half the positions packed into a few
    bins (hundreds per bin: several staged batches per bin), the rest spread out; orbital counts
    that need two slices (150 float, 70 double) or leave a slice ragged; against input order
    (the plain per-position kernel) and the oracle adjoint on the oracle's tables."""
    dims = (12, 13, 14)
    lat, mil, coef = inputs.random_cell(3300 + n_orb, dims, n_orb, 6.0, 5.0, NONORTHO)
    spl = splines(lat, dims, mil, coef, method="smooth", storage=storage, separate_lap=sep)
    rng = np.random.default_rng(3301)
    spread = inputs.positions(lat, 6000, 3302, -1, 2)
    # 6000 positions inside two bins' worth of cells (crystal coordinates in 0.05 .. 0.30)
    cluster = rng.uniform(0.05, 0.30, size=(6000, 3)) @ lat.T
    pos = np.ascontiguousarray(np.concatenate([spread, cluster])[rng.permutation(12000)])
    n = pos.shape[0]
    gv, gg, gl = inputs.upstream_weights(n, n_orb, 3303)
    if storage != "f64":
        gv, gg, gl = (x.astype(np.float32).astype(np.float64) for x in (gv, gg, gl))
    out = {}
    for order in ("input", "cell"):
        spl.set_order(order)
        out[order] = gpu_backward(spl, pos, gv, gg, gl)
    tol = 1e-12 if storage == "f64" else TOL["f32"]
    # two FP32 summation orders over up to hundreds of contributions per row: each within the
    # 2e-6 tolerance of the oracle, so within twice that of each other
    for a, b in zip(out["cell"], out["input"]):
        if a is not None:
            assert oracle.relative_error(a, b) < (1e-13 if storage == "f64" else 2 * TOL["f32"])
    beta, blap = oracle_tables(lat, mil, coef, dims, "smooth", storage, sep)
    rdc, rdcl, rdpos = oracle.bspline_adjoint(beta, lat, pos, gv, gg, gl, beta_lap=blap)
    dc, dcl, dpos = out["cell"]
    assert oracle.relative_error(dc, rdc) < tol
    if sep:
        assert oracle.relative_error(dcl, rdcl) < tol
    assert oracle.relative_error(dpos, rdpos) < tol
    spl.close()
