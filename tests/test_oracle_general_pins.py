"""Pins of the oracle's interpolating B-splines of any odd degree on uniform and non-uniform
periodic grids (Sec. II "Common features", "Grid"; the Appendix's recurrence).

Checks: the recurrence against the paper's printed cubic forms, the textbook central values
of the cardinal B-splines, partition of unity, derivatives by finite differences, exact
reproduction of the grid values, the degree-3 uniform case against the paper's cubic path,
trilinear interpolation for degree 1, convergence orders and continuity across knots."""
import math

import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs

NONORTHO = np.array([[5.0, 1.0, 0.5],
                     [0.0, 6.0, 0.3],
                     [0.0, 0.0, 7.0]])


def b_centred(xi):
    """Eq. (bsplinegridcenteredbasis)."""
    a = abs(xi)
    if a < 1:
        return 0.75 * a ** 3 - 1.5 * a ** 2 + 1
    if a < 2:
        return 0.25 * (2 - a) ** 3
    return 0.0


def test_recurrence_reproduces_the_printed_cubic_basis():
    """With C = 3/2 the recurrence gives Eq. (bsplinegridcenteredbasis) and the four
    polynomials of Eq. (b-splinebasis) on a uniform grid."""
    n = 16
    pts = np.arange(n) / n
    for xi in np.linspace(-2.5, 2.5, 41):
        x = xi / n                                  # grid point 0, grid units -> reduced
        got = oracle.recurrence_basis(pts, 3, np.array([-2]), x, 1.5)[0]
        assert got == pytest.approx(b_centred(xi), abs=1e-13)
    for t in (0.0, 0.13, 0.5, 0.77, 0.999):
        x = (5 + t) / n
        w = [oracle.recurrence_basis(pts, 3, np.array([5 + o - 2]), x, 1.5)[0] for o in (-1, 0, 1, 2)]
        np.testing.assert_allclose(w, oracle.basis("bspline", t), atol=1e-13)


def test_degree_constants_are_the_cardinal_central_values():
    """C_n = 1/B_n(0) with the textbook central values of the unit cardinal B-splines:
    B_1(0) = 1, B_3(0) = 2/3, B_5(0) = 11/20, B_7(0) = 151/315."""
    for n, b0 in ((1, 1.0), (3, 2.0 / 3.0), (5, 11.0 / 20.0), (7, 151.0 / 315.0)):
        assert oracle.degree_constant(n) == pytest.approx(1.0 / b0, rel=1e-13)


@pytest.mark.parametrize("degree", [1, 3, 5, 7])
@pytest.mark.parametrize("uniform", [True, False])
def test_partition_of_unity_and_derivatives(degree, uniform):
    """The periodic family sums to C everywhere; the derivative formula agrees with central
    differences of the recurrence (first and second derivatives)."""
    n = 11
    pts = np.arange(n) / n if uniform else inputs.graded_knots(n, 0.6, 0.1)
    C = 1.5 if degree == 3 else oracle.degree_constant(degree)
    rng = np.random.default_rng(degree)
    xs = rng.uniform(0, 1, 25)
    M = oracle.periodic_basis_matrix(pts, degree, xs, C)
    np.testing.assert_allclose(M.sum(axis=1), C, rtol=1e-13)
    h = 1e-6
    d1 = oracle.periodic_basis_matrix(pts, degree, xs, C, 1)
    fd1 = (oracle.periodic_basis_matrix(pts, degree, xs + h, C) -
           oracle.periodic_basis_matrix(pts, degree, xs - h, C)) / (2 * h)
    np.testing.assert_allclose(d1, fd1, atol=1e-6 * max(1.0, np.abs(d1).max()))
    if degree >= 3:
        d2 = oracle.periodic_basis_matrix(pts, degree, xs, C, 2)
        fd2 = (oracle.periodic_basis_matrix(pts, degree, xs + h, C, 1) -
               oracle.periodic_basis_matrix(pts, degree, xs - h, C, 1)) / (2 * h)
        np.testing.assert_allclose(d2, fd2, atol=1e-5 * max(1.0, np.abs(d2).max()))


@pytest.mark.parametrize("degree,graded", [(1, False), (3, False), (5, False), (7, False), (1, True), (3, True),
                                           (5, True), (7, True)])
def test_interpolation_reproduces_grid_values(degree, graded):
    dims = (9, 10, 11)
    knots = tuple(inputs.graded_knots(d, 0.5, 0.2 * a) for a, d in enumerate(dims)) if graded else (None,) * 3
    lat, mil, coef = inputs.random_cell(40 + degree, dims, 2, 4.0, 4.0, NONORTHO)
    beta, _ = oracle.general_interp_tables(lat, mil, coef, dims, degree, knots)
    pts = [oracle.axis_points(dims[a], knots[a]) for a in range(3)]
    rng = np.random.default_rng(degree)
    idx = rng.integers(0, dims, size=(12, 3))
    s = np.stack([pts[a][idx[:, a]] for a in range(3)], axis=1)
    pos = (s + np.array([1.0, -2.0, 0.0])) @ lat.T
    v, _, _ = oracle.general_eval(beta, lat, pos, degree, knots)
    pv, _, _, _ = oracle.pw_eval(lat, mil, coef, pos)
    assert oracle.relative_error(v, pv) < 1e-12


def test_cubic_uniform_equals_the_paper_path():
    """Degree 3 on a uniform grid with C = 3/2 is the paper's interpolating B-spline: the same
    coefficients and the same value, gradient and Laplacian (both Laplacian modes)."""
    dims = (8, 9, 10)
    lat, mil, coef = inputs.random_cell(50, dims, 3, 5.0, 4.0, NONORTHO)
    beta, blap = oracle.general_interp_tables(lat, mil, coef, dims, 3, laplacian=True)
    rb, rl = oracle.interpolating_tables(lat, mil, coef, dims, laplacian=True)
    assert oracle.relative_error(beta, rb) < 1e-12 and oracle.relative_error(blap, rl) < 1e-12
    pos = inputs.positions(lat, 15, 51, -1, 2)
    for bl in (None, blap):
        got = oracle.general_eval(beta, lat, pos, 3, beta_lap=bl)
        ref = oracle.bspline_eval(rb, lat, pos, beta_lap=None if bl is None else rl)
        for g, r in zip(got, ref):
            assert oracle.relative_error(g, r) < 1e-12


def test_degree_one_is_trilinear_interpolation():
    dims = (5, 6, 7)
    rng = np.random.default_rng(52)
    f = rng.standard_normal(dims + (2,))
    lat = np.diag([5.0, 6.0, 7.0])
    # linear interpolation: the coefficients are the grid values (C_1 = 1, B is the identity)
    pos = rng.uniform(0, 1, (10, 3)) * np.array([5.0, 6.0, 7.0])
    v, g, _ = oracle.general_eval(f, lat, pos, 1)
    for p in range(10):
        u = pos[p] / np.array([5.0, 6.0, 7.0]) * np.array(dims)
        i0 = np.floor(u).astype(int)
        t = u - i0
        ref = 0.0
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                    ref = ref + w * f[(i0[0] + dx) % 5, (i0[1] + dy) % 6, (i0[2] + dz) % 7]
        np.testing.assert_allclose(v[p], ref, atol=1e-13)


@pytest.mark.parametrize("degree,graded,ratio", [(1, False, 3.0), (3, False, 12.0), (5, False, 40.0),
                                                 (1, True, 3.0), (3, True, 11.0), (5, True, 35.0),
                                                 (7, True, 150.0)])
def test_convergence_order(degree, graded, ratio):
    """Refining the grid at a fixed planewave set converges the value as h^(n+1) (Sec. III A
    footnote for the cubic; the order of a degree-n spline in general), also on graded grids."""
    lat = np.eye(3) * 5.0
    mil = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 1], [0, -1, -1], [1, -1, 0], [-1, 1, 0]], dtype=np.int32)
    coef = np.array([[0.4 + 0.2j, 0.4 - 0.2j, 0.3, 0.3, -0.25j, 0.25j]])
    pos = inputs.positions(lat, 40, 53)
    pv, _, _, _ = oracle.pw_eval(lat, mil, coef, pos)
    errs = []
    for n in (12, 24):
        knots = tuple(inputs.graded_knots(n, 0.4, 0.1 * a) for a in range(3)) if graded else (None,) * 3
        beta, _ = oracle.general_interp_tables(lat, mil, coef, (n, n, n), degree, knots)
        v, _, _ = oracle.general_eval(beta, lat, pos, degree, knots)
        errs.append(np.abs(v - pv).max())
    assert errs[0] / errs[1] > ratio


@pytest.mark.parametrize("degree", [3, 5])
def test_graded_spline_is_smooth_across_knots_and_chain_rule(degree):
    """Splines of degree n are C^(n-1) (Sec. II): value, gradient and Laplacian agree on both
    sides of a non-uniform knot; the Cartesian gradient and Laplacian are the derivatives of
    the value (non-orthogonal cell)."""
    dims = (7, 8, 9)
    knots = tuple(inputs.graded_knots(d, 0.5, 0.15 * a) for a, d in enumerate(dims))
    rng = np.random.default_rng(54)
    beta = rng.standard_normal(dims + (2,))
    ainv = np.linalg.inv(NONORTHO)
    s0 = np.array([knots[0][3], 0.41, 0.77])
    eps = 1e-9
    lo = oracle.general_eval(beta, NONORTHO, (s0 - [eps, 0, 0]) @ NONORTHO.T, degree, knots)
    hi = oracle.general_eval(beta, NONORTHO, (s0 + [eps, 0, 0]) @ NONORTHO.T, degree, knots)
    for a, b in zip(lo, hi):
        assert np.abs(a - b).max() < 1e-5 * max(1.0, np.abs(a).max())
    pos = inputs.positions(NONORTHO, 6, 55)
    v, g, l = oracle.general_eval(beta, NONORTHO, pos, degree, knots)
    h = 1e-5
    fd_g, fd_l = np.zeros_like(g), np.zeros_like(l)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        vp, gp, _ = oracle.general_eval(beta, NONORTHO, pos + e, degree, knots)
        vm, gm, _ = oracle.general_eval(beta, NONORTHO, pos - e, degree, knots)
        fd_g[:, a] = (vp - vm) / (2 * h)
        fd_l += (gp[:, a] - gm[:, a]) / (2 * h)
    assert oracle.relative_error(g, fd_g) < 1e-7
    assert oracle.relative_error(l, fd_l) < 1e-5


def test_degree_one_graded_is_piecewise_linear_interpolation():
    """Degree 1 on a graded grid: the coefficients are the grid values (the collocation matrix
    is the identity) and the spline is trilinear interpolation between neighbouring grid
    points with weights (x - x_i) / (x_{i+1} - x_i) per axis."""
    dims = (5, 6, 7)
    knots = tuple(inputs.graded_knots(d, 0.5, 0.2 * a) for a, d in enumerate(dims))
    lat, mil, coef = inputs.random_cell(56, dims, 2, 3.0, 4.0, np.diag([5.0, 6.0, 7.0]))
    beta, _ = oracle.general_interp_tables(lat, mil, coef, dims, 1, knots)
    grid = oracle.general_grid_values(lat, mil, coef, [np.asarray(k) for k in knots])
    np.testing.assert_allclose(beta, grid, atol=1e-12 * np.abs(grid).max())
    rng = np.random.default_rng(57)
    s = rng.uniform(0, 1, (10, 3))
    v, _, _ = oracle.general_eval(beta, lat, s @ lat.T, 1, knots)
    for p in range(10):
        i0, t = [], []
        for a in range(3):
            k = np.asarray(knots[a])
            x = s[p, a]
            i = int(np.searchsorted(k, x, side="right")) - 1
            if i < 0:                               # below the first point: last interval
                i, x = dims[a] - 1, x + 1.0
            right = k[i + 1] if i + 1 < dims[a] else k[0] + 1.0
            i0.append(i)
            t.append((x - k[i]) / (right - k[i]))
        ref = 0.0
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = (t[0] if dx else 1 - t[0]) * (t[1] if dy else 1 - t[1]) * (t[2] if dz else 1 - t[2])
                    ref = ref + w * beta[(i0[0] + dx) % dims[0], (i0[1] + dy) % dims[1], (i0[2] + dz) % dims[2]]
        np.testing.assert_allclose(v[p], ref, atol=1e-13 * max(1.0, np.abs(ref).max()))


# ---------------------------------------------------------------------------
# smoothing B-splines of other odd degrees (Eq. b-splinecoefficients with the degree-n basis)
# ---------------------------------------------------------------------------

def fourier_of_recurrence_basis(theta, degree, nodes=32):
    """Integral over R of the recurrence's centred degree-n basis (with C_n) times
    cos(theta xi), by Gauss-Legendre on every unit piece of its support."""
    C = 1.5 if degree == 3 else oracle.degree_constant(degree)
    nb = 64
    pts = np.arange(nb) / nb
    x, w = np.polynomial.legendre.leggauss(nodes)
    half = (degree + 1) // 2
    total = 0.0
    for lo in range(-half, half):
        xi = lo + 0.5 * (x + 1)
        vals = np.array([oracle.recurrence_basis(pts, degree, np.array([-half]), v / nb, C)[0] for v in xi])
        total += 0.5 * np.sum(w * vals * np.cos(theta * xi))
    return total


@pytest.mark.parametrize("degree", [1, 3, 5, 7])
def test_degree_gamma_is_the_fourier_transform_of_the_basis(degree):
    """gamma for the degree-n basis is the Fourier transform of the recurrence's centred basis
    (the paper defines gamma this way for the cubic); degree 3 is the paper's gamma."""
    for th in (0.0, 0.3, 1.0, 2.0, np.pi, 4.5):
        assert oracle.gamma_degree_axis(np.array([th]), degree)[0] == pytest.approx(
            fourier_of_recurrence_basis(th, degree), rel=1e-10, abs=1e-13)
    th = np.linspace(0, 6, 25)
    if degree == 3:
        np.testing.assert_allclose(oracle.gamma_degree_axis(th, 3), oracle.gamma_axis(th), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("degree", [1, 5])
def test_degree_smoothing_fourier_components_are_exact(degree):
    """The smoothing spline of degree n reproduces every planewave coefficient c_G when no G
    aliases: its Fourier component (grid sum of beta times the basis transform) is c_G."""
    lat, mil, coef = inputs.random_cell(60 + degree, (9, 10, 11), 2, 4.0, 4.0, NONORTHO)
    dims = np.array((9, 10, 11))
    assert np.all(np.abs(mil).max(0) < dims / 2)
    beta, _ = oracle.smoothing_tables_degree(lat, mil, coef, tuple(dims), degree)
    bhat = np.fft.fftn(np.moveaxis(beta, -1, 0), axes=(1, 2, 3))
    cache = {}
    for idx, n in enumerate(mil[::7]):
        th = 2 * np.pi * n / dims
        Q = 1.0
        for a in range(3):
            key = round(float(th[a]), 14)
            if key not in cache:
                cache[key] = fourier_of_recurrence_basis(th[a], degree)
            Q *= cache[key]
        k = np.mod(n, dims)
        comp = bhat[:, k[0], k[1], k[2]] * Q / dims.prod()
        j = np.nonzero(np.all(mil == n, axis=1))[0][0]
        np.testing.assert_allclose(comp, coef[:, j], atol=1e-11 * np.abs(coef).max())


def test_degree_smoothing_cubic_is_the_paper_path_and_higher_degree_converges_faster():
    dims = (8, 9, 10)
    lat, mil, coef = inputs.random_cell(70, dims, 2, 5.0, 4.0, NONORTHO)
    b3, l3 = oracle.smoothing_tables_degree(lat, mil, coef, dims, 3, laplacian=True)
    rb, rl = oracle.smoothing_tables(lat, mil, coef, dims, laplacian=True)
    assert oracle.relative_error(b3, rb) < 1e-13 and oracle.relative_error(l3, rl) < 1e-13
    lat = np.eye(3) * 5.0
    mil = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 1], [0, -1, -1], [1, -1, 0], [-1, 1, 0]], dtype=np.int32)
    coef = np.array([[0.4 + 0.2j, 0.4 - 0.2j, 0.3, 0.3, -0.25j, 0.25j]])
    pos = inputs.positions(lat, 40, 71)
    pv, _, _, _ = oracle.pw_eval(lat, mil, coef, pos)
    for degree, grids, ratio in ((1, (24, 48), 3.0), (5, (12, 24), 40.0)):   # degree 1: past its pre-asymptotic range
        errs = []
        for n in grids:
            beta, _ = oracle.smoothing_tables_degree(lat, mil, coef, (n, n, n), degree)
            v, _, _ = oracle.general_eval(beta, lat, pos, degree)
            errs.append(np.abs(v - pv).max())
        assert errs[0] / errs[1] > ratio


# ---------------------------------------------------------------------------
# the adjoint of the general evaluation (general_adjoint)
# ---------------------------------------------------------------------------

def _general_loss(beta, pos, g, degree, knots, beta_lap=None):
    v, gr, l = oracle.general_eval(beta, NONORTHO, pos, degree, knots, beta_lap=beta_lap)
    return float(np.sum(g[0] * v) + np.sum(g[1] * gr) + np.sum(g[2] * l))


@pytest.mark.parametrize("sep", [False, True])
def test_general_adjoint_cubic_uniform_equals_the_cubic_adjoint(sep):
    """Degree 3 on a uniform grid is the paper's tricubic spline, whose adjoint the C oracle
    computes by its own loops: the two transposes agree."""
    dims = (6, 7, 8)
    rng = np.random.default_rng(60)
    beta = rng.standard_normal(dims + (3,))
    blap = rng.standard_normal(dims + (3,)) if sep else None
    pos = inputs.positions(NONORTHO, 7, 61, -1, 2)
    g = inputs.upstream_weights(7, 3, 62)
    dc, dcl, dp = oracle.general_adjoint(beta, NONORTHO, pos, *g, degree=3, beta_lap=blap)
    rdc, rdcl, rdp = oracle.bspline_adjoint(beta, NONORTHO, pos, *g, beta_lap=blap)
    assert oracle.relative_error(dc, rdc) < 1e-12
    if sep:
        assert oracle.relative_error(dcl, rdcl) < 1e-12
    assert oracle.relative_error(dp, rdp) < 1e-11


@pytest.mark.parametrize("degree,graded", [(1, False), (5, False), (7, False), (1, True), (3, True), (5, True)])
@pytest.mark.parametrize("sep", [False, True])
def test_general_adjoint_linearity_and_position_fd(degree, graded, sep):
    """The loss is linear in the coefficients: sum(dL/dbeta * beta') = L(beta') for random
    tables beta' through general_eval; and dL/dr against central differences of the loss
    (positions away from the grid planes, where the degree-1 spline has kinks)."""
    dims = (8, 9, 10)
    knots = tuple(inputs.graded_knots(d, 0.45, 0.2 * a) for a, d in enumerate(dims)) if graded \
        else (None, None, None)
    rng = np.random.default_rng(63 + degree + 10 * graded)
    beta = rng.standard_normal(dims + (2,))
    blap = rng.standard_normal(dims + (2,)) if sep else None
    pos = inputs.positions(NONORTHO, 6, 64 + degree, -1, 2)
    pts = [oracle.axis_points(d, k) for d, k in zip(dims, knots)]
    s = pos @ np.linalg.inv(NONORTHO).T
    s = s - np.floor(s)
    for a in range(3):      # keep every position 1e-3 away from a grid plane
        d = s[:, a, None] - np.concatenate([pts[a], [1.0]])[None, :]
        near = np.min(np.abs(d), axis=1) < 1e-3
        s[near, a] += 2e-3
    pos = s @ NONORTHO.T
    g = inputs.upstream_weights(6, 2, 65)
    dc, dcl, dp = oracle.general_adjoint(beta, NONORTHO, pos, *g, degree=degree, knots=knots, beta_lap=blap)
    for _ in range(2):
        b1 = rng.standard_normal(dims + (2,))
        b2 = rng.standard_normal(dims + (2,)) if sep else None
        lin = np.sum(dc * b1) + (np.sum(dcl * b2) if sep else 0.0)
        ref = _general_loss(b1, pos, g, degree, knots, b2)
        assert abs(lin - ref) <= 1e-11 * max(1.0, abs(ref))
    h = 1e-6
    fd = np.zeros_like(dp)
    for p in range(pos.shape[0]):
        gp = tuple(x[p:p + 1] for x in g)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd[p, a] = (_general_loss(beta, pos[p:p + 1] + e, gp, degree, knots, blap) -
                        _general_loss(beta, pos[p:p + 1] - e, gp, degree, knots, blap)) / (2 * h)
    assert oracle.relative_error(dp, fd) < 1e-6
