"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them compares the oracle with
itself: the checks are closed forms, the paper's second printed form of the same
object, brute-force dense solves, quadrature, invariants and convergence rates.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1309_6250_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")

NONORTHO = np.array([[5.0, 1.0, 0.5],
                     [0.0, 6.0, 0.3],
                     [0.0, 0.0, 7.0]])   # columns are a_1, a_2, a_3


def golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split("=")
                out[k.strip()] = float(v)
    return out


# ---------------------------------------------------------------------------
# grid-centred forms printed beside the polynomial forms (Appendix)
# ---------------------------------------------------------------------------

def b_centred(xi):
    """Eq. (bsplinegridcenteredbasis)."""
    a = abs(xi)
    if a < 1:
        return 0.75 * a ** 3 - 1.5 * xi ** 2 + 1.0
    if a < 2:
        return 0.25 * (2 - a) ** 3
    return 0.0


def l_centred(xi):
    """Eq. (lagrangegridcenteredbasis), the expanded polynomial of each branch."""
    a = abs(xi)
    if a < 1:
        return 0.5 * a ** 3 - xi ** 2 - 0.5 * a + 1.0
    if a < 2:
        return -a ** 3 / 6.0 + xi ** 2 - 11.0 / 6.0 * a + 1.0
    return 0.0


def l_centred_factored(xi):
    """Eq. (lagrangegridcenteredbasis), the factored form of each branch."""
    a = abs(xi)
    if a < 1:
        return 0.5 * (a + 1) * (a - 1) * (a - 2)
    if a < 2:
        return -(a - 1) * (a - 2) * (a - 3) / 6.0
    return 0.0


def s1_centred(xi):
    a = abs(xi)
    return 1.0 - a if a < 1 else 0.0


def s2_centred(xi):
    a = abs(xi)
    return (-a ** 3 / 6.0 + xi ** 2 / 2.0 - a / 3.0) if a < 1 else 0.0


TS = np.concatenate([np.linspace(0.0, 0.999, 37), [1e-9, 0.5, 0.999999]])


def test_bspline_basis_matches_grid_centred_form_and_sums():
    """Eq. (b-splinebasis) vs Eq. (bsplinegridcenteredbasis): b_l(t) = b(t - l);
    with C = 3/2 the weights sum to 3/2 and the derivative weights to 0."""
    for t in TS:
        w = oracle.basis("bspline", t, 0)
        for j in range(4):
            assert w[j] == pytest.approx(b_centred(t - (j - 1)), abs=1e-15)
        assert w.sum() == pytest.approx(1.5, abs=1e-15)
        assert oracle.basis("bspline", t, 1).sum() == pytest.approx(0.0, abs=1e-14)
        assert oracle.basis("bspline", t, 2).sum() == pytest.approx(0.0, abs=1e-14)
        assert oracle.basis("bspline", t, 3).sum() == pytest.approx(0.0, abs=1e-14)


@pytest.mark.parametrize("kind", ["bspline", "lagrange", "pp"])
def test_basis_derivatives_are_derivatives(kind):
    """The derivative weights are the t-derivatives of the weights (central differences)."""
    h = 1e-5
    for t in np.linspace(0.05, 0.95, 19):
        for d in range(3):
            fd = (oracle.basis(kind, t + h, d) - oracle.basis(kind, t - h, d)) / (2 * h)
            np.testing.assert_allclose(oracle.basis(kind, t, d + 1), fd, atol=1e-8)


def test_lagrange_basis_forms_and_exactness():
    """Eq. (lagrangebasis) vs both printed grid-centred forms; sum = 1; interpolation
    conditions l_i(j) = delta_ij; cubics are reproduced exactly (Appendix A)."""
    for t in TS:
        w = oracle.basis("lagrange", t, 0)
        for j in range(4):
            assert w[j] == pytest.approx(l_centred(t - (j - 1)), abs=1e-14)
            assert w[j] == pytest.approx(l_centred_factored(t - (j - 1)), abs=1e-14)
        assert w.sum() == pytest.approx(1.0, abs=1e-14)
        for p in ([1, 0, 0, 0], [0.3, -1.2, 0.7, 2.0], [0, 0, 0, 1]):
            poly = np.polynomial.Polynomial(p)
            assert np.dot(w, poly(np.arange(-1, 3))) == pytest.approx(poly(t), abs=1e-12)
    # interpolation at the nodes (the node t = 1 is the next cell's t = 0)
    np.testing.assert_allclose(oracle.basis("lagrange", 0.0, 0), [0, 1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(oracle.basis("lagrange", 1.0, 0), [0, 0, 1, 0], atol=1e-15)


def test_pp_basis_forms():
    """Eq. (pp-splinebasis) vs Eq. (pp-splinegridcenteredbasis); s_0^1 + s_1^1 = 1; a cubic
    with its exact second derivatives as sigma^2 is reproduced (Appendix B)."""
    for t in TS:
        w = oracle.basis("pp", t, 0)
        assert w[0] == pytest.approx(s1_centred(t), abs=1e-15)
        assert w[1] == pytest.approx(s1_centred(t - 1), abs=1e-15)
        assert w[2] == pytest.approx(s2_centred(t), abs=1e-15)
        assert w[3] == pytest.approx(s2_centred(t - 1), abs=1e-15)
        assert w[0] + w[1] == pytest.approx(1.0, abs=1e-15)
        poly = np.polynomial.Polynomial([0.2, -0.7, 1.3, 0.9])
        d2 = poly.deriv(2)
        val = w[0] * poly(0) + w[1] * poly(1) + w[2] * d2(0) + w[3] * d2(1)
        assert val == pytest.approx(poly(t), abs=1e-13)


def test_golden_paper_values():
    """Numbers printed in the paper (tests/golden/paper_values.txt)."""
    g = golden()
    b = oracle.basis("bspline", 0.0, 0)
    assert b[1] == g["bspline_b_at_0"]
    assert b[0] == g["bspline_b_at_1"] and b[2] == g["bspline_b_at_1"]
    assert b[3] == g["bspline_b_at_2"]
    tt = np.linspace(0, 1, 2001)
    assert max(oracle.basis("bspline", t, 0).max() for t in tt) == pytest.approx(g["bspline_max"])
    lg = oracle.basis("lagrange", 0.0, 0)
    assert lg[1] == g["lagrange_l_at_0"] and lg[2] == g["lagrange_l_at_1"]
    pp = oracle.basis("pp", 0.0, 0)
    assert pp[0] == g["pp_s1_at_0"] and pp[2] == g["pp_s2_at_0"]
    # the pp periodic system: diag 4, off-diagonals and corners 1, rhs 6 x second difference
    rng = np.random.default_rng(5)
    f = rng.standard_normal((9, 2, 3, 1))
    s = oracle.pp_second_derivative(f, 0)
    lhs = g["pp_matrix_diag"] * s + g["pp_matrix_off"] * (np.roll(s, 1, 0) + np.roll(s, -1, 0))
    rhs = g["pp_rhs_factor"] * (np.roll(f, 1, 0) - 2 * f + np.roll(f, -1, 0))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_natural_spacing_grid_to_pw_ratio():
    """Sec. III C footnote: at the natural spacing h = pi/G_max (Eq. natural_spacing) of a
    cubic cell, grid points / planewaves in a sphere -> 6/pi."""
    g = golden()
    a = 10.0
    ecut = 120.0
    gmax = math.sqrt(2 * ecut)
    n_pw = inputs.miller_set(np.eye(3) * a, ecut).shape[0]
    h = math.pi / gmax
    n_grid = (a / h) ** 3
    assert n_grid / n_pw == pytest.approx(g["grid_to_pw_ratio_natural"], rel=0.02)


# ---------------------------------------------------------------------------
# gamma of Eq. (b-splinecoefficients)
# ---------------------------------------------------------------------------

def gauss_fourier_of_b(theta, nodes=24):
    """Integral of b(xi) cos(theta xi) over R by Gauss-Legendre on the four unit pieces
    of Eq. (bsplinegridcenteredbasis)."""
    x, w = np.polynomial.legendre.leggauss(nodes)
    total = 0.0
    for lo in (-2, -1, 0, 1):
        xi = lo + 0.5 * (x + 1)
        total += 0.5 * np.sum(w * np.array([b_centred(v) for v in xi]) * np.cos(theta * xi))
    return total


def test_gamma_is_fourier_transform_of_b():
    """gamma per axis = Fourier transform of the grid-centred B-spline (Eq. b-splinecoefficients),
    the first printed form, and 3/2 at zero."""
    th = np.array([0.0, 1e-3, 0.05, 0.3, 1.0, 2.0, math.pi, 4.0, 6.0])
    gam = oracle.gamma_axis(th)
    for t, gv in zip(th, gam):
        # the quadrature integrates an O(1) integrand, so its error is absolute
        assert gv == pytest.approx(gauss_fourier_of_b(t), rel=1e-13, abs=1e-14)
    assert gam[0] == 1.5
    mid = th[(th > 0.2)]
    form1 = 3 * (3 - 4 * np.cos(mid) + np.cos(2 * mid)) / mid ** 4
    np.testing.assert_allclose(oracle.gamma_axis(mid), form1, rtol=1e-11)


# ---------------------------------------------------------------------------
# planewave sums, Eq. (pw_orbital)
# ---------------------------------------------------------------------------

def test_single_planewave_closed_form():
    """cos(G.r) and sin(G.r): analytic gradient -G sin / G cos, Laplacian -|G|^2 (.)"""
    mil = np.array([[1, 2, -1], [-1, -2, 1]], dtype=np.int32)
    coef = np.array([[0.5, 0.5], [-0.5j, 0.5j]])
    rng = np.random.default_rng(0)
    pos = rng.uniform(-10, 10, (50, 3))
    val, grad, lap, im = oracle.pw_eval(NONORTHO, mil, coef, pos)
    G = 2 * np.pi * np.linalg.inv(NONORTHO).T @ mil[0]
    ph = pos @ G
    np.testing.assert_allclose(val[:, 0], np.cos(ph), atol=1e-13)
    np.testing.assert_allclose(val[:, 1], np.sin(ph), atol=1e-13)
    np.testing.assert_allclose(grad[:, :, 0], -np.sin(ph)[:, None] * G[None], atol=1e-12)
    np.testing.assert_allclose(grad[:, :, 1], np.cos(ph)[:, None] * G[None], atol=1e-12)
    np.testing.assert_allclose(lap[:, 0], -G @ G * np.cos(ph), atol=1e-11)
    np.testing.assert_allclose(lap[:, 1], -G @ G * np.sin(ph), atol=1e-11)
    assert im < 1e-15


def test_generated_orbitals_are_real():
    """Gamma-point orbitals (Sec. III) from Hermitian coefficients have no imaginary part."""
    lat, mil, coef = inputs.random_cell(3, (8, 8, 8), 3, 5.0, 4.0, NONORTHO)
    pos = inputs.positions(lat, 40, 7, -1.0, 2.0)
    val, _, _, im = oracle.pw_eval(lat, mil, coef, pos)
    assert im < 1e-13 * np.abs(val).max()


def test_parseval_kinetic_energy():
    """-1/2 <phi lap phi>/<phi^2> over the cell = 1/2 sum |G|^2 |c|^2 / sum |c|^2, with the
    average taken exactly on a grid finer than twice the largest Miller index."""
    lat, mil, coef = inputs.random_cell(11, (8, 8, 8), 2, 4.0, 4.0, NONORTHO)
    M = 2 * int(np.abs(mil).max()) + 2
    idx = np.stack(np.meshgrid(*[np.arange(M)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = (idx / M) @ lat.T
    val, _, lap, _ = oracle.pw_eval(lat, mil, coef, pos)
    G = oracle.g_vectors(lat, mil)
    g2 = np.einsum("ij,ij->i", G, G)
    expect = 0.5 * np.sum(g2[None] * np.abs(coef) ** 2, 1) / np.sum(np.abs(coef) ** 2, 1)
    np.testing.assert_allclose(oracle.kinetic_energy(val, lap), expect, rtol=1e-12)


# ---------------------------------------------------------------------------
# coefficient construction
# ---------------------------------------------------------------------------

def test_fold_and_inverse_fft_equal_direct_sum():
    """The folded inverse FFT is the planewave sum at the grid points, also with aliases
    (Miller index N/2 and beyond)."""
    lat, mil, coef = inputs.random_cell(4, (6, 7, 8), 2, 9.0, 6.0, NONORTHO)
    assert np.abs(mil).max() >= 4          # some G alias on the 6- and 7-point axes
    dims = (6, 7, 8)
    f = oracle.grid_values(lat, mil, coef, dims)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, 3)
    pos = (idx / np.array(dims)) @ lat.T
    val, grad, lap, _ = oracle.pw_eval(lat, mil, coef, pos)
    np.testing.assert_allclose(f.reshape(-1, 2), val, atol=1e-12 * np.abs(val).max())
    for a, w in enumerate(("dx", "dy", "dz")):
        g = oracle.grid_values(lat, mil, coef, dims, w).reshape(-1, 2)
        np.testing.assert_allclose(g, grad[:, a], atol=1e-12 * np.abs(grad).max())
    fl = oracle.grid_values(lat, mil, coef, dims, "lap").reshape(-1, 2)
    np.testing.assert_allclose(fl, lap, atol=1e-12 * np.abs(lap).max())
    # the smoothing coefficients summed point by point
    beta = oracle.smoothing_coefficients(lat, mil, coef, dims)
    pts = idx[::7]
    direct = oracle.smoothing_coefficients_at(lat, mil, coef, dims, pts)
    np.testing.assert_allclose(beta[pts[:, 0], pts[:, 1], pts[:, 2]], direct,
                               atol=1e-12 * np.abs(beta).max())


def test_cyclic_solver_against_dense_solve():
    """Thomas + Sherman-Morrison equals a dense solve of the periodic tridiagonal system."""
    rng = np.random.default_rng(9)
    for n, d, o in ((3, 1.0, 0.25), (5, 4.0, 1.0), (16, 1.0, 0.25), (7, 2.5, -0.7)):
        A = np.zeros((n, n))
        for i in range(n):
            A[i, i] = d
            A[i, (i - 1) % n] += o
            A[i, (i + 1) % n] += o
        rhs = rng.standard_normal((n, 4))
        x = oracle.cyclic_tridiagonal_solve(rhs, 0, d, o)
        np.testing.assert_allclose(x, np.linalg.solve(A, rhs), atol=1e-13)


def test_interpolating_coefficients_against_dense_kronecker_solve():
    """Appendix, interpolating B-spline: the three-stage solve equals one dense solve of
    (B^x (x) B^y (x) B^z) beta = phi with B_il = b(i - l) periodic, on a 5x6x7 grid."""
    dims = (5, 6, 7)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal(dims + (2,))
    beta = oracle.interpolating_coefficients(phi)

    def B(n):
        M = np.zeros((n, n))
        for i in range(n):
            for l in range(n):
                for img in (-1, 0, 1):
                    M[i, l] += b_centred(i - l + img * n)
        return M
    K = np.kron(np.kron(B(dims[0]), B(dims[1])), B(dims[2]))
    dense = np.linalg.solve(K, phi.reshape(-1, 2)).reshape(phi.shape)
    np.testing.assert_allclose(beta, dense, atol=1e-12)


def brute_force_spline(beta, lattice, pos, basis_fn):
    """phi(u) = sum over every grid point and its periodic images of
    beta_l b(u_x - l_x) b(u_y - l_y) b(u_z - l_z), no stencil bookkeeping."""
    dims = beta.shape[:3]
    s = np.asarray(pos) @ np.linalg.inv(lattice).T
    out = np.zeros((len(pos), beta.shape[3]))
    for p, sp in enumerate(s):
        u = (sp - np.floor(sp)) * np.array(dims)
        wx = [np.array([basis_fn(u[a] - l - img * dims[a]) for l in range(dims[a])]).reshape(-1)
              for a in range(3) for img in (-1, 0, 1)]
        w = [sum(wx[3 * a + k] for k in range(3)) for a in range(3)]
        out[p] = np.einsum("i,j,k,ijko->o", w[0], w[1], w[2], beta)
    return out


def test_stencil_evaluation_equals_brute_force_sum():
    """Eq. (b-splineapproximation) through the 4x4x4 stencil equals the sum of every
    grid-centred basis function with periodic images (pins index, wrap and stencil)."""
    dims = (6, 5, 7)
    rng = np.random.default_rng(3)
    beta = rng.standard_normal(dims + (2,))
    pos = inputs.positions(NONORTHO, 25, 8, -2.0, 3.0)
    val, _, _ = oracle.bspline_eval(beta, NONORTHO, pos)
    np.testing.assert_allclose(val, brute_force_spline(beta, NONORTHO, pos, b_centred), atol=1e-12)
    tabs = np.stack([beta] * 5)
    lv, _, _ = oracle.lagrange_eval(tabs, NONORTHO, pos)
    np.testing.assert_allclose(lv, brute_force_spline(beta, NONORTHO, pos, l_centred), atol=1e-12)


def test_interpolating_spline_reproduces_grid_values():
    """Appendix: the interpolating B-spline takes the planewave values at the grid
    points (direct planewave sums, not the FFT route) to 1e-12."""
    lat, mil, coef = inputs.random_cell(5, (8, 9, 10), 3, 5.0, 4.0, NONORTHO)
    dims = (8, 9, 10)
    beta, _ = oracle.interpolating_tables(lat, mil, coef, dims)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, 3)
    pos = (idx / np.array(dims)) @ lat.T
    pw, _, _, _ = oracle.pw_eval(lat, mil, coef, pos)
    val, _, _ = oracle.bspline_eval(beta, lat, pos)
    assert oracle.relative_error(val, pw) < 1e-12


def test_tridiagonal_route_equals_fourier_division():
    """The interpolating coefficients equal the grid-value spectrum divided by the
    B-spline symbol prod_m (1 + cos(th_m)/2), from b(0) = 1, b(+-1) = 1/4."""
    lat, mil, coef = inputs.random_cell(6, (8, 8, 12), 2, 5.0, 4.0, NONORTHO)
    dims = (8, 8, 12)
    beta, _ = oracle.interpolating_tables(lat, mil, coef, dims)
    X = oracle.fold(mil, coef, dims)
    k = [np.arange(d) for d in dims]
    sym = [1 + 0.5 * np.cos(2 * np.pi * kk / d) for kk, d in zip(k, dims)]
    X = X / (sym[0][:, None, None] * sym[1][None, :, None] * sym[2][None, None, :])[None]
    viaf, _ = oracle.grid_sum(X)
    np.testing.assert_allclose(beta, viaf, atol=1e-12 * np.abs(beta).max())


def test_smoothing_spline_fourier_components_are_exact():
    """Sec. 'Smoothing B-spline coefficients': the spline's Fourier components equal c_G
    when no G aliases.  The component is integrated exactly: a discrete sum over grid
    points times a Gauss-Legendre integral of the grid-centred B-spline per axis."""
    lat, mil, coef = inputs.random_cell(7, (9, 10, 11), 2, 4.0, 4.0, NONORTHO)
    dims = np.array((9, 10, 11))
    assert np.all(np.abs(mil).max(0) < dims / 2)
    beta = oracle.smoothing_coefficients(lat, mil, coef, tuple(dims))
    bhat = np.fft.fftn(np.moveaxis(beta, -1, 0), axes=(1, 2, 3))  # sum_l beta_l e^{-i th.l}
    q = {}
    for n in mil:
        th = 2 * np.pi * n / dims
        Q = 1.0
        for a in range(3):
            key = round(float(th[a]), 15)
            if key not in q:
                q[key] = gauss_fourier_of_b(th[a])
            Q *= q[key]
        k = np.mod(n, dims)
        comp = bhat[:, k[0], k[1], k[2]] * Q / dims.prod()
        idx = np.nonzero(np.all(mil == n, axis=1))[0][0]
        np.testing.assert_allclose(comp, coef[:, idx], atol=1e-12 * np.abs(coef).max())


def test_constant_orbital_is_reproduced_exactly():
    """Only G = 0: smoothing and interpolating splines both return the constant, with zero
    gradient and Laplacian (gamma(0) = 27/8 = sum of the 64 weights)."""
    mil = np.zeros((1, 3), dtype=np.int32)
    coef = np.array([[1.7], [-0.3]])
    dims = (6, 7, 5)
    pos = inputs.positions(NONORTHO, 30, 1, -1, 2)
    for beta in (oracle.smoothing_coefficients(NONORTHO, mil, coef, dims),
                 oracle.interpolating_tables(NONORTHO, mil, coef, dims)[0]):
        val, grad, lap = oracle.bspline_eval(beta, NONORTHO, pos)
        np.testing.assert_allclose(val, np.broadcast_to([1.7, -0.3], val.shape), atol=1e-14)
        assert np.abs(grad).max() < 1e-13 and np.abs(lap).max() < 1e-12


def test_interpolating_bspline_equals_pp_spline():
    """Sec. II and III A: interpolating B-splines and pp-splines give identical values
    (and hence derivatives) for the same grid values and periodic boundaries."""
    lat, mil, coef = inputs.random_cell(8, (7, 8, 9), 2, 5.0, 4.0, NONORTHO)
    dims = (7, 8, 9)
    beta, _ = oracle.interpolating_tables(lat, mil, coef, dims)
    sig = oracle.pp_tables(oracle.grid_values(lat, mil, coef, dims))
    pos = inputs.positions(lat, 60, 4, -1, 2)
    vb, gb, lb = oracle.bspline_eval(beta, lat, pos)
    vp, gp, lp = oracle.pp_eval(sig, lat, pos)
    assert oracle.relative_error(vp, vb) < 1e-12
    assert oracle.relative_error(gp, gb) < 1e-12
    assert oracle.relative_error(lp, lb) < 1e-11


def test_pp_mixed_derivative_order_is_irrelevant():
    """The 1-D operators of Eq. (pp-splinecoefficients3) commute."""
    rng = np.random.default_rng(1)
    f = rng.standard_normal((6, 7, 8, 1))
    xy = oracle.pp_second_derivative(oracle.pp_second_derivative(f, 0), 1)
    yx = oracle.pp_second_derivative(oracle.pp_second_derivative(f, 1), 0)
    np.testing.assert_allclose(xy, yx, atol=1e-13)


def test_lagrange_tables_interpolate_planewave_derivatives():
    """Lagrange interpolation (Appendix A) of the five tables of Sec. III C returns the
    planewave value, gradient and Laplacian at the grid points."""
    lat, mil, coef = inputs.random_cell(12, (8, 8, 8), 2, 5.0, 4.0, NONORTHO)
    dims = (8, 8, 8)
    tabs = oracle.lagrange_tables(lat, mil, coef, dims)
    idx = np.stack(np.meshgrid(*[np.arange(d) for d in dims], indexing="ij"), -1).reshape(-1, 3)[::5]
    pos = (idx / np.array(dims)) @ lat.T
    v, g, l = oracle.lagrange_eval(tabs, lat, pos)
    pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
    assert oracle.relative_error(v, pv) < 1e-12
    assert oracle.relative_error(g, pg) < 1e-12
    assert oracle.relative_error(l, pl) < 1e-12


# ---------------------------------------------------------------------------
# evaluation: chain rule, continuity, periodicity, convergence
# ---------------------------------------------------------------------------

def test_chain_rule_by_finite_differences():
    """Sec. II (Coordinates): the Cartesian gradient is the derivative of the value and the
    Laplacian the divergence of the gradient, on a non-orthogonal cell with unequal N."""
    rng = np.random.default_rng(21)
    dims = (7, 9, 11)
    beta = rng.standard_normal(dims + (2,))
    pos = inputs.positions(NONORTHO, 20, 3)
    val, grad, lap = oracle.bspline_eval(beta, NONORTHO, pos)
    h = 1e-5
    fd_g = np.zeros_like(grad)
    fd_l = np.zeros_like(lap)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        vp, gp, _ = oracle.bspline_eval(beta, NONORTHO, pos + e)
        vm, gm, _ = oracle.bspline_eval(beta, NONORTHO, pos - e)
        fd_g[:, a] = (vp - vm) / (2 * h)
        fd_l += (gp[:, a] - gm[:, a]) / (2 * h)
    assert oracle.relative_error(grad, fd_g) < 1e-8
    assert oracle.relative_error(lap, fd_l) < 1e-6


def test_continuity_across_grid_planes_and_lagrange_negative_control():
    """B-splines are C2 (Appendix C): value, gradient and Hessian agree on both sides of a
    grid plane.  Lagrange interpolation has no continuous derivative (Appendix A)."""
    rng = np.random.default_rng(22)
    dims = (6, 6, 6)
    lat = np.eye(3) * 6.0
    beta = rng.standard_normal(dims + (1,))
    eps = 1e-9
    base = np.array([[3.0 + 0.37, 2.0 + 0.61, 4.0 + 0.13]])  # grid units
    for axis in range(3):
        lo = base.copy()
        hi = base.copy()
        lo[0, axis] = 3.0 - eps
        hi[0, axis] = 3.0 + eps
        pl = lo / 6.0 * 6.0  # grid spacing is 1 bohr
        ph = hi / 6.0 * 6.0
        for order in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (0, 2, 0),
                      (0, 0, 2), (1, 1, 0), (1, 0, 1), (0, 1, 1)]:
            a = oracle.bspline_reduced_derivative(beta, lat, pl, order)
            b = oracle.bspline_reduced_derivative(beta, lat, ph, order)
            assert abs(a - b).max() < 1e-6
        o = [0, 0, 0]
        o[axis] = 1
        a = oracle.lagrange_reduced_derivative(beta, lat, pl, o)
        b = oracle.lagrange_reduced_derivative(beta, lat, ph, o)
        assert abs(a - b).max() > 1e-3


def test_periodicity():
    """Shifting by lattice vectors leaves every output unchanged (Eq. reducedcoordinate)."""
    rng = np.random.default_rng(23)
    dims = (5, 6, 7)
    beta = rng.standard_normal(dims + (2,))
    pos = inputs.positions(NONORTHO, 30, 5)
    v0, g0, l0 = oracle.bspline_eval(beta, NONORTHO, pos)
    for shift in ([1, 0, 0], [0, -2, 1], [3, 1, -4]):
        v, g, l = oracle.bspline_eval(beta, NONORTHO, pos + NONORTHO @ np.array(shift, float))
        np.testing.assert_allclose(v, v0, atol=1e-11)
        np.testing.assert_allclose(g, g0, atol=1e-10)
        np.testing.assert_allclose(l, l0, atol=1e-9)


@pytest.mark.parametrize("method", ["smoothing", "interpolating"])
def test_convergence_order_under_refinement(method):
    """Sec. III A footnote: at a fixed cutoff the spline converges to the planewave sum as
    the grid is refined; cubic splines converge as h^4 for the value (h^3 gradient,
    h^2 Hessian-derived Laplacian, h^4 separate Laplacian table)."""
    lat = np.eye(3) * 5.0
    mil = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 1], [0, -1, -1], [1, -1, 0], [-1, 1, 0]],
                   dtype=np.int32)
    coef = np.array([[0.4 + 0.2j, 0.4 - 0.2j, 0.3, 0.3, -0.25j, 0.25j]])
    pos = inputs.positions(lat, 200, 13)
    pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
    errs = []
    for n in (8, 16, 32):
        dims = (n, n, n)
        tb = oracle.smoothing_tables if method == "smoothing" else oracle.interpolating_tables
        beta, blap = tb(lat, mil, coef, dims, laplacian=True)
        v, g, l = oracle.bspline_eval(beta, lat, pos)
        _, _, lt = oracle.bspline_eval(beta, lat, pos, beta_lap=blap)
        errs.append([np.abs(v - pv).max(), np.abs(g - pg).max(), np.abs(l - pl).max(),
                     np.abs(lt - pl).max()])
    errs = np.array(errs)
    ratio = errs[1] / errs[2]
    assert ratio[0] > 12 and ratio[3] > 12   # h^4
    assert ratio[1] > 6                        # h^3
    assert ratio[2] > 3                        # h^2


# ---------------------------------------------------------------------------
# adjoint (backward)
# ---------------------------------------------------------------------------

def _loss(beta, lat, pos, gv, gg, gl, beta_lap=None):
    v, g, l = oracle.bspline_eval(beta, lat, pos, beta_lap=beta_lap)
    return float(np.sum(gv * v) + np.sum(gg * g) + np.sum(gl * l))


@pytest.mark.parametrize("sep_lap", [False, True])
def test_adjoint_coefficients_dot_product_and_fd(sep_lap):
    """The loss is linear in beta: <dL/dbeta, dbeta> = L(dbeta) exactly, and a central
    difference on any entry is exact up to rounding."""
    rng = np.random.default_rng(30)
    dims = (5, 6, 7)
    beta = rng.standard_normal(dims + (3,))
    blap = rng.standard_normal(dims + (3,)) if sep_lap else None
    pos = inputs.positions(NONORTHO, 12, 6, -1, 2)
    gv, gg, gl = inputs.upstream_weights(12, 3, 31)
    db, dbl, _ = oracle.bspline_adjoint(beta, NONORTHO, pos, gv, gg, gl, beta_lap=blap)
    d = rng.standard_normal(beta.shape)
    zero = np.zeros_like(beta)
    lhs = np.sum(db * d)
    rhs = _loss(d, NONORTHO, pos, gv, gg, gl, beta_lap=zero if sep_lap else None)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    if sep_lap:
        lhs = np.sum(dbl * d)
        rhs = _loss(zero, NONORTHO, pos, gv, gg, gl, beta_lap=d)
        assert lhs == pytest.approx(rhs, rel=1e-12)
    for _ in range(5):
        idx = tuple(rng.integers(0, s) for s in beta.shape)
        bp = beta.copy()
        bm = beta.copy()
        bp[idx] += 0.5
        bm[idx] -= 0.5
        fd = (_loss(bp, NONORTHO, pos, gv, gg, gl, blap) - _loss(bm, NONORTHO, pos, gv, gg, gl, blap))
        assert db[idx] == pytest.approx(fd, rel=1e-9, abs=1e-11)


@pytest.mark.parametrize("sep_lap", [False, True])
def test_adjoint_positions_fd(sep_lap):
    """d loss / d r against central differences (h = 1e-5 bohr), away from grid planes
    where the Hessian-derived Laplacian has a kink."""
    rng = np.random.default_rng(32)
    dims = (6, 7, 8)
    lat = NONORTHO
    beta = rng.standard_normal(dims + (2,))
    blap = rng.standard_normal(dims + (2,)) if sep_lap else None
    pos = inputs.positions(lat, 40, 9)
    s = pos @ np.linalg.inv(lat).T * np.array(dims)
    t = s - np.floor(s)
    keep = np.all((t > 0.02) & (t < 0.98), axis=1)
    pos = pos[keep]
    gv, gg, gl = inputs.upstream_weights(len(pos), 2, 33)
    _, _, dpos = oracle.bspline_adjoint(beta, lat, pos, gv, gg, gl, beta_lap=blap)
    h = 1e-5
    fd = np.zeros_like(dpos)
    for p in range(len(pos)):
        for a in range(3):
            e = np.zeros_like(pos)
            e[p, a] = h
            fd[p, a] = (_loss(beta, lat, pos + e, gv, gg, gl, blap) -
                        _loss(beta, lat, pos - e, gv, gg, gl, blap)) / (2 * h)
    assert oracle.relative_error(dpos, fd) < 1e-6


# ---------------------------------------------------------------------------
# separate gradient tables for B-splines (Sec. III C)
# ---------------------------------------------------------------------------

def test_separate_gradient_tables_single_planewave_closed_form():
    """Smoothing spline of d_a phi for one planewave c e^{iG.r}, at grid points (weights
    [1/4, 1, 1/4, 0]): i G_a c e^{iG.r} prod_m (1 + cos th_m / 2)/gamma(th_m); the Laplacian
    table gives -|G|^2 times the same factor."""
    dims = np.array([8, 10, 12])
    n = np.array([2, -1, 3])
    mil = np.array([n, -n], dtype=np.int32)
    c = 0.7 - 0.2j
    coef = np.array([[c, np.conj(c)]])
    tabs = oracle.derivative_tables("smooth", NONORTHO, mil, coef, tuple(dims))
    rng = np.random.default_rng(31)
    j = rng.integers(0, dims, size=(20, 3))
    pos = (j / dims) @ NONORTHO.T
    v, g, l = oracle.bspline_eval_separate(tabs, NONORTHO, pos)
    th = 2 * np.pi * n / dims
    S = np.prod((1 + 0.5 * np.cos(th)) / oracle.gamma_axis(th))
    G = 2 * np.pi * np.linalg.inv(NONORTHO).T @ n
    e = c * np.exp(1j * pos @ G)
    np.testing.assert_allclose(v[:, 0], 2 * np.real(e) * S, atol=1e-12)
    np.testing.assert_allclose(g[:, :, 0], 2 * np.real(1j * e[:, None] * G[None, :]) * S, atol=1e-11)
    np.testing.assert_allclose(l[:, 0], -2 * (G @ G) * np.real(e) * S, atol=1e-10)


def test_interpolating_gradient_tables_reproduce_planewave_gradient_at_grid_points():
    """Interpolating B-splines pass through the grid values of the function they
    approximate, so separate gradient and Laplacian tables give the planewave gradient and
    Laplacian exactly at grid points."""
    dims = np.array([8, 9, 10])
    lat, mil, coef = inputs.random_cell(32, tuple(dims), 3, 5.0, 4.0, NONORTHO)
    tabs = oracle.derivative_tables("interp", lat, mil, coef, tuple(dims))
    rng = np.random.default_rng(33)
    pos = (rng.integers(0, dims, size=(20, 3)) / dims) @ lat.T
    v, g, l = oracle.bspline_eval_separate(tabs, lat, pos)
    pv, pg, pl, _ = oracle.pw_eval(lat, mil, coef, pos)
    assert oracle.relative_error(v, pv) < 1e-12
    assert oracle.relative_error(g, pg) < 1e-12
    assert oracle.relative_error(l, pl) < 1e-12


@pytest.mark.parametrize("method", ["smooth", "interp"])
def test_separate_gradient_converges_faster_than_derivative(method):
    """Sec. III C / Fig. 1: a separate approximation of the gradient converges like a
    value (h^4) where the derivative of the value spline converges as h^3."""
    lat = np.eye(3) * 5.0
    mil = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 1], [0, -1, -1], [1, -1, 0], [-1, 1, 0]],
                   dtype=np.int32)
    coef = np.array([[0.4 + 0.2j, 0.4 - 0.2j, 0.3, 0.3, -0.25j, 0.25j]])
    pos = inputs.positions(lat, 200, 34)
    _, pg, _, _ = oracle.pw_eval(lat, mil, coef, pos)
    sep, der = [], []
    for n in (8, 16, 32):
        tabs = oracle.derivative_tables(method, lat, mil, coef, (n, n, n))
        sep.append(np.abs(oracle.bspline_eval_separate(tabs, lat, pos)[1] - pg).max())
        der.append(np.abs(oracle.bspline_eval(tabs[0], lat, pos)[1] - pg).max())
    assert sep[1] / sep[2] > 12
    assert 6 < der[1] / der[2] < 12
    assert sep[2] < der[2]


# ---------------------------------------------------------------------------
# the paper's accuracy conclusions (Sec. III A, Fig. 1; Sec. IV) on the synthetic analogue
# ---------------------------------------------------------------------------

def test_fig1_conclusions_hold_for_the_oracle():
    """At natural spacing for every cutoff: smoothing B-splines are more accurate than
    interpolating splines, which are more accurate than Lagrange interpolation (values);
    pp-splines and interpolating B-splines give the same values; separate approximations of
    the gradient and Laplacian of the splines are more accurate than derivatives of the
    spline."""
    import fig1_analogue as f1
    rows = f1.run((10.0, 20.0, 40.0), use_oracle=True, n_orb=8, n_pos=500)
    for ecut in (10.0, 20.0, 40.0):
        r = {x["row"]: x for x in rows if x["ecut"] == ecut}
        assert r["smooth"]["value"] < r["interp"]["value"] < r["lagrange"]["value"]
        assert r["pp"]["value"] == pytest.approx(r["interp"]["value"], rel=1e-10)
        for m in ("smooth", "interp"):
            assert r[m + "_sep"]["lap"] < r[m]["lap"]
            assert r[m + "_sep"]["grad"] < r[m]["grad"]
        assert r["smooth_sep"]["lap"] < r["interp_sep"]["lap"] < r["lagrange"]["lap"]
        assert r["smooth_sep"]["grad"] < r["interp_sep"]["grad"] < r["lagrange"]["grad"]
    # the errors fall as the cutoff (and the natural grid) grows
    for lab in ("smooth", "interp", "lagrange"):
        v = [x["value"] for x in rows if x["row"] == lab]
        assert v[0] > v[1] > v[2]
